"""Pins of the oracle's FC-Gram continuation, derivative and filter (Sec. 2.2, Sec. 4.3)."""
import numpy as np
import pytest

from oracle import fc


def test_dft_matches_closed_forms():
    L = 37
    j = np.arange(L)
    delta = np.zeros(L)
    delta[0] = 1.0
    assert np.allclose(fc.dft(delta), np.ones(L), atol=1e-14)
    for m in (0, 1, 5, 36):
        X = fc.dft(np.exp(2j * np.pi * m * j / L))
        ref = np.zeros(L, complex)
        ref[m] = L
        assert np.abs(X - ref).max() < 1e-12
    x = np.random.default_rng(0).normal(size=L)
    assert np.abs(fc.idft(fc.dft(x)) - x).max() < 5e-14


@pytest.mark.parametrize("L", [7, 37, 64, 105, 378])
def test_dft_is_the_explicit_sum(L):
    # the library FFT on long-double data against the O(L^2) sum of the definition
    rng = np.random.default_rng(L)
    x = rng.normal(size=(3, L)) + 1j * rng.normal(size=(3, L))
    X, Xd = fc.dft(x), fc.dft_direct(x)
    assert X.dtype == np.clongdouble
    assert float(np.abs(X - Xd).max()) < 1e-16 * L
    xi = fc.idft(Xd)
    assert float(np.abs(xi - x).max()) < 1e-17 * L


def test_derivative_ignores_a_large_constant():
    # D(F + c) = D(F) exactly for a periodic derivative; with dyadic samples F + c is exact
    # in FP64, so any difference is the oracle's own evaluation error (an FP64 direct DFT
    # leaves about 1e-10 of max|D F| here)
    N = 384
    t = np.arange(N) / N
    F = np.round((np.sin(2 * np.pi * t) + 0.3 * np.cos(6 * np.pi * t + 1.0)) * 2.0**20) / 2.0**20
    c = 1024.0
    assert np.all((F + c) - c == F)
    D0 = fc.periodic_derivative(F, 1.0 / N)
    D1 = fc.periodic_derivative(F + c, 1.0 / N)
    assert np.abs(D1 - D0).max() < 1e-14 * np.abs(D0).max()


@pytest.mark.parametrize("d", [5, 2])
def test_gram_basis_orthogonal_and_polynomial(d):
    for C in (27, 40, 71):
        Q, AL, AR = fc.load_tables(d, C)
        assert AL.shape == (C, d) and AR.shape == (C, d)
        assert np.abs(Q.T @ Q - np.eye(d)).max() < 1e-14
        # columns of Q span the polynomials of degree < d on t = 0..d-1
        V = np.vander(np.arange(d, dtype=float), d, increasing=True)
        assert np.abs(Q @ (Q.T @ V) - V).max() < 1e-12 * np.abs(V).max()


@pytest.mark.parametrize("C", [27, 33, 40, 55, 71])
@pytest.mark.parametrize("N", [32, 100, 400])
def test_fc_derivative_polynomials_below_d(N, C):
    # Polynomial exactness of the Gram basis (Sec. 2.2): tolerance grows with N
    # (derivative amplification ~ pi N) from the tables' ~1e-14 continuation accuracy.
    d = 5
    x = np.linspace(0.0, 1.0, N)
    h = 1.0 / (N - 1)
    for deg in range(d):
        F = (x - 0.3) ** deg
        dF = deg * (x - 0.3) ** (deg - 1) if deg else 0 * x
        D = fc.fc_derivative(F, h, d, C)
        assert np.abs(D - dF).max() <= 1.5e-13 * N * max(1.0, np.abs(dF).max()), (deg, N, C)


def test_fc_derivative_degree_d_is_not_exact():
    # a planted check on the pin above: degree d is outside the exact class
    N, d, C = 64, 5, 27
    x = np.linspace(0.0, 1.0, N)
    D = fc.fc_derivative(x ** 9, 1.0 / (N - 1), d, C)
    assert np.abs(D - 9 * x ** 8).max() > 1e-8


def test_fc_derivative_convergence_smooth_nonperiodic():
    errs = []
    for N in (50, 100, 200, 400):
        x = np.linspace(0.0, 1.0, N)
        F = np.exp(np.sin(3 * x))
        D = fc.fc_derivative(F, 1.0 / (N - 1), 5, 27)
        errs.append(np.abs(D - 3 * np.cos(3 * x) * F).max())
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(3)]
    assert min(rates) > 3.5, (errs, rates)  # order d-1 = 4 for d = 5
    assert errs[-1] < 3e-8  # max |F'| is about 4.4


def test_fc_derivative_on_other_intervals_scales():
    # derivative on [a, b] with spacing h scales as 1/h (Sec. 2.2, re-scaling to [0,1])
    N = 80
    x = np.linspace(2.0, 5.0, N)
    F = np.sin(x)
    D = fc.fc_derivative(F, 3.0 / (N - 1), 5, 27)
    assert np.abs(D - np.cos(x)).max() < 5e-7  # fourth-order error at h = 3/79


def test_periodic_derivative_and_filter_closed_forms():
    N = 64
    x = np.arange(N) / N
    F = np.sin(2 * np.pi * 3 * x) + 0.5 * np.cos(2 * np.pi * 7 * x)
    dF = 2 * np.pi * 3 * np.cos(2 * np.pi * 3 * x) - 0.5 * 2 * np.pi * 7 * np.sin(2 * np.pi * 7 * x)
    assert np.abs(fc.periodic_derivative(F, 1.0 / N) - dF).max() < 1e-11
    # sigma(0) = 1, sigma(+-1) = exp(-alpha) (eq. filtering)
    assert fc.sigma(0, 10, 10.0, 14) == 1.0
    assert abs(fc.sigma(5, 10, 10.0, 14) - np.exp(-10.0)) < 1e-16
    assert abs(fc.sigma(-5, 10, 10.0, 14) - np.exp(-10.0)) < 1e-16
    # each Fourier mode k is multiplied by sigma(2k/N); the Nyquist mode by exp(-10)
    ref = np.exp(-10 * (6 / N) ** 14) * np.sin(2 * np.pi * 3 * x) + 0.5 * np.exp(-10 * (14 / N) ** 14) * np.cos(2 * np.pi * 7 * x)
    assert np.abs(fc.periodic_filter(F, 10.0, 14) - ref).max() < 1e-14
    nyq = np.cos(np.pi * np.arange(N))
    assert np.abs(fc.periodic_filter(nyq, 10.0, 14) - np.exp(-10.0) * nyq).max() < 1e-14


def test_fc_filter_keeps_smooth_lines():
    N = 120
    x = np.linspace(0, 1, N)
    F = 1.0 + 0.3 * x - 0.2 * x ** 2
    G = fc.fc_filter(F, 5, 27, 10.0, 14)
    assert np.abs(G - F).max() < 1e-11  # continuation high modes are tiny but not zero


def test_choose_C_policy_1_is_minimal():
    assert fc.choose_C(128, 27, 0) == 27
    for N in range(10, 1100):
        C = fc.choose_C(N, 27, 1)
        assert 27 <= C <= 71 and fc.is_7smooth(N + C)
        assert all(not fc.is_7smooth(N + c) for c in range(27, C))
    assert fc.choose_C(160, 27, 1) == 29  # 189 = 3^3 7


def test_choose_C_policies():
    # policy 1: smallest C >= 27 with N + C free of primes above 7
    assert fc.choose_C(160, 27, 1) == 29  # 189 = 3^3 7
    assert fc.choose_C(128, 27, 1) == 32  # 160
    # policy 2, worked by hand from the stated cost rule: N = 160 -> 189 = 3.3.3.7 costs
    # 3 (63 * 14) + 27 * 66 + 3 * 4 * 189 * 2/3 = 5940; 192 = 8.8.3 costs
    # 2 (24 * 52) + 64 * 14 + 2 * 4 * 24 * 7 = 4736, the least over C = 27..71
    assert fc.transform_cost(189) == 5940 and fc.transform_cost(192) == 4736
    assert fc.choose_C(160, 27, 2) == 32
    assert fc.transform_cost(187) is None  # 11 x 17
    assert fc.choose_C(48, 27, 2) == 32  # 80 = 8.2.5
    assert fc.choose_C(384, 27, 2) == 64  # 448 = 8.8.7
    lo, hi = fc.table_range(5)
    assert (lo, hi) == (27, 71)
    for n in range(10, 600, 7):
        C = fc.choose_C(n, 27, 2)
        assert lo <= C <= hi and fc.transform_cost(n + C) == min(
            fc.transform_cost(n + c) for c in range(27, hi + 1) if fc.transform_cost(n + c) is not None)


@pytest.mark.parametrize("d", [2, 5])
def test_neumann_continuation_reproduces_zero_slope_polynomials(d):
    # Sec. 2.2, Neumann variant: data (h F'_0 = 0, F_1, ..., F_{N-1}) of a polynomial of
    # degree < d with zero slope at the wall give back its wall value, and the continued
    # vector differentiates it (the continuation of a polynomial of degree < d is exact)
    N, C = 60, 31
    h = 1.0 / (N - 1)
    x = np.arange(N) * h
    p = 1.0 + 0.7 * x ** 2 if d > 2 else np.full(N, 1.3)
    dp = 1.4 * x if d > 2 else np.zeros(N)
    wall, ext = fc.neumann_extend_ld(p, 0.0, d, C)
    assert abs(float(wall) - p[0]) < 1e-13
    D = fc.spectral_derivative(ext, (N + C) * h)[:N].astype(np.float64)
    assert np.abs(D - dp).max() < 2e-10 * N


@pytest.mark.parametrize("d", [2, 5])  # the orders with tables
def test_neumann_wall_value_is_the_adiabatic_wall_temperature(d):
    # the wall value of the Neumann FC end data with zero derivative (Gram-basis
    # construction) equals the adiabatic wall temperature the solver imposes (polynomial
    # elimination, solver.adiabatic_weights), and the Neumann continued vector equals the
    # ordinary continuation of the line whose wall entry holds that temperature
    from oracle import solver as S
    rng = np.random.default_rng(d)
    N, C = 48, 27
    th = 1.0 + 0.1 * rng.normal(size=N)
    wall, ext = fc.neumann_extend_ld(th, 0.0, d, C)
    wts = S.adiabatic_weights(d)
    ref = sum(w * th[1 + j] for j, w in enumerate(wts))
    assert abs(float(wall) - ref) < 1e-14 * abs(ref)
    th2 = th.copy()
    th2[0] = float(wall)
    ext2 = fc.extend_ld(th2, d, C)
    assert np.abs((ext - ext2).astype(np.float64)).max() < 1e-11
