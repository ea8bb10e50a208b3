"""FC-Gram continuation, spectral derivative and spectral filter (oracle).

Test infrastructure only (see oracle/__init__.py).

Sec. 2.2: from N values F_j = F(x_j), x_j = j h, h = 1/(N-1), the FC-Gram
algorithm appends C continuation values (eq. (continuation)):
    F^c = [ F ; A_l Q^T F_l + A_r Q^T F_r ],
F_l / F_r = first / last d values. F^c is one period (length L = N + C, period
beta = L h) of a smooth periodic function whose Fourier coefficients are
differentiated by (2 pi i k / beta) (eq. (fc_der)) or filtered by
sigma(2k/(N+C)) = exp(-alpha_f (2k/(N+C))^p_f) (eq. (filtering), Sec. 4.3.1).

Precision: eq. (fc_der) and eq. (filtering) are exact linear maps of the data; the
oracle evaluates them in extended precision (numpy long double, 64-bit mantissa) and
rounds once to FP64 at the end, so that its own evaluation error stays far below the
FP64 rounding of any implementation it checks. The continued vector, the DFT, the
multipliers and the inverse DFT all stay in long double. The DFT is the definition
X_k = sum_j x_j exp(-2 pi i j k / L), computed by numpy's FFT routine on long-double
data as a library primitive (the test suite pins it against the explicit sum). An
FP64 direct sum is not accurate enough: on the Mach-25 fluxes (large mean, small
variation) every term is rounded at the size of the mean, and its error in a
derivative reaches 1.6e-10 of the result, where an FP64 FFT stays near 5e-12.
Mode numbers k run over the symmetric range -M..M; for even L the Nyquist
coefficient k = L/2 gets derivative factor 0 (keeps real data real) and filter
factor sigma(1).

Sec. 2.2 also admits end data with a derivative in place of the end value (the Neumann
variant, used for the adiabatic condition of Remark adiabatic): neumann_extend_ld builds
the Gram coefficients of (h F'_0, F_1, ..., F_{d-1}) and continues from them.
"""
import functools
import os

import numpy as np

_DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_2506_16076_gb300", "data")


@functools.lru_cache(maxsize=None)
def load_tables(d, C):
    """(Q, A_l, A_r) for matching order d and C continuation points (method data, Sec. 2.2)."""
    path = os.path.join(_DATA, f"fc_tables_d{d}.txt")
    with open(path) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines) and lines[i] != "end":
        assert lines[i] == f"d {d}", lines[i]
        c = int(lines[i + 1].split()[1])
        i += 2
        assert lines[i] == "Q"
        Q = np.array([[float(v) for v in lines[i + 1 + r].split()] for r in range(d)])
        i += 1 + d
        assert lines[i] == "AL"
        AL = np.array([[float(v) for v in lines[i + 1 + r].split()] for r in range(c)])
        i += 1 + c
        assert lines[i] == "AR"
        AR = np.array([[float(v) for v in lines[i + 1 + r].split()] for r in range(c)])
        i += 1 + c
        if c == C:
            return Q, AL, AR
    raise KeyError(f"no FC table for d={d}, C={C}")


def is_7smooth(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


@functools.lru_cache(maxsize=None)
def table_range(d):
    """Smallest and largest C with an FC table for order d."""
    path = os.path.join(_DATA, f"fc_tables_d{d}.txt")
    cs = []
    with open(path) as f:
        prev = None
        for ln in f:
            ln = ln.strip()
            if prev == f"d {d}" and ln.startswith("C "):
                cs.append(int(ln.split()[1]))
            prev = ln
    return min(cs), max(cs)


def transform_cost(L):
    """Cost rule of policy 2: L split greedily into factors 8, 4, 2, 3, 5, 7; each
    stage of radix R costs (L/R) B(R) with B(2, 4, 8, 3, 5, 7) = (4, 16, 52, 14, 36, 66),
    plus 4 (L/R)(R-1) on every stage except the last. None if a prime factor exceeds 7."""
    B = {2: 4, 4: 16, 8: 52, 3: 14, 5: 36, 7: 66}
    radices = []
    m = L
    for r in (8, 4, 2, 3, 5, 7):
        while m % r == 0:
            radices.append(r)
            m //= r
    if m != 1:
        return None
    total = 0
    for i, r in enumerate(radices):
        total += (L // r) * B[r]
        if i < len(radices) - 1:
            total += 4 * (L // r) * (r - 1)
    return total


def choose_C(N, C0, policy, d=5):
    """Continuation length for a line of N points (the paper leaves C free, Sec. 2.2).

    policy 0: C = C0 for every line (the paper uses one C per run).
    policy 1: smallest C >= C0 with N + C having no prime factor above 7.
    policy 2: among C0 <= C <= (largest tabulated C), the C whose N + C has the
    smallest transform_cost, ties to the smaller C; policy 1 if none qualifies."""
    if policy == 0:
        return C0
    if policy == 2:
        best = None
        for C in range(C0, table_range(d)[1] + 1):
            k = transform_cost(N + C)
            if k is not None and (best is None or k < best[0]):
                best = (k, C)
        if best is not None:
            return best[1]
    C = C0
    while not is_7smooth(N + C):
        C += 1
    return C


LD = np.longdouble
CLD = np.clongdouble
PI_LD = 4 * np.arctan(LD(1))  # pi to long-double precision


def continuation_ld(F, d, C):
    """Eq. (continuation): the C appended values of the FC-Gram continued vector, in
    long double. F: (..., N) real. Returns (..., C).

    The matrices A_l, A_r of an accurate d = 5 continuation have entries of order 1e4
    whose contributions cancel, which is one more reason to evaluate in extended
    precision."""
    Q, AL, AR = load_tables(d, C)
    Fl = np.asarray(F)[..., :d].astype(LD)
    Fr = np.asarray(F)[..., -d:].astype(LD)
    return (Fl @ Q.astype(LD)) @ AL.T.astype(LD) + (Fr @ Q.astype(LD)) @ AR.T.astype(LD)  # A_l Q^T F_l + A_r Q^T F_r


def continuation(F, d, C):
    """Eq. (continuation), rounded once to FP64."""
    return continuation_ld(F, d, C).astype(np.float64)


def extend_ld(F, d, C):
    """The continued vector F^c = [F; continuation] of length N + C, in long double."""
    return np.concatenate([np.asarray(F).astype(LD), continuation_ld(F, d, C)], axis=-1)


def neumann_coefficients(d, C):
    """Sec. 2.2, the Neumann variant of the FC-Gram continuation (end data with the
    derivative in place of the end value): the d x d matrix that maps the left-end data
    (h F'_0, F_1, ..., F_{d-1}) to the coefficients of the degree d-1 polynomial they fix
    in the Gram basis of the table (the columns of Q, orthonormal on the d matching
    points 0..d-1). Built as the inverse of the matrix whose row 0 holds the Gram
    polynomials' derivatives at point 0 (exact Lagrange derivative weights on the nodes
    0..d-1) and whose rows 1..d-1 hold their values, in long double."""
    from fractions import Fraction
    Q, _, _ = load_tables(d, C)
    nodes = range(d)
    w0 = []  # l_j'(0) for the Lagrange basis on the nodes 0..d-1
    for j in nodes:
        others = [m for m in nodes if m != j]
        den = Fraction(1)
        for m in others:
            den *= Fraction(j - m)
        num = Fraction(0)
        for skip in others:  # derivative of prod_m (x - m) at x = 0
            term = Fraction(1)
            for m in others:
                if m != skip:
                    term *= Fraction(0 - m)
            num += term
        w0.append(num / den)
    QL = Q.astype(LD)
    V = np.empty((d, d), dtype=LD)
    V[0] = sum(LD(w0[j].numerator) / LD(w0[j].denominator) * QL[j] for j in nodes)
    V[1:] = QL[1:]
    return _inv_ld(V)


def _inv_ld(V):
    """Gauss-Jordan inverse with partial pivoting in long double."""
    n = V.shape[0]
    A = np.concatenate([V.astype(LD), np.eye(n, dtype=LD)], axis=1)
    for col in range(n):
        piv = col + int(np.argmax(np.abs(A[col:, col])))
        A[[col, piv]] = A[[piv, col]]
        A[col] = A[col] / A[col, col]
        for r in range(n):
            if r != col:
                A[r] = A[r] - A[r, col] * A[col]
    return A[:, n:]


def neumann_extend_ld(F, dF0, d, C):
    """The Neumann-variant continued vector of a line whose left end carries a derivative
    condition (Sec. 2.2; Remark adiabatic): F[1:] are the values at points 1..N-1, dF0 the
    derivative at point 0 times the spacing. Returns (wall value, continued vector of
    length N + C) in long double: the wall value is that of the polynomial the left-end
    data fix, the continuation A_l c~ + A_r Q^T F_r with c~ its Gram coefficients."""
    Q, AL, AR = load_tables(d, C)
    Ft = np.asarray(F).astype(LD)
    data = np.concatenate([np.atleast_1d(LD(dF0)), Ft[1:d]])
    c = neumann_coefficients(d, C) @ data
    wall = c @ Q[0].astype(LD)
    ext = AL.astype(LD) @ c + AR.astype(LD) @ (Q.T.astype(LD) @ Ft[-d:])
    full = Ft.copy()
    full[0] = wall
    return wall, np.concatenate([full, ext])


def dft(x):
    """X_k = sum_j x_j exp(-2 pi i j k / L) along the last axis (definition), in long double."""
    return np.fft.fft(np.asarray(x).astype(CLD), axis=-1)


def idft(X):
    """x_j = (1/L) sum_k X_k exp(+2 pi i j k / L) along the last axis (definition), in long double."""
    return np.fft.ifft(np.asarray(X).astype(CLD), axis=-1)


def dft_direct(x):
    """The explicit sum of the DFT definition in long double (O(L^2); pins dft)."""
    x = np.asarray(x).astype(CLD)
    L = x.shape[-1]
    j = np.arange(L)
    a = -2 * PI_LD * (np.outer(j, j) % L).astype(LD) / L  # jk reduced mod L: same value, exact argument
    M = np.cos(a) + 1j * np.sin(a)
    return (x[..., None, :] * M).sum(axis=-1)


def mode_numbers(L):
    """Signed mode numbers of DFT index 0..L-1 in the symmetric range."""
    k = np.arange(L)
    return np.where(k <= L // 2, k, k - L).astype(float)


def spectral_derivative(Fc, beta):
    """Eq. (fc_der): differentiate the periodic extension of one period Fc of length beta.

    Evaluated in long double; returns long double (callers round once)."""
    L = Fc.shape[-1]
    k = mode_numbers(L).astype(LD)
    fac = 2j * PI_LD * k / LD(beta)
    if L % 2 == 0:
        fac[L // 2] = 0.0
    return idft(fac * dft(Fc)).real


def sigma(k, L, alpha, p):
    """Filter function of eq. (filtering): exp(-alpha (2k/(N+C))^p)."""
    return np.exp(-alpha * (2.0 * k / L) ** p)


def spectral_filter(Fc, alpha, p):
    """Eq. (filtering) on one period, in long double; returns long double."""
    L = Fc.shape[-1]
    k = mode_numbers(L)
    if L % 2 == 0:
        k[L // 2] = L / 2
    s = np.exp(-LD(alpha) * (LD(2) * k.astype(LD) / LD(L)) ** p)
    return idft(s * dft(Fc)).real


def _real_linear(op):
    """Apply a real linear operator to complex data part by part (complex-step derivatives)."""
    def wrapped(F, *a):
        if np.iscomplexobj(F):
            return op(F.real, *a) + 1j * op(F.imag, *a)
        return op(F, *a)
    wrapped.__doc__ = op.__doc__
    wrapped.__name__ = op.__name__
    return wrapped


@_real_linear
def fc_derivative(F, h, d, C):
    """FC derivative along the last axis of values on x_j = j h (Sec. 2.2).

    The continued vector has L = N + C entries and period beta = L h."""
    N = F.shape[-1]
    return spectral_derivative(extend_ld(F, d, C), (N + C) * h)[..., :N].astype(np.float64)


@_real_linear
def periodic_derivative(F, h):
    """Fourier derivative of samples of a periodic function (no continuation), period N h."""
    N = F.shape[-1]
    return spectral_derivative(np.asarray(F).astype(LD), N * h).astype(np.float64)


@_real_linear
def fc_filter(F, d, C, alpha, p):
    N = F.shape[-1]
    return spectral_filter(extend_ld(F, d, C), alpha, p)[..., :N].astype(np.float64)


@_real_linear
def periodic_filter(F, alpha, p):
    return spectral_filter(np.asarray(F).astype(LD), alpha, p).astype(np.float64)


@_real_linear
def fc_derivative_T(G, h, d, C):
    """Transpose of fc_derivative as a linear map R^N -> R^N.

    fc_derivative = restrict o (spectral derivative on the period) o extend, with
    extend = [I; M], M = continuation matrix (eq. continuation). The spectral
    derivative is a real skew-symmetric circulant, so the transpose is
    extend^T o (-spectral derivative) o zero-padding: the continuation part is folded
    back onto the first and last d points with (A_l Q^T)^T and (A_r Q^T)^T."""
    N = G.shape[-1]
    L = N + C
    Z = np.concatenate([np.asarray(G).astype(LD), np.zeros(G.shape[:-1] + (C,), LD)], axis=-1)
    W = -spectral_derivative(Z, L * h)
    Q, AL, AR = load_tables(d, C)
    out = W[..., :N].copy()
    ext = W[..., N:]
    out[..., :d] += (ext @ AL.astype(LD)) @ Q.T.astype(LD)  # (A_l Q^T)^T w
    out[..., N - d:] += (ext @ AR.astype(LD)) @ Q.T.astype(LD)  # (A_r Q^T)^T w
    return out.astype(np.float64)


@_real_linear
def fc_filter_T(G, d, C, alpha, p):
    """Transpose of fc_filter: extend^T o (spectral filter) o zero-padding. The filter
    multiplier is real and even in k, so the filter on the period is a symmetric circulant."""
    N = G.shape[-1]
    Z = np.concatenate([np.asarray(G).astype(LD), np.zeros(G.shape[:-1] + (C,), LD)], axis=-1)
    W = spectral_filter(Z, alpha, p)
    Q, AL, AR = load_tables(d, C)
    out = W[..., :N].copy()
    ext = W[..., N:]
    out[..., :d] += (ext @ AL.astype(LD)) @ Q.T.astype(LD)
    out[..., N - d:] += (ext @ AR.astype(LD)) @ Q.T.astype(LD)
    return out.astype(np.float64)


@_real_linear
def periodic_derivative_T(G, h):
    """Transpose of the periodic Fourier derivative: its negative (skew-symmetric circulant)."""
    return -periodic_derivative(G, h)
