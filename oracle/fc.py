"""FC-Gram continuation, spectral derivative and spectral filter (oracle).

Test infrastructure only (see oracle/__init__.py).

Sec. 2.2: from N values F_j = F(x_j), x_j = j h, h = 1/(N-1), the FC-Gram
algorithm appends C continuation values (eq. (continuation)):
    F^c = [ F ; A_l Q^T F_l + A_r Q^T F_r ],
F_l / F_r = first / last d values. F^c is one period (length L = N + C, period
beta = L h) of a smooth periodic function whose Fourier coefficients are
differentiated by (2 pi i k / beta) (eq. (fc_der)) or filtered by
sigma(2k/(N+C)) = exp(-alpha_f (2k/(N+C))^p_f) (eq. (filtering), Sec. 4.3.1).

The DFT here is the definition X_k = sum_j x_j exp(-2 pi i j k / L), written
as an explicit L x L matrix product, so this module shares nothing with an FFT.
Mode numbers k run over the symmetric range -M..M; for even L the Nyquist
coefficient k = L/2 gets derivative factor 0 (keeps real data real) and filter
factor sigma(1).
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


def choose_C(N, C0, policy):
    """Continuation length for a line of N points.

    policy 0: C = C0 for every line (the paper uses one C per run).
    policy 1: smallest C >= C0 with N + C having no prime factor above 7
    (a reading of the free parameter C; see the design notes)."""
    if policy == 0:
        return C0
    C = C0
    while not is_7smooth(N + C):
        C += 1
    return C


def continuation(F, d, C):
    """Eq. (continuation): the C appended values of the FC-Gram continued vector.

    F: (..., N) real. Returns (..., C). The matrices A_l, A_r of an accurate d = 5
    continuation have entries of order 1e4 whose contributions cancel, so the
    product is evaluated in extended precision and rounded once to FP64 (same
    formula, smaller evaluation error)."""
    Q, AL, AR = load_tables(d, C)
    ld = np.longdouble
    Fl = F[..., :d].astype(ld)
    Fr = F[..., -d:].astype(ld)
    ext = (Fl @ Q.astype(ld)) @ AL.T.astype(ld) + (Fr @ Q.astype(ld)) @ AR.T.astype(ld)  # A_l Q^T F_l + A_r Q^T F_r
    return ext.astype(np.float64)


@functools.lru_cache(maxsize=None)
def dft_matrix(L, sign):
    j = np.arange(L)
    return np.exp(sign * 2j * np.pi * (np.outer(j, j) % L) / L)  # jk reduced mod L: same value, exact argument


def dft(x):
    """X_k = sum_j x_j exp(-2 pi i j k / L) along the last axis (definition)."""
    L = x.shape[-1]
    return x @ dft_matrix(L, -1).T


def idft(X):
    """x_j = (1/L) sum_k X_k exp(+2 pi i j k / L) along the last axis (definition)."""
    L = X.shape[-1]
    return (X @ dft_matrix(L, +1).T) / L


def mode_numbers(L):
    """Signed mode numbers of DFT index 0..L-1 in the symmetric range."""
    k = np.arange(L)
    return np.where(k <= L // 2, k, k - L).astype(float)


def spectral_derivative(Fc, beta):
    """Eq. (fc_der): differentiate the periodic extension of one period Fc of length beta."""
    L = Fc.shape[-1]
    k = mode_numbers(L)
    fac = 2j * np.pi * k / beta
    if L % 2 == 0:
        fac[L // 2] = 0.0
    return idft(fac * dft(Fc)).real


def sigma(k, L, alpha, p):
    """Filter function of eq. (filtering): exp(-alpha (2k/(N+C))^p)."""
    return np.exp(-alpha * (2.0 * k / L) ** p)


def spectral_filter(Fc, alpha, p):
    L = Fc.shape[-1]
    k = mode_numbers(L)
    if L % 2 == 0:
        k[L // 2] = L / 2
    return idft(sigma(k, L, alpha, p) * dft(Fc)).real


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
    Fc = np.concatenate([F, continuation(F, d, C)], axis=-1)
    return spectral_derivative(Fc, (N + C) * h)[..., :N]


@_real_linear
def periodic_derivative(F, h):
    """Fourier derivative of samples of a periodic function (no continuation), period N h."""
    N = F.shape[-1]
    return spectral_derivative(F, N * h)


@_real_linear
def fc_filter(F, d, C, alpha, p):
    N = F.shape[-1]
    Fc = np.concatenate([F, continuation(F, d, C)], axis=-1)
    return spectral_filter(Fc, alpha, p)[..., :N]


@_real_linear
def periodic_filter(F, alpha, p):
    return spectral_filter(F, alpha, p)


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
    Z = np.concatenate([G, np.zeros(G.shape[:-1] + (C,))], axis=-1)
    W = -spectral_derivative(Z, L * h)
    Q, AL, AR = load_tables(d, C)
    out = W[..., :N].copy()
    ext = W[..., N:]
    out[..., :d] += (ext @ AL) @ Q.T  # (A_l Q^T)^T w
    out[..., N - d:] += (ext @ AR) @ Q.T  # (A_r Q^T)^T w
    return out


@_real_linear
def periodic_derivative_T(G, h):
    """Transpose of the periodic Fourier derivative: its negative (skew-symmetric circulant)."""
    return -periodic_derivative(G, h)
