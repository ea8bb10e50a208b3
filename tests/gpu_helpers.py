"""Helpers of the GPU parity tests: flat device state <-> oracle per-patch arrays, error measure."""
import numpy as np
import torch

from paper_2506_16076_gb300 import workloads as W


def to_dev(per_patch):
    return torch.from_numpy(np.ascontiguousarray(W.flatten(per_patch))).cuda()


def to_dev_scalar_field(per_patch):
    return torch.from_numpy(np.ascontiguousarray(np.concatenate([a.ravel() for a in per_patch]))).cuda()


def from_dev(t, w, ncomp=4):
    a = t.detach().cpu().numpy()
    if ncomp == 1:
        a = a[None]
    out = W.unflatten(a, w)
    return [o[0] for o in out] if ncomp == 1 else out


def rel_err(gpu, orc, mask=None, floor=1e-2):
    """Per component max|gpu - orc| / max(max|orc_c|, floor * max_c' max|orc_c'|), as a list.

    The floor keeps a component that is identically ~0 (e.g. the transverse momentum of
    a planar shock tube) from turning rounding noise into an O(1) "relative" error."""
    ncomp = gpu[0].shape[0]
    scale = [max(np.abs(o[c]).max() for o in orc) for c in range(ncomp)]
    top = max(scale)
    errs = []
    for c in range(ncomp):
        num = max(np.abs(np.where(m, g[c] - o[c], 0.0) if m is not None else g[c] - o[c]).max()
                  for g, o, m in zip(gpu, orc, mask or [None] * len(gpu)))
        errs.append(num / max(scale[c], floor * top, 1e-300))
    return errs


def smooth_mu(w, seed, scale):
    """Seeded smooth non-negative viscosity field (a frozen mu for RHS parity)."""
    rng = np.random.default_rng(seed)
    a, b, c = rng.uniform(1, 3, 3)
    out = []
    for p in w.patches:
        x, y = W.patch_xy(p)
        out.append(scale * (1.0 + np.sin(a * x) * np.cos(b * y + c)) ** 2)
    return out


def rel_err_normwise(gpu, orc):
    """max over points and components of |gpu - orc|, over max |orc| (all components)."""
    top = max(np.abs(o).max() for o in orc)
    return max(np.abs(g - o).max() for g, o in zip(gpu, orc)) / max(top, 1e-300)


def fp64_floor(sv, fn):
    """Error of an FP64 evaluation of the same operator (continued data rounded to
    double, numpy's double-precision FFT, multipliers in double) against the long-double
    oracle: the accuracy any FP64 implementation can be expected to reach. For lines of
    ~1000-2000 points it exceeds 1e-11 (the derivative amplifies rounding at the highest
    modes)."""
    from oracle import fc

    def deriv64(Fc, beta):
        L = Fc.shape[-1]
        fac = 2j * np.pi * fc.mode_numbers(L) / float(beta)
        if L % 2 == 0:
            fac[L // 2] = 0.0
        return np.fft.ifft(fac * np.fft.fft(np.asarray(Fc, dtype=np.float64), axis=-1), axis=-1).real

    def filter64(Fc, alpha, p):
        L = Fc.shape[-1]
        k = fc.mode_numbers(L)
        if L % 2 == 0:
            k[L // 2] = L / 2
        return np.fft.ifft(fc.sigma(k, L, alpha, p) * np.fft.fft(np.asarray(Fc, dtype=np.float64), axis=-1),
                           axis=-1).real

    saved = fc.spectral_derivative, fc.spectral_filter
    fc.spectral_derivative, fc.spectral_filter = deriv64, filter64
    try:
        return fn()
    finally:
        fc.spectral_derivative, fc.spectral_filter = saved


def ulp_floor(fn, states, seed=0):
    """Per-component sensitivity of an operator to one unit of FP64 rounding in its input:
    rel_err of fn(states perturbed by a relative 2^-52 uniform noise) against fn(states).
    Any FP64 implementation whose pointwise arithmetic rounds in another order differs from
    the oracle by about this much."""
    rng = np.random.default_rng(seed)
    pert = [s * (1.0 + 2.0 ** -52 * rng.uniform(-1.0, 1.0, s.shape)) for s in states]
    return rel_err(fn(pert), fn(states))
