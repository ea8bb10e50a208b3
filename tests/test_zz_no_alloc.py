"""The allocation-free single-patch RHS entry point against the context-based fc_rhs.

Callers that cannot allocate device memory (code inside a host memory manager that owns
all device memory, plug-ins whose host forbids allocation) use fc_rhs_patch_noalloc: its
scratch is a static device array, so the check here is that it reproduces fc_rhs of the
same patch (within the RHS tolerance of the other GPU tests) on two calls in a row, i.e.
that the shared array carries nothing from one call into the next; on a rectangular box
it is also held to the oracle."""
import numpy as np
import pytest
import torch

from oracle import solver as S
from paper_2506_16076_gb300 import workloads as W
from tests.gpu_helpers import fp64_floor, from_dev, rel_err, smooth_mu, to_dev, to_dev_scalar_field

RHS_TOL = 1e-11

pytestmark = pytest.mark.gpu


def test_noalloc_rhs_matches_context_rhs(gpu_lib):
    w = W.sod128(96)  # one affine patch, C = 27 on every line
    p = w.patches[0]
    ctx = gpu_lib.Context(w)
    refs = []
    for seed in (3, 4):
        st = W.random_smooth_state(w, seed=seed, amp=0.2)
        mu = smooth_mu(w, seed=seed, scale=0.01)
        e, m = to_dev(st), to_dev_scalar_field(mu)
        ref = torch.empty_like(e)
        ctx.rhs(e, ref, m)
        refs.append((e, m, ref))
    for e, m, ref in refs:  # two calls in a row, different inputs
        out = torch.full_like(e, float("nan"))
        gpu_lib.rhs_patch_noalloc(e, m, out, p.n1, p.n2, p.geom, w.params.d, w.params.C0, w.params.gamma)
        torch.cuda.synchronize()
        errs = rel_err(from_dev(out, w), from_dev(ref, w))
        assert max(errs) < 1e-11, errs


def _box(n1, n2, box, C):
    fs = (1.0, 0.0, 0.0, 1.0)
    p = W.PatchDesc(W.AFFINE, n1, n2, box, (W.DIRICHLET,) * 4, bc=(fs,) * 4)
    return W.Workload(f"box{n1}x{n2}", [p], W.Params(d=5, C0=C, c_policy=0), freestream=fs, init="freestream",
                      steps=1)


@pytest.mark.parametrize("n1,n2,box,C", [
    (160, 72, (-0.3, 1.9, 0.25, 0.9), 32),  # rectangular, non-unit box, another C (L = 192, 104)
    (997, 37, (0.0, 2.0, -0.5, 0.5), 27),   # the largest continued length, n1 + C = 1024
])
def test_noalloc_rectangular_and_longest(gpu_lib, n1, n2, box, C):
    # tolerance as for every RHS: 1e-11, or twice the error of an FP64-FFT evaluation of
    # the same operator where that is larger (lines of about 1000 points); the two entry
    # points transform with different FFT stage orders, so they round differently
    w = _box(n1, n2, box, C)
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    for seed in (7, 8):  # two calls in a row
        st = W.random_smooth_state(w, seed=seed, amp=0.2)
        mu = smooth_mu(w, seed=seed, scale=0.01)
        e, m = to_dev(st), to_dev_scalar_field(mu)
        ref = torch.empty_like(e)
        ctx.rhs(e, ref, m)
        out = torch.full_like(e, float("nan"))
        gpu_lib.rhs_patch_noalloc(e, m, out, n1, n2, box, 5, C, w.params.gamma)
        torch.cuda.synchronize()
        got = from_dev(out, w)
        orc = sv.rhs(st, mu)
        tol = max(RHS_TOL, 2 * max(rel_err(fp64_floor(sv, lambda: sv.rhs(st, mu)), orc)))
        errs = rel_err(got, from_dev(ref, w))
        assert max(errs) < 2 * tol, (errs, tol)
        errs = rel_err(got, orc)
        assert max(errs) < tol, (errs, tol)


def test_noalloc_rejects_bad_arguments(gpu_lib):
    n1, n2 = 64, 48
    e = torch.zeros(4, n1 * n2, dtype=torch.float64, device="cuda")
    m = torch.zeros(n1 * n2, dtype=torch.float64, device="cuda")
    box = (0.0, 1.0, 0.0, 1.0)
    with pytest.raises(gpu_lib.FcError):  # C outside the tabulated range
        gpu_lib.rhs_patch_noalloc(e, m, e.clone(), n1, n2, box, 5, 200)
    with pytest.raises(gpu_lib.FcError):  # state of the wrong size
        gpu_lib.rhs_patch_noalloc(e[:, :-1].contiguous(), m, e.clone(), n1, n2, box, 5, 27)
    with pytest.raises(gpu_lib.FcError):  # viscosity of the wrong dtype
        gpu_lib.rhs_patch_noalloc(e, m.float(), e.clone(), n1, n2, box, 5, 27)


def test_noalloc_rejects_oversized_patch(gpu_lib):
    e = torch.zeros(4, 600 * 600, dtype=torch.float64, device="cuda")
    m = torch.zeros(600 * 600, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.FcError):
        gpu_lib.rhs_patch_noalloc(e, m, e.clone(), 600, 600, (0.0, 1.0, 0.0, 1.0), 5, 27)
