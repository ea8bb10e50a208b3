"""The allocation-free single-patch RHS entry point against the context-based fc_rhs.

Callers that cannot allocate device memory use fc_rhs_patch_noalloc: its scratch is a
static device array, so the check here is that it reproduces fc_rhs of the same patch
(within the RHS tolerance of the other GPU tests) on two calls in a row, i.e. that the
shared array carries nothing from one call into the next."""
import numpy as np
import pytest
import torch

from paper_2506_16076_gb300 import workloads as W
from tests.gpu_helpers import from_dev, rel_err, smooth_mu, to_dev, to_dev_scalar_field

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


def test_noalloc_rejects_oversized_patch(gpu_lib):
    e = torch.zeros(4, 600 * 600, dtype=torch.float64, device="cuda")
    m = torch.zeros(600 * 600, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.FcError):
        gpu_lib.rhs_patch_noalloc(e, m, e.clone(), 600, 600, (0.0, 1.0, 0.0, 1.0), 5, 27)
