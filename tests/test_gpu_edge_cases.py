"""Edge cases of the line engine against the oracle: the shortest continued lines
(N = 2d), prime and long line lengths (generic-radix stages, continued lengths above
2000), both continuation-length policies. Ragged hole-cut segments and fully blanked
patches are covered by the multi-patch and full-size tests. Tolerance: 1e-11, or twice
the error of an FP64 FFT evaluation of the same operator where that is larger (long
lines: 7e-10 at N = 2047)."""
import numpy as np
import pytest
import torch

from oracle import solver as S
from paper_2506_16076_gb300 import workloads as W
from tests.gpu_helpers import fp64_floor, from_dev, rel_err, smooth_mu, to_dev, to_dev_scalar_field

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-11


def _box(n1, n2, policy):
    fs = (1.4, 1.0, 0.3, 1.0)
    p = W.PatchDesc(W.AFFINE, n1, n2, (0.0, 1.0, 0.0, 0.7), (W.DIRICHLET,) * 4, bc=(fs,) * 4)
    return W.Workload(f"box_{n1}x{n2}", [p], W.Params(c_policy=policy), fs, "freestream", 1)


CASES = [(10, 10, 0), (10, 10, 2), (11, 23, 0), (23, 11, 2), (2047, 12, 0), (12, 1021, 2), (97, 89, 0)]


@pytest.mark.parametrize("n1,n2,policy", CASES)
def test_rhs_and_filter_extreme_lengths(gpu_lib, n1, n2, policy):
    w = _box(n1, n2, policy)
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    st = W.random_smooth_state(w, seed=n1 + n2, amp=0.2)
    mu = smooth_mu(w, seed=2, scale=0.01)
    out = torch.empty_like(to_dev(st))
    ctx.rhs(to_dev(st), out, to_dev_scalar_field(mu))
    torch.cuda.synchronize()
    ref = sv.rhs(st, mu)
    tol = max(RHS_TOL, 2 * max(rel_err(fp64_floor(sv, lambda: sv.rhs(st, mu)), ref)))
    errs = rel_err(from_dev(out, w), ref)
    assert max(errs) < tol, (errs, tol)
    e = to_dev(st)
    ctx.filter(e)
    torch.cuda.synchronize()
    ref = sv.filter(st)
    tol = max(RHS_TOL, 2 * max(rel_err(fp64_floor(sv, lambda: sv.filter(st)), ref)))
    errs = rel_err(from_dev(e, w), ref)
    assert max(errs) < tol, (errs, tol)
