"""100 steps of Algorithm 1 on curvilinear overlapping patches against the oracle.

small_multipatch_grid (a stretched, twisted annulus with a no-slip adiabatic wall and four
bulged boxes cut by the hole, all given as GRID patches), from a seeded smooth state, with
the per-step filter and the time step of eq. CFL computed on each side and the viscosity
of the first step held fixed (the oracle's, stored with the state): within 1e-8 relative
per component after 100 steps. The expected state is the oracle's run stored by
tests/golden/make_multipatch_reference.py. Over 100 steps the smoothness classifier meets
decisions within the FP32 rounding of its logits (where either class is correct), so the
long run fixes the viscosity; the per-step classifier and viscosity are checked against
the oracle by tests/test_gpu_parity.py and tests/test_gpu_full_size.py."""
import os

import numpy as np
import pytest

from paper_2506_16076_gb300 import workloads as W
from tests.gpu_helpers import from_dev, rel_err, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_curved_multipatch_100_steps_parity(gpu_lib):
    import torch
    ref = np.load(os.path.join(GOLDEN, "multipatch_grid_100steps.npz"))
    nsteps = int(ref["nsteps"])
    assert nsteps == 100
    w = W.small_multipatch_grid()
    ctx = gpu_lib.Context(w)
    st0 = W.random_smooth_state(w, seed=int(ref["seed"]), amp=float(ref["amp"]))
    e = to_dev(st0)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.from_numpy(np.ascontiguousarray(ref["mu"])).cuda()
    dts = []
    for n in range(nsteps):
        ctx.rk_step(e, dt, mu, gpu_lib.STEP_FROZEN_MU | (gpu_lib.STEP_FILTER if n >= 1 else 0))
        dts.append(dt.item())
    assert np.allclose(dts, ref["dt"], rtol=1e-9, atol=0.0)
    errs = rel_err(from_dev(e, w), W.unflatten(ref["state"], w))
    assert max(errs) < 1e-8, errs
    assert ctx.sync_status(e) == 0
