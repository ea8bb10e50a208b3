"""Drag gradients of the adjoint configuration at its stated size: the Mach-3 cylinder
geometry at half resolution (O-grid 256 x 48, 4 x 4 affine 80 x 80 patches), Mach 2 at
2 degrees, J = wall pressure times n_x integrated over the wall after 400 steps,
checkpoints every 40 steps with recompute, the per-step filter on as in a plain run
(the run loses positivity at the rear of the cylinder after about 200 steps without
it). dJ/dMach, dJ/dalpha and dJ/drho_0 at 32 seeded points are checked against
central differences with step 1e-6, with the viscosity and the time step of every step
frozen at their forward values (the map the discrete adjoint differentiates)."""
import math

import numpy as np
import pytest
import torch

from paper_2506_16076_gb300 import adjoint as ADJ, workloads as W
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

NSTEPS, K, H = 400, 40, 1e-6


def _run_frozen(gpu_lib, ctx, e, mus, dts):
    for n in range(NSTEPS):
        f = gpu_lib.STEP_FILTER if n >= 1 else 0
        ctx.rk_step(e, dts[n], mus[n], gpu_lib.STEP_FROZEN_MU | gpu_lib.STEP_FIXED_DT | f)
    J, _ = ADJ.drag(ctx, e)
    return J.item()


def _J_params(gpu_lib, mach, alpha_deg, mus, dts):
    w = W.cyl_m2_half(mach, alpha_deg)
    ctx = gpu_lib.Context(w)
    return _run_frozen(gpu_lib, ctx, to_dev(W.initial_state(w)), mus, dts)


def _with_density(e0, drho):
    # perturb the initial density at fixed velocity and pressure
    rho = e0[0]
    u, v = e0[1] / rho, e0[2] / rho
    p = 0.4 * (e0[3] - 0.5 * rho * (u * u + v * v))
    r = rho + drho
    return torch.stack([r, r * u, r * v, p / 0.4 + 0.5 * r * (u * u + v * v)])


def test_config4_drag_gradients(gpu_lib):
    w = W.cyl_m2_half()
    ctx = gpu_lib.Context(w)
    e0 = to_dev(W.initial_state(w))
    J, dJdM, dJda, dJdrho, tr = ADJ.drag_gradients(w, ctx, e0, NSTEPS, K, filter=True)
    assert len(tr.checkpoints) == NSTEPS // K and math.isfinite(J)
    assert ctx.sync_status(e0) == 0
    fdM = (_J_params(gpu_lib, 2.0 + H, 2.0, tr.mus, tr.dts) - _J_params(gpu_lib, 2.0 - H, 2.0, tr.mus, tr.dts)) / (2 * H)
    ha = math.degrees(H)
    fda = (_J_params(gpu_lib, 2.0, 2.0 + ha, tr.mus, tr.dts) - _J_params(gpu_lib, 2.0, 2.0 - ha, tr.mus, tr.dts)) / (2 * H)
    assert abs(fdM - dJdM) <= 1e-5 * abs(dJdM), (fdM, dJdM)
    assert abs(fda - dJda) <= 1e-5 * max(abs(dJda), 1e-3 * abs(dJdM)), (fda, dJda)
    rng = np.random.default_rng(32)
    scale = dJdrho.abs().max().item()
    big = torch.nonzero(dJdrho.abs() > 1e-2 * scale).flatten().cpu().numpy()
    for p in rng.choice(big, size=min(32, len(big)), replace=False):
        d = torch.zeros(e0.shape[1], dtype=torch.float64, device="cuda")
        d[int(p)] = H
        fd = (_run_frozen(gpu_lib, ctx, _with_density(e0, d), tr.mus, tr.dts)
              - _run_frozen(gpu_lib, ctx, _with_density(e0, -d), tr.mus, tr.dts)) / (2 * H)
        assert abs(fd - dJdrho[int(p)].item()) <= 1e-5 * scale, (int(p), fd, dJdrho[int(p)].item())
