"""GPU discrete adjoint vs the oracle adjoint, the drag functional, and gradients vs
central finite differences (step 1e-6) with mu and dt frozen (through the C-ABI)."""
import dataclasses
import math

import numpy as np
import pytest
import torch

from oracle import adjoint as A, solver as S
from paper_2506_16076_gb300 import adjoint as ADJ, workloads as W
from tests.gpu_helpers import from_dev, rel_err, to_dev, to_dev_scalar_field

pytestmark = pytest.mark.gpu


def mach2_small(mach=2.0, alpha_deg=2.0):
    """The small cylinder workload under a Mach-M free stream at angle alpha (a tiny config-4 analogue)."""
    w = W.small_multipatch()
    a = math.radians(alpha_deg)
    fs = (1.4, mach * math.cos(a), mach * math.sin(a), 1.0)
    pts = [dataclasses.replace(p, bc=(fs,) * 4) for p in w.patches]
    return W.Workload(f"small_M{mach}", pts, w.params, fs, "freestream", 10)


@pytest.mark.parametrize("name", ["sod64", "multi", "multi_adiabatic", "grid_curved", "s_type"])
def test_adjoint_step_parity(gpu_lib, name):
    w = {"sod64": lambda: W.sod128(64), "multi": W.small_multipatch,
         "multi_adiabatic": lambda: W.small_multipatch(W.ADIABATIC),
         "grid_curved": W.small_multipatch_grid, "s_type": W.small_multipatch_stype}[name]()
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=41, amp=0.1))
    mu = [0.003 * (1 + np.cos(2 * g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    dt = 0.5 * sv.dt(st, mu)
    rng = np.random.default_rng(5)
    lam = [rng.normal(size=a.shape) for a in st]
    ref_lam, ref_gbc = A.step_adjoint(sv, st, mu, dt, lam)
    lam_n = torch.empty_like(to_dev(st))
    gbc = torch.zeros_like(lam_n)
    dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
    ctx.adjoint_step(to_dev(st), to_dev_scalar_field(mu), dtt, to_dev(lam), lam_n, gbc)
    torch.cuda.synchronize()
    errs = rel_err(from_dev(lam_n, w), ref_lam)
    assert max(errs) < 1e-11, errs
    if any(np.abs(g).max() > 0 for g in ref_gbc):
        errs = rel_err(from_dev(gbc, w), ref_gbc)
        assert max(errs) < 1e-11, errs


def test_adjoint_step_with_filter_parity(gpu_lib):
    w = W.small_multipatch(W.ADIABATIC)
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=43, amp=0.1))
    mu = [0.003 * (1 + np.cos(2 * g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    dt = 0.5 * sv.dt(st, mu)
    rng = np.random.default_rng(6)
    lam = [rng.normal(size=a.shape) for a in st]
    ref_lam, ref_gbc = A.step_adjoint(sv, st, mu, dt, lam, filt=True)
    lam_n = torch.empty_like(to_dev(st))
    gbc = torch.zeros_like(lam_n)
    dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
    ctx.adjoint_step(to_dev(st), to_dev_scalar_field(mu), dtt, to_dev(lam), lam_n, gbc, gpu_lib.STEP_FILTER)
    torch.cuda.synchronize()
    errs = rel_err(from_dev(lam_n, w), ref_lam)
    assert max(errs) < 1e-11, errs
    errs = rel_err(from_dev(gbc, w), ref_gbc)
    assert max(errs) < 1e-11, errs


@pytest.mark.parametrize("filt", [0, 1])
def test_parameter_sensitivity_parity(gpu_lib, filt):
    # dJ/d(Mach, angle) through the free-stream Dirichlet states of one adjoint step
    # (accumulated over two calls) and through a uniform free-stream initial state, and
    # dJ/drho_0, against the oracle adjoint
    w = mach2_small()
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=47, amp=0.1))
    mu = [0.003 * (1 + np.cos(2 * g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    dt = 0.5 * sv.dt(st, mu)
    rng = np.random.default_rng(8)
    lam = [rng.normal(size=a.shape) for a in st]
    ref_lam, ref_gbc = A.step_adjoint(sv, st, mu, dt, lam, filt=bool(filt))
    ref_par = A.dirichlet_param_sensitivity(sv, ref_gbc, w.freestream)
    dM, dA = A.freestream_jacobian(w.freestream, w.params.gamma)
    size = [sum(np.einsum("c,cji->", np.abs(v), np.abs(g)) for g in ref_gbc) for v in (dM, dA)]
    lam_n = torch.empty_like(to_dev(st))
    dparam = torch.zeros(2, dtype=torch.float64, device="cuda")
    dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
    for _ in range(2):
        ctx.adjoint_step(to_dev(st), to_dev_scalar_field(mu), dtt, to_dev(lam), lam_n, None,
                         gpu_lib.STEP_FILTER if filt else 0, dparam)
    torch.cuda.synchronize()
    got = dparam.cpu().numpy()
    for k in range(2):
        assert abs(got[k] - 2 * ref_par[k]) <= 1e-11 * 2 * size[k], (k, got, ref_par, size)
    # initial data: the oracle's adjoint state and a uniform free-stream e_0
    e0 = W.initial_state(w)
    drho_o, par0 = A.initial_sensitivity(sv, e0, ref_lam, w.freestream)
    drho = torch.empty(ctx.P, dtype=torch.float64, device="cuda")
    dp0 = torch.zeros(2, dtype=torch.float64, device="cuda")
    ctx.initial_sensitivity(to_dev(e0), to_dev(ref_lam), drho, dp0)
    torch.cuda.synchronize()
    got_rho = from_dev(drho, w, 1)
    scale = max(np.abs(d).max() for d in drho_o)
    assert max(np.abs(a - b).max() for a, b in zip(got_rho, drho_o)) <= 1e-13 * scale
    size0 = [sum(np.einsum("c,cji->", np.abs(v), np.abs(l)) for l in ref_lam) for v in (dM, dA)]
    got0 = dp0.cpu().numpy()
    for k in range(2):
        assert abs(got0[k] - par0[k]) <= 1e-12 * size0[k], (k, got0, par0)


def test_parameter_sensitivity_needs_a_free_stream(gpu_lib):
    w = W.sod128(32)
    w = dataclasses.replace(w, freestream=(0.0, 0.0, 0.0, 0.0))
    ctx = gpu_lib.Context(w)
    e = to_dev(W.initial_state(w))
    lam = torch.zeros_like(e)
    with pytest.raises(gpu_lib.FcError):
        ctx.initial_sensitivity(e, lam, None, torch.zeros(2, dtype=torch.float64, device="cuda"))


def test_drag_parity(gpu_lib):
    w = mach2_small()
    ctx = gpu_lib.Context(w)
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=3, amp=0.1))
    J, g = ADJ.drag(ctx, to_dev(st))
    assert abs(J.item() - A.wall_drag(sv, st)) <= 1e-13 * max(1.0, abs(J.item()))
    errs = rel_err(from_dev(g, w), A.wall_drag_grad(sv, st))
    assert max(errs) < 1e-14, errs


def _J_frozen(gpu_lib, mach, alpha, rho_pert, mus, dts, nsteps):
    w = mach2_small(mach, alpha)
    ctx = gpu_lib.Context(w)
    e = to_dev(W.initial_state(w))
    if rho_pert is not None:  # perturb the initial density at fixed velocity and pressure
        rho = e[0].clone()
        u, v = e[1] / rho, e[2] / rho
        p = 0.4 * (e[3] - 0.5 * rho * (u * u + v * v))
        rho = rho + rho_pert
        e = torch.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])
    for n in range(nsteps):
        ctx.rk_step(e, dts[n], mus[n], gpu_lib.STEP_FROZEN_MU | gpu_lib.STEP_FIXED_DT)
    J, _ = ADJ.drag(ctx, e)
    return J.item()


def test_drag_gradients_vs_central_differences(gpu_lib):
    nsteps, K, h = 8, 3, 1e-6
    w = mach2_small()
    ctx = gpu_lib.Context(w)
    e0 = to_dev(W.initial_state(w))
    J, dJdM, dJda, dJdrho, tr = ADJ.drag_gradients(w, ctx, e0, nsteps, K)
    fdM = (_J_frozen(gpu_lib, 2.0 + h, 2.0, None, tr.mus, tr.dts, nsteps)
           - _J_frozen(gpu_lib, 2.0 - h, 2.0, None, tr.mus, tr.dts, nsteps)) / (2 * h)
    assert abs(fdM - dJdM) <= 1e-5 * max(abs(dJdM), 1e-3), (fdM, dJdM)
    ha = math.degrees(h)
    fda = (_J_frozen(gpu_lib, 2.0, 2.0 + ha, None, tr.mus, tr.dts, nsteps)
           - _J_frozen(gpu_lib, 2.0, 2.0 - ha, None, tr.mus, tr.dts, nsteps)) / (2 * h)
    assert abs(fda - dJda) <= 1e-5 * max(abs(dJda), 1e-3), (fda, dJda)
    # a seeded set of initial-density points
    rng = np.random.default_rng(32)
    big = torch.nonzero(dJdrho.abs() > 1e-3 * dJdrho.abs().max()).flatten().cpu().numpy()
    for p in rng.choice(big, size=min(8, len(big)), replace=False):
        d = torch.zeros(e0.shape[1], dtype=torch.float64, device="cuda")
        d[int(p)] = h
        fd = (_J_frozen(gpu_lib, 2.0, 2.0, d, tr.mus, tr.dts, nsteps)
              - _J_frozen(gpu_lib, 2.0, 2.0, -d, tr.mus, tr.dts, nsteps)) / (2 * h)
        ad = dJdrho[int(p)].item()
        assert abs(fd - ad) <= 1e-5 * abs(dJdrho).max().item(), (p, fd, ad)


def test_lean_checkpointing_matches_stored_mu(gpu_lib):
    # recomputing each step's viscosity from the replayed state gives the same adjoint
    w = W.small_multipatch(W.ADIABATIC)
    ctx = gpu_lib.Context(w)
    e0 = to_dev(W.random_smooth_state(w, seed=19, amp=0.05))
    g = torch.randn_like(e0)
    _, tr = ADJ.forward(ctx, e0, 6, 3, filter=True)
    lam_a, gbc_a = ADJ.backward(ctx, tr, g)
    _, tr2 = ADJ.forward(ctx, e0, 6, 3, filter=True, store_mu=False)
    assert all(m is None for m in tr2.mus)
    lam_b, gbc_b = ADJ.backward(ctx, tr2, g)
    assert torch.equal(lam_a, lam_b) and torch.equal(gbc_a, gbc_b)


def test_autograd_function_matches_driver(gpu_lib):
    w = mach2_small()
    ctx = gpu_lib.Context(w)
    e0 = to_dev(W.random_smooth_state(w, seed=9, amp=0.05)).requires_grad_(True)
    eN = ADJ.FCSteps.apply(e0, ctx, 4, 2)
    g = torch.randn_like(eN)
    (eN * g).sum().backward()
    _, tr = ADJ.forward(ctx, e0.detach(), 4, 2)
    lam0, _ = ADJ.backward(ctx, tr, g)
    assert torch.allclose(e0.grad, lam0, rtol=0, atol=1e-12 * lam0.abs().max().item())
