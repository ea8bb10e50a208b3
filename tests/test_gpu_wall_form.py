"""Product-rule form of the operator on no-slip adiabatic wall patches (Remark adiabatic;
fc_params.wall_form = 1) on the GPU against the oracle, element by element on seeded
inputs: the RHS with a given viscosity on the O-grid, on the curved, twisted GRID annulus
and on the S-type arcs (1e-11 relative per component, as every RHS evaluation), ten
steps of Algorithm 1 with viscosity, filter and CFL step (1e-9), the wall patches' RHS
against the flux form's (different there, identical on every other patch), and the
discrete adjoint of a step with and without the filter (1e-11), and the wall-drag
gradients through the checkpointed adjoint against central differences. The oracle's
product-rule form is pinned against a symbolic operator of a manufactured state, its
transpose by dot-product identities (tests/test_oracle_wall_form.py)."""
import dataclasses
import math

import numpy as np
import pytest
import torch

from oracle import adjoint as A, solver as S
from paper_2506_16076_gb300 import adjoint as ADJ, workloads as W
from tests.gpu_helpers import from_dev, rel_err, smooth_mu, to_dev, to_dev_scalar_field

pytestmark = pytest.mark.gpu

RHS_TOL = 1e-11


def _pform(w, form=1):
    return dataclasses.replace(w, params=dataclasses.replace(w.params, wall_form=form))


CASES = {"multi_adiabatic": lambda: W.small_multipatch(W.ADIABATIC),
         "grid_curved": W.small_multipatch_grid,
         "s_type": W.small_multipatch_stype}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, gpu_lib):
    w = _pform(CASES[request.param]())
    return w, gpu_lib.Context(w), S.Solver(w)


def _rhs(ctx, st, mu):
    e = to_dev(st)
    out = torch.empty_like(e)
    ctx.rhs(e, out, to_dev_scalar_field(mu))
    torch.cuda.synchronize()
    return out


def test_rhs_parity_given_mu(case):
    w, ctx, sv = case
    assert any(sv.product_form(g) for g in sv.geos)
    st = W.random_smooth_state(w, seed=11, amp=0.2)
    mu = smooth_mu(w, seed=3, scale=0.01)
    errs = rel_err(from_dev(_rhs(ctx, st, mu), w), sv.rhs(st, mu))
    assert max(errs) < RHS_TOL, errs


def test_rhs_parity_zero_mu(case):
    w, ctx, sv = case
    st = W.random_smooth_state(w, seed=5, amp=0.2)
    mu = [np.zeros((p.n2, p.n1)) for p in w.patches]
    errs = rel_err(from_dev(_rhs(ctx, st, mu), w), sv.rhs(st, mu))
    assert max(errs) < RHS_TOL, errs


def test_only_wall_patches_change(case, gpu_lib):
    w, ctx, sv = case
    ctx0 = gpu_lib.Context(_pform(w, 0))
    st = W.random_smooth_state(w, seed=13, amp=0.2)
    mu = smooth_mu(w, seed=6, scale=0.01)
    a, b = _rhs(ctx, st, mu).cpu(), _rhs(ctx0, st, mu).cpu()
    offs = w.offsets
    for p, g in enumerate(sv.geos):
        sl = slice(offs[p], offs[p + 1])
        if sv.product_form(g):
            diff = (a[:, sl] - b[:, sl]).abs().max().item()
            assert 0.0 < diff < 5e-2 * a[:, sl].abs().max().item(), (p, diff)
        else:
            assert torch.equal(a[:, sl], b[:, sl]), p


def _run_gpu(ctx, e, nsteps, frozen=None):
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.zeros(e.shape[1], dtype=torch.float64, device="cuda")
    dts = []
    for n in range(nsteps):
        flags = 1 if n >= 1 else 0
        if frozen is not None:
            mu.copy_(frozen[n])
            flags |= 2
        ctx.rk_step(e, dt, mu, flags)
        dts.append(dt.item())
    return dts


def test_ten_steps_parity(case):
    # Algorithm 1 from a seeded smooth perturbation of the free stream: viscosity, filter
    # from step 1, CFL step, 5 stages with the wall overwrite and exchange. A classifier
    # tie (stated in the viscosity parity tests) is handled by injecting the oracle's
    # viscosity.
    w, ctx, sv = case
    st0 = W.random_smooth_state(w, seed=41, amp=0.05)
    st = [a.copy() for a in st0]
    mus, dts_ref = [], []
    for n in range(10):
        st = sv.step(st, n)
        mus.append(sv.last_mu)
        dts_ref.append(sv.last_dt)
    e = to_dev(st0)
    dts = _run_gpu(ctx, e, 10)
    assert abs(dts[0] - dts_ref[0]) <= 1e-13 * dts_ref[0]
    errs = rel_err(from_dev(e, w), st)
    if max(errs) >= 1e-9:
        e = to_dev(st0)
        _run_gpu(ctx, e, 10, frozen=[to_dev_scalar_field(m) for m in mus])
        errs = rel_err(from_dev(e, w), st)
    assert max(errs) < 1e-9, errs
    assert ctx.sync_status(e) == 0


@pytest.mark.parametrize("filt", [0, 1])
def test_adjoint_step_parity(case, gpu_lib, filt):
    # the discrete adjoint of a step with the product-rule wall patches (mu and dt frozen,
    # with and without the per-step filter) against the oracle's transpose, whose
    # pointwise Jacobians come from the complex step
    w, ctx, sv = case
    st = sv.project(W.random_smooth_state(w, seed=43 + filt, amp=0.1))
    mu = [0.003 * (1 + np.cos(2 * g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    dt = 0.5 * sv.dt(st, mu)
    rng = np.random.default_rng(7 + filt)
    lam = [rng.normal(size=a.shape) for a in st]
    ref_lam, ref_gbc = A.step_adjoint(sv, st, mu, dt, lam, filt=bool(filt))
    lam_n = torch.empty_like(to_dev(st))
    gbc = torch.zeros_like(lam_n)
    dtt = torch.tensor([dt], dtype=torch.float64, device="cuda")
    ctx.adjoint_step(to_dev(st), to_dev_scalar_field(mu), dtt, to_dev(lam), lam_n, gbc,
                     gpu_lib.STEP_FILTER if filt else 0)
    torch.cuda.synchronize()
    errs = rel_err(from_dev(lam_n, w), ref_lam)
    assert max(errs) < 1e-11, errs
    if any(np.abs(g).max() > 0 for g in ref_gbc):
        errs = rel_err(from_dev(gbc, w), ref_gbc)
        assert max(errs) < 1e-11, errs


def test_affine_wall_patch_is_refused(gpu_lib):
    fs = (1.4, 1.0, 0.0, 1.0)
    p = W.PatchDesc(W.AFFINE, 32, 32, (0.0, 1.0, 0.0, 1.0), (W.DIRICHLET, W.DIRICHLET, W.ADIABATIC, W.DIRICHLET),
                    bc=(fs,) * 4)
    w = W.Workload("affine_wall", [p], W.Params(d=5, C0=27, c_policy=2, wall_form=1), fs, "freestream", 1)
    with pytest.raises(gpu_lib.FcError):
        gpu_lib.Context(w)
    gpu_lib.Context(_pform(w, 0))  # the flux form accepts it


def _m2_wall(mach=2.0, alpha_deg=2.0):
    # the small cylinder with the no-slip adiabatic wall under a Mach-M stream at angle alpha
    w = W.small_multipatch(W.ADIABATIC)
    a = math.radians(alpha_deg)
    fs = (1.4, mach * math.cos(a), mach * math.sin(a), 1.0)
    pts = [dataclasses.replace(p, bc=(fs,) * 4) for p in w.patches]
    return _pform(W.Workload(f"small_M{mach}_wall", pts, w.params, fs, "freestream", 10))


def test_drag_gradients_vs_central_differences(gpu_lib):
    # dJ/dM and dJ/dalpha of the wall drag after a few steps with the viscosity and the
    # steps frozen (the checkpointed adjoint through the product-rule wall patch) against
    # central differences of the same frozen march
    nsteps, K, h = 6, 3, 1e-6
    w = _m2_wall()
    ctx = gpu_lib.Context(w)
    J, dJdM, dJda, dJdrho, tr = ADJ.drag_gradients(w, ctx, to_dev(W.initial_state(w)), nsteps, K)

    def J_frozen(mach, alpha):
        ww = _m2_wall(mach, alpha)
        c = gpu_lib.Context(ww)
        e = to_dev(W.initial_state(ww))
        for n in range(nsteps):
            c.rk_step(e, tr.dts[n], tr.mus[n], gpu_lib.STEP_FROZEN_MU | gpu_lib.STEP_FIXED_DT)
        return ADJ.drag(c, e)[0].item()

    assert abs(J_frozen(2.0, 2.0) - J) <= 1e-12 * max(abs(J), 1.0)
    fdM = (J_frozen(2.0 + h, 2.0) - J_frozen(2.0 - h, 2.0)) / (2 * h)
    assert abs(fdM - dJdM) <= 1e-5 * max(abs(dJdM), 1e-3), (fdM, dJdM)
    ha = math.degrees(h)
    fda = (J_frozen(2.0, 2.0 + ha) - J_frozen(2.0, 2.0 - ha)) / (2 * h)
    assert abs(fda - dJda) <= 1e-5 * max(abs(dJda), 1e-3), (fda, dJda)
