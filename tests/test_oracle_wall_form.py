"""Oracle pins for the product-rule form at no-slip adiabatic walls (Remark adiabatic):
on a patch with an adiabatic side the temperature theta replaces E among the
FC-differentiated quantities, the derivatives of E and p follow from the sum and product
rules applied to eq. p_T and eq. perfect_gas_T, and the convective flux divergence is
formed from them; the viscous fluxes mu grad e are FC-differentiated as elsewhere.

What fixes each result independently of the oracle's code:
- the product rules on analytic fields equal the symbolic derivatives of E and p
  (sympy), and the product-rule flux divergence, fed exact derivatives, equals the
  symbolic divergence of eq. euler 2d equation, both to rounding;
- the whole operator on a curved, non-orthogonal wall patch converges to the symbolic
  operator -div f(e) + div(mu grad e) of a smooth manufactured state (the error falls
  about tenfold per refinement and ends below 1e-3 of each component's scale, 6e-5 for
  E); a dropped term, a flipped sign or exchanged directions leaves an error of 1.6e-2
  (the kinetic term of dE) to O(1), and three such mistakes planted in the oracle are
  caught;
- a uniform state gives L = 0, and patches without an adiabatic side are unchanged;
- its transpose (the discrete adjoint) satisfies the dot-product identity against
  complex-step directional derivatives of the forward operator and of a whole filtered
  step, on the O-grid, the curved GRID annulus and the S-type arcs.
"""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint as A, euler, solver as S
from paper_2506_16076_gb300 import workloads as W

sp = pytest.importorskip("sympy")

GAM = 1.4
FS = (1.4, 1.0, 0.0, 1.0)


def _manufactured():
    x, y = sp.symbols("x y")
    rho = 1 + sp.Rational(1, 5) * sp.sin(1.3 * x + 0.4) * sp.cos(0.9 * y - 0.2)
    u = 0.4 + 0.2 * sp.cos(0.8 * x) * sp.sin(1.1 * y)
    v = -0.1 + 0.15 * sp.sin(0.7 * x + 1.1 * y)
    p = 1 + 0.1 * sp.cos(1.2 * x - 0.5 * y)
    mu = 0.02 * (1 + 0.5 * sp.sin(x + y))
    E = p / (GAM - 1) + rho * (u * u + v * v) / 2
    e = [rho, rho * u, rho * v, E]
    fx = [rho * u, rho * u * u + p, rho * u * v, u * (E + p)]
    fy = [rho * v, rho * u * v, rho * v * v + p, v * (E + p)]
    div = [sp.diff(fx[c], x) + sp.diff(fy[c], y) for c in range(4)]
    L = [-div[c] + sp.diff(mu * sp.diff(e[c], x), x) + sp.diff(mu * sp.diff(e[c], y), y) for c in range(4)]
    theta = p / rho
    Q = [rho, rho * u, rho * v, theta]
    lam = lambda ex: sp.lambdify((x, y), ex, "numpy")
    return dict(
        e=lam(e), mu=lam(mu), L=lam(L), div=lam(div), theta=lam(theta), Q=lam(Q),
        Qx=lam([sp.diff(q, x) for q in Q]), Qy=lam([sp.diff(q, y) for q in Q]),
        ex=lam([sp.diff(q, x) for q in e]), ey=lam([sp.diff(q, y) for q in e]),
        px=lam(sp.diff(p, x)), py=lam(sp.diff(p, y)))


MF = None


def _mf():
    global MF
    if MF is None:
        MF = _manufactured()
    return MF


def _ev(f, x, y):
    r = f(x, y)
    if isinstance(r, list):
        return np.array([np.broadcast_to(np.asarray(a, dtype=np.float64), x.shape) for a in r])
    return np.broadcast_to(np.asarray(r, dtype=np.float64), x.shape).copy()


def _wall_patch(n1, n2):
    # curved, non-orthogonal annulus (stretched radius, twisted angle), wall at q2 = 0
    return W.grid_patch(W.annulus_map(0.0, 0.0, 0.5, 1.5, 0.15, 0.3), n1, n2,
                        (W.PERIODIC, W.PERIODIC, W.ADIABATIC, W.DIRICHLET), (FS,) * 4, periodic1=True)


def _solver(pd, form):
    return S.Solver(W.Workload("wall_form", [pd], W.Params(d=5, C0=27, c_policy=2, wall_form=form), FS,
                               "freestream", 1))


def _rel_err(sv):
    m = _mf()
    g = sv.geos[0]
    e = _ev(m["e"], g.x, g.y)
    mu = _ev(m["mu"], g.x, g.y)
    Lx = _ev(m["L"], g.x, g.y)
    L = sv.rhs_patch(g, e, mu)
    return np.abs(L - Lx).max(axis=(1, 2)) / np.abs(Lx).max(axis=(1, 2))


def test_product_rules_equal_symbolic_derivatives():
    m = _mf()
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-1.5, 1.5, 200), rng.uniform(-1.5, 1.5, 200)
    Q = _ev(m["Q"], x, y)
    for D, key, pkey in (("Qx", "ex", "px"), ("Qy", "ey", "py")):
        De, Dp = euler.product_rule_derivatives(Q, _ev(m[D], x, y), GAM)
        ref, pref = _ev(m[key], x, y), _ev(m[pkey], x, y)
        assert np.abs(Dp - pref).max() <= 1e-13 * np.abs(pref).max()
        for c in range(4):
            assert np.abs(De[c] - ref[c]).max() <= 1e-13 * np.abs(ref[c]).max(), (key, c)


def test_product_rule_divergence_equals_symbolic_divergence():
    m = _mf()
    rng = np.random.default_rng(4)
    x, y = rng.uniform(-1.5, 1.5, 200), rng.uniform(-1.5, 1.5, 200)
    e, th = _ev(m["e"], x, y), _ev(m["theta"], x, y)
    div = euler.flux_divergence_product(e, th, _ev(m["ex"], x, y), _ev(m["px"], x, y),
                                        _ev(m["ey"], x, y), _ev(m["py"], x, y))
    ref = _ev(m["div"], x, y)
    for c in range(4):
        assert np.abs(div[c] - ref[c]).max() <= 1e-12 * np.abs(ref[c]).max(), c


@pytest.mark.parametrize("form", [0, 1])
def test_operator_converges_to_the_symbolic_operator(form):
    coarse = _rel_err(_solver(_wall_patch(192, 48), form))
    fine = _rel_err(_solver(_wall_patch(384, 96), form))
    assert (fine < 1e-3).all(), fine
    assert (coarse / fine > 6.0).all(), (coarse, fine)


def _planted(kind):
    good = euler.product_rule_derivatives

    def bad(Q, DQ, gamma):
        if kind == "dropped kinetic term":
            rho, mx, my, th = Q
            drho, dmx, dmy, dth = DQ
            dp = th * drho + rho * dth
            return np.stack([drho, dmx, dmy, dp / (gamma - 1.0) + (mx * dmx + my * dmy) / rho]), dp
        if kind == "sign of rho dtheta":
            rho, mx, my, th = Q
            De, dp = good(Q, DQ, gamma)
            dp2 = dp - 2.0 * rho * DQ[3]
            return np.stack([De[0], De[1], De[2], De[3] - 2.0 * rho * DQ[3] / (gamma - 1.0)]), dp2
        raise AssertionError(kind)
    return bad


@pytest.mark.parametrize("kind", ["dropped kinetic term", "sign of rho dtheta", "directions exchanged"])
def test_planted_mistakes_fail_the_pin(monkeypatch, kind):
    if kind == "directions exchanged":
        good = euler.flux_divergence_product
        monkeypatch.setattr(euler, "flux_divergence_product",
                            lambda e, th, ex, px, ey, py: good(e, th, ey, py, ex, px))
    else:
        monkeypatch.setattr(euler, "product_rule_derivatives", _planted(kind))
    err = _rel_err(_solver(_wall_patch(384, 96), 1))
    assert err.max() > 5e-3, (kind, err)


def test_uniform_state_and_patches_without_walls():
    pd = _wall_patch(128, 32)
    sv1 = _solver(pd, 1)
    g = sv1.geos[0]
    e = np.array(euler.cons_from_prim(*[np.full(g.x.shape, v) for v in (1.3, 0.7, -0.2, 0.9)], GAM))
    mu = 0.01 * (1.0 + g.x ** 2)
    assert np.abs(sv1.rhs_patch(g, e, mu)).max() <= 1e-10
    # without an adiabatic side the patch keeps the flux form bit for bit
    pd2 = W.grid_patch(W.annulus_map(0.0, 0.0, 0.5, 1.5, 0.15, 0.3), 128, 32,
                       (W.PERIODIC, W.PERIODIC, W.DIRICHLET, W.DIRICHLET), (FS,) * 4, periodic1=True)
    a, b = _solver(pd2, 1), _solver(pd2, 0)
    m = _mf()
    e2 = _ev(m["e"], a.geos[0].x, a.geos[0].y)
    mu2 = _ev(m["mu"], a.geos[0].x, a.geos[0].y)
    assert np.array_equal(a.rhs_patch(a.geos[0], e2, mu2), b.rhs_patch(b.geos[0], e2, mu2))
    assert sv1.product_form(g) and not a.product_form(a.geos[0])


def _dot(a, b):
    return sum(float(np.vdot(x, y).real) for x, y in zip(a, b))


@pytest.fixture(scope="module", params=["ogrid", "grid_curved", "s_type"])
def wall_case(request):
    w = {"ogrid": lambda: W.small_multipatch(W.ADIABATIC), "grid_curved": W.small_multipatch_grid,
         "s_type": W.small_multipatch_stype}[request.param]()
    w = dataclasses.replace(w, params=dataclasses.replace(w.params, wall_form=1))
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=7, amp=0.05))
    mu = [0.002 * (1 + np.cos(g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    return sv, st, mu


def _rand(states, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=a.shape) for a in states]


def test_rhs_adjoint_dot_product(wall_case):
    sv, st, mu = wall_case
    assert any(sv.product_form(g) for g in sv.geos)
    v, lam = _rand(st, 1), _rand(st, 2)
    lhs = _dot(A.rhs_jvp_complex(sv, st, mu, v), lam)
    rhs = _dot(v, A.rhs_adjoint(sv, st, mu, lam))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs), (lhs, rhs)


def test_step_adjoint_with_filter_dot_product(wall_case):
    sv, st, mu = wall_case
    dt = 0.5 * sv.dt(st, mu)
    v, lam = _rand(st, 3), _rand(st, 4)
    lhs = _dot(A.step_jvp_complex(sv, st, mu, dt, v, filt=True), lam)
    rhs = _dot(v, A.step_adjoint(sv, st, mu, dt, lam, filt=True)[0])
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)
