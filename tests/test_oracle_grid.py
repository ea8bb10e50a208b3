"""Oracle pins for GRID patches (general curvilinear patches given by their points and
metrics, Sec. 3.1-3.3): the inverse map by Newton's method on the local quadratic
interpolant, the spacings, and the whole operator against the closed-form AFFINE and
O-grid maps that the same points come from.

What fixes each result independently of the GRID code:
- the quadratic interpolant of an affine map is the map itself, so the inverse must be
  the affine closed form to rounding (a wrong Lagrange weight, derivative or sign in
  the Newton step breaks this);
- on a curved map the interpolant is third-order accurate: the parameter error against
  the exact inverse (found by bracketing) falls about eightfold per refinement;
- grid points map to their own indices;
- the GRID form of the AFFINE / O-grid workload reproduces that workload's geometry,
  donors, stencils, RHS and time step to rounding, and its interpolation weights to
  rounding where the donor is a box (the annulus's inverse carries the third-order
  interpolation error);
- a uniform state is preserved on a curved, non-orthogonal multi-patch grid
  (the FC derivative of a constant vanishes, Sec. 2.2, whatever the metrics).
"""
import dataclasses

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import geometry, solver as S
from paper_2506_16076_gb300 import workloads as W
from tests.gpu_helpers import smooth_mu

PRM = W.Params(d=5, C0=27, c_policy=2)
FS = (1.4, 1.0, 0.0, 1.0)


def _annulus(n1, n2, r0=0.5, r1=1.5, stretch=0.15, twist=0.3):
    return W.grid_patch(W.annulus_map(0.0, 0.0, r0, r1, stretch, twist), n1, n2,
                        (W.PERIODIC, W.PERIODIC, W.ADIABATIC, W.DIRICHLET), (FS,) * 4, periodic1=True)


def test_inverse_is_exact_on_an_affine_map():
    x0, x1, y0, y1 = -1.3, 0.7, 0.2, 1.45
    n1, n2 = 37, 23
    g = geometry.PatchGeo(W.as_grid(W.PatchDesc(W.AFFINE, n1, n2, (x0, x1, y0, y1), (W.DIRICHLET,) * 4,
                                                bc=(FS,) * 4)), PRM)
    rng = np.random.default_rng(3)
    # inside, plus a margin of half a cell outside (extrapolation by the edge stencils)
    hx, hy = (x1 - x0) / (n1 - 1), (y1 - y0) / (n2 - 1)
    x = rng.uniform(x0 - 0.5 * hx, x1 + 0.5 * hx, 500)
    y = rng.uniform(y0 - 0.5 * hy, y1 + 0.5 * hy, 500)
    s1, s2 = g.frac_index(x, y)
    assert np.abs(s1 - (x - x0) / hx).max() < 1e-11
    assert np.abs(s2 - (y - y0) / hy).max() < 1e-11


def test_inverse_reproduces_grid_points():
    for p in (_annulus(48, 12), W.small_multipatch_grid().patches[1]):
        g = geometry.PatchGeo(p, PRM)
        s1, s2 = g.frac_index(g.x.ravel(), g.y.ravel())
        I, J = np.meshgrid(np.arange(g.n1), np.arange(g.n2))
        d1 = s1 - I.ravel()
        if g.periodic1:
            d1 = np.mod(d1 + 0.5 * g.n1, g.n1) - 0.5 * g.n1
        assert np.abs(d1).max() < 1e-10 and np.abs(s2 - J.ravel()).max() < 1e-10


def _exact_annulus_inverse(x, y, r0=0.5, r1=1.5, stretch=0.15, twist=0.3):
    r = np.hypot(x, y)
    b = np.array([brentq(lambda t: r0 + (r1 - r0) * (t + stretch * np.sin(np.pi * t)) - rr, 0.0, 1.0,
                         xtol=1e-15) for rr in r])
    a = np.mod((np.arctan2(y, x) - twist * np.sin(np.pi * b) ** 2) / (2 * np.pi), 1.0)
    return a, b


def test_inverse_is_third_order_on_a_curved_map():
    rng = np.random.default_rng(1)
    r = rng.uniform(0.6, 1.4, 200)
    th = rng.uniform(0.0, 2 * np.pi, 200)
    x, y = r * np.cos(th), r * np.sin(th)
    a, b = _exact_annulus_inverse(x, y)
    errs = []
    for n1, n2 in ((32, 8), (64, 16), (128, 32)):
        g = geometry.PatchGeo(_annulus(n1, n2), PRM)
        s1, s2 = g.frac_index(x, y)
        assert g.contains(s1, s2).all()
        e1 = np.mod(s1 / n1 - a + 0.5, 1.0) - 0.5
        e2 = s2 / (n2 - 1) - b
        errs.append(max(np.abs(e1).max(), np.abs(e2).max()))
    assert errs[0] / errs[1] > 6.0 and errs[1] / errs[2] > 6.0, errs
    assert errs[2] < 1e-4, errs


def test_far_points_are_outside():
    g = geometry.PatchGeo(_annulus(32, 8), PRM)
    s1, s2 = g.frac_index(np.array([5.0, 0.0, -3.0]), np.array([0.0, 4.0, -3.0]))
    assert not g.contains(s1, s2).any()


def test_grid_form_reproduces_the_closed_form_maps():
    w0 = W.small_multipatch(W.ADIABATIC)
    w1 = W.small_multipatch_grid(curved=False)
    sv0, sv1 = S.Solver(w0), S.Solver(w1)
    for g0, g1 in zip(sv0.geos, sv1.geos):
        assert g1.kind == W.GRID and g1.periodic1 == g0.periodic1
        assert np.abs(g1.J - g0.J).max() <= 1e-14 * np.abs(g0.J).max()
        assert abs(g1.hhat - g0.hhat) <= 1e-13 * g0.hhat and abs(g1.htil - g0.htil) <= 1e-13 * g0.htil
        for m in ("blank", "receiver", "gen", "nodiff"):
            assert np.array_equal(getattr(g1, m), getattr(g0, m)), m
    for c0, c1 in zip(sv0.conn.items, sv1.conn.items):
        for k in ("j", "i", "donor", "a1", "a2"):
            assert np.array_equal(c0[k], c1[k]), k
        # boxes invert exactly; the annulus (patch 0) inverts its quadratic interpolant,
        # within the third-order interpolation error of the exact inverse
        ann = c0["donor"] == 0
        for k in ("t1", "t2"):
            dk = np.abs(c0[k] - c1[k])
            assert dk[~ann].max(initial=0.0) < 1e-11 and dk[ann].max(initial=0.0) < 1e-3, k
    assert not sv1.conn.errors
    st = W.random_smooth_state(w0, seed=5, amp=0.05)
    mu = smooth_mu(w0, seed=3, scale=1e-3)
    r0, r1 = sv0.rhs(st, mu), sv1.rhs(st, mu)
    for a, b in zip(r1, r0):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert abs(sv1.dt(st, mu) - sv0.dt(st, mu)) <= 1e-13 * sv0.dt(st, mu)


@pytest.mark.parametrize("make", [W.small_multipatch_grid, W.small_multipatch_stype], ids=["curved", "s_type"])
def test_uniform_state_preserved_on_curved_grid(make):
    w = make()
    w.patches = [dataclasses.replace(p, side=tuple(W.DIRICHLET if t == W.ADIABATIC else t for t in p.side))
                 for p in w.patches]
    sv = S.Solver(w)
    assert not sv.conn.errors
    u = np.array(W.prim_to_cons(*w.freestream))
    st = [np.broadcast_to(u[:, None, None], (4, p.n2, p.n1)).copy() for p in w.patches]
    out, _ = sv.run(st, 3)
    for g, o, f in zip(sv.geos, out, st):
        dev = np.abs(np.where(g.blank[None], 0, o - f)).max(axis=(1, 2))
        assert (dev <= 2e-12 * np.abs(f).max(axis=(1, 2)) + 1e-13).all(), dev


@pytest.mark.parametrize("kind", ["curved", "flat"])
def test_grid_spacings_are_the_point_distances(kind):
    p = W.small_multipatch_grid(curved=kind == "curved").patches[2]
    g = geometry.PatchGeo(p, PRM)
    d = [np.hypot(g.x[:, i + 1] - g.x[:, i], g.y[:, i + 1] - g.y[:, i]) for i in range(g.n1 - 1)]
    d += [np.hypot(g.x[j + 1] - g.x[j], g.y[j + 1] - g.y[j]) for j in range(g.n2 - 1)]
    d = np.concatenate(d)
    assert g.hhat == d.max() and g.htil == d.min()


def test_rhs_adjoint_dot_product_on_curved_grid():
    # the transpose of the operator on hole-cut, non-orthogonal patches (segments of
    # every length), against complex-step directional derivatives of the forward map
    from oracle import adjoint as A
    w = W.small_multipatch_grid()
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=2, amp=0.05))
    mu = [0.002 * (1 + np.cos(g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    rng = np.random.default_rng(1)
    v = [rng.normal(size=a.shape) for a in st]
    lam = [rng.normal(size=a.shape) for a in st]
    jv = A.rhs_jvp_complex(sv, st, mu, v)
    jtl = A.rhs_adjoint(sv, st, mu, lam)
    lhs = sum(float(np.vdot(a, b).real) for a, b in zip(jv, lam))
    rhs = sum(float(np.vdot(a, b).real) for a, b in zip(v, jtl))
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), 1.0), (lhs, rhs)


def test_metrics_from_points_exact_on_the_closed_form_maps():
    # FC differentiates the linear box maps and the trigonometric annulus map to rounding
    w1 = W.small_multipatch_grid(curved=False)
    w0 = W.small_multipatch_grid(curved=False, metrics=False)
    for p1, p0 in zip(w1.patches, w0.patches):
        assert p0.metrics is None
        g1, g0 = geometry.PatchGeo(p1, PRM), geometry.PatchGeo(p0, PRM)
        assert np.abs(g0.J - g1.J).max() <= 1e-12 * np.abs(g1.J).max()


def test_metrics_from_points_converge_at_high_order():
    errs = []
    for n1, n2 in ((64, 16), (128, 32), (256, 64)):
        p = _annulus(n1, n2)
        g1 = geometry.PatchGeo(p, PRM)
        g0 = geometry.PatchGeo(dataclasses.replace(p, metrics=None), PRM)
        errs.append(np.abs(g0.J - g1.J).max() / np.abs(g1.J).max())
    assert errs[0] / errs[1] > 12.0 and errs[1] / errs[2] > 12.0, errs
    assert errs[2] < 1e-4, errs


def test_s_type_ring_shares_grid_lines_and_connects():
    # neighbouring arcs share 2 half + 1 angular grid lines: the receivers near an arc's
    # end are located in its neighbour at integer angular indices (up to rounding)
    w = W.small_multipatch_stype(K=4, half=6)
    sv = S.Solver(w)
    assert not sv.conn.errors
    it = sv.conn.items[1]
    sel = (it["donor"] == 0) & (it["j"] > 0)  # receivers of arc 1 fed by arc 0
    assert sel.any()
    s1 = it["a1"][sel] + it["t1"][sel]
    assert np.abs(s1 - np.round(s1)).max() < 1e-9
    assert np.array_equal(np.round(s1).astype(int) - 32, it["i"][sel])


def test_s_type_arcs_agree_with_the_periodic_o_grid():
    # the same annulus as four FC-continued arcs and as one Fourier-differentiated
    # periodic O-grid (coincident points): on a smooth field the two RHS agree to the
    # FC error, smallest away from the arc ends
    w0 = W.small_multipatch(W.ADIABATIC)
    w1 = W.small_multipatch_stype(K=4, half=6)
    og = w0.patches[0]
    g0 = geometry.PatchGeo(og, w0.params)
    sv = S.Solver.__new__(S.Solver)
    sv.prm = w0.params

    def state(x, y):
        rho = 1.4 * (1 + 0.1 * np.sin(1.3 * x + 0.7) * np.cos(0.9 * y))
        u, v, p = 0.5 + 0.2 * np.cos(0.8 * y), 0.1 * np.sin(0.6 * x), 1.0 + 0.1 * np.cos(x - y)
        return np.stack(W.prim_to_cons(rho, u, v, p))

    def mu(x, y):
        return 1e-3 * (1 + np.sin(x) ** 2)

    r0 = sv.rhs_patch(g0, state(g0.x, g0.y), mu(g0.x, g0.y))
    for k, p in enumerate(w1.patches[:4]):
        g = geometry.PatchGeo(p, w1.params)
        idx = np.mod(k * 32 - 6 + np.arange(p.n1), og.n1)
        assert np.abs(g.x - g0.x[:, idx]).max() < 1e-13 and np.abs(g.y - g0.y[:, idx]).max() < 1e-13
        r = sv.rhs_patch(g, state(g.x, g.y), mu(g.x, g.y))
        ref = r0[:, :, idx]
        scale = np.abs(ref).max()
        assert np.abs(r[:, :, 8:-8] - ref[:, :, 8:-8]).max() < 2e-6 * scale
        assert np.abs(r - ref).max() < 2e-4 * scale
