"""Pins of the oracle's preliminary viscosity (Sec. 5.1, eq. V2D_unscaled) and time step
(Sec. 4.1, eq. CFL) against values worked out here by brute force from the definitions.

mu^_ij = R(tau~_ij) * max over the 7 x 7 index stencil around (i, j), clipped to the
patch grid (wrapped along a periodic angle) and over non-blanked points, of
S = |u| + |v| + a, times h^ (the largest distance between index-adjacent grid points),
on the generating points G~ only. The classes are forced, so that each of R(1..4) is
used next to planted maxima of S at index distances 3 and 4, next to the sides, across
the seam of a periodic line and on a blanked point.

dt = (1/pi) min_p CFL / (max S / h~_p + max mu / h~_p^2), h~_p the smallest distance
between index-adjacent points of patch p, maxima over its non-blanked points.
"""
import math

import numpy as np
import pytest

from oracle import solver as S
from oracle import viscosity as V
from paper_2506_16076_gb300 import workloads as W

GAMMA = 1.4
R_TAB = (1.5, 1.0, 0.5, 0.0)


def _spacings(p):
    """(largest, smallest) distance between index-adjacent points, from the coordinates."""
    x, y = W.patch_xy(p)
    d1 = np.hypot(np.diff(x, axis=1), np.diff(y, axis=1))
    d2 = np.hypot(np.diff(x, axis=0), np.diff(y, axis=0))
    ds = [d1.ravel(), d2.ravel()]
    if p.side[0] == W.PERIODIC:
        ds.append(np.hypot(x[:, 0] - x[:, -1], y[:, 0] - y[:, -1]))
    allv = np.concatenate(ds)
    return allv.max(), allv.min()


def _state(prim):
    rho, u, v, p = prim
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)])


def _brute_muhat(p, prim, tau, gen, blank):
    rho, u, v, pr = prim
    n2, n1 = rho.shape
    spd = np.abs(u) + np.abs(v) + np.sqrt(GAMMA * pr / rho)
    hhat, _ = _spacings(p)
    per = p.side[0] == W.PERIODIC
    out = np.zeros((n2, n1))
    for j in range(n2):
        for i in range(n1):
            if not gen[j, i]:
                continue
            best = 0.0
            for dj in range(-3, 4):
                for di in range(-3, 4):
                    jj, ii = j + dj, i + di
                    if per:
                        ii %= n1
                    if not (0 <= jj < n2 and 0 <= ii < n1) or blank[jj, ii]:
                        continue
                    best = max(best, spd[jj, ii])
            out[j, i] = R_TAB[tau[j, i] - 1] * best * hhat
    return out


def _forced_tau(n2, n1):
    j, i = np.mgrid[0:n2, 0:n1]
    return 1 + (i + 2 * j) % 4


def _check_preliminary(monkeypatch, p, prim, gen_expected, params=None):
    w = W.Workload("pin", [p], params or W.Params(), freestream=(1.0, 0.0, 0.0, 1.0), init="freestream", steps=1)
    g = S.Solver(w).geos[0]
    assert np.array_equal(g.gen, gen_expected)
    tau = _forced_tau(p.n2, p.n1)
    monkeypatch.setattr(V, "tau_patch", lambda g_, phi: (tau, np.full(tau.shape, np.inf)))
    muhat, t, _ = V.preliminary(g, _state(prim), w.params)
    assert np.array_equal(t, tau)
    ref = _brute_muhat(p, prim, tau, gen_expected, g.blank)
    assert np.abs(muhat - ref).max() <= 1e-13 * np.abs(ref).max()
    return muhat, ref


def _uniform_prim(n2, n1, rho=1.0, u=0.3, v=0.1, p=1.0):
    return [np.full((n2, n1), c, dtype=float) for c in (rho, u, v, p)]


def test_preliminary_affine_box(monkeypatch):
    # non-square spacing (h^ = 0.1 along x, 0.0647 along y), q1 = 0 side internal: the
    # generating points are i >= n_v = 9
    n1, n2 = 24, 18
    p = W.PatchDesc(W.AFFINE, n1, n2, (0.0, 2.3, 0.0, 1.1),
                    (W.INTERNAL, W.DIRICHLET, W.DIRICHLET, W.DIRICHLET), bc=((1.0, 0.0, 0.0, 1.0),) * 4)
    prim = _uniform_prim(n2, n1)
    prim[1][8, 13] = 3.0     # interior maximum: reaches i = 10..16, j = 5..11 and no further
    prim[1][0, 22] = 2.0     # next to two sides: the stencil is clipped, not wrapped
    prim[2][15, 5] = -1.5    # outside G~ and 4 columns from it: reaches no generating point
    prim[2][14, 6] = -1.2    # reaches i = 9, the first generating column
    prim[3][3, 18] = 4.0     # pressure maximum (sound speed)
    gen = np.zeros((n2, n1), bool)
    gen[:, 9:] = True
    muhat, ref = _check_preliminary(monkeypatch, p, prim, gen)
    # the planted interior maximum is seen at index distance 3 and not at 4
    s_peak = 3.0 + 0.1 + math.sqrt(GAMMA)
    tau = _forced_tau(n2, n1)
    assert muhat[8, 16] == pytest.approx(R_TAB[tau[8, 16] - 1] * s_peak * 0.1, rel=1e-14)
    assert muhat[11, 10] == pytest.approx(R_TAB[tau[11, 10] - 1] * s_peak * 0.1, rel=1e-14)
    if tau[8, 17] < 4:
        assert muhat[8, 17] < R_TAB[tau[8, 17] - 1] * s_peak * 0.1 * 0.99
    assert np.all(muhat[:, :9] == 0.0)


def test_preliminary_periodic_ogrid(monkeypatch):
    # periodic angle: a maximum at i = 1 reaches i = n1 - 2 across the seam; h^ is the
    # outer chord 2 r1 sin(pi / n1) or the radial spacing, whichever is larger
    n1, n2 = 40, 20
    p = W.PatchDesc(W.OGRID, n1, n2, (0.0, 0.0, 0.5, 1.5), (W.PERIODIC, W.PERIODIC, W.SLIPWALL, W.INTERNAL),
                    bc=((1.0, 0.0, 0.0, 1.0),) * 4)
    prim = _uniform_prim(n2, n1, u=0.2, v=-0.4)
    prim[1][4, 1] = 5.0
    prim[3][9, n1 - 1] = 3.0
    gen = np.zeros((n2, n1), bool)
    gen[:n2 - 9, :] = True
    hhat, _ = _spacings(p)
    assert hhat == pytest.approx(max(1.0 / (n2 - 1), 2 * 1.5 * math.sin(math.pi / n1)), rel=1e-14)
    muhat, ref = _check_preliminary(monkeypatch, p, prim, gen)
    tau = _forced_tau(n2, n1)
    s_peak = 5.0 + 0.4 + math.sqrt(GAMMA)
    for i in (n1 - 2, n1 - 1, 0, 1, 2, 3, 4):
        assert muhat[4, i] == pytest.approx(R_TAB[tau[4, i] - 1] * s_peak * hhat, rel=1e-14)


def test_preliminary_skips_blanked_points(monkeypatch):
    # a hole blanks the box's lower-left corner; a huge speed planted on a blanked point
    # must not reach any generating point (n_v = 2 here, so that generating points sit
    # within 3 points of the hole)
    n1, n2 = 20, 20
    prm = W.Params(n_v=2)
    p = W.PatchDesc(W.AFFINE, n1, n2, (0.0, 1.0, 0.0, 1.0),
                    (W.DIRICHLET, W.DIRICHLET, W.DIRICHLET, W.DIRICHLET), bc=((1.0, 0.0, 0.0, 1.0),) * 4,
                    hole=(0.0, 0.0, 0.3))
    prim = _uniform_prim(n2, n1)
    prim[1][5, 2] = 50.0  # blanked (distance 0.283 < 0.3), 3 points from generating points
    w = W.Workload("pin", [p], prm, freestream=(1.0, 0.0, 0.0, 1.0), init="freestream", steps=1)
    g = S.Solver(w).geos[0]
    assert g.blank[5, 2] and not g.blank[n2 - 1, n1 - 1]
    assert g.gen[8, 1] and _forced_tau(n2, n1)[8, 1] < 4
    muhat, ref = _check_preliminary(monkeypatch, p, prim, g.gen.copy(), prm)
    s_bg = 0.4 + math.sqrt(GAMMA)
    tau = _forced_tau(n2, n1)
    assert np.all(muhat[g.gen] <= np.array(R_TAB)[tau[g.gen] - 1] * s_bg / 19 * (1 + 1e-14))


def test_dt_uniform_single_patch():
    w = W.sod128(32)
    sv = S.Solver(w)
    rho, u, v, pr, mu = 1.3, 0.4, -0.2, 0.9, 3e-3
    n = 32
    e = _state([np.full((n, n), c) for c in (rho, u, v, pr)])
    s_ = abs(u) + abs(v) + math.sqrt(GAMMA * pr / rho)
    h = 1.0 / 31
    ref = 0.5 / (s_ / h + mu / h ** 2) / math.pi
    assert sv.dt([e], [np.full((n, n), mu)]) == pytest.approx(ref, rel=1e-14)
    # with mu = 0 the step is the plain wave-speed limit
    assert sv.dt([e], [np.zeros((n, n))]) == pytest.approx(0.5 * h / s_ / math.pi, rel=1e-14)


@pytest.mark.parametrize("fast_patch", [0, 3])
def test_dt_minimum_over_patches(fast_patch):
    # piecewise-uniform states on the O-grid + 2 x 2 boxes; the patch that sets the step
    # changes with the planted speed, and blanked points (with a huge mu) do not count
    w = W.small_multipatch()
    sv = S.Solver(w)
    states, mus, cand = [], [], []
    for k, p in enumerate(w.patches):
        u = 9.0 if k == fast_patch else 0.5 + 0.1 * k
        prim = (1.0 + 0.05 * k, u, 0.2, 1.0 + 0.1 * k)
        states.append(_state([np.full((p.n2, p.n1), c) for c in prim]))
        mval = 1e-3 * (k + 1)
        m = np.full((p.n2, p.n1), mval)
        g = sv.geos[k]
        if g.blank.any():
            m[g.blank] = 1e3
        mus.append(m)
        _, htil = _spacings(p)
        if p.kind == W.OGRID:
            assert htil == pytest.approx(min(1.0 / (p.n2 - 1), 2 * 0.5 * math.sin(math.pi / p.n1)), rel=1e-14)
        else:
            x0, x1, y0, y1 = p.geom
            assert htil == pytest.approx(min((x1 - x0) / (p.n1 - 1), (y1 - y0) / (p.n2 - 1)), rel=1e-14)
        spd = abs(u) + 0.2 + math.sqrt(GAMMA * prim[3] / prim[0])
        cand.append(w.params.cfl / (spd / htil + mval / htil ** 2))
    ref = min(cand) / math.pi
    assert int(np.argmin(cand)) == fast_patch
    assert sv.dt(states, mus) == pytest.approx(ref, rel=1e-14)
