"""Pins of the oracle's geometry: fringes, donors, Neville, windows, SB operator."""
import numpy as np
import pytest

from oracle import geometry as G, viscosity as V
from paper_2506_16076_gb300 import workloads as W


def test_rnd_rounds_half_up():
    assert list(G.rnd([0.5, 1.5, -0.5, 2.49, 2.51])) == [1, 2, 0, 2, 3]


def test_neville_matches_lagrange_and_is_exact_on_quadratics():
    t = np.linspace(-0.5, 2.5, 13)
    f = lambda s: 3 - 2 * s + 0.7 * s * s
    vals = [np.full_like(t, f(k)) for k in (0.0, 1.0, 2.0)]
    assert np.abs(G.neville((0.0, 1.0, 2.0), vals, t) - f(t)).max() < 1e-13


def test_fringe_counts_closed_form():
    prm = W.Params()
    n1, n2 = 40, 30
    d = W.PatchDesc(W.AFFINE, n1, n2, (0, 1, 0, 1), (W.INTERNAL,) * 4)
    g = G.PatchGeo(d, prm)
    nf, nv = prm.n_f, prm.n_v
    assert g.receiver.sum() == n1 * n2 - (n1 - 2 * nf) * (n2 - 2 * nf)
    assert g.gen.sum() == (n1 - 2 * nv) * (n2 - 2 * nv)
    # external sides do not generate fringes
    d2 = W.PatchDesc(W.AFFINE, n1, n2, (0, 1, 0, 1), (W.DIRICHLET, W.INTERNAL, W.SLIPWALL, W.SLIPWALL))
    g2 = G.PatchGeo(d2, prm)
    assert g2.receiver.sum() == nf * n2 and g2.gen.sum() == (n1 - nv) * n2


@pytest.fixture(scope="module")
def small():
    w = W.small_multipatch()
    geos, conn = G.build(w)
    return w, geos, conn


def test_donor_receiver_condition_holds(small):
    w, geos, conn = small
    assert conn.errors == []
    for p, it in enumerate(conn.items):
        for q in np.unique(it["donor"]):
            sel = it["donor"] == q
            h = geos[q]
            assert q != p
            for m2 in range(3):
                for m1 in range(3):
                    i1 = it["a1"][sel] + m1
                    i1 = np.mod(i1, h.n1) if h.periodic1 else i1
                    i2 = it["a2"][sel] + m2
                    assert not (h.receiver[i2, i1] | h.blank[i2, i1]).any()


def test_exchange_exact_for_quadratics_from_affine_donors(small):
    w, geos, conn = small
    f = lambda x, y: 1.0 + 0.3 * x - 0.2 * y + 0.05 * x * x - 0.04 * x * y + 0.02 * y * y
    states = [np.stack([f(g.x, g.y)] * 4) for g in geos]
    states = conn.exchange(states)
    for g, it, e in zip(geos, conn.items, states):
        aff = np.array([geos[q].kind == W.AFFINE for q in it["donor"]], bool)
        err = np.abs(e[0][it["j"], it["i"]] - f(g.x[it["j"], it["i"]], g.y[it["j"], it["i"]]))
        if aff.any():
            assert err[aff].max() < 1e-12
        if (~aff).any():  # curvilinear donor: third-order accurate only
            assert err[~aff].max() < 2e-3


def test_window_weights():
    k = np.arange(-12, 13)
    w = V.window_weight(k, 0, 9)
    assert w[k == 0] == 1.0 and (w[np.abs(k) >= 9] == 0).all() and (w > 0).sum() == 17
    assert np.allclose(w, w[::-1]) and (np.diff(w[12:]) <= 0).all()
    # c = 18: flat top of width 18 cells, then a cos^2 roll-off over 9 cells
    ws = V.window_weight(np.array([0, 8.9, 9.0, 13.5, 18.0, 19.0]), 18, 9)
    assert np.allclose(ws, [1, 1, 1, 0.5, 0, 0])


def test_sb_operator_partition_of_unity(small):
    w, geos, conn = small
    sb = V.SBOperator(geos, w.params)
    muhat = [np.where(g.gen, 2.5, 0.0) for g in geos]
    mu = sb.apply(muhat)
    for g, m, den in zip(geos, mu, sb.den):
        covered = (den > 0) & ~g.blank
        assert covered.sum() == (~g.blank).sum()
        assert np.abs(m[covered] - 2.5).max() < 1e-13


def test_sdnn_standin_on_synthetic_classes():
    import importlib.util, os
    path = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2506_16076_gb300", "data", "train_sdnn.py")
    spec = importlib.util.spec_from_file_location("train_sdnn", path)
    ts = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(ts)
    X, y = ts.windows(np.random.default_rng(7), 4000)
    cls, _, _ = V.classify(X * 3.0 + 0.5)  # min-max normalisation makes the class scale-free
    assert (cls - 1 == y).mean() > 0.9
    flat = np.full((3, 7), 2.0)
    assert (V.classify(flat)[0] == 4).all()


def test_every_point_of_a_periodic_line_has_its_centred_window():
    # Sec. 5: each point's classifier input is the 7-point stencil centred on it; along
    # a periodic q1 line it wraps, so the points next to the seam (i = 0, 1, 2 and
    # n - 3 .. n - 1) keep a centred window too
    og = W.small_multipatch().patches[0]
    g = G.PatchGeo(og, W.Params(d=5, C0=27, c_policy=2))
    st = V.window_starts(g, 1)
    assert (st >= 0).all()
    i = np.arange(g.n1)
    assert np.array_equal(st[0], np.mod(i - 3, g.n1))
    # the non-periodic q2 lines: windows clamped inside the line
    s2 = V.window_starts(g, 2)
    j = np.arange(g.n2)
    assert np.array_equal(s2[:, 0], np.clip(j - 3, 0, g.n2 - 7))


def test_intra_patch_exchange_copies_shared_points():
    # sub-patches of one patch share their overlap grid points (Sec. 3.2.1); the exchange
    # between them copies values (Sec. 3.4.2): every such receiver's stencil offsets are
    # integers and its value equals the coincident donor point's bit for bit
    from oracle import geometry as G
    w = W.subpatched(W.sod128(185))  # 2 x 2 sub-patches of 101 x 101 sharing 17 lines
    geos, conn = G.build(w)
    rng = np.random.default_rng(4)
    states = [rng.normal(size=(4, g.n2, g.n1)) for g in geos]
    before = [s.copy() for s in states]
    conn.exchange(states)
    ncopy = 0
    for p, it in enumerate(conn.items):
        for k in range(len(it["j"])):
            q = it["donor"][k]
            if q < 0:
                continue
            assert float(it["t1"][k]).is_integer() and float(it["t2"][k]).is_integer()
            i1 = int(it["a1"][k] + it["t1"][k])
            i2 = int(it["a2"][k] + it["t2"][k])
            got = states[p][:, it["j"][k], it["i"][k]]
            assert np.array_equal(got, before[q][:, i2, i1])
            ncopy += 1
    assert ncopy > 1000
