"""Pins of the oracle's physics, time stepping and whole-solver behaviour."""
import dataclasses
import os

import numpy as np
import pytest

from oracle import euler, riemann, solver as S, viscosity as V
from paper_2506_16076_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()[:2]
                out[k] = float(v)
    return out


def test_defaults_follow_the_paper():
    g = golden_constants()
    p = W.Params()
    assert p.gamma == g["gamma"] and p.n_v == g["n_v"] and p.n_f == g["n_f"]
    assert p.alpha_f == g["alpha_f"] and p.p_f == g["p_f"] and p.cfl == g["cfl"]
    assert tuple(p.R) == (g["R1"], g["R2"], g["R3"], g["R4"])
    assert p.loc == g["loc_stencil"] and p.win_r == g["sb_r"]
    assert len(S.SSP54_ALPHA) == g["rk_stages"]
    assert abs(1 / np.pi - g["dt_prefactor"]) < 1e-16


def test_flux_closed_form():
    gam = 1.4
    rho, u, v, p = 2.0, 3.0, -1.0, 5.0
    e = euler.cons_from_prim(np.array(rho), np.array(u), np.array(v), np.array(p), gam)
    E = p / 0.4 + 0.5 * rho * (u * u + v * v)
    assert np.allclose(e, [2.0, 6.0, -2.0, E])
    assert np.allclose(euler.flux_x(e, gam), [rho * u, rho * u * u + p, rho * u * v, u * (E + p)])
    assert np.allclose(euler.flux_y(e, gam), [rho * v, rho * u * v, rho * v * v + p, v * (E + p)])
    a = np.sqrt(gam * p / rho)
    assert np.isclose(euler.sound_speed(e, gam), a)
    assert np.isclose(euler.mwsb(e, gam), abs(u) + abs(v) + a)
    assert np.isclose(euler.proxy_mach(e, gam), np.hypot(u, v) / a)
    assert np.isclose(euler.temperature(e, gam), p / rho)
    assert np.isclose(euler.energy_from_theta(e[0], e[1], e[2], p / rho, gam), E)


@pytest.mark.parametrize("M", [3.0, 10.0, 25.0])
def test_mach_shock_ic_satisfies_rankine_hugoniot(M):
    # eq. mach_shock_ic: a shock moving at speed M into (1.4, 0, 0, 1) (sound speed 1).
    # Reading: the printed post-shock density (gamma+1)M^2/((gamma-1)M^2+2) is the
    # density RATIO; with pre-shock density 1.4 the state is 1.4 times it.
    gam = 1.4
    zeta = (2 * gam * M * M - gam + 1) / (gam + 1)
    ratio = (gam + 1) * M * M / ((gam - 1) * M * M + 2)
    printed = np.array([ratio, (zeta - 1) / (gam * M), 0.0, zeta])
    eP = euler.cons_from_prim(*printed, gam)
    eR0 = euler.cons_from_prim(1.4, 0.0, 0.0, 1.0, gam)
    assert abs((euler.flux_x(eP, gam) - euler.flux_x(eR0, gam))[0] - M * (eP - eR0)[0]) > 0.1  # printed form fails mass
    post = np.array([1.4 * ratio, (zeta - 1) / (gam * M), 0.0, zeta])
    pre = np.array([1.4, 0.0, 0.0, 1.0])
    eL = euler.cons_from_prim(*post, gam)
    eR = euler.cons_from_prim(*pre, gam)
    jump_f = euler.flux_x(eL, gam) - euler.flux_x(eR, gam)
    assert np.allclose(jump_f, M * (eL - eR), rtol=1e-12, atol=1e-12)


def test_ssprk54_order_conditions_and_ssp():
    A, b, c = S.butcher_from_shu_osher()
    tol = 1e-13
    assert abs(b.sum() - 1) < tol
    assert abs(b @ c - 1 / 2) < tol
    assert abs(b @ c ** 2 - 1 / 3) < tol
    assert abs(b @ (A @ c) - 1 / 6) < tol
    assert abs(b @ c ** 3 - 1 / 4) < tol
    assert abs(b @ (c * (A @ c)) - 1 / 8) < tol
    assert abs(b @ (A @ c ** 2) - 1 / 12) < tol
    assert abs(b @ (A @ (A @ c)) - 1 / 24) < tol
    # SSP: all Shu-Osher coefficients non-negative, each row of alpha sums to 1
    for al, be in zip(S.SSP54_ALPHA, S.SSP54_BETA):
        assert min(al) >= 0 and min(be) >= 0 and abs(sum(al) - 1) < 1e-14


def test_ssprk54_fourth_order_on_linear_ode():
    lam = -1.0 + 2.0j
    errs = []
    for n in (10, 20, 40, 80):
        dt = 1.0 / n
        y = 1.0 + 0j
        for _ in range(n):
            u = [y]
            Ls = []
            for i in range(5):
                Ls.append(lam * u[i])
                u.append(sum(S.SSP54_ALPHA[i][k] * u[k] + S.SSP54_BETA[i][k] * dt * Ls[k] for k in range(i + 1)))
            y = u[5]
        errs.append(abs(y - np.exp(lam)))
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(3)]
    assert min(rates) > 3.8, rates


def test_riemann_solver_sod_star_state():
    # closed-form Sod star state (textbook values p* = 0.30313, u* = 0.92745)
    p, u = riemann.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(p - 0.30313) < 1e-5 and abs(u - 0.92745) < 1e-5


@pytest.mark.slow
def test_sod_against_exact_riemann_and_invariants():
    w = W.sod128(128)
    sv = S.Solver(w)
    st0 = S.smear_initial(sv, W.initial_state(w), 0.5)
    g = sv.geos[0]
    hx = hy = 1.0 / 127

    def integ(a):  # trapezoid over the unit square
        wx = np.full(128, hx); wx[[0, -1]] *= 0.5
        wy = np.full(128, hy); wy[[0, -1]] *= 0.5
        return wy @ a @ wx

    out, dts = sv.run(st0, 100)
    T = sum(dts)
    e = out[0]
    rho, u, v, p = euler.primitives(e, 1.4)
    # y-invariance and vanishing transverse velocity
    assert np.abs(e - e[:, 64:65]).max() < 1e-9
    assert np.abs(v).max() < 1e-9
    r_ex, u_ex, p_ex = riemann.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (g.x[64] - 0.5) / T)
    assert np.mean(np.abs(rho[64] - r_ex)) < 2e-2
    assert np.mean(np.abs(p[64] - p_ex)) < 2e-2
    # conservation before the waves reach x = 0, 1: mass and energy constant,
    # x-momentum grows at rate p_L - p_R = 0.9 (non-conservative chain-rule form: not exact)
    m0, m1 = integ(st0[0][0]), integ(e[0])
    E0, E1 = integ(st0[0][3]), integ(e[3])
    P1 = integ(e[1])
    assert abs(m1 - m0) / m0 < 1e-3
    assert abs(E1 - E0) / E0 < 1e-3
    assert abs(P1 - 0.9 * T) / (0.9 * T) < 2e-2
    assert np.all(np.isfinite(e)) and rho.min() > 0.1 and p.min() > 0.09


def test_free_stream_preserved_on_curvilinear_multipatch():
    w = W.small_multipatch()
    og = w.patches[0]
    w.patches[0] = dataclasses.replace(og, side=(W.PERIODIC, W.PERIODIC, W.DIRICHLET, W.INTERNAL))
    sv = S.Solver(w)
    st = W.initial_state(w)
    out, dts = sv.run(st, 3)
    for g, o, f in zip(sv.geos, out, st):
        dev = np.abs(np.where(g.blank[None], 0, o - f)).max(axis=(1, 2))
        assert (dev <= 2e-12 * np.abs(f).max(axis=(1, 2)) + 1e-13).all(), dev


def test_slip_wall_zeroes_normal_momentum():
    w = W.small_multipatch()
    sv = S.Solver(w)
    out = sv.step(W.initial_state(w), 0)
    g = sv.geos[0]
    mn = out[0][1][0] * g.cos[0] + out[0][2][0] * g.sin[0]
    assert np.abs(mn).max() < 1e-13


def test_stored_sod_reference_matches_oracle():
    # the stored 100-step shock-tube state (tests/golden/sod128_100steps.npz) comes from
    # this oracle: its first two CFL steps are recomputed here
    from tests.golden.make_sod128_reference import OUT
    ref = np.load(OUT)
    w = W.sod128(128)
    sv = S.Solver(w)
    st = S.smear_initial(sv, W.initial_state(w), 0.5)
    for n in range(2):
        st = sv.step(st, n)
        assert abs(sv.last_dt - ref["dt"][n]) <= 1e-15 * ref["dt"][n]
    assert ref["state"].shape == (4, 128, 128) and np.isfinite(ref["state"]).all()


def test_adiabatic_weights():
    # d = 2: p = a0 (p'(0) = 0) through theta_1; d = 3: p = a0 + a2 x^2 through
    # theta_1, theta_2 gives a0 = (4 theta_1 - theta_2) / 3
    assert S.adiabatic_weights(2) == (1.0,)
    w3 = S.adiabatic_weights(3)
    assert abs(w3[0] - 4 / 3) < 1e-15 and abs(w3[1] + 1 / 3) < 1e-15
    for d in (2, 3, 4, 5, 6):
        w = np.array(S.adiabatic_weights(d))
        j = np.arange(1, d, dtype=float)
        assert abs(w.sum() - 1.0) < 1e-13  # constants
        for k in range(2, d):  # x^k has zero slope at 0 and value 0 there
            assert abs(w @ j ** k) < 1e-11 * j.max() ** k


def test_adiabatic_wall_condition():
    # after the wall overwrite: zero momenta at the wall, and the temperature along each
    # wall-normal line has zero slope at the wall (degree d-1 fit through the wall value
    # and the d-1 inward values)
    w = W.small_multipatch(W.ADIABATIC)
    sv = S.Solver(w)
    st = sv.apply_bc(W.random_smooth_state(w, seed=3, amp=0.1))
    e = st[0]
    assert np.all(e[1][0] == 0.0) and np.all(e[2][0] == 0.0)
    th = euler.temperature(e, w.params.gamma)
    d = w.params.d
    x = np.arange(d, dtype=float)
    for i in range(0, e.shape[2], 7):
        c = np.polyfit(x, th[:d, i], d - 1)
        assert abs(c[-2]) < 1e-9 * np.abs(th[:d, i]).max(), c  # slope at the wall
