"""Pins of the oracle's discrete adjoint: dot-product identities against complex-step
directional derivatives of the forward map, and a central-difference check of a
functional gradient on a tiny grid."""
import dataclasses

import numpy as np
import pytest

from oracle import adjoint as A, fc, solver as S
from paper_2506_16076_gb300 import workloads as W


def dot(a, b):
    return sum(float(np.vdot(x, y).real) for x, y in zip(a, b))


def rand_like(states, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=a.shape) for a in states]


@pytest.mark.parametrize("N,C", [(10, 27), (37, 29), (64, 27)])
def test_fc_derivative_transpose(N, C):
    rng = np.random.default_rng(N)
    x, y = rng.normal(size=(3, N)), rng.normal(size=(3, N))
    h = 1.0 / (N - 1)
    lhs = np.sum(fc.fc_derivative(x, h, 5, C) * y)
    rhs = np.sum(x * fc.fc_derivative_T(y, h, 5, C))
    assert abs(lhs - rhs) < 1e-11 * np.abs(fc.fc_derivative(x, h, 5, C)).max() * np.abs(y).sum()
    xp = rng.normal(size=(2, 48))
    yp = rng.normal(size=(2, 48))
    assert abs(np.sum(fc.periodic_derivative(xp, 1 / 48) * yp) - np.sum(xp * fc.periodic_derivative_T(yp, 1 / 48))) < 1e-10


@pytest.fixture(scope="module")
def small():
    w = W.small_multipatch()
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=2, amp=0.05))
    mu = [0.002 * (1 + np.cos(g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    return w, sv, st, mu


def test_rhs_adjoint_dot_product(small):
    w, sv, st, mu = small
    v = rand_like(st, 1)
    lam = rand_like(st, 2)
    jv = A.rhs_jvp_complex(sv, st, mu, v)
    jtl = A.rhs_adjoint(sv, st, mu, lam)
    lhs, rhs = dot(jv, lam), dot(v, jtl)
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0) * 1e2, (lhs, rhs)


def test_project_adjoint_dot_product(small):
    w, sv, st, mu = small
    v = rand_like(st, 3)
    lam = rand_like(st, 4)
    jv = A.project_jvp_complex(sv, st, v)
    lhs, rhs = dot(jv, lam), dot(v, A.project_T(sv, lam))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


@pytest.fixture(scope="module")
def small_adiabatic():
    w = W.small_multipatch(W.ADIABATIC)
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=12, amp=0.05))
    mu = [0.002 * (1 + np.cos(g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    return w, sv, st, mu


def test_project_adjoint_dot_product_adiabatic_wall(small_adiabatic):
    w, sv, st, mu = small_adiabatic
    v = rand_like(st, 13)
    lam = rand_like(st, 14)
    jv = A.project_jvp_complex(sv, st, v)
    lhs, rhs = dot(jv, lam), dot(v, A.project_T(sv, lam, None, st))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


def test_step_adjoint_dot_product_adiabatic_wall(small_adiabatic):
    w, sv, st, mu = small_adiabatic
    dt = 0.5 * sv.dt(st, mu)
    v = rand_like(st, 15)
    lam = rand_like(st, 16)
    jv = A.step_jvp_complex(sv, st, mu, dt, v)
    lam_n, _ = A.step_adjoint(sv, st, mu, dt, lam)
    lhs, rhs = dot(jv, lam), dot(v, lam_n)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("N,C", [(10, 27), (37, 29), (64, 27)])
def test_fc_filter_transpose(N, C):
    rng = np.random.default_rng(N + 1)
    x, y = rng.normal(size=(3, N)), rng.normal(size=(3, N))
    lhs = np.sum(fc.fc_filter(x, 5, C, 10.0, 14) * y)
    rhs = np.sum(x * fc.fc_filter_T(y, 5, C, 10.0, 14))
    assert abs(lhs - rhs) < 1e-13 * np.abs(x).sum() * np.abs(y).max() * 10


@pytest.mark.parametrize("fix", ["small", "small_adiabatic"])
def test_filter_adjoint_dot_product(fix, request):
    w, sv, st, mu = request.getfixturevalue(fix)
    v = rand_like(st, 21)
    lam = rand_like(st, 22)
    jv = A.filter_jvp_complex(sv, st, v)
    lhs, rhs = dot(jv, lam), dot(v, A.filter_T(sv, lam, st))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs), (lhs, rhs)


def test_step_adjoint_with_filter_dot_product(small_adiabatic):
    w, sv, st, mu = small_adiabatic
    dt = 0.5 * sv.dt(st, mu)
    v = rand_like(st, 23)
    lam = rand_like(st, 24)
    jv = A.step_jvp_complex(sv, st, mu, dt, v, filt=True)
    lam_n, _ = A.step_adjoint(sv, st, mu, dt, lam, filt=True)
    lhs, rhs = dot(jv, lam), dot(v, lam_n)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)


def test_step_adjoint_dot_product(small):
    w, sv, st, mu = small
    dt = 0.5 * sv.dt(st, mu)
    v = rand_like(st, 5)
    lam = rand_like(st, 6)
    jv = A.step_jvp_complex(sv, st, mu, dt, v)
    lam_n, _ = A.step_adjoint(sv, st, mu, dt, lam)
    lhs, rhs = dot(jv, lam), dot(v, lam_n)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)


def test_drag_gradient_central_differences():
    # tiny cylinder grid, frozen mu and dt: dJ/de_0 . v against central differences (step 1e-6)
    w = W.small_multipatch()
    sv = S.Solver(w)
    st0 = sv.project(W.random_smooth_state(w, seed=7, amp=0.02))
    mu = [np.zeros((p.n2, p.n1)) for p in w.patches]
    dt = 0.5 * sv.dt(st0, mu)
    nsteps = 2

    def J_of(st):
        for _ in range(nsteps):
            st = A.step_forward(sv, st, mu, dt)[5]
        return A.wall_drag(sv, st)

    traj = [st0]
    for _ in range(nsteps):
        traj.append(A.step_forward(sv, traj[-1], mu, dt)[5])
    lam = A.wall_drag_grad(sv, traj[-1])
    for n in range(nsteps - 1, -1, -1):
        lam, _ = A.step_adjoint(sv, traj[n], mu, dt, lam)
    v = rand_like(st0, 8)
    h = 1e-6
    fd = (J_of([a + h * b for a, b in zip(st0, v)]) - J_of([a - h * b for a, b in zip(st0, v)])) / (2 * h)
    ad = dot(lam, v)
    assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-3), (fd, ad)


@pytest.mark.parametrize("make", [W.small_multipatch_grid, W.small_multipatch_stype], ids=["grid_curved", "s_type"])
def test_step_adjoint_with_filter_dot_product_on_grid_patches(make):
    # the adjoint of a filtered step on hole-cut curved GRID patches and on S-type arcs
    # (exchange into and out of GRID donors, adiabatic wall on a GRID side)
    w = make()
    sv = S.Solver(w)
    st = sv.project(W.random_smooth_state(w, seed=32, amp=0.05))
    mu = [0.002 * (1 + np.cos(g.x) * np.sin(g.y)) ** 2 for g in sv.geos]
    dt = 0.5 * sv.dt(st, mu)
    v = rand_like(st, 33)
    lam = rand_like(st, 34)
    jv = A.step_jvp_complex(sv, st, mu, dt, v, filt=True)
    lam_n, _ = A.step_adjoint(sv, st, mu, dt, lam, filt=True)
    lhs, rhs = dot(jv, lam), dot(v, lam_n)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)


def _mach_workload(mach, alpha):
    import dataclasses
    w = W.small_multipatch()
    fs = (1.4, mach * np.cos(alpha), mach * np.sin(alpha), 1.0)
    return W.Workload("small_mach", [dataclasses.replace(p, bc=(fs,) * 4) for p in w.patches], w.params, fs,
                      "freestream", 2)


def test_freestream_jacobian_against_differences():
    fs = (1.4, 2.0 * np.cos(0.05), 2.0 * np.sin(0.05), 1.0)  # a = 1: Mach 2 at 0.05 rad
    a = np.sqrt(1.4 * 1.0 / 1.4)
    e = A.freestream_state(2.0, 0.05, 1.4, 1.0, 1.4)
    assert np.allclose(e, [1.4, 1.4 * fs[1], 1.4 * fs[2], 1.0 / 0.4 + 0.7 * 4.0], rtol=1e-15)
    dM, dA = A.freestream_jacobian(fs, 1.4)
    h = 1e-6
    fdM = (A.freestream_state(2.0 + h, 0.05, 1.4, 1.0, 1.4) - A.freestream_state(2.0 - h, 0.05, 1.4, 1.0, 1.4)) / (2 * h)
    fdA = (A.freestream_state(2.0, 0.05 + h, 1.4, 1.0, 1.4) - A.freestream_state(2.0, 0.05 - h, 1.4, 1.0, 1.4)) / (2 * h)
    assert np.allclose(dM, fdM, rtol=1e-8, atol=1e-9) and np.allclose(dA, fdA, rtol=1e-8, atol=1e-9)
    assert dM[0] == 0.0 and dA[0] == 0.0 and abs(dA[3]) < 1e-15 and a == 1.0  # energy: |u| fixed


def test_parameter_gradients_central_differences():
    # J = wall drag after 2 steps (mu = 0, dt frozen) from the uniform free stream of
    # (Mach, alpha), with the Dirichlet sides holding the same free stream: dJ/dMach and
    # dJ/dalpha from the adjoint (Dirichlet part + initial-state part) against central
    # differences, and dJ/drho_0 at a few points against density perturbations
    M0, a0, nsteps, h = 2.0, 0.04, 2, 1e-6
    w = _mach_workload(M0, a0)
    sv = S.Solver(w)
    st0 = W.initial_state(w)
    mu = [np.zeros((p.n2, p.n1)) for p in w.patches]
    dt = 0.5 * sv.dt(sv.project([a.copy() for a in st0]), mu)

    def J_of(mach, alpha, drho=None):
        ww = _mach_workload(mach, alpha)
        s2 = S.Solver(ww)
        st = W.initial_state(ww)
        if drho is not None:
            from oracle import euler
            out = []
            for e, d in zip(st, drho):
                rho, u, v, p = euler.primitives(e, 1.4)
                out.append(euler.cons_from_prim(rho + d, u, v, p, 1.4))
            st = out
        for _ in range(nsteps):
            st = A.step_forward(s2, st, mu, dt)[5]
        return A.wall_drag(s2, st)

    traj = [st0]
    for _ in range(nsteps):
        traj.append(A.step_forward(sv, traj[-1], mu, dt)[5])
    lam = A.wall_drag_grad(sv, traj[-1])
    par = np.zeros(2)
    for n in range(nsteps - 1, -1, -1):
        lam, gbc = A.step_adjoint(sv, traj[n], mu, dt, lam)
        par += A.dirichlet_param_sensitivity(sv, gbc, w.freestream)
    drho, par0 = A.initial_sensitivity(sv, st0, lam, w.freestream)
    par += par0
    fdM = (J_of(M0 + h, a0) - J_of(M0 - h, a0)) / (2 * h)
    fdA = (J_of(M0, a0 + h) - J_of(M0, a0 - h)) / (2 * h)
    assert abs(fdM - par[0]) <= 1e-6 * max(abs(par[0]), 1e-3), (fdM, par[0])
    assert abs(fdA - par[1]) <= 1e-6 * max(abs(par[1]), 1e-3), (fdA, par[1])
    scale = max(np.abs(d).max() for d in drho)
    k = 0  # points on the O-grid next to the wall, where the drag is most sensitive
    for (j, i) in ((1, 3), (2, 40), (4, 77)):
        d = [np.zeros((p.n2, p.n1)) for p in w.patches]
        d[k][j, i] = h
        fd = (J_of(M0, a0, d) - J_of(M0, a0, [-x for x in d])) / (2 * h)
        assert abs(fd - drho[k][j, i]) <= 1e-6 * scale, (j, i, fd, drho[k][j, i])
