"""Discrete adjoint of the semi-discrete operator and of one SSPRK-4 step (oracle).

Test infrastructure only (see oracle/__init__.py).

The forward map is the step of Algorithm 1 with the viscosity mu and the time
step dt frozen (the smoothness classifier is not differentiable) and no filter:
    u_0 = P(e_n),  u_i = P( sum_k alpha_ik u_k + beta_ik dt L(u_k) ),  e_{n+1} = u_5,
with P the boundary overwrite followed by the inter-patch exchange (Sec. 4.2,
Sec. 3.4.1) and L the operator of eq. (semi-discrete) in the curvilinear form of
eq. (general_curvilinear):
    L(u) = -N sum_k sum_i J_ki D_k( f_i(u) - mu sum_m J_mi D_m u ),
N = zeroing on points where a derivative is undefined. Its linearisation
transposes to
    eta_i = -sum_k D_k^T (J_ki N lam),
    L'(u)^T lam = sum_i A_i(u)^T eta_i - sum_m D_m^T ( mu sum_i J_mi eta_i ),
A_i = d f_i / d e the flux Jacobians, D^T the transposed FC derivative
(fc.fc_derivative_T). P^T: the exchange transpose scatters each receiver's
adjoint to its donors with the Neville (Lagrange) weights and zeroes the
receiver; the boundary transpose zeroes Dirichlet points (their adjoint is the
sensitivity to the imposed state) and projects out the wall-normal momentum.
"""
import numpy as np

from paper_2506_16076_gb300 import workloads as W
from . import fc
from .geometry import neville
from .solver import SSP54_ALPHA, SSP54_BETA


def flux_jacobians(e, gam):
    """A_x, A_y with A[c][j] = d f_c / d e_j (eq. euler 2d equation), arrays (4, 4, ...)."""
    rho, m, n, E = e
    u, v = m / rho, n / rho
    g1 = gam - 1.0
    p = g1 * (E - 0.5 * rho * (u * u + v * v))
    pr, pm, pn, pE = 0.5 * g1 * (u * u + v * v), -g1 * u, -g1 * v, g1 + 0 * u
    H = (E + p) / rho
    z, o = 0 * u, 1 + 0 * u
    Ax = np.array([[z, o, z, z],
                   [-u * u + pr, 2 * u + pm, pn, pE],
                   [-u * v, v, u, z],
                   [-u * H + u * pr, H + u * pm, u * pn, u * (1 + pE)]])
    Ay = np.array([[z, z, o, z],
                   [-u * v, v, u, z],
                   [-v * v + pr, pm, 2 * v + pn, pE],
                   [-v * H + v * pr, v * pm, H + v * pn, v * (1 + pE)]])
    return Ax, Ay


def d1T(sv, g, G):
    out = np.zeros_like(G)
    prm = sv.prm
    for (j, a, n, per) in g.seg1:
        if per:
            out[..., j, a:a + n] = fc.periodic_derivative_T(G[..., j, a:a + n], g.h1)
        elif n >= 2 * prm.d:
            out[..., j, a:a + n] = fc.fc_derivative_T(G[..., j, a:a + n], g.h1, prm.d,
                                                      fc.choose_C(n, prm.C0, prm.c_policy, prm.d))
    return out


def d2T(sv, g, G):
    out = np.zeros_like(G)
    prm = sv.prm
    for (i, a, n, per) in g.seg2:
        if n >= 2 * prm.d:
            out[..., a:a + n, i] = fc.fc_derivative_T(G[..., a:a + n, i], g.h2, prm.d,
                                                      fc.choose_C(n, prm.C0, prm.c_policy, prm.d))
    return out


def rhs_adjoint_patch(sv, g, u, mu, lam):
    """L'(u)^T lam on one patch."""
    if sv.product_form(g):
        return rhs_adjoint_patch_product(sv, g, u, mu, lam)
    J1x, J1y, J2x, J2y = g.J
    lm = np.where(g.nodiff[None], 0.0, lam)
    eta_x = -(d1T(sv, g, J1x * lm) + d2T(sv, g, J2x * lm))
    eta_y = -(d1T(sv, g, J1y * lm) + d2T(sv, g, J2y * lm))
    Ax, Ay = flux_jacobians(u, sv.prm.gamma)
    out = np.einsum("cj...,c...->j...", Ax, eta_x) + np.einsum("cj...,c...->j...", Ay, eta_y)
    out -= d1T(sv, g, mu * (J1x * eta_x + J1y * eta_y))
    out -= d2T(sv, g, mu * (J2x * eta_x + J2y * eta_y))
    return out


def rhs_adjoint_patch_product(sv, g, u, mu, lam, h=1e-30):
    """L'(u)^T lam on a patch in the product-rule form (Remark adiabatic):
        L(u) = -N ( c(u, Qx, Qy) + sum_k sum_i J_ki D_k H_i(u, Qx, Qy) ),
        Qx = sum_k J_kx D_k Q(u),  Qy = sum_k J_ky D_k Q(u),
    with Q = (rho, rho u, rho v, theta) and (c, H_x, H_y) the pointwise map of
    solver.wall_pointwise. Transposed in reverse order: eta_i = -sum_k D_k^T (J_ki N lam)
    are the adjoints of H_i and -N lam that of c; the transpose of the pointwise map's
    Jacobian (its 12 columns by the complex step, exact to rounding for this analytic
    map) gives the adjoints of u, Qx and Qy; Qbar = sum_k D_k^T (sum_i J_ki Qbar_i); and
    the Jacobian of Q(u) carries Qbar back to u."""
    from .solver import wall_pointwise, wall_quantities
    gam = sv.prm.gamma
    J1x, J1y, J2x, J2y = g.J
    lm = np.where(g.nodiff[None], 0.0, lam)
    eta_x = -(d1T(sv, g, J1x * lm) + d2T(sv, g, J2x * lm))
    eta_y = -(d1T(sv, g, J1y * lm) + d2T(sv, g, J2y * lm))
    Q = wall_quantities(u, gam)
    D1, D2 = sv.d1(g, Q), sv.d2(g, Q)
    inp = np.concatenate([u, J1x * D1 + J2x * D2, J1y * D1 + J2y * D2]).astype(complex)
    wbar = np.concatenate([-lm, eta_x, eta_y])  # adjoints of the outputs (c, H_x, H_y)
    bar = np.zeros(inp.shape)
    for j in range(12):
        z = inp.copy()
        z[j] += 1j * h
        out = np.concatenate(wall_pointwise(z[:4], z[4:8], z[8:], mu, gam))
        bar[j] = np.sum(wbar * (out.imag / h), axis=0)
    ubar, qxbar, qybar = bar[:4], bar[4:8], bar[8:]
    Qbar = d1T(sv, g, J1x * qxbar + J1y * qybar) + d2T(sv, g, J2x * qxbar + J2y * qybar)
    for j in range(4):  # dQ/du: identity on rho, rho u, rho v; d theta / d u_j
        z = u.astype(complex)
        z[j] += 1j * h
        ubar[j] += (Qbar[j] if j < 3 else 0.0) + (wall_quantities(z, gam)[3].imag / h) * Qbar[3]
    return ubar


def rhs_adjoint(sv, states, mus, lams):
    return [rhs_adjoint_patch(sv, g, u, m, l) for g, u, m, l in zip(sv.geos, states, mus, lams)]


def exchange_T(sv, lams):
    """Transpose of the exchange: receiver adjoints scattered to donors, receivers zeroed."""
    out = [l.copy() for l in lams]
    nodes = (0.0, 1.0, 2.0)
    for p, it in enumerate(sv.conn.items):
        if len(it["j"]) == 0:
            continue
        lr = lams[p][:, it["j"], it["i"]]
        for q in np.unique(it["donor"]):
            sel = it["donor"] == q
            h = sv.geos[q]
            t1, t2 = it["t1"][sel], it["t2"][sel]
            for m2 in range(3):
                w2 = neville(nodes, [np.full_like(t2, float(k == m2)) for k in range(3)], t2)
                for m1 in range(3):
                    w1 = neville(nodes, [np.full_like(t1, float(k == m1)) for k in range(3)], t1)
                    i1 = it["a1"][sel] + m1
                    i1 = np.mod(i1, h.n1) if h.periodic1 else i1
                    i2 = it["a2"][sel] + m2
                    np.add.at(out[q], (slice(None), i2, i1), w2 * w1 * lr[:, sel])
    for p, it in enumerate(sv.conn.items):
        if len(it["j"]):
            out[p][:, it["j"], it["i"]] = 0.0
    return out


def bc_T(sv, lams, gbc=None):
    """Transpose of the boundary overwrite (slip then Dirichlet); gbc accumulates the
    adjoint arriving at Dirichlet points (sensitivity to the imposed states)."""
    from .solver import _side_slice
    out = [l.copy() for l in lams]
    for k, (g, lam) in enumerate(zip(sv.geos, out)):
        side = g.desc.side
        for s in range(4):
            if side[s] != W.DIRICHLET:
                continue
            sl = _side_slice(s)
            keep = g.blank[sl]
            if gbc is not None:
                gbc[k][(slice(None),) + sl] += np.where(keep, 0.0, lam[(slice(None),) + sl])
            lam[(slice(None),) + sl] = np.where(keep, lam[(slice(None),) + sl], 0.0)
        for s in range(4):
            if side[s] != W.SLIPWALL:
                continue
            sl = _side_slice(s)
            if g.kind == W.AFFINE:
                comp = 1 if s < 2 else 2
                lam[comp][sl] = np.where(g.blank[sl], lam[comp][sl], 0.0)
            else:
                c, sn = g.cos[sl], g.sin[sl]
                mn = lam[1][sl] * c + lam[2][sl] * sn
                lam[1][sl] = lam[1][sl] - mn * c
                lam[2][sl] = lam[2][sl] - mn * sn
    return out


def wall_T(sv, lams, states):
    """Transpose of the linearised no-slip adiabatic wall condition at the state it was
    applied to (the wall density and the inward points are not changed by it):
    E_w = rho_w theta_w / (gamma - 1), theta_w = sum_j w_j theta(e_j), momenta set to 0."""
    from . import euler
    from .solver import _side_slice, _inward_slice, adiabatic_weights
    gam = sv.prm.gamma
    g1 = gam - 1.0
    out = [l.copy() for l in lams]
    for k, (g, lam) in enumerate(zip(sv.geos, out)):
        side = g.desc.side
        e = states[k]
        for s in range(4):
            if side[s] != W.ADIABATIC:
                continue
            sl = _side_slice(s)
            live = ~g.blank[sl]
            w = adiabatic_weights(sv.prm.d)
            lamE = np.where(live, lam[3][sl], 0.0)
            rho_w = e[0][sl]
            th_w = sum(wj * euler.temperature(e[(slice(None),) + _inward_slice(s, j + 1)], gam) for j, wj in enumerate(w))
            for c in (1, 2, 3):
                lam[c][sl] = np.where(live, 0.0, lam[c][sl])
            lam[0][sl] = lam[0][sl] + lamE * th_w / g1
            for j, wj in enumerate(w):
                isl = _inward_slice(s, j + 1)
                r, mx, my, E = (e[c][isl] for c in range(4))
                gcoef = lamE * rho_w / g1 * wj
                lam[0][isl] = lam[0][isl] + gcoef * g1 * (-E / r ** 2 + (mx * mx + my * my) / r ** 3)
                lam[1][isl] = lam[1][isl] + gcoef * (-g1 * mx / r ** 2)
                lam[2][isl] = lam[2][isl] + gcoef * (-g1 * my / r ** 2)
                lam[3][isl] = lam[3][isl] + gcoef * (g1 / r)
    return out


def project_T(sv, lams, gbc=None, states=None):
    """P = exchange o wall o bc  =>  P^T = bc^T o wall^T o exchange^T; the wall term needs
    the state at which P was applied (states, any time the walls are adiabatic)."""
    lam = exchange_T(sv, lams)
    if any(W.ADIABATIC in g.desc.side for g in sv.geos):
        lam = wall_T(sv, lam, states)
    return bc_T(sv, lam, gbc)


def filter_T(sv, lams, states):
    """Transpose of the linearised per-step filter (Sec. 4.3.1) at the state it was applied
    to: Q = (rho, rho u, rho v, theta(e)) is filtered along q1 lines, then q2 lines, and E
    is rebuilt from the filtered Q (eq. perfect_gas_T); blanked points are unchanged."""
    from . import euler
    prm = sv.prm
    gam, a, pf, d = prm.gamma, prm.alpha_f, prm.p_f, prm.d
    g1 = gam - 1.0
    out = []
    for g, lam, e in zip(sv.geos, lams, states):
        Fq = np.stack([e[0], e[1], e[2], euler.temperature(e, gam)])
        # forward values: G after q1, H after q2
        H = sv.filter_patch(g, e)
        r2, m2, n2 = H[0], H[1], H[2]
        th2 = euler.temperature(H, gam)
        # E' = r th/(g-1) + (m^2 + n^2)/(2 r): adjoint of the rebuild
        mu = np.stack([lam[0] + lam[3] * (th2 / g1 - 0.5 * (m2 * m2 + n2 * n2) / r2 ** 2),
                       lam[1] + lam[3] * m2 / r2,
                       lam[2] + lam[3] * n2 / r2,
                       lam[3] * r2 / g1])
        # q2 lines (transposed), then q1 lines
        muG = mu.copy()
        for (i, s, n, per) in g.seg2:
            if n >= 2 * d:
                muG[:, s:s + n, i] = fc_filter_T_lines(mu[:, s:s + n, i], d, fc.choose_C(n, prm.C0, prm.c_policy, d), a, pf)
        muQ = muG.copy()
        for (j, s, n, per) in g.seg1:
            if per:
                muQ[:, j, s:s + n] = fc.periodic_filter(muG[:, j, s:s + n], a, pf)
            elif n >= 2 * d:
                muQ[:, j, s:s + n] = fc_filter_T_lines(muG[:, j, s:s + n], d, fc.choose_C(n, prm.C0, prm.c_policy, d), a, pf)
        # Q_theta = theta(e): adjoint through theta = (g-1)(E/r - (m^2+n^2)/(2 r^2))
        r, m, n_, E = e
        lt = muQ[3]
        res = np.stack([muQ[0] + lt * g1 * (-E / r ** 2 + (m * m + n_ * n_) / r ** 3),
                        muQ[1] + lt * (-g1 * m / r ** 2),
                        muQ[2] + lt * (-g1 * n_ / r ** 2),
                        lt * g1 / r])
        out.append(np.where(g.blank[None], lam, res))
    return out


def fc_filter_T_lines(G, d, C, a, pf):
    return fc.fc_filter_T(G, d, C, a, pf)


def filter_jvp_complex(sv, u, v, h=1e-30):
    z = [x + 1j * h * y for x, y in zip(u, v)]
    return [np.imag(a) / h for a in sv.filter(z)]


def step_forward(sv, e_n, mu, dt, filt=False):
    """The differentiated step (mu, dt frozen; the per-step filter if filt); returns the
    stage states u_0..u_5 and, with the filter, the projected state it was applied to."""
    pre = sv.project([a.copy() for a in e_n])
    u = [sv.project(sv.filter(pre)) if filt else pre]
    Ls = {}
    for i in range(5):
        new = []
        for p in range(len(sv.geos)):
            acc = np.zeros_like(u[0][p])
            for k in range(i + 1):
                if SSP54_ALPHA[i][k] != 0.0:
                    acc = acc + SSP54_ALPHA[i][k] * u[k][p]
                if SSP54_BETA[i][k] != 0.0:
                    if k not in Ls:
                        Ls[k] = sv.rhs(u[k], mu)
                    acc = acc + SSP54_BETA[i][k] * dt * Ls[k][p]
            new.append(acc)
        u.append(sv.project(new))
    return (u, pre) if filt else u


def step_adjoint(sv, e_n, mu, dt, lam_np1, filt=False):
    """lam_n = (d e_{n+1}/d e_n)^T lam_{n+1} and the Dirichlet sensitivity of the step."""
    if filt:
        u, pre = step_forward(sv, e_n, mu, dt, filt=True)
    else:
        u = step_forward(sv, e_n, mu, dt)
    npch = len(sv.geos)
    gbc = [np.zeros_like(a) for a in e_n]
    lam_u = [[np.zeros_like(a) for a in e_n] for _ in range(6)]
    psi = [[np.zeros_like(a) for a in e_n] for _ in range(6)]  # sum_i beta_ik lam_v_i
    lam_u[5] = [l.copy() for l in lam_np1]
    for i in range(5, 0, -1):
        if any(np.any(x) for x in psi[i]):
            add = rhs_adjoint(sv, u[i], mu, psi[i])
            lam_u[i] = [a + dt * b for a, b in zip(lam_u[i], add)]
        lam_v = project_T(sv, lam_u[i], gbc, u[i])
        for k in range(i):
            al, be = SSP54_ALPHA[i - 1][k], SSP54_BETA[i - 1][k]
            for p in range(npch):
                if al != 0.0:
                    lam_u[k][p] = lam_u[k][p] + al * lam_v[p]
                if be != 0.0:
                    psi[k][p] = psi[k][p] + be * lam_v[p]
    add = rhs_adjoint(sv, u[0], mu, psi[0])
    lam_u[0] = [a + dt * b for a, b in zip(lam_u[0], add)]
    lam_n = project_T(sv, lam_u[0], gbc, u[0])
    if filt:
        lam_n = project_T(sv, filter_T(sv, lam_n, pre), gbc, pre)
    return lam_n, gbc


def step_jvp_complex(sv, e_n, mu, dt, v, h=1e-30, filt=False):
    """Directional derivative of the frozen step by the complex step: Im(step(e + i h v)) / h."""
    z = [a + 1j * h * b for a, b in zip(e_n, v)]
    out = (step_forward(sv, z, mu, dt, filt=True)[0] if filt else step_forward(sv, z, mu, dt))[5]
    return [np.imag(a) / h for a in out]


def rhs_jvp_complex(sv, u, mu, v, h=1e-30):
    z = [a + 1j * h * b for a, b in zip(u, v)]
    return [np.imag(a) / h for a in sv.rhs(z, mu)]


def project_jvp_complex(sv, u, v, h=1e-30):
    z = [a + 1j * h * b for a, b in zip(u, v)]
    return [np.imag(a) / h for a in sv.project(z)]


def wall_drag(sv, states):
    """J = sum over the wall ring of the first curvilinear patch of p n_x r0 dtheta
    (periodic trapezoid of the integral of wall pressure times n_x, outward body normal)."""
    from . import euler
    for g, e in zip(sv.geos, states):
        if g.kind == W.OGRID and g.desc.side[2] in (W.SLIPWALL, W.ADIABATIC):
            r0 = g.desc.geom[2]
            p = euler.primitives(e[:, 0, :], sv.prm.gamma)[3]
            return np.sum(p * g.cos[0]) * r0 * 2 * np.pi / g.n1
    raise ValueError("no wall")


def wall_drag_grad(sv, states):
    """dJ/de for wall_drag (same layout as states)."""
    from . import euler
    out = [np.zeros_like(e) for e in states]
    gam = sv.prm.gamma
    for k, (g, e) in enumerate(zip(sv.geos, states)):
        if g.kind == W.OGRID and g.desc.side[2] in (W.SLIPWALL, W.ADIABATIC):
            r0 = g.desc.geom[2]
            rho, m, n, E = e[:, 0, :]
            w = g.cos[0] * r0 * 2 * np.pi / g.n1
            g1 = gam - 1.0
            u, v = m / rho, n / rho
            out[k][0, 0, :] = w * g1 * 0.5 * (u * u + v * v)
            out[k][1, 0, :] = -w * g1 * u
            out[k][2, 0, :] = -w * g1 * v
            out[k][3, 0, :] = w * g1
            return out
    raise ValueError("no wall")


# ---- sensitivities to the problem parameters (build addition; Sec. 7, eq. mach_flow_ic) ------

def freestream_state(mach, alpha, rho, p, gamma):
    """Conserved free stream (rho, M a cos alpha, M a sin alpha, p) with a = sqrt(gamma p / rho)."""
    from . import euler
    a = np.sqrt(gamma * p / rho)
    return euler.cons_from_prim(rho, mach * a * np.cos(alpha), mach * a * np.sin(alpha), p, gamma)


def freestream_jacobian(fs, gamma, h=1e-30):
    """d e_fs / dM and d e_fs / dalpha at fixed density and pressure, by complex-step
    differentiation of freestream_state (fs = primitive (rho, u, v, p))."""
    rho, u, v, p = fs
    a = np.sqrt(gamma * p / rho)
    M, al = np.hypot(u, v) / a, np.arctan2(v, u)
    dM = np.imag(freestream_state(M + 1j * h, al, rho, p, gamma)) / h
    dA = np.imag(freestream_state(M, al + 1j * h, rho, p, gamma)) / h
    return np.real(dM), np.real(dA)


def dirichlet_param_sensitivity(sv, gbc, fs):
    """(dJ/dM, dJ/dalpha) carried by the Dirichlet adjoint gbc of free-stream sides: the sum
    over the Dirichlet points of sides whose state is fs of gbc . d e_fs / d(M, alpha)."""
    dM, dA = freestream_jacobian(fs, sv.prm.gamma)
    out = np.zeros(2)
    for g, lam in zip(sv.geos, gbc):
        mask = np.zeros((g.n2, g.n1), bool)
        for s in range(4):
            if g.desc.side[s] == W.DIRICHLET and tuple(g.desc.bc[s]) == tuple(fs):
                if s == 0:
                    mask[:, 0] = True
                elif s == 1:
                    mask[:, -1] = True
                elif s == 2:
                    mask[0, :] = True
                else:
                    mask[-1, :] = True
        mask &= ~g.blank
        out[0] += np.einsum("c,cji->", dM, np.where(mask, lam, 0.0))
        out[1] += np.einsum("c,cji->", dA, np.where(mask, lam, 0.0))
    return out


def initial_sensitivity(sv, states, lams, fs):
    """dJ/drho_0 at fixed velocity and pressure (complex step of the conserved state in rho)
    per patch, and the (dJ/dM, dJ/dalpha) part through a uniform free-stream e_0: the sum
    over non-blanked points of lam . d e_fs / d(M, alpha)."""
    from . import euler
    gam = sv.prm.gamma
    h = 1e-30
    drho = []
    for g, e, lam in zip(sv.geos, states, lams):
        rho, u, v, p = euler.primitives(e, gam)
        de = np.imag(euler.cons_from_prim(rho + 1j * h, u, v, p, gam)) / h
        drho.append(np.where(g.blank, 0.0, np.einsum("cji,cji->ji", lam, de)))
    dM, dA = freestream_jacobian(fs, gam)
    par = np.zeros(2)
    for g, lam in zip(sv.geos, lams):
        live = np.where(g.blank, 0.0, lam)
        par[0] += np.einsum("c,cji->", dM, live)
        par[1] += np.einsum("c,cji->", dA, live)
    return drho, par
