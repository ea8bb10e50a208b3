"""Semi-discrete operator, boundary conditions, filter, time step (oracle).

Test infrastructure only (see oracle/__init__.py).

Sec. 4.1 eq. (semi-discrete): de_h/dt = L[e_h], with L assembled from 1-D FC
derivatives in q1 and q2 in the curvilinear form eq. (general_curvilinear):
    L = -sum_k sum_i J_ki d/dq^k ( f_i(e) - mu sum_m J_mi d/dq^m e ),
i.e. the viscous flux f_visc = mu grad_x e (eq. f_visc, convection diffusion).
Time stepping: SSPRK-4 (5 stages, Sec. 4.1; coefficients of the published
SSPRK(5,4) scheme the paper cites, gottlieb2005high), adaptive dt of eq. (CFL),
Dirichlet / slip-wall overwrite at every stage (Sec. 4.2), inter-patch
exchange at every stage (Sec. 4.2, Alg. 1 line sol_comm), per-step spectral
filter of rho, rho u, rho v, theta with E rebuilt (Sec. 4.3.1), and the
Algorithm 1 order per step: viscosity, filter, dt, 5 stages.

On patches with a no-slip adiabatic side, Params.wall_form = 1 selects the form of
Remark adiabatic: theta in place of E among the FC-differentiated quantities, the
derivatives of E and p by the sum and product rules, the convective divergence from them
(Solver.rhs_patch_product).

Readings (see the design notes): derivatives are 0 on blanked points and on
segments too short for FC (fewer than 2d points), where L is set to 0; the
filter acts on steps n >= 1 ("every time step following the initial time")
and is followed by the boundary overwrite and the exchange; every step starts
by applying the boundary overwrite and the exchange to its input (idempotent
on a consistent state); slip walls zero the wall-normal momentum.
"""
import functools

import numpy as np

from paper_2506_16076_gb300 import workloads as W
from . import euler, fc, geometry, viscosity

# SSPRK(5,4) in Shu-Osher form (Spiteri & Ruuth 2002; Gottlieb, Ketcheson & Shu):
#   u^(i) = sum_k alpha_ik u^(k) + beta_ik dt L(u^(k))
SSP54_ALPHA = [
    [1.0],
    [0.444370493651235, 0.555629506348765],
    [0.620101851488403, 0.0, 0.379898148511597],
    [0.178079954393132, 0.0, 0.0, 0.821920045606868],
    [0.0, 0.0, 0.517231671970585, 0.096059710526147, 0.386708617503269],
]
SSP54_BETA = [
    [0.391752226571890],
    [0.0, 0.368410593050371],
    [0.0, 0.0, 0.251891774271694],
    [0.0, 0.0, 0.0, 0.544974750228521],
    [0.0, 0.0, 0.0, 0.063692468666290, 0.226007483236906],
]


def butcher_from_shu_osher(alpha=SSP54_ALPHA, beta=SSP54_BETA):
    """Butcher (A, b, c) of the Shu-Osher scheme (for the order-condition pins)."""
    s = len(alpha)
    # stage i+1 value = u0 + dt sum_j A'[i+1][j] L(u^(j)); A'[0] = 0
    A = np.zeros((s + 1, s))
    for i in range(s):
        row = np.zeros(s)
        for k in range(i + 1):
            row += alpha[i][k] * A[k]
            row[k] += beta[i][k]
        A[i + 1] = row
    return A[:s], A[s], A[:s].sum(axis=1)


class Solver:
    def __init__(self, w: W.Workload, filter_from_step=1):
        self.w = w
        self.prm = w.params
        self.geos, self.conn = geometry.build(w)
        self.sb = viscosity.SBOperator(self.geos, self.prm)
        self.filter_from_step = filter_from_step
        self.last_dt = None

    # ---- 1-D derivatives along segments (Sec. 2.2, Sec. 4.1) -------------------------
    def d1(self, g, F):
        """d/dq1 of F (..., n2, n1) on every q1 segment; 0 where undefined."""
        out = np.zeros_like(F)
        d, C0, pol = self.prm.d, self.prm.C0, self.prm.c_policy
        groups = {}
        for (j, a, n, per) in g.seg1:
            groups.setdefault((a, n, per), []).append(j)
        for (a, n, per), rows in groups.items():
            rows = np.array(rows)
            lines = F[..., rows, a:a + n]
            if per:
                out[..., rows, a:a + n] = fc.periodic_derivative(lines, g.h1)
            elif n >= 2 * d:
                out[..., rows, a:a + n] = fc.fc_derivative(lines, g.h1, d, fc.choose_C(n, C0, pol, d))
        return out

    def d2(self, g, F):
        Ft = np.swapaxes(F, -1, -2)
        out = np.zeros_like(Ft)
        d, C0, pol = self.prm.d, self.prm.C0, self.prm.c_policy
        groups = {}
        for (i, a, n, per) in g.seg2:
            groups.setdefault((a, n), []).append(i)
        for (a, n), cols in groups.items():
            cols = np.array(cols)
            if n >= 2 * d:
                out[..., cols, a:a + n] = fc.fc_derivative(Ft[..., cols, a:a + n], g.h2, d, fc.choose_C(n, C0, pol, d))
        return np.swapaxes(out, -1, -2)

    # ---- eq. (semi-discrete) ------------------------------------------------------------
    def rhs_patch(self, g, e, mu):
        if self.product_form(g):
            return self.rhs_patch_product(g, e, mu)
        gam = self.prm.gamma
        J1x, J1y, J2x, J2y = g.J
        D1, D2 = self.d1(g, e), self.d2(g, e)
        dx = J1x * D1 + J2x * D2
        dy = J1y * D1 + J2y * D2
        Hx = euler.flux_x(e, gam) - mu * dx
        Hy = euler.flux_y(e, gam) - mu * dy
        L = -(J1x * self.d1(g, Hx) + J1y * self.d1(g, Hy) + J2x * self.d2(g, Hx) + J2y * self.d2(g, Hy))
        return np.where(g.nodiff[None], 0.0, L)

    def product_form(self, g):
        return getattr(self.prm, "wall_form", 0) == 1 and W.ADIABATIC in tuple(g.desc.side)

    def rhs_patch_product(self, g, e, mu):
        """L on a patch with a no-slip adiabatic wall in the form of Remark adiabatic: the
        temperature theta = p/rho replaces E among the FC-differentiated quantities (its
        continuation along the wall-normal lines is the Neumann expansion, since the wall
        overwrite puts the Neumann end data's value at the wall); the x and y derivatives
        of E and p follow from those of rho, rho u, rho v and theta by the sum and product
        rules, the convective flux divergence from the same rules, and the viscous fluxes
        mu grad e, with grad E from the product rule, are FC-differentiated as elsewhere:
            L = -( div f(e) - sum_k sum_i J_ki d/dq^k (mu sum_m J_mi d/dq^m e) )."""
        gam = self.prm.gamma
        J1x, J1y, J2x, J2y = g.J
        Q = wall_quantities(e, gam)
        D1, D2 = self.d1(g, Q), self.d2(g, Q)
        conv, Hx, Hy = wall_pointwise(e, J1x * D1 + J2x * D2, J1y * D1 + J2y * D2, mu, gam)
        L = -(conv + J1x * self.d1(g, Hx) + J1y * self.d1(g, Hy) + J2x * self.d2(g, Hx) + J2y * self.d2(g, Hy))
        return np.where(g.nodiff[None], 0.0, L)

    def rhs(self, states, mus):
        return [self.rhs_patch(g, e, m) for g, e, m in zip(self.geos, states, mus)]

    # ---- Sec. 4.2: boundary overwrite ----------------------------------------------------
    def apply_bc(self, states):
        gam = self.prm.gamma
        for g, e in zip(self.geos, states):
            side = g.desc.side
            for s in range(4):
                if side[s] != W.SLIPWALL:
                    continue
                sl = _side_slice(s)
                if g.kind == W.AFFINE:
                    comp = 1 if s < 2 else 2
                    e[comp][sl] = np.where(g.blank[sl], e[comp][sl], 0.0)
                else:
                    c, sn = g.cos[sl], g.sin[sl]
                    mn = e[1][sl] * c + e[2][sl] * sn
                    e[1][sl] = e[1][sl] - mn * c
                    e[2][sl] = e[2][sl] - mn * sn
            for s in range(4):
                if side[s] != W.DIRICHLET:
                    continue
                sl = _side_slice(s)
                val = euler.cons_from_prim(*[np.float64(v) for v in g.desc.bc[s]], gam)
                for k in range(4):
                    e[k][sl] = np.where(g.blank[sl], e[k][sl], val[k])
            for s in range(4):
                if side[s] != W.ADIABATIC:
                    continue
                # no-slip adiabatic wall (Sec. 4.2, Remarks adiabatic_th and adiabatic)
                sl = _side_slice(s)
                th_w = sum(wj * euler.temperature(e[(slice(None),) + _inward_slice(s, j + 1)], gam)
                           for j, wj in enumerate(adiabatic_weights(self.prm.d)))
                keep = g.blank[sl]
                e[1][sl] = np.where(keep, e[1][sl], 0.0)
                e[2][sl] = np.where(keep, e[2][sl], 0.0)
                e[3][sl] = np.where(keep, e[3][sl], e[0][sl] * th_w / (gam - 1.0))
        return states

    def project(self, states):
        """Boundary overwrite then inter-patch exchange (Sec. 4.2, Alg. 1 line sol_comm)."""
        self.apply_bc(states)
        self.conn.exchange(states)
        return states

    # ---- Sec. 4.3.1: per-step filter ---------------------------------------------------------
    def filter_patch(self, g, e):
        gam, a, p = self.prm.gamma, self.prm.alpha_f, self.prm.p_f
        d, C0, pol = self.prm.d, self.prm.C0, self.prm.c_policy
        F = np.stack([e[0], e[1], e[2], euler.temperature(e, gam)])
        G = F.copy()
        for (j, s, n, per) in g.seg1:
            if per:
                G[:, j, s:s + n] = fc.periodic_filter(F[:, j, s:s + n], a, p)
            elif n >= 2 * d:
                G[:, j, s:s + n] = fc.fc_filter(F[:, j, s:s + n], d, fc.choose_C(n, C0, pol, d), a, p)
        H = G.copy()
        for (i, s, n, per) in g.seg2:
            if n >= 2 * d:
                H[:, s:s + n, i] = fc.fc_filter(G[:, s:s + n, i], d, fc.choose_C(n, C0, pol, d), a, p)
        out = np.stack([H[0], H[1], H[2], euler.energy_from_theta(H[0], H[1], H[2], H[3], gam)])
        return np.where(g.blank[None], e, out)

    def filter(self, states):
        return [self.filter_patch(g, e) for g, e in zip(self.geos, states)]

    # ---- eq. (CFL) -------------------------------------------------------------------------
    def dt(self, states, mus):
        best = np.inf
        for g, e, m in zip(self.geos, states, mus):
            v = ~g.blank
            if not v.any():
                continue
            S = euler.mwsb(e, self.prm.gamma)[v].max()
            M = m[v].max()
            best = min(best, self.prm.cfl / (S / g.htil + M / g.htil ** 2))
        return best / np.pi

    # ---- Algorithm 1, one time step ------------------------------------------------------------
    def step(self, states, n_step, mu=None, dt=None, filt=True):
        states = [e.copy() for e in states]
        self.project(states)
        if mu is None:
            mu = viscosity.viscosity(self.geos, self.sb, states, self.prm)[0]
        if filt and n_step >= self.filter_from_step:
            states = self.filter(states)
            self.project(states)
        if dt is None:
            dt = self.dt(states, mu)
        self.last_dt = dt
        self.last_mu = mu
        u = [states]
        Ls = []
        for i in range(5):
            Ls.append(self.rhs(u[i], mu))
            new = []
            for p in range(len(self.geos)):
                acc = np.zeros_like(states[p])
                for k in range(i + 1):
                    if SSP54_ALPHA[i][k] != 0.0:
                        acc = acc + SSP54_ALPHA[i][k] * u[k][p]
                    if SSP54_BETA[i][k] != 0.0:
                        acc = acc + SSP54_BETA[i][k] * dt * Ls[k][p]
                new.append(acc)
            self.project(new)
            u.append(new)
        return u[5]

    def run(self, states, nsteps, start=0, **kw):
        dts = []
        for n in range(start, start + nsteps):
            states = self.step(states, n, **kw)
            dts.append(self.last_dt)
        return states, dts


def wall_quantities(e, gam):
    """Q = (rho, rho u, rho v, theta): the FC-differentiated quantities of the product-rule
    form (Remark adiabatic), theta = p / rho (eq. p_T)."""
    return np.stack([e[0], e[1], e[2], euler.temperature(e, gam)])


def wall_pointwise(e, Qx, Qy, mu, gam):
    """The pointwise part of the product-rule form (Remark adiabatic) from the state e and
    the x and y derivatives Qx, Qy of Q = (rho, rho u, rho v, theta): the convective
    divergence div f(e) and the viscous fluxes H_x = -mu d/dx e, H_y = -mu d/dy e, the
    derivatives of E and p by the sum and product rules."""
    Q = wall_quantities(e, gam)
    ex, px = euler.product_rule_derivatives(Q, Qx, gam)
    ey, py = euler.product_rule_derivatives(Q, Qy, gam)
    return euler.flux_divergence_product(e, Q[3], ex, px, ey, py), -mu * ex, -mu * ey


def _side_slice(s):
    return [(slice(None), 0), (slice(None), -1), (0, slice(None)), (-1, slice(None))][s]


def _inward_slice(s, j):
    """Grid points j steps inward from side s (along the wall-normal grid lines)."""
    return [(slice(None), j), (slice(None), -1 - j), (j, slice(None)), (-1 - j, slice(None))][s]


@functools.lru_cache(maxsize=None)
def adiabatic_weights(d):
    """Weights w_1..w_{d-1} with sum_j w_j theta_j = p(0) for the polynomial p of degree
    d-1 with p'(0) = 0 and p(j) = theta_j, j = 1..d-1 (unit spacing): the wall value of
    the Neumann FC end data (Sec. 2.2, Remark adiabatic). Exact rational elimination."""
    from fractions import Fraction
    m = d - 1
    powers = [0] + list(range(2, d))  # p'(0) = 0 removes the linear term
    A = [[Fraction(j) ** k for k in powers] + [Fraction(int(r == j)) for r in range(1, d)] for j in range(1, d)]
    for col in range(m):  # Gauss-Jordan on [A | I]
        piv = next(r for r in range(col, m) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        pv = A[col][col]
        A[col] = [x / pv for x in A[col]]
        for r in range(m):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [x - f * y for x, y in zip(A[r], A[col])]
    return tuple(float(x) for x in A[0][m:])  # row of a_0 in the inverse


# ---- Sec. 4.3.2: localised smearing of discontinuous initial data ----------------------------
def smear_initial(solver, states, x_disc, direction=1):
    """Blend a strong filter (alpha_f=10, p_f=2) into a window w_{18,9} around x = x_disc
    along q1 lines of affine patches (eq. q, eq. qf); E is rebuilt from theta."""
    prm = solver.prm
    gam = prm.gamma
    out = []
    for g, e in zip(solver.geos, states):
        if g.kind != W.AFFINE:
            out.append(e)
            continue
        x0, x1, _, _ = g.desc.geom
        h = (x1 - x0) / (g.n1 - 1)
        if not (x0 < x_disc < x1):
            out.append(e)
            continue
        F = np.stack([e[0], e[1], e[2], euler.temperature(e, gam)])
        C = fc.choose_C(g.n1, prm.C0, prm.c_policy, prm.d)
        Ff = fc.fc_filter(F, prm.d, C, 10.0, 2)
        w = viscosity.window_weight((g.x - x_disc) / h, 18, 9)
        G = w[None] * Ff + (1.0 - w[None]) * F
        out.append(np.stack([G[0], G[1], G[2], euler.energy_from_theta(G[0], G[1], G[2], G[3], gam)]))
    return out
