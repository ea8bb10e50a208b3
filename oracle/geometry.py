"""Patch geometry, fringes, donor search and Neville interpolation (oracle).

Test infrastructure only (see oracle/__init__.py).

Sec. 3.1-3.2: each patch is the image of Q = [0,1]^2 under a smooth map M_p;
its grid is the image of a Cartesian parameter grid (eq. param-grid). Three
kinds: affine boxes (C/I-type patches), an annulus around the cylinder whose
angular direction is periodic (a reading: the paper would use S-type patches,
eq. param_S), and GRID patches given by their points (S-type arcs and other
curvilinear patches), with metrics given or computed by FC derivatives of the
points and the inverse map by Newton's method on the local quadratic interpolant.
Sec. 3.3: Jacobian J = dq/dx of the inverse map, grad_x = J^T grad_q
(eq. general_curvilinear).
Sec. 3.4: n-point fringe regions from the maximum-index-norm distance to the
grid points on internal sides (eq. fringe_region, read with "< n"), donor
choice (the patch where the receiver is farthest from the boundary) and a 3x3
donor stencil with iterated 1-D quadratic interpolation in parameter space,
evaluated by Neville's algorithm (Sec. 3.4.1). Donor points must not be
receivers (Remark overlap_cond); the testing phase reports a violation.

Readings (paper silent): patches that cover the obstacle are blanked inside a
hole radius and their grid lines split into segments at blanked points; points
next to blanked points count as internal-boundary points; the index distance
is capped at `depth_cap`; the stencil is centred at rnd(s) (half up, as in
eq. zeta) and, if it would touch a donor receiver or blanked point, shifted by
the first valid offset in the order 0, -1, +1, -2, +2 (smallest |o1|+|o2|
first); donor ties go to the lowest patch index.
"""
import numpy as np

from paper_2506_16076_gb300 import workloads as W

CONTAIN_TOL = 1e-9
OFFSETS = (0, -1, 1, -2, 2)


def rnd(t):
    """Nearest integer with rnd(n + 1/2) = n + 1 (Sec. 5.2, after eq. zeta)."""
    return np.floor(np.asarray(t) + 0.5).astype(np.int64)


class PatchGeo:
    def __init__(self, desc: W.PatchDesc, params: W.Params):
        self.desc = desc
        self.kind = desc.kind
        self.n1, self.n2 = desc.n1, desc.n2
        self.periodic1 = desc.kind == W.OGRID or (
            desc.kind == W.GRID and desc.side[0] == W.PERIODIC and desc.side[1] == W.PERIODIC)
        # parameter spacings (eq. param-grid without the sub-patch vicinity; periodic: 1/n)
        self.h1 = 1.0 / self.n1 if self.periodic1 else 1.0 / (self.n1 - 1)
        self.h2 = 1.0 / (self.n2 - 1)
        self.params = params
        self.x, self.y = W.patch_xy(desc)
        self._metrics()
        self._spacings()
        self._blank()
        self._depth(params)
        self.receiver = (~self.blank) & (self.depth < params.n_f)
        self.gen = (~self.blank) & (self.depth >= params.n_v)
        self._segments(params)

    # Sec. 3.3: J = dq/dx
    def _metrics(self):
        if self.kind == W.GRID:
            if self.desc.metrics is not None:  # given with the grid (Sec. 3.3)
                self.J = np.array(self.desc.metrics, dtype=np.float64)
            else:
                self.J = self._grid_metrics()
            return
        if self.kind == W.AFFINE:
            x0, x1, y0, y1 = self.desc.geom
            z = np.zeros((self.n2, self.n1))
            self.J = np.stack([z + 1.0 / (x1 - x0), z, z, z + 1.0 / (y1 - y0)])  # J1x, J1y, J2x, J2y
        else:
            xc, yc, r0, r1 = self.desc.geom
            dx, dy = self.x - xc, self.y - yc
            r = np.hypot(dx, dy)
            c, s = dx / r, dy / r
            self.J = np.stack([-s / (2 * np.pi * r), c / (2 * np.pi * r), c / (r1 - r0), s / (r1 - r0)])
            self.cos, self.sin = c, s

    def _grid_metrics(self):
        """dq/dx of a GRID patch given without metrics (Sec. 3.3): the Jacobian
        d(x, y)/d(q1, q2) by FC derivatives of the coordinates along the full grid lines
        (Fourier along a periodic q1; the continuation length of each line by the run's C
        policy), inverted point by point."""
        from . import fc
        p = self.params
        d = p.d

        def dq1(F):
            if self.periodic1:
                return fc.periodic_derivative(F, self.h1)
            return fc.fc_derivative(F, self.h1, d, fc.choose_C(self.n1, p.C0, p.c_policy, d))

        def dq2(F):
            return fc.fc_derivative(F.T, self.h2, d, fc.choose_C(self.n2, p.C0, p.c_policy, d)).T

        xa, ya, xb, yb = dq1(self.x), dq1(self.y), dq2(self.x), dq2(self.y)
        det = xa * yb - xb * ya
        return np.stack([yb / det, -xb / det, -ya / det, xa / det])

    def _spacings(self):
        """h_hat (max) and h_tilde (min) distance between index-adjacent points (Sec. 5.1, eq. CFL)."""
        if self.kind == W.GRID:  # from the points (wrapped along a periodic q1)
            x, y = self.x, self.y
            if self.periodic1:
                d1 = np.hypot(np.roll(x, -1, axis=1) - x, np.roll(y, -1, axis=1) - y)
            else:
                d1 = np.hypot(x[:, 1:] - x[:, :-1], y[:, 1:] - y[:, :-1])
            d2 = np.hypot(x[1:] - x[:-1], y[1:] - y[:-1])
            self.hhat = float(max(d1.max(), d2.max()))
            self.htil = float(min(d1.min(), d2.min()))
        elif self.kind == W.AFFINE:
            x0, x1, y0, y1 = self.desc.geom
            hx, hy = (x1 - x0) / (self.n1 - 1), (y1 - y0) / (self.n2 - 1)
            self.hhat, self.htil = max(hx, hy), min(hx, hy)
        else:
            xc, yc, r0, r1 = self.desc.geom
            dr = (r1 - r0) / (self.n2 - 1)
            ch = 2.0 * np.sin(np.pi / self.n1)
            self.hhat, self.htil = max(dr, r1 * ch), min(dr, r0 * ch)

    def _blank(self):
        hx, hy, R = self.desc.hole
        if R > 0 and self.kind != W.OGRID:
            dx, dy = self.x - hx, self.y - hy
            self.blank = (dx * dx + dy * dy) < R * R
        else:
            self.blank = np.zeros((self.n2, self.n1), bool)

    def _dilate(self, m):
        out = m.copy()
        if self.periodic1:
            for s in (-1, 1):
                out |= np.roll(m, s, axis=1)
        else:
            out[:, 1:] |= m[:, :-1]
            out[:, :-1] |= m[:, 1:]
        o2 = out.copy()
        o2[1:, :] |= out[:-1, :]
        o2[:-1, :] |= out[1:, :]
        return o2

    def _depth(self, params):
        """Capped max-index-norm distance to internal-boundary points (eq. fringe_region)."""
        side = self.desc.side
        I = np.zeros((self.n2, self.n1), bool)
        if side[0] == W.INTERNAL:
            I[:, 0] = True
        if side[1] == W.INTERNAL:
            I[:, -1] = True
        if side[2] == W.INTERNAL:
            I[0, :] = True
        if side[3] == W.INTERNAL:
            I[-1, :] = True
        I |= self._dilate(self.blank) & ~self.blank
        I &= ~self.blank
        cap = params.depth_cap
        depth = np.full((self.n2, self.n1), cap, np.int64)
        reached = I.copy()
        depth[I] = 0
        for k in range(1, cap):
            nxt = self._dilate(reached)
            new = nxt & ~reached
            depth[new] = k
            reached = nxt
            if reached.all():
                break
        depth[self.blank] = 0
        self.depth = depth

    def _segments(self, params):
        """Maximal runs of non-blanked points along each grid line (q1 rows, q2 columns)."""
        self.seg1, self.seg2 = [], []  # (line index, start, length, periodic)
        for j in range(self.n2):
            if self.periodic1:
                self.seg1.append((j, 0, self.n1, True))
            else:
                self.seg1 += [(j, a, n, False) for a, n in _runs(~self.blank[j, :])]
        for i in range(self.n1):
            self.seg2 += [(i, a, n, False) for a, n in _runs(~self.blank[:, i])]
        d = params.d
        self.nodiff = self.blank.copy()  # points where a derivative is not defined (set to 0)
        for (j, a, n, per) in self.seg1:
            if not per and n < 2 * d:
                self.nodiff[j, a:a + n] = True
        for (i, a, n, per) in self.seg2:
            if n < 2 * d:
                self.nodiff[a:a + n, i] = True

    # inverse map: physical point -> fractional grid indices (s1, s2)
    def frac_index(self, x, y):
        if self.kind == W.GRID:
            return self._grid_inverse(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
        if self.kind == W.AFFINE:
            x0, x1, y0, y1 = self.desc.geom
            return (x - x0) / (x1 - x0) * (self.n1 - 1), (y - y0) / (y1 - y0) * (self.n2 - 1)
        xc, yc, r0, r1 = self.desc.geom
        th = np.mod(np.arctan2(y - yc, x - xc), 2 * np.pi)
        r = np.hypot(x - xc, y - yc)
        return th / (2 * np.pi) * self.n1, (r - r0) / (r1 - r0) * (self.n2 - 1)

    def _grid_inverse(self, x, y):
        """GRID patches: Newton's method on the 3 x 3 quadratic (Lagrange) interpolant of
        the grid around a stencil centre c, started at the nearest grid point (ties:
        smallest flat index), which is also the first centre (clamped to [1, n - 2] along
        a non-periodic direction). A direction's centre moves to rnd(s) (clamped) only when
        the estimate is more than 0.75 from it, so that Newton cannot cycle between two
        neighbouring stencils across a half-integer. At most 30 steps, stopping after a
        step with |ds1| + |ds2| < 1e-11 (Newton's quadratic convergence leaves an error
        at rounding level). Queries more than the largest spacing outside the bounding
        box, and failed iterations, get indices far outside the grid."""
        shape = np.shape(x)
        xq, yq = np.ravel(x), np.ravel(y)
        n1, n2 = self.n1, self.n2
        X, Y = self.x.ravel(), self.y.ravel()
        h = self.hhat
        s1 = np.full(xq.shape, -1e9)
        s2 = np.full(xq.shape, -1e9)
        x0, x1, y0, y1 = X.min(), X.max(), Y.min(), Y.max()
        near = (xq >= x0 - h) & (xq <= x1 + h) & (yq >= y0 - h) & (yq <= y1 + h)
        idx = np.nonzero(near)[0]
        if idx.size == 0:
            return s1.reshape(shape), s2.reshape(shape)
        k0 = np.array([int(np.argmin((X - xq[q]) ** 2 + (Y - yq[q]) ** 2)) for q in idx])
        a1 = (k0 % n1).astype(np.float64)
        a2 = (k0 // n1).astype(np.float64)
        active = np.ones(idx.size, bool)
        done = np.zeros(idx.size, bool)
        xs, ys = xq[idx], yq[idx]

        def centre1(a):
            c = rnd(a)
            return c if self.periodic1 else np.clip(c, 1, n1 - 2)

        c1 = centre1(a1)
        c2 = np.clip(rnd(a2), 1, n2 - 2)
        for _ in range(30):
            if not active.any():
                break
            c1 = np.where(np.abs(a1 - c1) > 0.75, centre1(a1), c1)
            c2 = np.where(np.abs(a2 - c2) > 0.75, np.clip(rnd(a2), 1, n2 - 2), c2)
            t1, t2 = a1 - c1, a2 - c2
            L = [0.5 * t1 * (t1 - 1.0), 1.0 - t1 * t1, 0.5 * t1 * (t1 + 1.0)]
            dL = [t1 - 0.5, -2.0 * t1, t1 + 0.5]
            M = [0.5 * t2 * (t2 - 1.0), 1.0 - t2 * t2, 0.5 * t2 * (t2 + 1.0)]
            dM = [t2 - 0.5, -2.0 * t2, t2 + 0.5]
            Xv = np.zeros_like(a1); Yv = np.zeros_like(a1)
            Xa = np.zeros_like(a1); Xb = np.zeros_like(a1); Ya = np.zeros_like(a1); Yb = np.zeros_like(a1)
            for b in range(3):
                jj = c2 + b - 1
                for a in range(3):
                    ii = c1 + a - 1
                    if self.periodic1:
                        ii = np.mod(ii, n1)
                    k = jj * n1 + ii
                    w, wa, wb = L[a] * M[b], dL[a] * M[b], L[a] * dM[b]
                    Xv = Xv + w * X[k]; Yv = Yv + w * Y[k]
                    Xa = Xa + wa * X[k]; Xb = Xb + wb * X[k]
                    Ya = Ya + wa * Y[k]; Yb = Yb + wb * Y[k]
            rx, ry = Xv - xs, Yv - ys
            det = Xa * Yb - Xb * Ya
            ok = active & (np.abs(det) > 0.0)
            active &= ok
            safe = np.where(ok, det, 1.0)
            d1 = -(Yb * rx - Xb * ry) / safe
            d2 = -(-Ya * rx + Xa * ry) / safe
            a1 = np.where(active, a1 + d1, a1)
            a2 = np.where(active, a2 + d2, a2)
            active &= (np.abs(a1) < 1e12) & (np.abs(a2) < 1e12)
            conv = active & (np.abs(d1) + np.abs(d2) < 1e-11)
            done |= conv
            active &= ~conv
        res1 = np.where(done, np.mod(a1, n1) if self.periodic1 else a1, -1e9)
        res2 = np.where(done, a2, -1e9)
        s1[idx], s2[idx] = res1, res2
        return s1.reshape(shape), s2.reshape(shape)

    def contains(self, s1, s2):
        ok2 = (s2 >= -CONTAIN_TOL) & (s2 <= self.n2 - 1 + CONTAIN_TOL)
        if self.periodic1:
            ok1 = np.ones_like(ok2)
        else:
            ok1 = (s1 >= -CONTAIN_TOL) & (s1 <= self.n1 - 1 + CONTAIN_TOL)
        ok = ok1 & ok2
        z1, z2 = self.nearest(s1, s2)
        ok &= ~self.blank[z2, z1]
        return ok

    def nearest(self, s1, s2):
        """zeta of eq. zeta as integer indices (clamped / wrapped into the grid)."""
        z1, z2 = rnd(s1), rnd(s2)
        z1 = np.mod(z1, self.n1) if self.periodic1 else np.clip(z1, 0, self.n1 - 1)
        return z1, np.clip(z2, 0, self.n2 - 1)

    def bbox(self):
        return self.x.min(), self.x.max(), self.y.min(), self.y.max()


def _runs(mask):
    out, a = [], None
    for i, m in enumerate(mask):
        if m and a is None:
            a = i
        if not m and a is not None:
            out.append((a, i - a))
            a = None
    if a is not None:
        out.append((a, len(mask) - a))
    return out


def stencil_search(g: PatchGeo, s1, s2):
    """Stencil start (a1, a2) and validity for fractional indices s1, s2 (arrays)."""
    c1, c2 = rnd(s1), rnd(s2)
    bad = g.blank | g.receiver
    cands = sorted(((o1, o2) for o1 in OFFSETS for o2 in OFFSETS),
                   key=lambda o: (abs(o[0]) + abs(o[1]), OFFSETS.index(o[0]), OFFSETS.index(o[1])))
    a1 = np.zeros_like(c1)
    a2 = np.zeros_like(c2)
    found = np.zeros(c1.shape, bool)
    for o1, o2 in cands:
        b1, b2 = c1 - 1 + o1, c2 - 1 + o2
        ok = ~found & (b2 >= 0) & (b2 <= g.n2 - 3)
        if not g.periodic1:
            ok &= (b1 >= 0) & (b1 <= g.n1 - 3)
        for m2 in range(3):
            for m1 in range(3):
                i1 = np.mod(b1 + m1, g.n1) if g.periodic1 else np.clip(b1 + m1, 0, g.n1 - 1)
                i2 = np.clip(b2 + m2, 0, g.n2 - 1)
                ok &= ~bad[i2, i1]
        a1 = np.where(ok, b1, a1)
        a2 = np.where(ok, b2, a2)
        found |= ok
    return a1, a2, found


def neville(nodes, vals, t):
    """Neville's algorithm: value at t of the polynomial through (nodes[i], vals[i]).

    vals: list of arrays (one per node); t: array. (Sec. 3.4.1.)"""
    P = [v.copy() for v in vals]
    n = len(nodes)
    for m in range(1, n):
        for i in range(n - m):
            xi, xj = nodes[i], nodes[i + m]
            P[i] = ((t - xj) * P[i] - (t - xi) * P[i + 1]) / (xi - xj)
    return P[0]


SNAP = 1e-9  # index units: fractional stencil offsets this close to an integer are that integer


class Connectivity:
    """Receivers of every patch with their donors and stencils (Sec. 3.4.1)."""

    def __init__(self, geos, params):
        self.geos = geos
        self.items = []  # per patch: dict(recv flat idx, donor, a1, a2, t1, t2)
        self.errors = []
        boxes = [g.bbox() for g in geos]
        for p, g in enumerate(geos):
            rj, ri = np.nonzero(g.receiver)
            n = len(rj)
            xr, yr = g.x[rj, ri], g.y[rj, ri]
            best_depth = np.full(n, -1, np.int64)
            donor = np.full(n, -1, np.int64)
            A1 = np.zeros(n, np.int64)
            A2 = np.zeros(n, np.int64)
            T1 = np.zeros(n)
            T2 = np.zeros(n)
            for q, h in enumerate(geos):
                if q == p or n == 0 or not _overlap(boxes[p], boxes[q]):
                    continue
                s1, s2 = h.frac_index(xr, yr)
                ok = h.contains(s1, s2)
                a1, a2, found = stencil_search(h, s1, s2)
                ok &= found
                z1, z2 = h.nearest(s1, s2)
                dep = h.depth[z2, z1]
                better = ok & (dep > best_depth)  # strict: ties keep the lower patch index
                best_depth = np.where(better, dep, best_depth)
                donor = np.where(better, q, donor)
                A1 = np.where(better, a1, A1)
                A2 = np.where(better, a2, A2)
                t1 = s1 - a1
                if h.periodic1:
                    t1 = np.mod(s1 - a1 + 0.5 * h.n1, h.n1) - 0.5 * h.n1  # unwrap across theta = 0
                T1 = np.where(better, t1, T1)
                T2 = np.where(better, s2 - a2, T2)
            if n and (donor < 0).any():
                self.errors.append((p, int((donor < 0).sum())))
            # a receiver that coincides with a donor grid point (sub-patches of one patch
            # share their overlap points, Sec. 3.4.2) takes that point's value: its offsets
            # within the stencil are snapped to the integer they equal up to rounding, where
            # the quadratic interpolation reduces to the node value
            T1 = np.where(np.abs(T1 - np.round(T1)) < SNAP, np.round(T1), T1)
            T2 = np.where(np.abs(T2 - np.round(T2)) < SNAP, np.round(T2), T2)
            self.items.append(dict(j=rj, i=ri, donor=donor, a1=A1, a2=A2, t1=T1, t2=T2))

    def exchange(self, states):
        """Overwrite every receiver with its interpolated donor value (Sec. 3.4.1), in place."""
        nodes = (0.0, 1.0, 2.0)
        new = []
        for p, it in enumerate(self.items):
            vals = np.zeros((states[p].shape[0], len(it["j"])), dtype=states[p].dtype)
            for q in np.unique(it["donor"]):
                if q < 0:
                    continue
                sel = it["donor"] == q
                h, e = self.geos[q], states[q]
                a1, a2, t1, t2 = it["a1"][sel], it["a2"][sel], it["t1"][sel], it["t2"][sel]
                rows = []
                for m2 in range(3):
                    i2 = a2 + m2
                    pts = []
                    for m1 in range(3):
                        i1 = np.mod(a1 + m1, h.n1) if h.periodic1 else a1 + m1
                        pts.append(e[:, i2, i1])
                    rows.append(neville(nodes, pts, t1))  # along q1 for each of 3 rows
                vals[:, sel] = neville(nodes, rows, t2)  # then along q2
            new.append(vals)
        for p, it in enumerate(self.items):
            if len(it["j"]):
                states[p][:, it["j"], it["i"]] = new[p]
        return states


def _overlap(a, b):
    return not (a[1] < b[0] or b[1] < a[0] or a[3] < b[2] or b[3] < a[2])


def build(w: W.Workload):
    geos = [PatchGeo(p, w.params) for p in w.patches]
    conn = Connectivity(geos, w.params)
    return geos, conn
