"""Multi-patch artificial viscosity (oracle). Test infrastructure only.

Sec. 5.1: smoothness classification tau~ of the proxy Phi (local Mach number)
on the viscosity-generation subgrid G~ = G minus the n_v-fringe
(eq. viscosity_generation); preliminary viscosity
    mu^_ij = R(tau~_ij) * max_{7x7 stencil} S * h^      (eq. V2D_unscaled)
with R = (1.5, 1, 0.5, 0), S = |u|+|v|+a, h^ the largest grid spacing.
Sec. 5.2: smoothing-blending operator
    Lambda[b](x) = sum_{p,(i,j) in G~_p} W~_{p,ij}(x) b_{p,ij}     (eq. Lambda)
with windows W_{p,ij} = w_{0,9}(q1 - q1_i) w_{0,9}(q2 - q2_j) evaluated at the
nearest grid point zeta_p(x) of each patch containing x (eq. W, multipatch_W,
zeta), normalised over all generating points of all patches
(eq. multipatch_W_norm); mu = Lambda[mu^] (eq. viscosity).

Readings: window eq. (qf) read as cos^2(pi (|x|/h - c/2) / (2 r)) so it falls
smoothly to 0 at |x| = (c/2 + r) h (17 taps for c=0, r=9); the classifier is a
stand-in (7-point windows of Phi along each direction, min-max normalised,
ReLU MLP 7-16-16-4 in FP32, class = argmax + 1, tau~ = min over the two
directions; a window with range below 1e-6 max(1, max|Phi|) is class 4;
windows are shifted inside a segment at its ends; segments shorter than 7
points give class 4); points with zero normaliser get mu = 0.
Parity unpinned: the stand-in is not the paper's detector.
"""
import functools
import os

import numpy as np

from paper_2506_16076_gb300 import workloads as W
from . import euler
from .geometry import _overlap

_DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_2506_16076_gb300", "data")
SMOOTH_TOL = 1e-6


@functools.lru_cache(maxsize=None)
def load_sdnn():
    with open(os.path.join(_DATA, "sdnn_standin.txt")) as f:
        lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    out, i = {}, 0
    while i < len(lines):
        name, r, c = lines[i][0], int(lines[i][1]), int(lines[i][2])
        out[name] = np.array([[float(v) for v in lines[i + 1 + k]] for k in range(r)], dtype=np.float32)
        i += 1 + r
    return out


def window_weight(k, c, r):
    """w_{c,r} at offset k grid cells (eq. qf, read smoothly; see module doc)."""
    a = np.abs(np.asarray(k, dtype=float))
    w = np.where(a < c / 2.0, 1.0, np.cos(np.pi * (a - c / 2.0) / (2.0 * r)) ** 2)
    return np.where(a >= c / 2.0 + r, 0.0, w)


def mlp_logits(x64):
    """Stand-in network on normalised windows (n, 7): FP32 ReLU MLP 7-16-16-4."""
    P = load_sdnn()
    x = x64.astype(np.float32)
    h = np.maximum(x @ P["W1"].T + P["b1"][:, 0], np.float32(0))
    h = np.maximum(h @ P["W2"].T + P["b2"][:, 0], np.float32(0))
    return h @ P["W3"].T + P["b3"][:, 0]


def classify(win):
    """Class in {1,2,3,4} for each 7-point window (n, 7) of Phi, plus the logit margin."""
    lo = win.min(axis=1)
    hi = win.max(axis=1)
    rg = hi - lo
    flat = rg < SMOOTH_TOL * np.maximum(1.0, np.abs(win).max(axis=1))
    x = (win - lo[:, None]) / np.where(flat, 1.0, rg)[:, None]
    o = mlp_logits(x).astype(np.float64)
    cls = o.argmax(axis=1) + 1
    srt = np.sort(o, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    cls = np.where(flat, 4, cls)
    margin = np.where(flat, np.inf, margin)
    return cls, margin, o


def window_starts(g, direction):
    """Start index (along the line) of the 7-point window of every point; -1: no window."""
    st = np.full((g.n2, g.n1), -1, np.int64)
    segs = g.seg1 if direction == 1 else g.seg2
    for (line, a, n, per) in segs:
        if per:  # centred, wrapped: the start is stored modulo n (negative marks "no window")
            idx = np.mod(np.arange(n) - 3, n)
        elif n < 7:
            continue
        else:
            idx = np.clip(np.arange(a, a + n) - 3, a, a + n - 7)
        if direction == 1:
            st[line, a:a + n] = idx
        else:
            st[a:a + n, line] = idx
    return st


def tau_patch(g, phi):
    """tau~ on every point (meaningful on generating points) and the min logit margin."""
    taus, margins = [], []
    for dirn in (1, 2):
        st = window_starts(g, dirn)
        sel = g.gen & (st >= 0)
        jj, ii = np.nonzero(sel)
        s = st[jj, ii]
        if dirn == 1:
            cols = (s[:, None] + np.arange(7)[None, :])
            if g.periodic1:
                cols = np.mod(cols, g.n1)
            win = phi[jj[:, None], cols]
        else:
            win = phi[s[:, None] + np.arange(7)[None, :], ii[:, None]]
        t = np.full((g.n2, g.n1), 4, np.int64)
        m = np.full((g.n2, g.n1), np.inf)
        if len(jj):
            c, mg, _ = classify(win)
            t[jj, ii] = c
            m[jj, ii] = mg
        taus.append(t)
        margins.append(m)
    return np.minimum(taus[0], taus[1]), np.minimum(margins[0], margins[1])


def max7x7(g, S):
    half = 3
    Sb = np.where(g.blank, 0.0, S)
    out = Sb.copy()
    for a in range(-half, half + 1):
        for b in range(-half, half + 1):
            out = np.maximum(out, _shift(Sb, a, b, g.periodic1, 0.0))
    return out


def _shift(A, di, dj, per1, fill):
    """B[j, i] = A[j + dj, i + di] (fill outside; wrap along q1 if periodic)."""
    n2, n1 = A.shape
    B = np.full_like(A, fill)
    if per1:
        A = np.roll(A, -di, axis=1)
        di = 0
    j0, j1 = max(0, -dj), min(n2, n2 - dj)
    i0, i1 = max(0, -di), min(n1, n1 - di)
    if j0 < j1 and i0 < i1:
        B[j0:j1, i0:i1] = A[j0 + dj:j1 + dj, i0 + di:i1 + di]
    return B


def preliminary(g, e, params):
    """mu^ on the generating points of one patch (eq. V2D_unscaled); 0 elsewhere."""
    phi = np.where(g.blank, 0.0, euler.proxy_mach(e, params.gamma))
    S = euler.mwsb(e, params.gamma)
    tau, margin = tau_patch(g, phi)
    R = np.asarray(params.R)[tau - 1]
    muhat = np.where(g.gen, R * max7x7(g, S) * g.hhat, 0.0)
    return muhat, tau, margin


class SBOperator:
    """Geometry part of Lambda: windows, nearest points in other patches, normaliser."""

    def __init__(self, geos, params):
        self.geos = geos
        r = params.win_r
        k = np.arange(-(r - 1), r)
        self.taps = k
        self.w = window_weight(k, 0, r)
        self.cross = []  # per patch: list of (q, j_idx, i_idx, z2, z1) for foreign patches containing the point
        boxes = [g.bbox() for g in geos]
        for p, g in enumerate(geos):
            lst = []
            valid = ~g.blank
            for q, h in enumerate(geos):
                if q == p or not _overlap(boxes[p], boxes[q]):
                    continue
                s1, s2 = h.frac_index(g.x, g.y)
                inside = h.contains(s1, s2) & valid
                jj, ii = np.nonzero(inside)
                if len(jj):
                    z1, z2 = h.nearest(s1[jj, ii], s2[jj, ii])
                    lst.append((q, jj, ii, z2, z1))
            self.cross.append(lst)
        self.den_own = [self.window_sum(g, g.gen.astype(float)) for g in geos]
        self.den = []
        for p, g in enumerate(geos):
            d = self.den_own[p].copy()
            for (q, jj, ii, z2, z1) in self.cross[p]:
                d[jj, ii] += self.den_own[q][z2, z1]
            self.den.append(d)

    def window_sum(self, g, b):
        """sum over (i',j') of w(i-i') w(j-j') b[j',i'] (b already zero off G~)."""
        out = np.zeros_like(b)
        for a, wa in zip(self.taps, self.w):
            for c, wc in zip(self.taps, self.w):
                out += (wa * wc) * _shift(b, a, c, g.periodic1, 0.0)
        return out

    def apply(self, muhats):
        num_own = [self.window_sum(g, m) for g, m in zip(self.geos, muhats)]
        out = []
        for p, g in enumerate(self.geos):
            num = num_own[p].copy()
            for (q, jj, ii, z2, z1) in self.cross[p]:
                num[jj, ii] += num_own[q][z2, z1]
            den = self.den[p]
            mu = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
            out.append(np.where(g.blank, 0.0, mu))
        return out


def viscosity(geos, sb, states, params):
    """mu = Lambda[mu^] on every patch; also returns tau~ and margins for tie checks."""
    pre = [preliminary(g, e, params) for g, e in zip(geos, states)]
    mu = sb.apply([m for m, _, _ in pre])
    return mu, [t for _, t, _ in pre], [mg for _, _, mg in pre], [m for m, _, _ in pre]
