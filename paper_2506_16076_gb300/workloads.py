"""Seeded synthetic inputs: patch layouts, initial states, parameters.

This module holds no arithmetic of the FC-SDNN method. It only describes
geometry (patch kinds, point counts, bounds, side types, the blanked hole),
the initial primitive states, and the flat state layout. Both the oracle
(test infrastructure) and the CUDA path consume what it produces.

Workloads (stand-ins for the paper's meshes, which are not published):
  sod128      single affine patch [0,1]^2, 128x128, Sod tube along x
  cyl_m3      O-grid r in [0.5,1.5] (512 theta x 96 r) + 4x4 affine 160x160
              patches on [-4,8]x[-6,6] with 10-point overlaps, Mach 3 free stream,
              no-slip adiabatic cylinder wall
  cyl_m2_half same geometry at half resolution (256x48, 80x80), Mach 2 at 2 deg,
              no-slip adiabatic cylinder wall
  cyl_m25_32  [-8,16]x[-12,12] as 32x32 affine patches with seeded uneven sizes
              48..384 (refined toward the body) + 1024x192 O-grid, Mach 25, no-slip
              adiabatic wall, potential-flow start with a near-wall layer
  cyl_m25_4096 64x64 affine patches with seeded sizes 64..512 + O-grid, Mach 25
  cyl_m25_32_sub cyl_m25_32 split into the paper's 101 x 101 sub-patches (subpatched)
  The two seeded arrays use the rule n = nmin + round((nmax-nmin)*u*(1-a*dc/dmax)),
  u ~ U[0,1) from numpy.random.default_rng(seed), dc = distance from the patch
  centre to the cylinder centre; a is the taper coefficient.
"""
from dataclasses import dataclass, field, replace
import math
import numpy as np

# patch kinds
AFFINE, OGRID, GRID = 0, 1, 2
# side types (side order: q1=0, q1=1, q2=0, q2=1)
INTERNAL, DIRICHLET, SLIPWALL, OUTFLOW, PERIODIC, ADIABATIC = 0, 1, 2, 3, 4, 5

GAMMA = 1.4


@dataclass
class PatchDesc:
    kind: int
    n1: int
    n2: int
    geom: tuple  # AFFINE: (x0, x1, y0, y1); OGRID: (xc, yc, r0, r1)
    side: tuple  # 4 side types
    bc: tuple = ((0.0, 0.0, 0.0, 0.0),) * 4  # Dirichlet primitive (rho,u,v,p) per side
    hole: tuple = (0.0, 0.0, -1.0)  # (xc, yc, R): blank points closer than R; R<=0: none
    # GRID only: coordinates (n2, n1) and metrics dq/dx (4, n2, n1) = (q1_x, q1_y, q2_x, q2_y)
    x: object = None
    y: object = None
    metrics: object = None

    @property
    def npts(self):
        return self.n1 * self.n2


@dataclass
class Params:
    d: int = 5
    C0: int = 27
    c_policy: int = 0  # 0: C = C0 on every line; 1: smallest C >= C0 with N+C 7-smooth;
    #                    2: C in [C0, largest tabulated C] with the cheapest transform of N+C
    gamma: float = GAMMA
    alpha_f: float = 10.0
    p_f: int = 14
    cfl: float = 0.5
    n_f: int = 5
    n_v: int = 9
    win_r: int = 9
    loc: int = 7
    R: tuple = (1.5, 1.0, 0.5, 0.0)
    depth_cap: int = 64
    wall_form: int = 0  # 0: flux form on every patch; 1: on patches with an ADIABATIC side the
    #                     product-rule form of Remark adiabatic (derivatives of E and p from FC
    #                     derivatives of rho, rho u, rho v and theta)


@dataclass
class Workload:
    name: str
    patches: list
    params: Params
    freestream: tuple  # primitive (rho, u, v, p)
    init: str  # 'sod' or 'freestream'
    steps: int
    extra: dict = field(default_factory=dict)

    @property
    def offsets(self):
        off = [0]
        for p in self.patches:
            off.append(off[-1] + p.npts)
        return off

    @property
    def total_points(self):
        return self.offsets[-1]


def sod128(n=128):
    left, right = (1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1)
    p = PatchDesc(AFFINE, n, n, (0.0, 1.0, 0.0, 1.0), (DIRICHLET, DIRICHLET, SLIPWALL, SLIPWALL),
                  bc=(left, right, left, left))
    return Workload("sod128" if n == 128 else f"sod{n}", [p], Params(d=5, C0=27, c_policy=0),
                    freestream=left, init="sod", steps=100, extra={"left": left, "right": right, "x_split": 0.5})


def mach_shock_state(M, gamma=GAMMA):
    """Post-shock primitive state of a Mach-M shock moving at speed M into (1.4, 0, 0, 1)
    (eq. mach_shock_ic; the printed density is read as the density ratio, so the
    post-shock density is 1.4 times it)."""
    zeta = (2 * gamma * M * M - gamma + 1) / (gamma + 1)
    ratio = (gamma + 1) * M * M / ((gamma - 1) * M * M + 2)
    return (1.4 * ratio, (zeta - 1) / (gamma * M), 0.0, zeta)


def moving_shock(M, n1=256, n2=16, x_split=0.25):
    """A planar Mach-M shock at x = x_split moving right into gas at rest (Sec. 7,
    eq. mach_shock_ic) on one affine patch [0, 1] x [0, (n2-1)/(n1-1)] with square cells;
    x-ends hold the two states, y-sides are slip walls."""
    post, pre = mach_shock_state(M), (1.4, 0.0, 0.0, 1.0)
    ly = (n2 - 1) / (n1 - 1)
    p = PatchDesc(AFFINE, n1, n2, (0.0, 1.0, 0.0, ly), (DIRICHLET, DIRICHLET, SLIPWALL, SLIPWALL),
                  bc=(post, pre, post, post))
    return Workload(f"shock_M{M:g}", [p], Params(d=5, C0=27, c_policy=2), freestream=pre, init="sod", steps=0,
                    extra={"left": post, "right": pre, "x_split": x_split, "mach": M})


def _cart_array(nx, ny, x0, x1, y0, y1, nper, overlap, fs, hole, sizes=None):
    """nx*ny affine patches tiling [x0,x1]x[y0,y1].

    Uniform case (sizes None): every patch has nper points per side on one global
    grid; neighbours share `overlap` grid lines. Seeded case: sizes[i][j] = (n1, n2)
    and neighbouring patches overlap by `overlap` points of the coarser neighbour.
    Outer sides: left/bottom/top Dirichlet free stream, right outflow.
    """
    patches = []
    if sizes is None:
        ntot = nx * nper - (nx - 1) * overlap
        hx = (x1 - x0) / (ntot - 1)
        mty = ny * nper - (ny - 1) * overlap
        hy = (y1 - y0) / (mty - 1)
    for j in range(ny):
        for i in range(nx):
            if sizes is None:
                n1 = n2 = nper
                a = x0 + i * (nper - overlap) * hx
                b = a + (nper - 1) * hx
                c = y0 + j * (nper - overlap) * hy
                e = c + (nper - 1) * hy
            else:
                n1, n2 = sizes[j][i]
                wx, wy = (x1 - x0) / nx, (y1 - y0) / ny
                # overlap half-width on each internal side: `overlap` points of the coarser
                # neighbour, so both patches keep an (overlap)-point layer inside the other
                def half(nself, nnb, w):
                    return 0.5 * overlap * w / (min(nself, nnb) - 1)
                lx = half(n1, sizes[j][i - 1][0], wx) if i > 0 else 0.0
                rx = half(n1, sizes[j][i + 1][0], wx) if i < nx - 1 else 0.0
                ly = half(n2, sizes[j - 1][i][1], wy) if j > 0 else 0.0
                ry = half(n2, sizes[j + 1][i][1], wy) if j < ny - 1 else 0.0
                a, b = x0 + i * wx - lx, x0 + (i + 1) * wx + rx
                c, e = y0 + j * wy - ly, y0 + (j + 1) * wy + ry
            side = (DIRICHLET if i == 0 else INTERNAL, OUTFLOW if i == nx - 1 else INTERNAL,
                    DIRICHLET if j == 0 else INTERNAL, DIRICHLET if j == ny - 1 else INTERNAL)
            patches.append(PatchDesc(AFFINE, n1, n2, (a, b, c, e), side, bc=(fs,) * 4, hole=hole))
    return patches


def _ogrid(nth, nr, r0, r1, fs, wall=SLIPWALL):
    return PatchDesc(OGRID, nth, nr, (0.0, 0.0, r0, r1), (PERIODIC, PERIODIC, wall, INTERNAL), bc=(fs,) * 4)


def cyl_m3(scale=1.0):
    fs = (1.4, 3.0, 0.0, 1.0)
    nc = int(round(160 * scale))
    og = _ogrid(int(round(512 * scale)), int(round(96 * scale)), 0.5, 1.5, fs, ADIABATIC)
    cart = _cart_array(4, 4, -4.0, 8.0, -6.0, 6.0, nc, 10, fs, hole=(0.0, 0.0, 1.0))
    return Workload("cyl_m3" if scale == 1.0 else f"cyl_m3_x{scale}", [og] + cart,
                    Params(d=5, C0=27, c_policy=2), freestream=fs, init="freestream", steps=2000)


def cyl_m2_half(mach=2.0, alpha_deg=2.0):
    """The Mach-3 cylinder geometry at half resolution under a Mach-2 free stream at 2
    degrees angle of attack (the adjoint configuration); mach and alpha_deg vary the
    free stream (and the Dirichlet states) for finite-difference checks."""
    a = math.radians(alpha_deg)
    fs = (1.4, mach * math.cos(a), mach * math.sin(a), 1.0)
    og = _ogrid(256, 48, 0.5, 1.5, fs, ADIABATIC)
    cart = _cart_array(4, 4, -4.0, 8.0, -6.0, 6.0, 80, 10, fs, hole=(0.0, 0.0, 1.0))
    return Workload("cyl_m2_half", [og] + cart, Params(d=5, C0=27, c_policy=2), freestream=fs,
                    init="freestream", steps=400, extra={"mach": mach, "alpha_deg": alpha_deg})


def seeded_sizes(nx, ny, nmin, nmax, seed, x0, x1, y0, y1, taper):
    rng = np.random.default_rng(seed)
    u = rng.random((ny, nx, 2))
    wx, wy = (x1 - x0) / nx, (y1 - y0) / ny
    cx = x0 + (np.arange(nx) + 0.5) * wx
    cy = y0 + (np.arange(ny) + 0.5) * wy
    dc = np.hypot(cx[None, :], cy[:, None])
    f = 1.0 - taper * dc / dc.max()
    n = nmin + np.round((nmax - nmin) * u * f[:, :, None]).astype(int)
    return [[(int(n[j, i, 0]), int(n[j, i, 1])) for i in range(nx)] for j in range(ny)]


def cyl_m25_array(nx, nmin, nmax, seed, taper, nth, nr, name):
    fs = (1.4, 25.0, 0.0, 1.0)
    sizes = seeded_sizes(nx, nx, nmin, nmax, seed, -8.0, 16.0, -12.0, 12.0, taper)
    og = _ogrid(nth, nr, 0.5, 1.5, fs, ADIABATIC)
    cart = _cart_array(nx, nx, -8.0, 16.0, -12.0, 12.0, None, 19, fs, hole=(0.0, 0.0, 1.0), sizes=sizes)
    return Workload(name, [og] + cart, Params(d=5, C0=27, c_policy=2), freestream=fs, init="potential", steps=200,
                    extra={"taper": taper, "seed": seed, "cyl_radius": 0.5, "cutoff": 3.0, "wall_layer": 0.05})


def cyl_m25_32():
    """32x32 uneven affine patches + 1024x192 O-grid, Mach 25 (about 30M points)."""
    return cyl_m25_array(32, 48, 384, 3, 0.6, 1024, 192, "cyl_m25_32")


def cyl_m25_4096():
    """64x64 uneven affine patches + O-grid, Mach 25 (about 64M points with the taper below)."""
    return cyl_m25_array(64, 64, 512, 5, 0.95, 1024, 192, "cyl_m25_4096")


def small_multipatch(wall=SLIPWALL):
    """A tiny O-grid + 2x2 affine array around a cylinder: the oracle finishes it in seconds.
    wall: SLIPWALL or ADIABATIC (no-slip adiabatic) on the cylinder."""
    fs = (1.4, 3.0, 0.0, 1.0)
    og = _ogrid(128, 32, 0.5, 1.5, fs, wall)
    cart = _cart_array(2, 2, -2.5, 2.5, -2.5, 2.5, 64, 10, fs, hole=(0.0, 0.0, 0.85))
    name = "small_multipatch" if wall == SLIPWALL else "small_multipatch_adiabatic"
    return Workload(name, [og] + cart, Params(d=5, C0=27, c_policy=2), freestream=fs, init="freestream", steps=20)


def subpatched(w: Workload, n0=83, nv=9):
    """The paper's sub-patch decomposition (Sec. 3.2.1, eqs. rect, discretization,
    subpatchesQ) applied to the affine patches of a workload: a line of more than
    n0 + 2 nv points is re-gridded to N = r (n0 + 1) - 1 + 2 nv points (the smallest r
    with N >= n; same physical extent) and split into r overlapping sub-patches of
    n0 + 2 nv points each, starting every n0 + 1 points (neighbours share 2 nv - 1 grid
    lines). Sub-patch sides inside the parent patch are internal (the exchange copies
    the coincident grid values); the parent's outer sides keep their types. Shorter
    lines and the O-grid are kept as they are."""
    m = n0 + 2 * nv
    step = n0 + 1

    def split(n, a, b):
        if n <= m:
            return [(n, a, b, True, True)]
        r = -(-(n - m) // step) + 1  # smallest r with r (n0 + 1) - 1 + 2 nv >= n
        N = r * step - 1 + 2 * nv
        h = (b - a) / (N - 1)
        return [(m, a + k * step * h, a + (k * step + m - 1) * h, k == 0, k == r - 1) for k in range(r)]

    out = []
    for p in w.patches:
        if p.kind != AFFINE:
            out.append(p)
            continue
        x0, x1, y0, y1 = p.geom
        for (n2, c, d, lo2, hi2) in split(p.n2, y0, y1):
            for (n1, a, b, lo1, hi1) in split(p.n1, x0, x1):
                side = (p.side[0] if lo1 else INTERNAL, p.side[1] if hi1 else INTERNAL,
                        p.side[2] if lo2 else INTERNAL, p.side[3] if hi2 else INTERNAL)
                out.append(PatchDesc(AFFINE, n1, n2, (a, b, c, d), side, bc=p.bc, hole=p.hole))
    return Workload(w.name + "_sub", out, w.params, w.freestream, w.init, w.steps,
                    {**w.extra, "subpatch": (n0, nv)})


def cyl_m25_32_sub():
    """cyl_m25_32 with its patches split into the paper's 101 x 101 sub-patches."""
    return subpatched(cyl_m25_32())


WORKLOADS = {
    "cyl_m25_32_sub": cyl_m25_32_sub,
    "sod128": sod128,
    "cyl_m3": cyl_m3,
    "cyl_m2_half": cyl_m2_half,
    "cyl_m25_32": cyl_m25_32,
    "cyl_m25_4096": cyl_m25_4096,
    "small_multipatch": small_multipatch,
}


# ---------------------------------------------------------------- grids (geometry only)

def grid_patch(mapping, n1, n2, side, bc, periodic1=False, hole=(0.0, 0.0, -1.0)):
    """A GRID patch from a smooth mapping (q1, q2) -> (x, y, x_q1, x_q2, y_q1, y_q2) on
    q1 = i / (n1 - 1) (i / n1 if periodic1), q2 = j / (n2 - 1): coordinates and the
    metrics dq/dx as the inverse of the mapping's Jacobian (geometry input only)."""
    q1 = np.arange(n1) / (n1 if periodic1 else n1 - 1)
    q2 = np.arange(n2) / (n2 - 1)
    Q1, Q2 = np.meshgrid(q1, q2)
    x, y, xa, xb, ya, yb = mapping(Q1, Q2)
    det = xa * yb - xb * ya
    metrics = np.stack([yb / det, -xb / det, -ya / det, xa / det])
    return PatchDesc(GRID, n1, n2, (0.0, 0.0, 0.0, 0.0), side, bc=bc, hole=hole,
                     x=np.ascontiguousarray(x), y=np.ascontiguousarray(y), metrics=np.ascontiguousarray(metrics))


def affine_map(x0, x1, y0, y1, bump=0.0):
    """(q1, q2) -> box [x0, x1] x [y0, y1], displaced inside by
    bump * (x1 - x0, y1 - y0) * sin(pi q1) sin(pi q2) (zero on the box's edges)."""
    def f(a, b):
        lx, ly = x1 - x0, y1 - y0
        s = bump * np.sin(np.pi * a) * np.sin(np.pi * b)
        sa = bump * np.pi * np.cos(np.pi * a) * np.sin(np.pi * b)
        sb = bump * np.pi * np.sin(np.pi * a) * np.cos(np.pi * b)
        return (x0 + lx * (a + s), y0 + ly * (b + s), lx * (1.0 + sa), lx * sb, ly * sa, ly * (1.0 + sb))
    return f


def annulus_map(xc, yc, r0, r1, stretch=0.0, twist=0.0):
    """(q1, q2) -> annulus r0 <= r <= r1 around (xc, yc), q1 periodic (angle), with
    r = r0 + (r1 - r0) (q2 + stretch sin(pi q2)) and angle 2 pi q1 + twist sin(pi q2)^2
    (grid lines leave both circles along the normal)."""
    def f(a, b):
        dr = r1 - r0
        r = r0 + dr * (b + stretch * np.sin(np.pi * b))
        rb = dr * (1.0 + stretch * np.pi * np.cos(np.pi * b))
        th = 2.0 * np.pi * a + twist * np.sin(np.pi * b) ** 2
        tha = 2.0 * np.pi
        thb = twist * np.pi * np.sin(2.0 * np.pi * b)
        c, s = np.cos(th), np.sin(th)
        return (xc + r * c, yc + r * s, -r * s * tha, rb * c - r * s * thb, r * c * tha, rb * s + r * c * thb)
    return f


def arc_map(xc, yc, r0, r1, th0, th1):
    """(q1, q2) -> the annular sector th0 <= angle <= th1, r0 <= r <= r1 around (xc, yc):
    an S-type patch along a circle (Sec. 3.1), angle along q1, radius along q2."""
    def f(a, b):
        dr, dth = r1 - r0, th1 - th0
        r = r0 + dr * b
        th = th0 + dth * a
        c, s = np.cos(th), np.sin(th)
        return (xc + r * c, yc + r * s, -r * s * dth, dr * c, r * c * dth, dr * s)
    return f


def s_type_ring(xc, yc, r0, r1, K, nth, nr, half, fs, wall):
    """K non-periodic arc patches (GRID, S-type) covering the annulus r0 <= r <= r1 in
    place of one periodic O-grid of nth angular points: arc k spans the angles
    [k P - half, (k + 1) P + half] (P = nth / K spacings of 2 pi / nth), so neighbours
    share 2 half + 1 angular grid lines; q1 ends internal, the wall at q2 = 0, the outer
    circle internal. Every line is FC-continued (no Fourier shortcut)."""
    assert nth % K == 0
    dth = 2.0 * np.pi / nth
    per = nth // K
    out = []
    for k in range(K):
        th0, th1 = (k * per - half) * dth, ((k + 1) * per + half) * dth
        out.append(grid_patch(arc_map(xc, yc, r0, r1, th0, th1), per + 2 * half + 1, nr,
                              (INTERNAL, INTERNAL, wall, INTERNAL), (fs,) * 4))
    return out


def small_multipatch_stype(K=4, half=6):
    """small_multipatch (adiabatic cylinder wall) with its periodic O-grid replaced by K
    overlapping S-type arc patches of the same spacing (s_type_ring)."""
    w = small_multipatch(ADIABATIC)
    og = w.patches[0]
    xc, yc, r0, r1 = og.geom
    ring = s_type_ring(xc, yc, r0, r1, K, og.n1, og.n2, half, w.freestream, ADIABATIC)
    return Workload("small_multipatch_stype", ring + w.patches[1:], w.params, w.freestream, w.init, w.steps,
                    dict(w.extra))


def as_grid(p: PatchDesc, bump=0.0, stretch=0.0, twist=0.0, metrics=True):
    """The GRID form of an AFFINE or OGRID patch: the same map (plus the optional
    smooth displacements of affine_map / annulus_map), sides, states and hole.
    metrics=False: the points only (the library computes the metrics)."""
    if p.kind == AFFINE:
        g = grid_patch(affine_map(*p.geom, bump=bump), p.n1, p.n2, p.side, p.bc, hole=p.hole)
    elif p.kind == OGRID:
        g = grid_patch(annulus_map(*p.geom, stretch=stretch, twist=twist), p.n1, p.n2, p.side, p.bc,
                       periodic1=True, hole=p.hole)
    else:
        return p
    return g if metrics else replace(g, metrics=None)


def small_multipatch_grid(curved=True, metrics=True):
    """small_multipatch (adiabatic cylinder wall) with every patch given as a GRID patch;
    curved: the annulus stretched and twisted and the boxes bulged inside, so that the
    grids are non-orthogonal and the metrics vary from point to point; metrics=False:
    points only, the metrics left to the library."""
    w = small_multipatch(ADIABATIC)
    ps = [as_grid(p, bump=0.04 if curved else 0.0, stretch=0.15 if curved else 0.0,
                  twist=0.3 if curved else 0.0, metrics=metrics) for p in w.patches]
    name = "small_multipatch_grid" + ("_curved" if curved else "") + ("" if metrics else "_points")
    return Workload(name, ps, w.params, w.freestream, w.init, w.steps, dict(w.extra))


def patch_xy(p: PatchDesc):
    """Physical coordinates (x, y), each shape (n2, n1), of a patch's grid points."""
    if p.kind == GRID:
        return np.array(p.x, dtype=np.float64), np.array(p.y, dtype=np.float64)
    i = np.arange(p.n1)
    j = np.arange(p.n2)
    if p.kind == AFFINE:
        x0, x1, y0, y1 = p.geom
        x = x0 + (x1 - x0) * i / (p.n1 - 1)
        y = y0 + (y1 - y0) * j / (p.n2 - 1)
        return np.broadcast_to(x[None, :], (p.n2, p.n1)).copy(), np.broadcast_to(y[:, None], (p.n2, p.n1)).copy()
    xc, yc, r0, r1 = p.geom
    th = 2.0 * np.pi * i / p.n1
    r = r0 + (r1 - r0) * j / (p.n2 - 1)
    return xc + r[:, None] * np.cos(th)[None, :], yc + r[:, None] * np.sin(th)[None, :]


def prim_to_cons(rho, u, v, p, gamma=GAMMA):
    """Initial-condition construction from primitive states (eq. perfect_gas)."""
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def initial_state(w: Workload):
    """List of per-patch conserved states, each (4, n2, n1), for the workload's IC.

    Blanked points get the free-stream state (they never change)."""
    out = []
    for p in w.patches:
        x, y = patch_xy(p)
        if w.init == "sod":
            L, R = w.extra["left"], w.extra["right"]
            left = x < w.extra["x_split"]
            prim = [np.where(left, L[k], R[k]) for k in range(4)]
        elif w.init == "potential":
            prim = potential_flow_prim(x, y, w.freestream, w.extra["cyl_radius"], w.extra["cutoff"],
                                       w.extra.get("wall_layer", 0.0))
        else:
            prim = [np.full(x.shape, w.freestream[k]) for k in range(4)]
        out.append(prim_to_cons(*prim, gamma=w.params.gamma))
    return out


def potential_flow_prim(x, y, fs, R, cutoff, wall_layer=0.0):
    """Free-stream density and pressure with the incompressible potential-flow velocity
    around a cylinder of radius R at the origin, u - i v = U (e^{-ia} - R^2 e^{ia} / z^2),
    whose wall-normal velocity vanishes on r = R. The disturbance is switched off smoothly
    between r = cutoff and 2 cutoff so that the outer boundaries see the free stream.
    wall_layer > 0: the velocity is multiplied by 1 - exp(-((r - R) / wall_layer)^2), so
    that it also vanishes at the wall (a start consistent with a no-slip wall)."""
    rho, u0, v0, p = fs
    U = np.hypot(u0, v0)
    a = np.arctan2(v0, u0)
    z = x + 1j * y
    r = np.abs(z)
    zs = np.where(r > 0, z, 1.0)
    dist = -U * R * R * np.exp(1j * a) / (zs * zs)  # disturbance of u - i v
    t = np.clip((r - cutoff) / cutoff, 0.0, 1.0)
    sw = np.where(t <= 0, 1.0, np.where(t >= 1, 0.0, 0.5 * (1 + np.cos(np.pi * t))))
    w = u0 - 1j * v0 + sw * dist
    if wall_layer > 0:
        w = w * np.where(r > R, 1.0 - np.exp(-(((r - R) / wall_layer) ** 2)), 0.0)
    return [np.full(x.shape, rho), w.real, -w.imag, np.full(x.shape, p)]


def flatten(per_patch):
    """[4][P_tot] flat SoA layout: per patch, row-major (n2, n1), q1 fastest."""
    return np.concatenate([a.reshape(a.shape[0], -1) for a in per_patch], axis=1)


def unflatten(flat, w: Workload):
    off = w.offsets
    return [flat[:, off[k]:off[k + 1]].reshape(flat.shape[0], p.n2, p.n1) for k, p in enumerate(w.patches)]


def random_smooth_state(w: Workload, seed, amp=0.05):
    """Seeded smooth perturbation of the free stream (for RHS parity tests)."""
    rng = np.random.default_rng(seed)
    fs = w.freestream
    out = []
    kx, ky, ph = rng.uniform(0.5, 2.0, 4), rng.uniform(0.5, 2.0, 4), rng.uniform(0, 2 * np.pi, 4)
    for p in w.patches:
        x, y = patch_xy(p)
        prim = []
        for c in range(4):
            pert = np.sin(kx[c] * x + ph[c]) * np.cos(ky[c] * y + 0.3 * ph[c])
            # density and pressure: relative perturbation; velocities: 3 amp (sound speed ~ 1)
            prim.append(fs[c] * (1.0 + amp * pert) if c in (0, 3) else fs[c] + 3.0 * amp * pert)
        out.append(prim_to_cons(*prim, gamma=w.params.gamma))
    return out


def cyl_m3_stype(K=8, half=8):
    """cyl_m3 with its 512 x 96 periodic O-grid replaced by K overlapping S-type arc
    patches of the same spacing (s_type_ring): every line FC-continued."""
    w = cyl_m3()
    og = w.patches[0]
    xc, yc, r0, r1 = og.geom
    ring = s_type_ring(xc, yc, r0, r1, K, og.n1, og.n2, half, w.freestream, ADIABATIC)
    return Workload("cyl_m3_stype", ring + w.patches[1:], w.params, w.freestream, w.init, w.steps, dict(w.extra))


WORKLOADS["small_multipatch_stype"] = small_multipatch_stype
WORKLOADS["cyl_m3_stype"] = cyl_m3_stype
