"""The kernels' line arithmetic compiled for the host (tests/line_engine_host.cpp: the same
fc_line.cuh and plan builder the GPU runs, one lane per line) checked on the CPU:

- every candidate FFT stage order of every continued length the autotuner may choose
  differentiates random trigonometric polynomials to rounding (exact spectral
  derivative as the reference);
- the FC derivative (detrended two-phase continuation, in-place transforms, digit-
  reversed multiplier) of every candidate order matches the oracle's long-double FC
  derivative (Sec. 2.2, eq. fc_der) on smooth lines, and differentiates polynomials of
  degree below d exactly up to rounding;
- the FC filter (Sec. 4.3.1, eq. filtering) of every candidate order matches the
  oracle's.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import fc as F
from paper_2506_16076_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
CUDA_LIB = "/usr/local/cuda/lib64"


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    from paper_2506_16076_gb300 import build
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ and the CUDA headers are needed to build the host harness")
    lib = build.build()
    out = str(tmp_path_factory.mktemp("le") / "line_engine_host")
    cmd = [gxx, "-O2", "-std=c++17", "-w", f"-I{CUDA_INC}", "-o", out, os.path.join(ROOT, "tests", "line_engine_host.cpp"),
           f"-L{os.path.dirname(lib)}", "-lfcsdnn", f"-L{CUDA_LIB}", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = ":".join([os.path.dirname(lib), CUDA_LIB, env.get("LD_LIBRARY_PATH", "")])
    return out, env


def _smooth7(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def test_every_candidate_stage_order_differentiates_exactly(harness):
    exe, env = harness
    lengths = [L for L in range(16, 1200) if _smooth7(L)] + [176, 297, 143 * 2]  # also generic primes 11, 13
    r = subprocess.run([exe, "plans", *map(str, lengths)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    rows = [ln.split() for ln in r.stdout.splitlines()]
    assert len(rows) >= len(lengths)
    worst = max(rows, key=lambda x: float(x[2]))
    # FP64 transforms: a few units of rounding times log L
    assert float(worst[2]) < 2e-14, worst


def test_fma_records_encode_their_twiddles(harness):
    # the ratio-form records of the FMA butterflies (every candidate stage order): each
    # twiddle rebuilt from S, t and its flag equals exp(+-2 pi i e / L) to rounding, with
    # |t| <= 1 and |S| >= 1/sqrt 2 (the bounds that keep the ratio form accurate)
    exe, env = harness
    lengths = [L for L in range(16, 1200) if _smooth7(L)] + [4096, 2187, 3125, 2401]
    r = subprocess.run([exe, "records", *map(str, lengths)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    rows = [ln.split() for ln in r.stdout.splitlines()]
    assert len(rows) >= len(lengths)
    assert max(float(x[2]) for x in rows) < 1e-15, max(rows, key=lambda x: float(x[2]))
    assert max(float(x[3]) for x in rows) <= 1.0 + 1e-15
    assert min(float(x[4]) for x in rows) >= 0.7071067


ALPHA_F, P_F = 10.0, 14  # the paper's filter parameters (Sec. 4.3.1)


def _run_fc(exe, env, tmp, lines, d=5, op=0):
    from paper_2506_16076_gb300 import fcsdnn
    tab = np.asarray(fcsdnn.fc_table_blob(d), dtype=np.float64)
    fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("<idii", d, ALPHA_F, P_F, tab.size))
        f.write(tab.tobytes())
        f.write(struct.pack("<i", len(lines)))
        for (N, C, h, data) in lines:
            f.write(struct.pack("<iiid", op, N, C, h))
            f.write(np.ascontiguousarray(data, dtype=np.float64).tobytes())
    r = subprocess.run([exe, "fc", fin, fout], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    raw = open(fout, "rb").read()
    pos, res = 0, []
    for (N, C, h, data) in lines:
        nc = struct.unpack_from("<i", raw, pos)[0]
        pos += 4
        outs = []
        for _ in range(nc):
            outs.append(np.frombuffer(raw, dtype=np.float64, count=4 * N, offset=pos).reshape(4, N))
            pos += 8 * 4 * N
        res.append(outs)
    return res


def _smooth_lines(seed):
    rng = np.random.default_rng(seed)
    lines = []
    for N in (10, 37, 64, 101, 160, 257, 384, 640):
        C = F.choose_C(N, 27, 2, 5)
        x = np.arange(N) / (N - 1)
        comps = []
        for _ in range(4):
            a, b, c, k = rng.uniform(-1, 1, 4)
            comps.append(5.0 + a * np.sin(3.0 * k * x + b) + c * np.exp(x) * np.cos(2.0 * x))
        lines.append((N, C, 1.0 / (N - 1), np.stack(comps)))
    return lines


def test_fc_filter_matches_the_oracle(harness, tmp_path):
    exe, env = harness
    lines = _smooth_lines(9)
    res = _run_fc(exe, env, str(tmp_path), lines, op=1)
    for (N, C, h, data), outs in zip(lines, res):
        ref = F.fc_filter(data, 5, C, ALPHA_F, P_F)
        for o in outs:
            err = np.abs(o - ref).max() / np.abs(ref).max()
            assert err < 1e-14 * max(1.0, N / 64), (N, C, err)


def test_fc_derivative_matches_the_oracle(harness, tmp_path):
    exe, env = harness
    lines = _smooth_lines(8)
    res = _run_fc(exe, env, str(tmp_path), lines)
    for (N, C, h, data), outs in zip(lines, res):
        ref = F.fc_derivative(data, h, 5, C)
        for o in outs:
            err = np.abs(o - ref).max() / np.abs(ref).max()
            # FP64 transforms of lines with a mean 5 times their variation: rounding at the
            # top modes grows with the length (the floor measured for the GPU kernels)
            assert err < 1e-12 * max(1.0, N / 256), (N, C, err)


def test_fc_derivative_exact_on_polynomials(harness, tmp_path):
    exe, env = harness
    lines = []
    for N in (10, 41, 128, 333):
        C = F.choose_C(N, 27, 2, 5)
        x = np.arange(N) / (N - 1)
        data = np.stack([1.0 + 0 * x, 2.0 * x - 1.0, x ** 3 - 0.5 * x ** 2, x ** 4])
        lines.append((N, C, 1.0 / (N - 1), data))
    res = _run_fc(exe, env, str(tmp_path), lines)
    for (N, C, h, data), outs in zip(lines, res):
        x = np.arange(N) / (N - 1)
        exact = np.stack([0 * x, 2.0 + 0 * x, 3 * x ** 2 - x, 4 * x ** 3])
        for o in outs:
            assert np.abs(o - exact).max() < 1e-11 * N, (N, np.abs(o - exact).max())


def _run_grid(exe, env, tmp, p, xq, yq):
    fin, fout = os.path.join(tmp, "g.bin"), os.path.join(tmp, "go.bin")
    periodic = int(p.side[0] == W.PERIODIC)
    with open(fin, "wb") as f:
        f.write(struct.pack("<iii", p.n1, p.n2, periodic))
        f.write(np.ascontiguousarray(p.x, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(p.y, dtype=np.float64).tobytes())
        f.write(struct.pack("<i", len(xq)))
        f.write(np.asarray(xq, dtype=np.float64).tobytes())
        f.write(np.asarray(yq, dtype=np.float64).tobytes())
    r = subprocess.run([exe, "grid", fin, fout], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    v = np.fromfile(fout, dtype=np.float64)
    nq = len(xq)
    return v[0], v[1], v[2:2 + nq], v[2 + nq:2 + 2 * nq]


@pytest.mark.parametrize("kind", ["annulus", "bulged_box", "thin_strip"])
def test_host_grid_inverse_matches_the_oracle(harness, tmp_path, kind):
    # the library's host geometry of a GRID patch (bucketed nearest point, Newton on the
    # local quadratic interpolant) locates points exactly where the oracle does
    from oracle import geometry
    exe, env = harness
    fs = (1.4, 1.0, 0.0, 1.0)
    if kind == "annulus":
        p = W.grid_patch(W.annulus_map(0.0, 0.0, 0.5, 1.5, 0.15, 0.3), 96, 24,
                         (W.PERIODIC, W.PERIODIC, W.DIRICHLET, W.DIRICHLET), (fs,) * 4, periodic1=True)
    elif kind == "bulged_box":
        p = W.grid_patch(W.affine_map(-1.0, 2.0, -0.5, 1.0, bump=0.05), 61, 33, (W.DIRICHLET,) * 4, (fs,) * 4)
    else:  # a long thin diagonal strip: its bounding box is large against its spacings
        def strip(a, b):
            return (10.0 * a + 0.02 * b, 10.0 * a - 0.02 * b, 10.0 + 0 * a, 0.02 + 0 * a, 10.0 + 0 * a,
                    -0.02 + 0 * a)
        p = W.grid_patch(strip, 2000, 4, (W.DIRICHLET,) * 4, (fs,) * 4)
    g = geometry.PatchGeo(p, W.Params(d=5, C0=27, c_policy=2))
    rng = np.random.default_rng(4)
    x0, x1, y0, y1 = g.bbox()
    wx, wy = x1 - x0, y1 - y0
    xq = np.concatenate([rng.uniform(x0 - 0.1 * wx, x1 + 0.1 * wx, 400), g.x.ravel()[::37]])
    yq = np.concatenate([rng.uniform(y0 - 0.1 * wy, y1 + 0.1 * wy, 400), g.y.ravel()[::37]])
    hhat, htil, s1, s2 = _run_grid(exe, env, str(tmp_path), p, xq, yq)
    assert abs(hhat - g.hhat) <= 1e-15 * g.hhat and abs(htil - g.htil) <= 1e-15 * g.htil
    o1, o2 = g.frac_index(xq, yq)
    found_o, found_h = o1 > -1e8, s1 > -1e8
    assert np.array_equal(found_o, found_h)
    assert found_o.sum() > 20
    d1 = s1[found_o] - o1[found_o]
    if g.periodic1:
        d1 = np.mod(d1 + 0.5 * g.n1, g.n1) - 0.5 * g.n1
    assert np.abs(d1).max() < 1e-10 and np.abs(s2[found_o] - o2[found_o]).max() < 1e-10
    assert np.array_equal(g.contains(o1, o2), g.contains(s1, s2))


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_host_continuation_length_matches_the_oracle(harness, policy):
    # both sides implement the C rules (the paper leaves C free, Sec. 2.2) independently
    exe, env = harness
    lo, hi = F.table_range(5)
    r = subprocess.run([exe, "policy", "27", str(policy), str(hi), "10", "2100"], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    got = dict(tuple(map(int, ln.split())) for ln in r.stdout.splitlines())
    bad = [(N, C, F.choose_C(N, 27, policy, 5)) for N, C in got.items() if C != F.choose_C(N, 27, policy, 5)]
    assert not bad, bad[:10]


@pytest.mark.parametrize("d", [3, 4, 5, 6])
def test_host_adiabatic_weights_match_the_oracle(harness, d):
    from oracle import solver as S
    exe, env = harness
    r = subprocess.run([exe, "adw", str(d)], capture_output=True, text=True, env=env, timeout=60)
    assert r.returncode == 0, r.stderr
    got = np.array([float(v) for v in r.stdout.split()])
    ref = np.array([float(v) for v in S.adiabatic_weights(d)])
    assert got.shape == ref.shape and np.abs(got - ref).max() <= 1e-15 * np.abs(ref).max()


def _patches_for_geometry():
    w = W.small_multipatch()
    wc = W.small_multipatch_grid(curved=True)
    st = W.small_multipatch_stype()
    m25 = W.cyl_m25_32()
    holed = [p for p in m25.patches[1:] if p.hole[2] > 0 and 0 < int(
        np.sum(np.hypot(*W.patch_xy(p)) < p.hole[2])) < p.npts][:2]
    return {"ogrid": w.patches[0], "box_hole": w.patches[1], "grid_annulus": wc.patches[0],
            "grid_bulged_hole": wc.patches[2], "s_type_arc": st.patches[0], "m25_holed_a": holed[0],
            "m25_holed_b": holed[1]}


@pytest.mark.parametrize("name", list(_patches_for_geometry().keys()))
def test_host_patch_geometry_matches_the_oracle(harness, tmp_path, name):
    # blanking, the fringe/depth distances (eq. fringe_region), receivers, generating
    # points and no-derivative points of the library's build_patch against the oracle's
    from oracle import geometry
    exe, env = harness
    p = _patches_for_geometry()[name]
    fin, fout = os.path.join(str(tmp_path), "p.bin"), os.path.join(str(tmp_path), "po.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("<iii", p.kind, p.n1, p.n2))
        f.write(struct.pack("<4d", *p.geom))
        f.write(struct.pack("<4i", *p.side))
        f.write(struct.pack("<3d", *p.hole))
        if p.kind == W.GRID:
            f.write(np.ascontiguousarray(p.x, dtype=np.float64).tobytes())
            f.write(np.ascontiguousarray(p.y, dtype=np.float64).tobytes())
    r = subprocess.run([exe, "patch", fin, fout], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    raw = open(fout, "rb").read()
    N = p.n1 * p.n2
    hhat, htil = struct.unpack_from("<2d", raw, 0)
    off = 16
    arrs = {}
    for k in ("blank", "receiver", "gen", "nodiff"):
        arrs[k] = np.frombuffer(raw, dtype=np.uint8, count=N, offset=off).reshape(p.n2, p.n1).astype(bool)
        off += N
    depth = np.frombuffer(raw, dtype=np.int32, count=N, offset=off).reshape(p.n2, p.n1)
    g = geometry.PatchGeo(p, W.Params(d=5, C0=27, c_policy=2))
    assert abs(hhat - g.hhat) <= 1e-14 * g.hhat and abs(htil - g.htil) <= 1e-14 * g.htil
    for k in ("blank", "receiver", "gen", "nodiff"):
        assert np.array_equal(arrs[k], getattr(g, k)), k
    nb = ~g.blank
    assert np.array_equal(depth[nb], g.depth[nb])
