"""The reference arm of bench.py (the CPU oracle, no GPU): one JSON line with the
contract's keys, on a bounded sample."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "small_multipatch"],
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "Euler RHS point-updates/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["higher_is_better"] is True and d["steps"] == 1


def test_reference_sample_is_bounded():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2506_16076_gb300 import workloads as W
    w = W.cyl_m25_32()
    ws = bench.oracle_sample_workload(w, 1, max_points=64000)
    assert len(ws.patches) == 1 and ws.patches[0].npts <= 64000
    big = bench.oracle_sample_workload(w, 1)
    assert big.patches[0].npts == max(p.npts for p in w.patches if p.kind == W.AFFINE)
