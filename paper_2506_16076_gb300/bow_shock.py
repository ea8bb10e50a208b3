"""Supersonic flow past the cylinder: stagnation pressure and bow-shock stand-off.

Runs the Mach-M cylinder workload (the 512 x 96 O-grid + 4 x 4 Cartesian patches of
cyl_m3, free stream (1.4, M, 0, 1), no-slip adiabatic wall) through fc_rk_step and,
every `--report-every` steps, prints one JSON line with the simulated time, the wall
pressure at the front stagnation point, the stand-off distance d0 of the bow shock
along the stagnation line, and their reference values: the Rayleigh pitot pressure
behind a normal shock and the experimental fit d0 / (2 R) = 0.193 exp(4.67 / M^2) the
paper validates against (Sec. 7, eq. cylinder_bow).

  python -m paper_2506_16076_gb300.bow_shock --mach 3 --steps 40000 --report-every 5000
  python -m paper_2506_16076_gb300.bow_shock --workload cyl_m25_32 --steps 8000 --report-every 1000
  python -m paper_2506_16076_gb300.bow_shock --mach 25 --wall-form product --steps 60000

A uniform hypersonic stream switched on against the no-slip wall loses positivity in the
first filtered steps, so from Mach 10 on (or with --potential-start) the run starts as
the Mach-25 workloads do: free-stream density and pressure with the potential-flow
velocity around the cylinder, damped to zero in a 0.05-thick layer at the wall.

The shock is located on the O-grid's radial line through the front stagnation point
(angle pi): the outermost radius where the density exceeds the midpoint between the
free-stream density and the line's maximum.
"""
import argparse
import dataclasses
import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

GAMMA = 1.4


def pitot_pressure(M, p_inf=1.0, gamma=GAMMA):
    """Stagnation pressure behind a normal shock (Rayleigh pitot formula)."""
    g = gamma
    a = ((g + 1) ** 2 * M * M / (4 * g * M * M - 2 * (g - 1))) ** (g / (g - 1))
    return p_inf * a * (1 - g + 2 * g * M * M) / (g + 1)


def billig_standoff(M, lam1=0.193, lam2=4.67):
    """d0 / (2 R) of the experimental fit for cylinders (Sec. 7, eq. cylinder_bow)."""
    return lam1 * math.exp(lam2 / (M * M))


def shock_radius(r, rho, rho_inf):
    """Outermost r with rho above the midpoint of rho_inf and max(rho); nan if none."""
    thr = 0.5 * (rho_inf + float(np.max(rho)))
    k = np.nonzero(rho > thr)[0]
    return float(r[k.max()]) if len(k) else float("nan")


def workload(mach, potential_start=False):
    from paper_2506_16076_gb300 import workloads as W
    w = W.cyl_m3()
    fs = (1.4, float(mach), 0.0, 1.0)
    pts = [dataclasses.replace(p, bc=(fs,) * 4) for p in w.patches]
    w = dataclasses.replace(w, name=f"cyl_m{mach:g}", patches=pts, freestream=fs)
    if potential_start:
        w = dataclasses.replace(w, init="potential",
                                extra={"cyl_radius": 0.5, "cutoff": 3.0, "wall_layer": 0.05})
    return w


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mach", type=float, default=3.0)
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--report-every", type=int, default=5000)
    ap.add_argument("--potential-start", action="store_true",
                    help="start from the potential flow with a no-slip wall layer (default from Mach 10 on)")
    ap.add_argument("--d", type=int, default=None,
                    help="FC order d of the continuation (the paper uses d = 2 throughout; default: the workload's)")
    ap.add_argument("--wall-form", choices=["flux", "product"], default="flux",
                    help="operator on the wall patch: the flux form, or the product-rule form of Remark adiabatic "
                         "(fc_params.wall_form = 1)")
    ap.add_argument("--workload", default=None,
                    help="a named workload with an O-grid around the cylinder (e.g. cyl_m25_32) instead of the "
                         "Mach-M cylinder on the 4 x 4 array")
    args = ap.parse_args()
    import torch
    from paper_2506_16076_gb300 import fcsdnn, workloads as W

    if args.workload:
        w = W.WORKLOADS[args.workload]()
        args.mach = float(np.hypot(w.freestream[1], w.freestream[2]) / math.sqrt(GAMMA * w.freestream[3] /
                                                                                w.freestream[0]))
    else:
        w = workload(args.mach, args.potential_start or args.mach >= 10.0)
    if args.d is not None:
        w = dataclasses.replace(w, params=dataclasses.replace(w.params, d=args.d))
    if args.wall_form == "product":
        w = dataclasses.replace(w, params=dataclasses.replace(w.params, wall_form=1))
    og = w.patches[0]
    assert og.kind == W.OGRID
    xc, yc, r0, r1 = og.geom
    R = r0
    ctx = fcsdnn.Context(w)
    e = torch.from_numpy(W.flatten(W.initial_state(w))).cuda()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.zeros(e.shape[1], dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    r = np.linspace(r0, r1, og.n2)
    i_front = og.n1 // 2  # angle pi: upstream of the cylinder
    t = 0.0
    dts = torch.zeros(args.report_every, dtype=torch.float64, device="cuda")
    for n in range(args.steps):
        with torch.cuda.stream(s):
            ctx.rk_step(e, dt, mu, fcsdnn.STEP_GRAPH | (fcsdnn.STEP_FILTER if n else 0))
            dts[n % args.report_every].copy_(dt[0])
        if (n + 1) % args.report_every == 0:
            s.synchronize()
            t += float(dts.sum())
            a = W.unflatten(e.cpu().numpy(), w)[0]
            rho = a[0][:, i_front]
            p = (GAMMA - 1.0) * (a[3][:, i_front] - 0.5 * (a[1][:, i_front] ** 2 + a[2][:, i_front] ** 2) / rho)
            rs = shock_radius(r, rho, w.freestream[0])
            status = ctx.sync_status(e)
            print(json.dumps({"step": n + 1, "t": round(t, 5), "status": status,
                              "p_stagnation_wall": round(float(p[0]), 4),
                              "p_pitot": round(pitot_pressure(args.mach, w.freestream[3]), 4),
                              "standoff_over_2R": round((rs - R) / (2 * R), 4),
                              "billig_fit": round(billig_standoff(args.mach), 4)}), flush=True)
            if status != 0:  # a non-finite or non-physical state: nothing further to measure
                break


if __name__ == "__main__":
    main()
