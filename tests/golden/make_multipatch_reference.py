"""Write the oracle's state after 100 steps of the curved multi-patch workload.

small_multipatch_grid: a stretched, twisted annulus around the cylinder (no-slip adiabatic
wall) and four bulged boxes cut by the hole, all given as GRID patches, from the seeded
smooth state W.random_smooth_state(seed=29, amp=0.05); Algorithm 1 with the per-step
filter and the time step of eq. CFL, and the viscosity of the first step (computed by the
oracle from the projected initial state, then held fixed): over 100 steps the smoothness
classifier meets decisions within the FP32 rounding of its logits, where either class is
a correct result, so the long run fixes the viscosity and the per-step classifier and
viscosity are checked elsewhere. Calls only oracle/ and the seeded input generators;
computed once on a host whose long double is fast, so that the GPU parity test of the
100-step run does not recompute it. Run from the repository root:

    python -m tests.golden.make_multipatch_reference
"""
import os

import numpy as np

from oracle import solver as S, viscosity as V
from paper_2506_16076_gb300 import workloads as W

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "multipatch_grid_100steps.npz")
NSTEPS = 100
SEED, AMP = 29, 0.05


def compute(nsteps=NSTEPS):
    w = W.small_multipatch_grid()
    sv = S.Solver(w)
    st = W.random_smooth_state(w, seed=SEED, amp=AMP)
    mu0 = V.viscosity(sv.geos, sv.sb, sv.project([a.copy() for a in st]), w.params)[0]
    dts = []
    for n in range(nsteps):
        st = sv.step(st, n, mu=mu0)
        dts.append(sv.last_dt)
    return W.flatten(st), np.array(dts), np.concatenate([m.ravel() for m in mu0])


if __name__ == "__main__":
    state, dts, mu0 = compute()
    np.savez_compressed(OUT, state=state, dt=dts, mu=mu0, nsteps=NSTEPS, seed=SEED, amp=AMP)
    print(OUT, os.path.getsize(OUT), "bytes")
