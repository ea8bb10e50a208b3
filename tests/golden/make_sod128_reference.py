"""Write the oracle's Sod shock-tube state after 100 steps (128 x 128, d = 5, C = 27).

Calls only oracle/ and the seeded input generators: the stored array is the oracle's
result, computed once on a host whose long double is fast, so that the GPU parity test
of the 100-step run does not recompute it (the oracle's extended-precision FFT is slow
where long double is emulated in software). Run from the repository root:

    python -m tests.golden.make_sod128_reference
"""
import os

import numpy as np

from oracle import solver as S
from paper_2506_16076_gb300 import workloads as W

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sod128_100steps.npz")
NSTEPS = 100


def compute(nsteps=NSTEPS):
    w = W.sod128(128)
    sv = S.Solver(w)
    st = S.smear_initial(sv, W.initial_state(w), 0.5)
    dts = []
    for n in range(nsteps):
        st = sv.step(st, n)
        dts.append(sv.last_dt)
    return st[0], np.array(dts)


if __name__ == "__main__":
    state, dts = compute()
    np.savez_compressed(OUT, state=state, dt=dts, nsteps=NSTEPS)
    print(OUT, os.path.getsize(OUT), "bytes")
