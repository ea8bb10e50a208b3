"""Generate the FC-Gram continuation matrices (Q, A_l, A_r) used by the FC method.

Method data, produced once and stored on disc as the paper prescribes for these
matrices (Sec. 2.2, eq. (continuation)): "computed once and stored on disc".
The paper does not print the construction (it cites the FC-Gram literature), so
this script implements the classical FC-Gram recipe from the mathematics:

* Q: the d x d orthogonal factor of the QR decomposition of the Vandermonde
  matrix on the d equispaced matching points t = 0..d-1 (grid units), i.e. the
  Gram polynomial basis of degree < d, with R's diagonal made positive.
* For every Gram polynomial g_j (continuous, degree j), a "blend-to-zero"
  trigonometric polynomial T(t) of period P and K modes is fitted, in the
  least-squares sense on an oversampled set, to g_j on the matching interval
  [0, d-1] and to zero on the interval of Z points where the opposite end's
  matching points sit once the continued line wraps around. The fit is solved
  by a truncated SVD in mpmath at 40 decimal digits.
* A_r[c, j] = T_j^right(d + c): the C continuation points that follow the last
  data point F_{N-1}; A_l[c, j] = T_j^left(c - C): the same points seen from the
  first data point F_0 (they precede it periodically).

With these, eq. (continuation) reads  F^c = [F ; A_l Q^T F_l + A_r Q^T F_r].

Output: fc_tables_d{d}.txt, one block per C in [C_MIN, C_MAX]. Each block is
"d <d>", "C <C>", then the matrices Q (d rows), AL (C rows), AR (C rows) with
17 significant digits. The fit parameters are written in each block's header.
Run:  python gen_fc_tables.py   (needs mpmath; about a minute on 8 cores)
"""
import math
import os
import sys
from multiprocessing import get_context

import mpmath as mp

C_MIN, C_MAX = 27, 71
DPS = 40


def fit_params(d, C):
    Z = d if d > 2 else 2
    P = round(1.73 * (C + d + Z))
    K = round(0.36 * P)
    nos = 40 if d == 2 else max(10, math.ceil(1.75 * (2 * K + 1) / (d + Z - 2)))
    return Z, P, K, nos


def gram_basis(d):
    V = mp.matrix(d, d)
    for i in range(d):
        for k in range(d):
            V[i, k] = mp.mpf(i) ** k
    Q, R = mp.qr(V)
    for j in range(d):
        if R[j, j] < 0:
            for i in range(d):
                Q[i, j] = -Q[i, j]
            for k in range(d):
                R[j, k] = -R[j, k]
    return Q, R ** -1


def trig_row(t, K, P):
    row = [mp.mpf(1)]
    for k in range(1, K + 1):
        a = 2 * mp.pi * k * t / P
        row += [mp.cos(a), mp.sin(a)]
    return row


def blend(d, C, side):
    Z, P, K, nos = fit_params(d, C)
    _, Rinv = gram_basis(d)
    match = [mp.mpf(m) / nos for m in range((d - 1) * nos + 1)]
    if side == "r":
        zero = [d + C + mp.mpf(m) / nos for m in range((Z - 1) * nos + 1)]
        evalpts = [mp.mpf(d + c) for c in range(C)]
    else:
        zero = [-(C + Z) + mp.mpf(m) / nos for m in range((Z - 1) * nos + 1)]
        evalpts = [mp.mpf(c - C) for c in range(C)]
    pts = match + zero
    ncol = 2 * K + 1
    A = mp.matrix([trig_row(t, K, P) for t in pts])
    U, S, V = mp.svd_r(A)
    cut = S[0] * mp.mpf(10) ** (-(DPS - 8))
    E = mp.matrix([trig_row(t, K, P) for t in evalpts])
    out = [[None] * d for _ in range(C)]
    worst = mp.mpf(0)
    for j in range(d):
        b = [mp.fsum(t ** k * Rinv[k, j] for k in range(d)) for t in match] + [mp.mpf(0)] * len(zero)
        x = [mp.mpf(0)] * ncol
        for s in range(min(A.rows, ncol)):
            if S[s] < cut:
                continue
            ub = mp.fsum(U[i, s] * b[i] for i in range(A.rows)) / S[s]
            for k in range(ncol):
                x[k] += V[s, k] * ub
        res = max(abs(mp.fsum(A[i, k] * x[k] for k in range(ncol)) - b[i]) for i in range(A.rows))
        worst = max(worst, res)
        for c in range(C):
            out[c][j] = mp.fsum(E[c, k] * x[k] for k in range(ncol))
    return out, worst


def one_block(args):
    d, C = args
    mp.mp.dps = DPS
    Q, _ = gram_basis(d)
    AL, rl = blend(d, C, "l")
    AR, rr = blend(d, C, "r")
    Z, P, K, nos = fit_params(d, C)
    lines = [f"# fit: Z={Z} P={P} K={K} oversampling={nos} dps={DPS} max_fit_residual={float(max(rl, rr)):.3e}",
             f"d {d}", f"C {C}", "Q"]
    fmt = lambda v: repr(float(v))
    lines += [" ".join(fmt(Q[i, j]) for j in range(d)) for i in range(d)]
    lines.append("AL")
    lines += [" ".join(fmt(v) for v in row) for row in AL]
    lines.append("AR")
    lines += [" ".join(fmt(v) for v in row) for row in AR]
    return "\n".join(lines)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    ds = [int(a) for a in sys.argv[1:]] or [5, 2]
    with get_context("spawn").Pool() as pool:
        for d in ds:
            blocks = pool.map(one_block, [(d, C) for C in range(C_MIN, C_MAX + 1)])
            path = os.path.join(here, f"fc_tables_d{d}.txt")
            with open(path, "w") as f:
                f.write(f"# FC-Gram continuation tables, d={d}, C={C_MIN}..{C_MAX}; written by gen_fc_tables.py\n")
                f.write("\n".join(blocks) + "\nend\n")
            print("wrote", path)


if __name__ == "__main__":
    main()
