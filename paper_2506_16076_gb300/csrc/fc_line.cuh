// Per-line building blocks of the FC derivative and filter: in-place mixed-radix FFT
// stages in shared memory, FC-Gram continuation, spectral multipliers.
//
// Every function takes (lane, nl): lane index and lane count of the group that
// processes the line (a warp: nl = 32). Work is split with strided loops and all
// cross-lane exchange goes through shared memory separated by FC_SYNC(), so the
// functions have no intra-warp register dependencies.
#pragma once
#include <math.h>
#include <string.h>

#include "fc_internal.h"

#ifdef __CUDA_ARCH__
#define FC_SYNC() __syncwarp()
#else
#define FC_SYNC() \
  do {            \
  } while (0)
#endif
#define FC_HD __host__ __device__ __forceinline__

namespace fcx {

constexpr double TWO_PI = 6.283185307179586;

FC_HD double2 cpx(double x, double y) {
  double2 r;
  r.x = x;
  r.y = y;
  return r;
}
FC_HD double2 cadd(double2 a, double2 b) { return cpx(a.x + b.x, a.y + b.y); }
FC_HD double2 csub(double2 a, double2 b) { return cpx(a.x - b.x, a.y - b.y); }
FC_HD double2 cscl(double2 a, double s) { return cpx(a.x * s, a.y * s); }
FC_HD double2 cmul(double2 a, double2 w) { return cpx(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x)); }
// s i b with s = -1 (forward transform) or +1 (inverse transform)
template <bool INV>
FC_HD double2 mul_si(double2 b) {
  return INV ? cpx(-b.y, b.x) : cpx(b.y, -b.x);
}

// ---- small DFTs: y_q = sum_m x_m exp(s 2 pi i q m / R) ----
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  FC_HD static void run(double2* v) {
    double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  FC_HD static void run(double2* v) {
    double2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    double2 c = cadd(v[1], v[3]), d = mul_si<INV>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <bool INV>
struct Dft<8, INV> {
  FC_HD static void run(double2* v) {
    double2 e[4] = {v[0], v[2], v[4], v[6]};
    double2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    const double r = 0.7071067811865476;
    // w8^1 o1 = r a1, w8^3 o3 = r a3 with the sums below; r folded into the FMAs
    const double2 a1 = INV ? cpx(o[1].x - o[1].y, o[1].y + o[1].x)   // o1.x - s o1.y, o1.y + s o1.x
                           : cpx(o[1].x + o[1].y, o[1].y - o[1].x);
    const double2 a3 = INV ? cpx(-(o[3].x + o[3].y), o[3].x - o[3].y)  // -o3.x - s o3.y, -o3.y + s o3.x
                           : cpx(o[3].y - o[3].x, -(o[3].y + o[3].x));
    const double2 t2 = mul_si<INV>(o[2]);  // w8^2 o2
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cpx(fma(r, a1.x, e[1].x), fma(r, a1.y, e[1].y));
    v[5] = cpx(fma(-r, a1.x, e[1].x), fma(-r, a1.y, e[1].y));
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = cpx(fma(r, a3.x, e[3].x), fma(r, a3.y, e[3].y));
    v[7] = cpx(fma(-r, a3.x, e[3].x), fma(-r, a3.y, e[3].y));
  }
};

// odd R: pairs (x_m, x_{R-m}); y_q = x0 + sum_m cos(2 pi q m/R) a_m + s i sum_m sin(2 pi q m/R) b_m
template <int R>
struct OddConst;
template <>
struct OddConst<3> {
  FC_HD static double c(int k) { return -0.5; }
  FC_HD static double s(int k) { return 0.8660254037844387; }
};
template <>
struct OddConst<5> {
  FC_HD static double c(int k) { return k == 1 ? 0.30901699437494745 : -0.8090169943749473; }
  FC_HD static double s(int k) { return k == 1 ? 0.9510565162951535 : 0.5877852522924732; }
};
template <>
struct OddConst<7> {
  FC_HD static double c(int k) {
    return k == 1 ? 0.6234898018587336 : (k == 2 ? -0.22252093395631434 : -0.900968867902419);
  }
  FC_HD static double s(int k) {
    return k == 1 ? 0.7818314824680298 : (k == 2 ? 0.9749279121818236 : 0.43388373911755823);
  }
};

template <int R, bool INV>
struct DftOdd {
  FC_HD static void run(double2* v) {
    constexpr int H = (R - 1) / 2;
    double2 a[H], b[H];
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      a[m - 1] = cadd(v[m], v[R - m]);
      b[m - 1] = csub(v[m], v[R - m]);
    }
    double2 x0 = v[0];
    double2 y0 = x0;
#pragma unroll
    for (int m = 0; m < H; ++m) y0 = cadd(y0, a[m]);
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      double2 t = x0;
      double2 u;
#pragma unroll
      for (int m = 1; m <= H; ++m) {
        int km = (q * m) % R;  // angle index in 1..R-1
        double cc, ss;
        if (km <= H) {
          cc = OddConst<R>::c(km);
          ss = OddConst<R>::s(km);
        } else {
          cc = OddConst<R>::c(R - km);
          ss = -OddConst<R>::s(R - km);
        }
        t = cpx(fma(cc, a[m - 1].x, t.x), fma(cc, a[m - 1].y, t.y));
        u = (m == 1) ? cpx(ss * b[0].x, ss * b[0].y) : cpx(fma(ss, b[m - 1].x, u.x), fma(ss, b[m - 1].y, u.y));
      }
      double2 iu = mul_si<INV>(u);
      v[q] = cadd(t, iu);
      v[R - q] = csub(t, iu);
    }
    v[0] = y0;
  }
};
template <bool INV>
struct Dft<3, INV> : DftOdd<3, INV> {};
template <bool INV>
struct Dft<5, INV> : DftOdd<5, INV> {};
template <bool INV>
struct Dft<7, INV> : DftOdd<7, INV> {};

// ---- in-place transforms (one buffer): decimation in frequency forward, decimation in
// time inverse. With stage radices R_0..R_{m-1} and spans L/(R_0..R_s), the forward
// transform leaves mode k at slot p where p = sum_s d_s L/(R_0..R_s) and
// k = sum_s d_s R_0..R_{s-1} (digit-reversed order, table Plan::rev); the inverse
// transform takes that order back to natural order, so no permutation pass is needed
// and spectral multipliers look up each slot's mode number.
// spectral multipliers folded into the last stage of a forward transform (span 1, where
// the R outputs of butterfly bb land in slots bb R + r), from per-slot tables that also
// hold the transform's pending factors (fc_tables.h): MUL_DERIV: i fac dmul[slot] (eq.
// fc_der, dmul = k P), MUL_FILTER: sigp[slot] (eq. filtering, sigp = sigma(2k/L)/L P)
enum { MUL_NONE = 0, MUL_DERIV = 1, MUL_FILTER = 2 };
template <int MUL>
FC_HD double2 apply_mult(double2 z, double m, double fac) {
  if (MUL == MUL_DERIV) {
    const double f = fac * m;
    return cpx(-f * z.y, f * z.x);
  }
  return cscl(z, m);
}
template <int MUL>
FC_HD double2 apply_out(double2 z, const double* __restrict__ mt, int slot, double fac) {
  return MUL == MUL_NONE ? z : apply_mult<MUL>(z, mt[slot], fac);
}

// psc (forward only, may be null): pending factors of the inputs, multiplied in first;
// mt: the multiplier table of MUL
template <int R, bool INV, bool DIF, int MUL = MUL_NONE>
FC_HD void inplace_stage_r(double2* a, int L, int span, int nseq, const double2* __restrict__ tw, int lane, int nl,
                           double fac = 0.0, const double* __restrict__ mt = nullptr,
                           const double* __restrict__ psc = nullptr) {
  const int nbf = L / R;
  const int tws = L / (R * span);
  for (int idx = lane; idx < nseq * nbf; idx += nl) {
    const int s = idx / nbf;
    const int t = idx - s * nbf;
    const int bb = t / span;
    const int j = t - bb * span;
    double2* x = a + s * L + bb * R * span + j;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[r * span];
    if (DIF && psc) {
      const double* ps = psc + bb * R * span + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = cscl(v[r], ps[r * span]);
    }
    if (!DIF && j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        double2 w = tw[q * j * tws];
        if (INV) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    Dft<R, INV>::run(v);
    if (DIF && j != 0) {
#pragma unroll
      for (int q = 1; q < R; ++q) {
        double2 w = tw[q * j * tws];
        if (INV) w.y = -w.y;
        v[q] = cmul(v[q], w);
      }
    }
    if (MUL != MUL_NONE) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = apply_mult<MUL>(v[r], mt[bb * R + r], fac);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) x[r * span] = v[r];
  }
}

// ---- FMA-form inverse (decimation in time) stages of radix 2, 4, 8 (span > 1): each
// twiddled input w_q x_q is S_q u_q with u_q = x'_q + i t_q x'_q (x' = x, or i x when
// the record's flag bit q-1 is set: the ratio form of w_q in the plan's records), two
// FMAs, and the real S_q (or its ratio to a partner's) multiplies inside the butterfly's
// FMAs, so a radix-4 butterfly with twiddles is 22 FMAs instead of 16 adds and 3
// complex products (28), a radix-8 one 62 FMAs and 4 adds instead of 80 operations. The
// records (Builder::fma_tables) hold t_q, the flags and the scale ratios per offset j.
FC_HD long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long v;
  memcpy(&v, &x, sizeof(v));
  return v;
#endif
}
FC_HD double2 rot_u(double2 b, double t, bool f) {
  const double bx = f ? -b.y : b.x, by = f ? b.x : b.y;
  return cpx(fma(-t, by, bx), fma(t, bx, by));
}
FC_HD double2 fma2(double s, double2 u, double2 a) { return cpx(fma(s, u.x, a.x), fma(s, u.y, a.y)); }
// a + s i u and a - s i u
FC_HD double2 fma2_pi(double s, double2 u, double2 a) { return cpx(fma(-s, u.y, a.x), fma(s, u.x, a.y)); }
FC_HD double2 fma2_mi(double s, double2 u, double2 a) { return cpx(fma(s, u.y, a.x), fma(-s, u.x, a.y)); }

template <int R>
FC_HD void inplace_stage_dit_fma(double2* a, int L, int span, int nseq, const double2* __restrict__ rec, int lane,
                                 int nl) {
  constexpr int RS = R == 2 ? 2 : (R == 4 ? 4 : 8);  // record length in double2
  const int nbf = L / R;
  for (int idx = lane; idx < nseq * nbf; idx += nl) {
    const int s = idx / nbf;
    const int t = idx - s * nbf;
    const int bb = t / span;
    const int j = t - bb * span;
    double2* x = a + s * L + bb * R * span + j;
    const double2* q = rec + j * RS;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[r * span];
    const double2 h0 = q[0];
    const long long fl = dbits(h0.x);
    if (R == 2) {
      const double2 u1 = rot_u(v[1], h0.y, fl & 1);
      const double S1 = q[1].x;
      x[0] = fma2(S1, u1, v[0]);
      x[span] = fma2(-S1, u1, v[0]);
    } else if (R == 4) {
      const double2 h1 = q[1], h2 = q[2], h3 = q[3];
      const double2 u1 = rot_u(v[1], h0.y, fl & 1), u2 = rot_u(v[2], h1.x, fl & 2), u3 = rot_u(v[3], h1.y, fl & 4);
      const double S2 = h2.x, S1 = h2.y, rho = h3.x;
      const double2 A = fma2(S2, u2, v[0]), B = fma2(-S2, u2, v[0]);
      const double2 p = fma2(rho, u3, u1), m = fma2(-rho, u3, u1);  // (v1 + v3) / S1, (v1 - v3) / S1
      x[0] = fma2(S1, p, A);
      x[2 * span] = fma2(-S1, p, A);
      x[span] = fma2_pi(S1, m, B);
      x[3 * span] = fma2_mi(S1, m, B);
    } else {
      const double2 h1 = q[1], h2 = q[2], h3 = q[3], h4 = q[4], h5 = q[5], h6 = q[6], h7 = q[7];
      // even half: DFT4 of (x0, S2 u2, S4 u4, S6 u6)
      const double2 u2 = rot_u(v[2], h1.x, fl & 2), u4 = rot_u(v[4], h2.x, fl & 8), u6 = rot_u(v[6], h3.x, fl & 32);
      const double S4 = h4.x, S2 = h4.y, r62 = h5.x;
      const double2 A = fma2(S4, u4, v[0]), B = fma2(-S4, u4, v[0]);
      const double2 p = fma2(r62, u6, u2), m = fma2(-r62, u6, u2);
      const double2 E0 = fma2(S2, p, A), E2 = fma2(-S2, p, A), E1 = fma2_pi(S2, m, B), E3 = fma2_mi(S2, m, B);
      // odd half: DFT4 of (S1 u1, S3 u3, S5 u5, S7 u7) / S1
      const double2 u1 = rot_u(v[1], h0.y, fl & 1), u3 = rot_u(v[3], h1.y, fl & 4);
      const double2 u5 = rot_u(v[5], h2.y, fl & 16), u7 = rot_u(v[7], h3.y, fl & 64);
      const double r51 = h5.y, r73 = h6.x, r31 = h6.y, S1 = h7.x, S1r = h7.y;
      const double2 al = fma2(r51, u5, u1), be = fma2(-r51, u5, u1);
      const double2 ga = fma2(r73, u7, u3), de = fma2(-r73, u7, u3);
      const double2 o0 = fma2(r31, ga, al), o2 = fma2(-r31, ga, al);
      const double2 o1 = fma2_pi(r31, de, be), o3 = fma2_mi(r31, de, be);
      // y_k = E_k + W^k S1 o_k, y_{k+4} = E_k - W^k S1 o_k, W = exp(2 pi i / 8)
      x[0] = fma2(S1, o0, E0);
      x[4 * span] = fma2(-S1, o0, E0);
      x[2 * span] = fma2_pi(S1, o2, E2);
      x[6 * span] = fma2_mi(S1, o2, E2);
      const double2 w1 = cpx(o1.x - o1.y, o1.x + o1.y), w3 = cpx(-(o3.x + o3.y), o3.x - o3.y);
      x[span] = fma2(S1r, w1, E1);
      x[5 * span] = fma2(-S1r, w1, E1);
      x[3 * span] = fma2(S1r, w3, E3);
      x[7 * span] = fma2(-S1r, w3, E3);
    }
  }
}

// FMA-form forward (decimation in frequency) stage of radix 2, 4, 8: the inputs carry
// pending real factors, combined through the ratios of the butterfly's record rat (per
// butterfly); the outputs keep the factor of the first input; outputs 1..R-1 are then
// rotated by u = y' + i t y' with the rotation record rot (per offset j, span > 1) and
// their factor multiplied by the twiddle's S (host-side bookkeeping, fc_tables.h). A
// radix-4 butterfly with twiddles is 22 FMAs instead of 28 operations. In the last stage
// (span 1) the multiplier table mt applies MUL with the final factors folded in.
template <int R, int MUL>
FC_HD void inplace_stage_dif_fma(double2* a, int L, int span, int nseq, const double2* __restrict__ rot,
                                 const double2* __restrict__ rat, int lane, int nl, double fac,
                                 const double* __restrict__ mt) {
  constexpr int RH = R / 2;  // rotation and ratio record lengths in double2
  const int nbf = L / R;
  for (int idx = lane; idx < nseq * nbf; idx += nl) {
    const int s = idx / nbf;
    const int t = idx - s * nbf;
    const int bb = t / span;
    const int j = t - bb * span;
    double2* x = a + s * L + bb * R * span + j;
    const double2* g = rat + t * RH;
    double2 v[R], y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[r * span];
    if (R == 2) {
      const double r10 = g[0].x;
      y[0] = fma2(r10, v[1], v[0]);
      y[1] = fma2(-r10, v[1], v[0]);
    } else if (R == 4) {
      const double2 g0 = g[0];
      const double s10 = g[1].x;
      const double2 A = fma2(g0.x, v[2], v[0]), B = fma2(-g0.x, v[2], v[0]);
      const double2 C = fma2(g0.y, v[3], v[1]), M = fma2(-g0.y, v[3], v[1]);
      y[0] = fma2(s10, C, A);
      y[2] = fma2(-s10, C, A);
      y[1] = fma2_mi(s10, M, B);
      y[3] = fma2_pi(s10, M, B);
    } else {
      const double2 g0 = g[0], g1 = g[1], g2 = g[2], g3 = g[3];
      // even half: DFT4 of (v0, v2, v4, v6) with factors relative to v0's
      const double2 A = fma2(g0.x, v[4], v[0]), B = fma2(-g0.x, v[4], v[0]);
      const double2 C = fma2(g0.y, v[6], v[2]), M = fma2(-g0.y, v[6], v[2]);
      const double2 E0 = fma2(g1.x, C, A), E2 = fma2(-g1.x, C, A);
      const double2 E1 = fma2_mi(g1.x, M, B), E3 = fma2_pi(g1.x, M, B);
      // odd half: DFT4 of (v1, v3, v5, v7) relative to v1's factor
      const double2 al = fma2(g1.y, v[5], v[1]), be = fma2(-g1.y, v[5], v[1]);
      const double2 ga = fma2(g2.x, v[7], v[3]), de = fma2(-g2.x, v[7], v[3]);
      const double2 o0 = fma2(g2.y, ga, al), o2 = fma2(-g2.y, ga, al);
      const double2 o1 = fma2_mi(g2.y, de, be), o3 = fma2_pi(g2.y, de, be);
      // y_k = E_k + W^k (P1/P0) o_k, y_{k+4} = E_k - W^k (P1/P0) o_k, W = exp(-2 pi i / 8)
      const double tau = g3.x, taur = g3.y;
      y[0] = fma2(tau, o0, E0);
      y[4] = fma2(-tau, o0, E0);
      y[2] = fma2_mi(tau, o2, E2);
      y[6] = fma2_pi(tau, o2, E2);
      const double2 w1 = cpx(o1.x + o1.y, o1.y - o1.x), w3 = cpx(o3.y - o3.x, -(o3.x + o3.y));
      y[1] = fma2(taur, w1, E1);
      y[5] = fma2(-taur, w1, E1);
      y[3] = fma2(taur, w3, E3);
      y[7] = fma2(-taur, w3, E3);
    }
    if (span > 1) {
      const double2* h = rot + j * RH;
      const long long fl = dbits(h[0].x);
      y[1] = rot_u(y[1], h[0].y, fl & 1);
#pragma unroll
      for (int q = 2; q < R; q += 2) {
        const double2 hq = h[q / 2];
        y[q] = rot_u(y[q], hq.x, (fl >> (q - 1)) & 1);
        y[q + 1] = rot_u(y[q + 1], hq.y, (fl >> q) & 1);
      }
    }
    if (MUL != MUL_NONE) {
#pragma unroll
      for (int r = 0; r < R; ++r) y[r] = apply_mult<MUL>(y[r], mt[bb * R + r], fac);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) x[r * span] = y[r];
  }
}

// last forward stage (span 1) of odd radix R with the inputs' pending factors folded
// into the butterfly (records of fc_tables.h): the DftOdd computation with every
// coefficient multiplied by the factor ratios, the outputs left with the first input's
// factor (in the multiplier table mt)
template <int R, int MUL>
FC_HD void inplace_stage_odd_fold(double2* a, int L, int nseq, const double2* __restrict__ rec, int lane, int nl,
                                  double fac, const double* __restrict__ mt) {
  constexpr int H = (R - 1) / 2;
  constexpr int RS2 = (2 * H + 2 * H * H + 1) / 2;  // record length in double2
  const int nbf = L / R;
  for (int idx = lane; idx < nseq * nbf; idx += nl) {
    const int s = idx / nbf;
    const int bb = idx - s * nbf;
    double2* x = a + s * L + bb * R;
    const double* c = (const double*)(rec + bb * RS2);
    double2 v[R], ap[H], bp[H];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[r];
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      ap[m - 1] = fma2(c[m - 1], v[R - m], v[m]);
      bp[m - 1] = fma2(-c[m - 1], v[R - m], v[m]);
    }
    double2 y0 = v[0];
#pragma unroll
    for (int m = 0; m < H; ++m) y0 = fma2(c[H + m], ap[m], y0);
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      double2 t = v[0], u;
#pragma unroll
      for (int m = 0; m < H; ++m) {
        t = fma2(c[2 * H + (q - 1) * H + m], ap[m], t);
        const double sq = c[2 * H + H * H + (q - 1) * H + m];
        u = m == 0 ? cscl(bp[0], sq) : fma2(sq, bp[m], u);
      }
      const double2 iu = mul_si<false>(u);
      x[q] = apply_out<MUL>(cadd(t, iu), mt, bb * R + q, fac);
      x[R - q] = apply_out<MUL>(csub(t, iu), mt, bb * R + R - q, fac);
    }
    x[0] = apply_out<MUL>(y0, mt, bb * R, fac);
  }
}

template <bool INV, bool DIF>
FC_HD void inplace_stage_gen(double2* a, int L, int span, int R, int nseq, const double2* __restrict__ tw, int lane,
                             int nl, const double* __restrict__ psc = nullptr) {
  const int nbf = L / R;
  const int tws = L / (R * span);
  const int wr = L / R;  // exp(s 2 pi i / R) = tw[wr]
  for (int idx = lane; idx < nseq * nbf; idx += nl) {
    const int s = idx / nbf;
    const int t = idx - s * nbf;
    const int bb = t / span;
    const int j = t - bb * span;
    double2* x = a + s * L + bb * R * span + j;
    double2 v[MAX_GENERIC_RADIX], y[MAX_GENERIC_RADIX];
    for (int r = 0; r < R; ++r) {
      v[r] = x[r * span];
      if (DIF && psc) v[r] = cscl(v[r], psc[bb * R * span + r * span + j]);
      if (!DIF && j != 0 && r) {
        double2 w = tw[r * j * tws];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    for (int q = 0; q < R; ++q) {
      double ax = 0.0, ay = 0.0;
      int e = 0;
      for (int m = 0; m < R; ++m) {
        double2 w = tw[e * wr];
        if (INV) w.y = -w.y;
        ax = fma(v[m].x, w.x, fma(-v[m].y, w.y, ax));
        ay = fma(v[m].x, w.y, fma(v[m].y, w.x, ay));
        e += q;
        if (e >= R) e -= R;
      }
      y[q] = cpx(ax, ay);
    }
    for (int q = 0; q < R; ++q) {
      double2 o = y[q];
      if (DIF && j != 0 && q) {
        double2 w = tw[q * j * tws];
        if (INV) w.y = -w.y;
        o = cmul(o, w);
      }
      x[q * span] = o;
    }
  }
}

template <int MUL>
FC_HD void fft_forward_mul(double2* a, const Plan& P, int nseq, const double2* twpool, const double* rp, double fac,
                           int lane, int nl);

// forward (DIF) or inverse (DIT) in-place transform of nseq sequences of length P.L in a.
// The forward transform's outputs carry the plan's per-slot pending factors (fc_tables.h):
// its consumers multiply through the per-slot tables (mul_deriv_slot, mul_filter_slot).
template <bool INV>
FC_HD void fft_inplace(double2* a, const Plan& P, int nseq, const double2* twpool, const double* rp, int lane,
                       int nl) {
  const double2* tw = twpool + P.tw;
  const int L = P.L;
  if (!INV) {
    fft_forward_mul<MUL_NONE>(a, P, nseq, twpool, rp, 0.0, lane, nl);
  } else {
    int span = 1;
    const double2* rec = twpool + P.fmd;
    for (int st = P.nst - 1; st >= 0; --st) {
      const int R = P.rad[st];
      if (span > 1 && (R == 2 || R == 4 || R == 8)) {
        if (R == 2)
          inplace_stage_dit_fma<2>(a, L, span, nseq, rec, lane, nl);
        else if (R == 4)
          inplace_stage_dit_fma<4>(a, L, span, nseq, rec, lane, nl);
        else
          inplace_stage_dit_fma<8>(a, L, span, nseq, rec, lane, nl);
        rec += span * (R == 2 ? 2 : (R == 4 ? 4 : 8));
        FC_SYNC();
        span *= R;
        continue;
      }
      switch (R) {
        case 2: inplace_stage_r<2, true, false>(a, L, span, nseq, tw, lane, nl); break;
        case 3: inplace_stage_r<3, true, false>(a, L, span, nseq, tw, lane, nl); break;
        case 4: inplace_stage_r<4, true, false>(a, L, span, nseq, tw, lane, nl); break;
        case 5: inplace_stage_r<5, true, false>(a, L, span, nseq, tw, lane, nl); break;
        case 7: inplace_stage_r<7, true, false>(a, L, span, nseq, tw, lane, nl); break;
        case 8: inplace_stage_r<8, true, false>(a, L, span, nseq, tw, lane, nl); break;
        default: inplace_stage_gen<true, false>(a, L, span, R, nseq, tw, lane, nl); break;
      }
      FC_SYNC();
      span *= R;
    }
  }
}

// the multipliers as a pass of their own after fft_inplace<false> (per-slot tables with
// the pending factors folded in): derivative i fac dmul[slot] (eq. fc_der), filter
// sigp[slot] (eq. filtering)
FC_HD void mul_deriv_slot(double2* a, int L, int nseq, double fac, const double* __restrict__ dmul, int lane, int nl) {
  for (int idx = lane; idx < nseq * L; idx += nl) a[idx] = apply_mult<MUL_DERIV>(a[idx], dmul[idx % L], fac);
}
FC_HD void mul_filter_slot(double2* a, int L, int nseq, const double* __restrict__ sigp, int lane, int nl) {
  for (int idx = lane; idx < nseq * L; idx += nl) a[idx] = apply_mult<MUL_FILTER>(a[idx], sigp[idx % L], 0.0);
}

// forward transform followed by the derivative (MUL_DERIV) or filter (MUL_FILTER)
// multiplier (MUL_NONE: the transform alone, outputs with pending factors), the
// multiplier applied inside the last stage when its radix has a fixed butterfly (one
// shared-memory pass and one barrier fewer); radix-2/4/8 stages in the FMA form
template <int MUL>
FC_HD void fft_forward_mul(double2* a, const Plan& P, int nseq, const double2* twpool, const double* rp, double fac,
                           int lane, int nl) {
  const double2* tw = twpool + P.tw;
  const double2* rec = twpool + P.fmf;
  const double* psc = rp + P.psc;
  const double* mt = MUL == MUL_DERIV ? rp + P.dmul : (MUL == MUL_FILTER ? rp + P.sigp : nullptr);
  const int L = P.L;
  int span = L;
  for (int st = 0; st < P.nst; ++st) {
    const int R = P.rad[st];
    span /= R;
    const bool last = st == P.nst - 1;
    if (R == 2 || R == 4 || R == 8) {
      const double2* rot = rec;
      if (span > 1) rec += span * (R / 2);
      const double2* rat = rec;
      rec += (L / R) * (R / 2);
      if (last) {
        if (R == 2)
          inplace_stage_dif_fma<2, MUL>(a, L, span, nseq, rot, rat, lane, nl, fac, mt);
        else if (R == 4)
          inplace_stage_dif_fma<4, MUL>(a, L, span, nseq, rot, rat, lane, nl, fac, mt);
        else
          inplace_stage_dif_fma<8, MUL>(a, L, span, nseq, rot, rat, lane, nl, fac, mt);
      } else {
        if (R == 2)
          inplace_stage_dif_fma<2, MUL_NONE>(a, L, span, nseq, rot, rat, lane, nl, 0.0, nullptr);
        else if (R == 4)
          inplace_stage_dif_fma<4, MUL_NONE>(a, L, span, nseq, rot, rat, lane, nl, 0.0, nullptr);
        else
          inplace_stage_dif_fma<8, MUL_NONE>(a, L, span, nseq, rot, rat, lane, nl, 0.0, nullptr);
      }
      FC_SYNC();
      continue;
    }
    if ((P.fmod >> st) & 1) {  // odd last stage with the pending factors folded in
      const int rs2 = (R - 1 + (R - 1) * (R - 1) / 2 + 1) / 2;
      const double2* rr = rec;
      rec += (L / R) * rs2;
      if (R == 3)
        inplace_stage_odd_fold<3, MUL>(a, L, nseq, rr, lane, nl, fac, mt);
      else if (R == 5)
        inplace_stage_odd_fold<5, MUL>(a, L, nseq, rr, lane, nl, fac, mt);
      else
        inplace_stage_odd_fold<7, MUL>(a, L, nseq, rr, lane, nl, fac, mt);
      FC_SYNC();
      continue;
    }
    const double* ps = nullptr;
    if ((P.fmsc >> st) & 1) {
      ps = psc;
      psc += L;
    }
    if (last && MUL != MUL_NONE) {
      switch (R) {
        case 3: inplace_stage_r<3, false, true, MUL>(a, L, span, nseq, tw, lane, nl, fac, mt, ps); break;
        case 5: inplace_stage_r<5, false, true, MUL>(a, L, span, nseq, tw, lane, nl, fac, mt, ps); break;
        case 7: inplace_stage_r<7, false, true, MUL>(a, L, span, nseq, tw, lane, nl, fac, mt, ps); break;
        default:
          inplace_stage_gen<false, true>(a, L, span, R, nseq, tw, lane, nl, ps);
          FC_SYNC();
          if (MUL == MUL_DERIV)
            mul_deriv_slot(a, L, nseq, fac, mt, lane, nl);
          else
            mul_filter_slot(a, L, nseq, mt, lane, nl);
          break;
      }
    } else {
      switch (R) {
        case 3: inplace_stage_r<3, false, true>(a, L, span, nseq, tw, lane, nl, 0.0, nullptr, ps); break;
        case 5: inplace_stage_r<5, false, true>(a, L, span, nseq, tw, lane, nl, 0.0, nullptr, ps); break;
        case 7: inplace_stage_r<7, false, true>(a, L, span, nseq, tw, lane, nl, 0.0, nullptr, ps); break;
        default: inplace_stage_gen<false, true>(a, L, span, R, nseq, tw, lane, nl, ps); break;
      }
    }
    FC_SYNC();
  }
}

// FC-Gram continuation (eq. continuation) of the nseq complex sequences in a: entries
// [0, n) hold the data (two real lines packed as re/im); entries [n, n+C) receive
//   ext = ML F_l + MR F_r,   ML = A_l Q^T, MR = A_r Q^T (C x d).
// ML and MR have entries of order 1e4 (d = 5) whose contributions cancel, so the same
// linear map is evaluated in detrended form: with F~_l = F_l - F_0 - (F_1 - F_0) tau_l
// (tau_l = 0..d-1) and F~_r = F_r - F_{n-1} - (F_{n-1} - F_{n-2}) tau_r (tau_r = 1-d..0),
//   ext = ML F~_l + MR F~_r + F_0 uL + (F_1 - F_0) vL + F_{n-1} uR + (F_{n-1} - F_{n-2}) vR
// with uL = ML 1, vL = ML tau_l, uR = MR 1, vR = MR tau_r precomputed. The detrended
// values are differences of nearby samples (exact or nearly so), so the large
// coefficients multiply only second differences. Layout of M: ML, MR, uL, vL, uR, vR.
// tmp: 2 d nseq complex scratch (the detrended end data, computed once per line).
FC_HD void continue_lines(double2* a, int L, int n, int C, int d, const double* __restrict__ M, int nseq, int lane,
                          int nl, double2* tmp) {
  const double* ML = M;
  const double* MR = M + C * d;
  const double* uL = MR + C * d;
  const double* vL = uL + C;
  const double* uR = vL + C;
  const double* vR = uR + C;
  // phase 1: per sequence, the detrended end values F~_l[2..d-1], F~_r[0..d-3] and the
  // end value / end slope of both ends, 2d complex values per sequence, into tmp
  for (int idx = lane; idx < nseq * 2 * d; idx += nl) {
    const int s = idx / (2 * d);
    const int q = idx - s * 2 * d;
    const double2* x = a + s * L;
    const double2 f0 = x[0], f1 = x[1], fn = x[n - 1], fm = x[n - 2];
    const double2 dl = csub(f1, f0), dr = csub(fn, fm);
    double2 v;
    if (q < d - 2) {  // left, j = q + 2
      const double j = (double)(q + 2);
      v = cpx(fma(-j, dl.x, (x[q + 2].x - f0.x)), fma(-j, dl.y, (x[q + 2].y - f0.y)));
    } else if (q < 2 * d - 4) {  // right, j = q - (d - 2)
      const int j = q - (d - 2);
      const double t = (double)(d - 1 - j);
      v = cpx(fma(t, dr.x, (x[n - d + j].x - fn.x)), fma(t, dr.y, (x[n - d + j].y - fn.y)));
    } else {
      const int w = q - (2 * d - 4);  // 0: f0, 1: dl, 2: fn, 3: dr
      v = w == 0 ? f0 : (w == 1 ? dl : (w == 2 ? fn : dr));
    }
    tmp[idx] = v;
  }
  FC_SYNC();
  // phase 2: ext_k = ML F~_l + MR F~_r + F_0 uL + dl vL + F_{n-1} uR + dr vR
  for (int idx = lane; idx < nseq * C; idx += nl) {
    const int s = idx / C;
    const int k = idx - s * C;
    const double2* e = tmp + s * 2 * d;
    double ex = 0.0, ey = 0.0;
    for (int j = 2; j < d; ++j) {
      const double ml = ML[k * d + j];
      ex = fma(ml, e[j - 2].x, ex);
      ey = fma(ml, e[j - 2].y, ey);
    }
    for (int j = 0; j < d - 2; ++j) {
      const double mr = MR[k * d + j];
      ex = fma(mr, e[d - 2 + j].x, ex);
      ey = fma(mr, e[d - 2 + j].y, ey);
    }
    const double2 f0 = e[2 * d - 4], dl = e[2 * d - 3], fn = e[2 * d - 2], dr = e[2 * d - 1];
    ex = fma(f0.x, uL[k], fma(dl.x, vL[k], fma(fn.x, uR[k], fma(dr.x, vR[k], ex))));
    ey = fma(f0.y, uL[k], fma(dl.y, vL[k], fma(fn.y, uR[k], fma(dr.y, vR[k], ey))));
    a[s * L + n + k] = cpx(ex, ey);
  }
}

// ---- Euler physics (Sec. 2.1) ----
struct Prim {
  double rho, u, v, p;
};
FC_HD Prim primitives(double r, double mx, double my, double E, double gam) {
  Prim q;
  const double ir = 1.0 / r;
  q.rho = r;
  q.u = mx * ir;
  q.v = my * ir;
  q.p = (gam - 1.0) * (E - 0.5 * (mx * q.u + my * q.v));
  return q;
}

}  // namespace fcx
