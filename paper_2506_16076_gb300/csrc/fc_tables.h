// Host-side builders of the FMA-form transform records (fc_line.cuh), shared by the
// context's plan builder (fc_host.cpp) and the allocation-free entry (fc_noalloc.cu).
//
// A twiddle w = (c, s) is stored in ratio form: w = S (1 + i t) with S = c, t = s / c
// when |c| >= |s|, else w = S i (1 + i t) with S = s, t = -c / s (flag set), so that
// w b = S u with u = b' + i t b' (b' = b, or i b when flagged): two FMAs, |t| <= 1 and
// |S| >= 1/sqrt 2, the real factor S left to the butterfly's FMAs.
//
// Inverse transform (decimation in time, twiddles on the inputs): per radix-2/4/8 stage
// of span > 1, in the inverse stage order, one record per offset j (double2 units):
//   R = 2: (flags, t1), (S1, 0)
//   R = 4: (flags, t1), (t2, t3), (S2, S1), (S3/S1, 0)
//   R = 8: (flags, t1), (t2, t3), (t4, t5), (t6, t7), (S4, S2), (S6/S2, S5/S1),
//          (S7/S3, S3/S1), (S1, S1/sqrt 2)
// Forward transform (decimation in frequency, twiddles on the outputs): every element
// carries a pending real factor P (1 at the start); a radix-2/4/8 butterfly combines its
// inputs with the ratios of their factors and leaves its outputs with the factor of its
// first input times the S of the output twiddle's ratio form. Per radix-2/4/8 stage, in
// stage order: if span > 1 one rotation record per offset j, R/2 double2: (flags, t1),
// (t2, t3), ...; then one ratio record per butterfly (index bb span + j), R/2 double2:
//   R = 2: (P1/P0, 0)
//   R = 4: (P2/P0, P3/P1), (P1/P0, 0)
//   R = 8: (P4/P0, P6/P2), (P2/P0, P5/P1), (P7/P3, P3/P1), (P1/P0, P1/P0/sqrt 2)
// A last stage (span 1) of radix 3, 5 or 7 whose inputs carry factors folds them into its
// FMAs (bit st of Plan::fmod): per butterfly, H = (R-1)/2, the doubles rho_m =
// P_{R-m}/P_m, pi_m = P_m/P_0, cos(2 pi q m/R) pi_m and sin(2 pi q m/R) pi_m (q, m = 1..H,
// q major), padded to whole double2; its outputs keep P_0. A stage of another radix whose
// inputs carry factors other than 1 multiplies them in first (bit st of Plan::fmsc, L
// factors per such stage in the real pool from Plan::psc). The factors left after the last stage are folded into the per-slot
// derivative table (Plan::dmul: k P for the mode k held at the slot, 0 for the Nyquist
// mode) and filter table (Plan::sigp: sigma(2k/L)/L P).
#pragma once
#include <cmath>
#include <cstring>
#include <vector>

#include "fc_internal.h"

namespace fcx {

constexpr long double TABLE_PI = 3.14159265358979323846264338327950288L;
constexpr long double TABLE_RSQRT2 = 0.70710678118654752440084436210484903928L;

// ratio form of exp(i ang): S, t and the flag
inline void ratio_form(long double ang, long double& S, long double& t, bool& flag) {
  const long double c = cosl(ang), s = sinl(ang);
  flag = !(fabsl(c) >= fabsl(s));
  if (!flag) {
    S = c;
    t = s / c;
  } else {
    S = s;
    t = -c / s;
  }
}

inline double2 table_pair(long double x, long double y) {
  double2 v;
  v.x = (double)x;
  v.y = (double)y;
  return v;
}

inline double flag_word(long long flags) {
  double f;
  std::memcpy(&f, &flags, sizeof(f));
  return f;
}

inline bool fma_radix(int R) { return R == 2 || R == 4 || R == 8; }

// records of the inverse transform (appended to tw); sets p.fmd
inline void fma_inverse_records(Plan& p, std::vector<double2>& tw) {
  const int L = p.L;
  p.fmd = (int)tw.size();
  int span = 1;
  for (int st = p.nst - 1; st >= 0; --st) {
    const int R = p.rad[st];
    if (span > 1 && fma_radix(R)) {
      const int tws = L / (R * span);
      for (int j = 0; j < span; ++j) {
        long double S[8] = {1.0L}, t[8] = {0.0L};
        long long flags = 0;
        for (int q = 1; q < R; ++q) {
          const long long e = ((long long)q * j * tws) % L;
          bool f;
          ratio_form(2.0L * TABLE_PI * (long double)e / (long double)L, S[q], t[q], f);
          if (f) flags |= 1LL << (q - 1);
        }
        tw.push_back(table_pair(0.0L, t[1]));
        tw.back().x = flag_word(flags);
        if (R == 2) {
          tw.push_back(table_pair(S[1], 0.0L));
        } else if (R == 4) {
          tw.push_back(table_pair(t[2], t[3]));
          tw.push_back(table_pair(S[2], S[1]));
          tw.push_back(table_pair(S[3] / S[1], 0.0L));
        } else {
          tw.push_back(table_pair(t[2], t[3]));
          tw.push_back(table_pair(t[4], t[5]));
          tw.push_back(table_pair(t[6], t[7]));
          tw.push_back(table_pair(S[4], S[2]));
          tw.push_back(table_pair(S[6] / S[2], S[5] / S[1]));
          tw.push_back(table_pair(S[7] / S[3], S[3] / S[1]));
          tw.push_back(table_pair(S[1], S[1] * TABLE_RSQRT2));
        }
      }
    }
    span *= R;
  }
}

// records of the forward transform (tw) and its scale tables (rp); rev: the plan's slot ->
// mode table; sig: the filter factor per mode (null: no filter table). Sets p.fmf, p.fmsc,
// p.psc, p.dmul, p.sigp.
inline void fma_forward_records(Plan& p, std::vector<double2>& tw, std::vector<double>& rp, const int* rev,
                                const double* sig) {
  const int L = p.L;
  std::vector<long double> P((size_t)L, 1.0L);
  p.fmf = (int)tw.size();
  p.fmsc = 0;
  p.fmod = 0;
  p.psc = (int)rp.size();
  int span = L;
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.rad[st];
    span /= R;
    if (!fma_radix(R)) {
      bool scaled = false;
      for (long double v : P) scaled = scaled || v != 1.0L;
      if (scaled && span == 1 && (R == 3 || R == 5 || R == 7)) {
        p.fmod |= 1 << st;
        const int H = (R - 1) / 2;
        for (int bb = 0; bb < L / R; ++bb) {
          const long double* Pr = P.data() + (size_t)bb * R;
          std::vector<long double> rec;
          for (int m = 1; m <= H; ++m) rec.push_back(Pr[R - m] / Pr[m]);
          for (int m = 1; m <= H; ++m) rec.push_back(Pr[m] / Pr[0]);
          for (int q = 1; q <= H; ++q)
            for (int m = 1; m <= H; ++m)
              rec.push_back(cosl(2.0L * TABLE_PI * (long double)(q * m) / (long double)R) * (Pr[m] / Pr[0]));
          for (int q = 1; q <= H; ++q)
            for (int m = 1; m <= H; ++m)
              rec.push_back(sinl(2.0L * TABLE_PI * (long double)(q * m) / (long double)R) * (Pr[m] / Pr[0]));
          if (rec.size() % 2) rec.push_back(0.0L);
          for (size_t i = 0; i < rec.size(); i += 2) tw.push_back(table_pair(rec[i], rec[i + 1]));
        }
        for (int bb = 0; bb < L / R; ++bb)
          for (int r = 1; r < R; ++r) P[(size_t)(bb * R + r)] = P[(size_t)(bb * R)];
        continue;
      }
      if (scaled) {
        p.fmsc |= 1 << st;
        for (long double v : P) rp.push_back((double)v);
        for (long double& v : P) v = 1.0L;
      }
      continue;
    }
    const int tws = L / (R * span);
    std::vector<long double> Sj((size_t)span * R, 1.0L);
    if (span > 1) {
      for (int j = 0; j < span; ++j) {
        long double t[8] = {0.0L};
        long long flags = 0;
        for (int q = 1; q < R; ++q) {
          const long long e = ((long long)q * j * tws) % L;
          bool f;
          ratio_form(-2.0L * TABLE_PI * (long double)e / (long double)L, Sj[(size_t)j * R + q], t[q], f);
          if (f) flags |= 1LL << (q - 1);
        }
        tw.push_back(table_pair(0.0L, t[1]));
        tw.back().x = flag_word(flags);
        for (int q = 2; q < R; q += 2) tw.push_back(table_pair(t[q], t[q + 1]));
      }
    }
    for (int bb = 0; bb < L / (R * span); ++bb)
      for (int j = 0; j < span; ++j) {
        const int base = bb * R * span + j;
        long double Pr[8];
        for (int r = 0; r < R; ++r) Pr[r] = P[(size_t)(base + r * span)];
        if (R == 2) {
          tw.push_back(table_pair(Pr[1] / Pr[0], 0.0L));
        } else if (R == 4) {
          tw.push_back(table_pair(Pr[2] / Pr[0], Pr[3] / Pr[1]));
          tw.push_back(table_pair(Pr[1] / Pr[0], 0.0L));
        } else {
          tw.push_back(table_pair(Pr[4] / Pr[0], Pr[6] / Pr[2]));
          tw.push_back(table_pair(Pr[2] / Pr[0], Pr[5] / Pr[1]));
          tw.push_back(table_pair(Pr[7] / Pr[3], Pr[3] / Pr[1]));
          tw.push_back(table_pair(Pr[1] / Pr[0], Pr[1] / Pr[0] * TABLE_RSQRT2));
        }
        for (int q = 0; q < R; ++q) P[(size_t)(base + q * span)] = Pr[0] * Sj[(size_t)j * R + q];
      }
  }
  p.dmul = (int)rp.size();
  for (int slot = 0; slot < L; ++slot) {
    const int k = rev[slot];
    long double kk = (2 * k <= L) ? k : k - L;
    if (2 * k == L) kk = 0.0L;
    rp.push_back((double)(kk * P[(size_t)slot]));
  }
  p.sigp = -1;
  if (sig) {
    p.sigp = (int)rp.size();
    for (int slot = 0; slot < L; ++slot) rp.push_back((double)((long double)sig[rev[slot]] * P[(size_t)slot]));
  }
}

}  // namespace fcx
