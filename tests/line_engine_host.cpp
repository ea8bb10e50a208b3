// Host build of the line engine (fc_line.cuh) and of the plan and table builder
// (fc_host.cpp) for CPU tests of the kernels' arithmetic: the same source the GPU runs,
// compiled as plain C++ with one "lane" per line (the warp-level barriers compile to
// nothing on the host).
//
//   line_engine_host plans L1 L2 ...
//     for every continued length L and every candidate stage order the autotuner may
//     pick, the derivative of a random trigonometric polynomial of two packed sequences
//     (forward transform, derivative multiplier, inverse transform) against its exact
//     derivative; prints "L order max_rel_err" per candidate.
//
//   line_engine_host fc <in> <out>
//     FC derivatives or FC filters (continuation + transform) of lines read from <in>:
//       int32 d, double alpha_f, int32 p_f, int32 ntab, double tab[ntab] (the packed
//       FC-Gram tables), int32 nlines, then per line int32 op (0: derivative, 1: filter),
//       int32 N, int32 C, double h, double data[4][N];
//     <out> gets, per line, int32 ncand and ncand x double result[4][N] (one per
//     candidate stage order of the continued length N + C).
//
//   line_engine_host patch <in> <out>
//     the host geometry of one patch (build_patch): <in> holds int32 kind, n1, n2,
//     double geom[4], int32 side[4], double hole[3], and for GRID double x[n2][n1],
//     y[n2][n1]; <out> gets double hhat, htil, then uint8 blank, receiver, generating,
//     no-derivative [n2][n1] and int32 depth [n2][n1].
//
//   line_engine_host policy C0 policy Cmax N0 N1
//     the continuation length the library picks for every line length N0..N1
//     (choose_continuation), one "N C" pair per line.
//
//   line_engine_host records L1 L2 ...
//     the FMA-form butterfly records of every candidate stage order (fc_tables.h) read
//     back and checked against the twiddles they encode; prints "L order max_err max_t
//     min_S" per candidate.
//
//   line_engine_host adw d
//     the no-slip adiabatic wall weights (adiabatic_weights) for d, one per line.
//
//   line_engine_host grid <in> <out>
//     the host geometry of a GRID patch (fc_host.cpp build_patch, frac_index): <in> holds
//       int32 n1, int32 n2, int32 periodic1, double x[n2][n1], double y[n2][n1],
//       int32 nq, double xq[nq], double yq[nq];
//     <out> gets double hhat, double htil, double s1[nq], double s2[nq] (the fractional
//     indices of the query points; far outside the grid when not located).
#include "../paper_2506_16076_gb300/csrc/fc_host.cpp"
#include "../paper_2506_16076_gb300/csrc/fc_line.cuh"

#include <complex>
#include <cstdio>
#include <cstring>
#include <random>

namespace {

// derivative (filter: the spectral filter) of the 4 components of one line (two packed
// sequences) with plan P, as the kernels' deriv2 (filter2) does
void derive(double2* A, int Lmax, const fcx::Plan& P, int n, int C, int fcm, double scale, int d,
            const Builder& B, bool filter = false) {
  using namespace fcx;
  if (fcm >= 0) continue_lines(A, P.L, n, C, d, B.rp.data() + fcm, 2, 0, 1, A + 2 * Lmax);
  fft_inplace<false>(A, P, 2, B.tw.data(), B.rp.data(), 0, 1);
  if (filter)
    mul_filter_slot(A, P.L, 2, B.rp.data() + P.sigp, 0, 1);
  else
    mul_deriv_slot(A, P.L, 2, scale * TWO_PI / ((double)P.L * (double)P.L), B.rp.data() + P.dmul, 0, 1);
  fft_inplace<true>(A, P, 2, B.tw.data(), B.rp.data(), 0, 1);
}

// the FMA-form records of every candidate stage order of each length (fc_tables.h), read
// back in the device kernels' order: each twiddle rebuilt from its ratio form against
// exp(+-2 pi i e / L), the inverse records with their stored scales S (S3 = (S3/S1) S1 and
// so on), the forward rotations up to their real factor; prints "L order max_err max_t min_S"
int run_records(int argc, char** argv) {
  using namespace fcx;
  fc_ctx c;
  Builder B{&c};
  const long double PI = 3.14159265358979323846264338327950288L;
  for (int a = 2; a < argc; ++a) {
    const int L = atoi(argv[a]);
    const int pi = B.plan(L);
    for (const Plan& P : B.cands[pi]) {
      long double err = 0, tmax = 0, smin = 1e30L;
      auto rebuild = [&](long double S, long double t, bool f) {  // S (1 + i t) or S i (1 + i t)
        tmax = std::max(tmax, fabsl(t));
        return f ? std::complex<long double>(-S * t, S) : std::complex<long double>(S, S * t);
      };
      // inverse records
      const double2* rec = B.tw.data() + P.fmd;
      int span = 1;
      for (int st = P.nst - 1; st >= 0; --st) {
        const int R = P.rad[st];
        if (span > 1 && (R == 2 || R == 4 || R == 8)) {
          const int RS = R == 2 ? 2 : (R == 4 ? 4 : 8);
          const int tws = L / (R * span);
          for (int j = 0; j < span; ++j) {
            const double2* q = rec + j * RS;
            long long fl;
            memcpy(&fl, &q[0].x, sizeof(fl));
            long double t[8] = {0}, S[8] = {1};
            t[1] = q[0].y;
            if (R == 2) {
              S[1] = q[1].x;
            } else if (R == 4) {
              t[2] = q[1].x, t[3] = q[1].y, S[2] = q[2].x, S[1] = q[2].y, S[3] = (long double)q[3].x * S[1];
            } else {
              t[2] = q[1].x, t[3] = q[1].y, t[4] = q[2].x, t[5] = q[2].y, t[6] = q[3].x, t[7] = q[3].y;
              S[4] = q[4].x, S[2] = q[4].y, S[1] = q[7].x;
              S[6] = (long double)q[5].x * S[2], S[5] = (long double)q[5].y * S[1];
              S[3] = (long double)q[6].y * S[1], S[7] = (long double)q[6].x * S[3];
              err = std::max(err, fabsl((long double)q[7].y - S[1] * 0.70710678118654752440L));
            }
            for (int r = 1; r < R; ++r) {
              smin = std::min(smin, fabsl(S[r]));
              const long double ang = 2.0L * PI * (long double)(((long long)r * j * tws) % L) / L;
              const std::complex<long double> w = rebuild(S[r], t[r], (fl >> (r - 1)) & 1);
              err = std::max(err, std::abs(w - std::complex<long double>(cosl(ang), sinl(ang))));
            }
          }
          rec += span * RS;
        }
        span *= R;
      }
      // forward rotation records (factors folded elsewhere): direction only
      rec = B.tw.data() + P.fmf;
      span = L;
      for (int st = 0; st < P.nst; ++st) {
        const int R = P.rad[st];
        span /= R;
        if (R == 2 || R == 4 || R == 8) {
          const int tws = L / (R * span);
          if (span > 1) {
            for (int j = 0; j < span; ++j) {
              const double2* h = rec + j * (R / 2);
              long long fl;
              memcpy(&fl, &h[0].x, sizeof(fl));
              for (int r = 1; r < R; ++r) {
                const double tr = r == 1 ? h[0].y : (r % 2 == 0 ? h[r / 2].x : h[r / 2].y);
                const std::complex<long double> d = rebuild(1.0L, tr, (fl >> (r - 1)) & 1);
                const long double ang = -2.0L * PI * (long double)(((long long)r * j * tws) % L) / L;
                const std::complex<long double> w(cosl(ang), sinl(ang));
                err = std::max(err, fabsl(std::imag(w * std::conj(d))) / std::abs(d));
              }
            }
            rec += span * (R / 2);
          }
          rec += (L / R) * (R / 2);
        } else if ((P.fmod >> st) & 1) {
          const int H = (R - 1) / 2;
          rec += (L / R) * ((2 * H + 2 * H * H + 1) / 2);
        }
      }
      printf("%d ", L);
      for (int s = 0; s < P.nst; ++s) printf("%s%d", s ? "." : "", P.rad[s]);
      printf(" %.3Le %.6Lf %.6Lf\n", err, tmax, smin == 1e30L ? 1.0L : smin);
    }
  }
  return 0;
}

int run_plans(int argc, char** argv) {
  using namespace fcx;
  fc_ctx c;
  Builder B{&c};
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (int a = 2; a < argc; ++a) {
    const int L = atoi(argv[a]);
    const int pi = B.plan(L);
    const std::vector<Plan> cands = B.cands[pi];
    // random modes |k| < L/2 on both sequences (complex coefficients)
    const int K = (L - 1) / 2;
    std::vector<double> cr(2 * (2 * K + 1)), ci(2 * (2 * K + 1));
    for (size_t q = 0; q < cr.size(); ++q) {
      cr[q] = U(rng);
      ci[q] = U(rng);
    }
    std::vector<double2> f(2 * L), df(2 * L);
    double dmax = 0;
    for (int s = 0; s < 2; ++s)
      for (int t = 0; t < L; ++t) {
        long double fx = 0, fy = 0, gx = 0, gy = 0;
        for (int k = -K; k <= K; ++k) {
          const long double ang = 2.0L * 3.14159265358979323846264338327950288L * k * t / L;
          const long double cs = cosl(ang), sn = sinl(ang);
          const long double ar = cr[s * (2 * K + 1) + k + K], ai = ci[s * (2 * K + 1) + k + K];
          const long double vr = ar * cs - ai * sn, vi = ar * sn + ai * cs;  // c_k e^{i ang}
          const long double w = 2.0L * 3.14159265358979323846264338327950288L * k / L;
          fx += vr;
          fy += vi;
          gx += -w * vi;  // i w (vr + i vi)
          gy += w * vr;
        }
        f[s * L + t] = cpx((double)fx, (double)fy);
        df[s * L + t] = cpx((double)gx, (double)gy);
        dmax = std::max(dmax, (double)std::max(fabsl(gx), fabsl(gy)));
      }
    for (const Plan& P : cands) {
      std::vector<double2> A(2 * L + CONT_TMP);
      for (int q = 0; q < 2 * L; ++q) A[q] = f[q];
      derive(A.data(), L, P, L, 0, -1, 1.0, 0, B);
      double err = 0;
      for (int q = 0; q < 2 * L; ++q)
        err = std::max(err, std::max(fabs(A[q].x - df[q].x), fabs(A[q].y - df[q].y)));
      printf("%d ", L);
      for (int s = 0; s < P.nst; ++s) printf("%s%d", s ? "." : "", P.rad[s]);
      printf(" %.3e\n", err / dmax);
    }
  }
  return 0;
}

int run_fc(const char* in, const char* out) {
  using namespace fcx;
  FILE* fi = fopen(in, "rb");
  FILE* fo = fopen(out, "wb");
  if (!fi || !fo) return 2;
  int d = 0, ntab = 0, nlines = 0, pf = 0;
  double af = 0;
  if (fread(&d, 4, 1, fi) != 1 || fread(&af, 8, 1, fi) != 1 || fread(&pf, 4, 1, fi) != 1 ||
      fread(&ntab, 4, 1, fi) != 1)
    return 3;
  fc_ctx c;
  c.prm.alpha_f = af;
  c.prm.p_f = pf;
  c.fctab.resize(ntab);
  if (fread(c.fctab.data(), 8, ntab, fi) != (size_t)ntab) return 3;
  c.d = d;
  c.Cmin = (int)c.fctab[1];
  c.Cmax = (int)c.fctab[2];
  Builder B{&c};
  if (fread(&nlines, 4, 1, fi) != 1) return 3;
  for (int l = 0; l < nlines; ++l) {
    int op = 0, N = 0, C = 0;
    double h = 0;
    if (fread(&op, 4, 1, fi) != 1 || fread(&N, 4, 1, fi) != 1 || fread(&C, 4, 1, fi) != 1 ||
        fread(&h, 8, 1, fi) != 1)
      return 3;
    std::vector<double> data(4 * (size_t)N);
    if (fread(data.data(), 8, data.size(), fi) != data.size()) return 3;
    const int fcm = B.fcm(C);
    const int pi = B.plan(N + C);
    const std::vector<Plan> cands = B.cands[pi];
    const int L = N + C, nc = (int)cands.size();
    fwrite(&nc, 4, 1, fo);
    for (const Plan& P : cands) {
      std::vector<double2> A(2 * L + CONT_TMP);
      for (int t = 0; t < N; ++t) {
        A[t] = cpx(data[t], data[N + t]);
        A[L + t] = cpx(data[2 * N + t], data[3 * N + t]);
      }
      derive(A.data(), L, P, N, C, fcm, 1.0 / h, d, B, op == 1);
      std::vector<double> o(4 * (size_t)N);
      for (int t = 0; t < N; ++t) {
        o[t] = A[t].x;
        o[N + t] = A[t].y;
        o[2 * N + t] = A[L + t].x;
        o[3 * N + t] = A[L + t].y;
      }
      fwrite(o.data(), 8, o.size(), fo);
    }
  }
  fclose(fi);
  fclose(fo);
  return 0;
}

int run_grid(const char* in, const char* out) {
  FILE* fi = fopen(in, "rb");
  FILE* fo = fopen(out, "wb");
  if (!fi || !fo) return 2;
  int n1 = 0, n2 = 0, per = 0, nq = 0;
  if (fread(&n1, 4, 1, fi) != 1 || fread(&n2, 4, 1, fi) != 1 || fread(&per, 4, 1, fi) != 1) return 3;
  const size_t N = (size_t)n1 * n2;
  std::vector<double> x(N), y(N);
  if (fread(x.data(), 8, N, fi) != N || fread(y.data(), 8, N, fi) != N || fread(&nq, 4, 1, fi) != 1) return 3;
  std::vector<double> xq(nq), yq(nq);
  if (fread(xq.data(), 8, nq, fi) != (size_t)nq || fread(yq.data(), 8, nq, fi) != (size_t)nq) return 3;
  HPatch h;
  std::memset(&h.d, 0, sizeof(h.d));
  h.d.kind = FC_PATCH_GRID;
  h.d.n1 = n1;
  h.d.n2 = n2;
  for (int s = 0; s < 4; ++s) h.d.side[s] = (per && s < 2) ? FC_SIDE_PERIODIC : FC_SIDE_DIRICHLET;
  h.d.hole[2] = -1.0;
  h.d.x = x.data();
  h.d.y = y.data();
  fc_params prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.d = 5;
  prm.n_f = 5;
  prm.n_v = 9;
  prm.depth_cap = 64;
  build_patch(h, prm);
  fwrite(&h.hhat, 8, 1, fo);
  fwrite(&h.htil, 8, 1, fo);
  std::vector<double> s1(nq), s2(nq);
  for (int q = 0; q < nq; ++q) frac_index(h, xq[q], yq[q], s1[q], s2[q]);
  fwrite(s1.data(), 8, nq, fo);
  fwrite(s2.data(), 8, nq, fo);
  fclose(fi);
  fclose(fo);
  return 0;
}

int run_patch(const char* in, const char* out) {
  FILE* fi = fopen(in, "rb");
  FILE* fo = fopen(out, "wb");
  if (!fi || !fo) return 2;
  HPatch h;
  std::memset(&h.d, 0, sizeof(h.d));
  int hdr[3];
  if (fread(hdr, 4, 3, fi) != 3 || fread(h.d.geom, 8, 4, fi) != 4 || fread(h.d.side, 4, 4, fi) != 4 ||
      fread(h.d.hole, 8, 3, fi) != 3)
    return 3;
  h.d.kind = hdr[0];
  h.d.n1 = hdr[1];
  h.d.n2 = hdr[2];
  const size_t N = (size_t)hdr[1] * hdr[2];
  std::vector<double> x, y;
  if (h.d.kind == FC_PATCH_GRID) {
    x.resize(N);
    y.resize(N);
    if (fread(x.data(), 8, N, fi) != N || fread(y.data(), 8, N, fi) != N) return 3;
    h.d.x = x.data();
    h.d.y = y.data();
  }
  fc_params prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.d = 5;
  prm.n_f = 5;
  prm.n_v = 9;
  prm.depth_cap = 64;
  build_patch(h, prm);
  fwrite(&h.hhat, 8, 1, fo);
  fwrite(&h.htil, 8, 1, fo);
  fwrite(h.blank.data(), 1, N, fo);
  fwrite(h.recv.data(), 1, N, fo);
  fwrite(h.gen.data(), 1, N, fo);
  fwrite(h.nodiff.data(), 1, N, fo);
  fwrite(h.depth.data(), 4, N, fo);
  fclose(fi);
  fclose(fo);
  return 0;
}

int run_policy(char** argv) {
  fc_params prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.C0 = atoi(argv[2]);
  prm.c_policy = atoi(argv[3]);
  prm.d = 5;
  const int Cmax = atoi(argv[4]);
  for (int N = atoi(argv[5]); N <= atoi(argv[6]); ++N) printf("%d %d\n", N, choose_continuation(N, prm, Cmax));
  return 0;
}

int run_adw(char** argv) {
  for (double w : adiabatic_weights(atoi(argv[2]))) printf("%.17g\n", w);
  return 0;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc >= 2 && std::string(argv[1]) == "plans") return run_plans(argc, argv);
  if (argc >= 2 && std::string(argv[1]) == "records") return run_records(argc, argv);
  if (argc == 4 && std::string(argv[1]) == "fc") return run_fc(argv[2], argv[3]);
  if (argc == 4 && std::string(argv[1]) == "grid") return run_grid(argv[2], argv[3]);
  if (argc == 7 && std::string(argv[1]) == "policy") return run_policy(argv);
  if (argc == 4 && std::string(argv[1]) == "patch") return run_patch(argv[2], argv[3]);
  if (argc == 3 && std::string(argv[1]) == "adw") return run_adw(argv);
  fprintf(stderr, "usage: line_engine_host plans L... | fc <in> <out> | grid <in> <out> | policy ... | adw d\n");
  return 1;
}
