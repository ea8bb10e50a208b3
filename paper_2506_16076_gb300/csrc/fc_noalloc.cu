// fc_rhs_patch_noalloc: the RHS of one stand-alone affine patch without any device
// allocation, for callers that cannot allocate device memory (code running inside a
// host memory manager or allocator that owns all device memory, plug-ins whose host
// forbids allocation, code paths that must not allocate once set up). Everything the
// two line kernels need beyond the caller's inputs and outputs (partial sums, per-point
// flags, twiddles, continuation matrices, plans, line records) lives in one file-scope
// static device array, which every GPU that loads the library holds until exit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fc_internal.h"
#include "fc_tables.h"

using namespace fcx;

namespace {

// Maximum patch: 262144 points (e.g. 512 x 512), continued lengths up to 1024.
constexpr long long NA_MAX_POINTS = 262144;
constexpr int NA_MAX_L = 1024;
constexpr int NA_MAX_C = 128;
constexpr int NA_MAX_D = 8;
constexpr size_t NA_R1 = 4 * NA_MAX_POINTS * sizeof(double);
constexpr size_t NA_INFO = NA_MAX_POINTS * sizeof(uint32_t);
// per continued length: the twiddles (L) and the FMA-form records (fc_tables.h: at most
// 2 L inverse, L forward rotation and L/2 per forward stage), and in the real pool its
// per-slot derivative factors (L) and pending-factor tables (at most L per stage)
constexpr int NA_TW_PER_L = 9;
constexpr int NA_RP_PER_L = 8;
constexpr size_t NA_TW = 2 * NA_TW_PER_L * NA_MAX_L * sizeof(double2);
constexpr size_t NA_RP = (2 * NA_MAX_C * NA_MAX_D + 4 * NA_MAX_C + 2 * NA_RP_PER_L * NA_MAX_L) * sizeof(double);
constexpr size_t NA_PLANS = 2 * sizeof(Plan);
constexpr size_t NA_JOBS = 2 * NA_MAX_L * sizeof(Job);
constexpr size_t NA_IP = 2 * NA_MAX_L * sizeof(int);
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_R1 = 0;
constexpr size_t OFF_INFO = align256(OFF_R1 + NA_R1);
constexpr size_t OFF_TW = align256(OFF_INFO + NA_INFO);
constexpr size_t OFF_RP = align256(OFF_TW + NA_TW);
constexpr size_t OFF_PLANS = align256(OFF_RP + NA_RP);
constexpr size_t OFF_JOBS = align256(OFF_PLANS + NA_PLANS);
constexpr size_t OFF_IP = align256(OFF_JOBS + NA_JOBS);
constexpr size_t NA_BYTES = align256(OFF_IP + NA_IP);

}  // namespace

static __device__ __align__(256) unsigned char fc_noalloc_scratch[NA_BYTES];

namespace {

constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_scratch[NA_MAX_DEVICES] = {nullptr};

std::vector<int> na_factorize(int L) {
  std::vector<int> f;
  int m = L;
  for (int r : {8, 4, 2, 3, 5, 7})
    while (m % r == 0) {
      f.push_back(r);
      m /= r;
    }
  for (int p = 11; m > 1; p += 2)
    while (m % p == 0) {
      f.push_back(p);
      m /= p;
    }
  return f;
}

}  // namespace

extern "C" fc_status fc_rhs_patch_noalloc(const double* e_dev, const double* mu_dev, double* rhs_dev, int n1, int n2,
                                          const double* box, int d, int C, const double* table, int table_len,
                                          double gamma, void* stream) {
  if (!e_dev || !mu_dev || !rhs_dev || !box || !table) return FC_ERR_INVALID;
  if ((long long)n1 * n2 > NA_MAX_POINTS || n1 + C > NA_MAX_L || n2 + C > NA_MAX_L || C > NA_MAX_C || d > NA_MAX_D) {
    fprintf(stderr,
            "fc_rhs_patch_noalloc: %d x %d points with C = %d, d = %d exceeds the static scratch limits "
            "(%lld points, continued length %d, C %d, d %d)\n",
            n1, n2, C, d, NA_MAX_POINTS, NA_MAX_L, NA_MAX_C, NA_MAX_D);
    return FC_ERR_INVALID;
  }
  if (n1 < 2 * d || n2 < 2 * d || C < 1 || d < 2 || !(box[1] > box[0]) || !(box[3] > box[2])) return FC_ERR_INVALID;
  if (table_len != d * d + 2 * C * d) {  // one (Q, A_l, A_r) block of this d and C, nothing else
    fprintf(stderr, "fc_rhs_patch_noalloc: table holds %d values, the d = %d, C = %d block needs %d\n", table_len, d,
            C, d * d + 2 * C * d);
    return FC_ERR_INVALID;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return FC_ERR_CUDA;
  if (!g_scratch[dev]) {  // set-up, once per device, with that device current
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, fc_noalloc_scratch) != cudaSuccess || !p) return FC_ERR_CUDA;
    set_kernel_attributes();
    g_scratch[dev] = (unsigned char*)p;
  }
  unsigned char* S = g_scratch[dev];
  cudaStream_t st = (cudaStream_t)stream;
  const long long P = (long long)n1 * n2;

  // host-built tables: twiddles of the two continued lengths, continuation matrices in the
  // detrended layout (ML, MR, ML 1, ML tau_l, MR 1, MR tau_r), plans, one job per line
  const int L[2] = {n1 + C, n2 + C};
  std::vector<double2> tw;
  std::vector<int> ip;
  std::vector<Plan> plans(2);
  for (int k = 0; k < 2; ++k) {
    Plan& pl = plans[k];
    std::memset(&pl, 0, sizeof(Plan));
    pl.L = L[k];
    std::vector<int> f = na_factorize(L[k]);
    if ((int)f.size() > MAXST) return FC_ERR_INVALID;
    for (int r : f)
      if (r > MAX_GENERIC_RADIX) return FC_ERR_INVALID;
    pl.nst = (int)f.size();
    for (int s = 0; s < pl.nst; ++s) pl.rad[s] = f[s];
    pl.tw = (int)tw.size();
    pl.sig = -1;
    pl.rev = (int)ip.size();
    for (int slot = 0; slot < L[k]; ++slot) {  // slot -> mode table of the in-place transforms
      int rem = slot, mode = 0, w = 1, span = L[k];
      for (int s2 = 0; s2 < pl.nst; ++s2) {
        span /= pl.rad[s2];
        const int dgt = rem / span;
        rem -= dgt * span;
        mode += dgt * w;
        w *= pl.rad[s2];
      }
      ip.push_back(mode);
    }
    for (int e = 0; e < L[k]; ++e) {
      const long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)e / (long double)L[k];
      double2 w;
      w.x = (double)cosl(a);
      w.y = (double)sinl(a);
      tw.push_back(w);
    }
    fma_inverse_records(pl, tw);
  }
  const double* Q = table;
  const double* AL = Q + d * d;
  const double* AR = AL + C * d;
  std::vector<double> rp;
  std::vector<long double> M[2];
  for (int which = 0; which < 2; ++which) {
    const double* A = which ? AR : AL;
    M[which].assign((size_t)C * d, 0.0L);
    for (int k = 0; k < C; ++k)
      for (int i = 0; i < d; ++i) {
        long double s = 0;
        for (int j = 0; j < d; ++j) s += (long double)A[k * d + j] * (long double)Q[i * d + j];
        M[which][(size_t)k * d + i] = s;
      }
    for (long double v : M[which]) rp.push_back((double)v);
  }
  for (int which = 0; which < 2; ++which)
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < C; ++k) {
        long double s = 0;
        for (int i = 0; i < d; ++i) {
          const long double tau = which == 0 ? (long double)i : (long double)(i - (d - 1));
          s += M[which][(size_t)k * d + i] * (pass == 0 ? 1.0L : tau);
        }
        rp.push_back((double)s);
      }
  for (int k = 0; k < 2; ++k) {  // forward records after the continuation matrices (fcm = 0)
    const std::vector<int> rev(ip.begin() + plans[k].rev, ip.begin() + plans[k].rev + L[k]);
    fma_forward_records(plans[k], tw, rp, rev.data(), nullptr);
  }
  if (tw.size() * sizeof(double2) > NA_TW || rp.size() * sizeof(double) > NA_RP) {
    fprintf(stderr, "fc_rhs_patch_noalloc: the transform tables exceed the static scratch\n");
    return FC_ERR_INVALID;
  }
  std::vector<Job> jobs;
  for (int dir = 0; dir < 2; ++dir) {
    const int nl = dir ? n1 : n2, n = dir ? n2 : n1;
    const double scale = dir ? (n2 - 1) / (box[3] - box[2]) : (n1 - 1) / (box[1] - box[0]);
    for (int line = 0; line < nl; ++line) {
      Job J;
      std::memset(&J, 0, sizeof(Job));
      J.base = dir ? line : (long long)line * n1;
      J.stride = dir ? n1 : 1;
      J.n = n;
      J.plan = dir;
      J.fcm = 0;
      J.C = C;
      J.patch = 0;
      J.gbase = -1;
      J.scale = scale;
      jobs.push_back(J);
    }
  }
  // the tables and the flag words are rewritten on every call (the array keeps the last
  // call's contents); R1 needs no clearing: the row pass writes every point before the
  // column pass reads it
  if (cudaMemsetAsync(S + OFF_INFO, 0, (size_t)P * sizeof(uint32_t), st) != cudaSuccess ||
      cudaMemcpyAsync(S + OFF_TW, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(S + OFF_RP, rp.data(), rp.size() * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(S + OFF_PLANS, plans.data(), plans.size() * sizeof(Plan), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(S + OFF_JOBS, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(S + OFF_IP, ip.data(), ip.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FC_ERR_CUDA;
  // the host vectors above are released on return: wait for the copies from them
  if (cudaStreamSynchronize(st) != cudaSuccess) return FC_ERR_CUDA;

  DevTables T;
  std::memset(&T, 0, sizeof(T));
  T.tw = (const double2*)(S + OFF_TW);
  T.rp = (const double*)(S + OFF_RP);
  T.ip = (const int*)(S + OFF_IP);
  T.plans = (const Plan*)(S + OFF_PLANS);
  T.info = (const uint32_t*)(S + OFF_INFO);
  T.patches = nullptr;
  T.npatch = 1;
  T.P = P;
  T.Pg = 1;
  T.gamma = gamma;
  T.d = d;
  const Job* jq1 = (const Job*)(S + OFF_JOBS);
  const Job* jq2 = jq1 + n2;
  double* R1 = (double*)(S + OFF_R1);
  StageCoef sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.Ucur = e_dev;
  sc.out = rhs_dev;
  sc.rhs_only = 1;
  launch_cart_q1(T, jq1, n2, L[0], e_dev, mu_dev, R1, nullptr, st);  // no y-flux buffer: q2 computes the fluxes
  launch_cart_q2(T, jq2, n1, L[1], mu_dev, R1, nullptr, sc, st);
  return cudaGetLastError() == cudaSuccess ? FC_OK : FC_ERR_CUDA;
}
