// Host runtime of the C ABI (include/fcsdnn.h): geometry processing at initialisation
// (Sec. 3, Alg. 1 line 2), FFT plans, line job queues, device workspaces, and the
// orchestration of the per-step passes (Alg. 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "fc_internal.h"
#include "fc_tables.h"

using namespace fcx;

namespace {

constexpr double PI = 3.141592653589793;
constexpr int AUTOTUNE_PLANS = 4;  // stage orders per continued length offered to the autotuner
constexpr double CONTAIN_TOL = 1e-9;

// SSPRK(5,4), Shu-Osher form (Sec. 4.1: the SSPRK-4 scheme the paper cites)
constexpr double A20 = 0.444370493651235, A21 = 0.555629506348765, B1 = 0.391752226571890, B2 = 0.368410593050371;
constexpr double A30 = 0.620101851488403, A32 = 0.379898148511597, B3 = 0.251891774271694;
constexpr double A40 = 0.178079954393132, A43 = 0.821920045606868, B4 = 0.544974750228521;
constexpr double A52 = 0.517231671970585, A53 = 0.096059710526147, B53 = 0.063692468666290;
constexpr double A54 = 0.386708617503269, B54 = 0.226007483236906;

struct Seg {
  int line, a, n;
  bool periodic;
};

struct HPatch {
  fc_patch_desc d;
  long long off = 0, gbase = -1;
  int n1 = 0, n2 = 0;
  bool periodic1 = false;
  double h1 = 0, h2 = 0;       // parameter spacings
  double hhat = 0, htil = 0;   // largest / smallest distance between index-adjacent points
  std::vector<double> x, y;    // physical coordinates (n2*n1)
  std::vector<uint8_t> blank, recv, gen, nodiff;
  std::vector<int> depth;
  std::vector<Seg> seg1, seg2;
  double bx0, bx1, by0, by1;   // bounding box
  // GRID patches: metrics [4][n2*n1] as given, and a uniform bucket grid over the points
  std::vector<double> jm;
  double hcell = 0;
  int hnx = 0, hny = 0;
  std::vector<int> hstart, hidx;  // points of bucket b: hidx[hstart[b] .. hstart[b+1])
};

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
};

inline long long rnd_half_up(double t) { return (long long)std::floor(t + 0.5); }
constexpr double SNAP_IDX = 1e-9;  // index units: stencil offsets this close to an integer are that integer

// receivers whose weights are unit vectors (a coincident donor point) go to the copy list
void split_exchange(const std::vector<Recv>& all, std::vector<Recv>& interp, std::vector<PtCopy>& copies) {
  interp.clear();
  copies.clear();
  for (const Recv& r : all) {
    int m1 = -1, m2 = -1;
    for (int m = 0; m < 3; ++m) {
      const bool u1 = r.w1[m] == 1.0 && r.w1[(m + 1) % 3] == 0.0 && r.w1[(m + 2) % 3] == 0.0;
      const bool u2 = r.w2[m] == 1.0 && r.w2[(m + 1) % 3] == 0.0 && r.w2[(m + 2) % 3] == 0.0;
      if (u1) m1 = m;
      if (u2) m2 = m;
    }
    if (m1 >= 0 && m2 >= 0)
      copies.push_back(PtCopy{r.dst, r.src[3 * m2 + m1]});
    else
      interp.push_back(r);
  }
}
inline double pymod(double a, double n) { return a - n * std::floor(a / n); }

}  // namespace

struct fc_ctx {
  std::string err;
  fc_params prm{};
  std::vector<double> fctab;  // copy of the packed tables
  std::vector<float> sdnn;
  int d = 5, Cmin = 0, Cmax = -1;
  std::vector<HPatch> hp;
  long long P = 0, Pg = 0, active = 0;
  uint64_t launches = 0;

  // FFT plans as uploaded and, per plan, the stage orders the autotuner may choose from
  std::vector<Plan> plans_h;
  std::vector<std::vector<Plan>> plan_cands;
  double tune_report[6] = {0, 0, 0, 0, 0, 0};
  Job* d_tune_jobs = nullptr;  // the autotuner's timing batch (allocated on first use)

  // device tables
  std::vector<void*> allocs;
  DevTables T{};
  Plan* d_plans = nullptr;
  double2* d_tw = nullptr;
  double* d_rp = nullptr;
  int* d_ip = nullptr;
  uint32_t* d_info = nullptr;
  PatchDev* d_patches = nullptr;
  double* d_J = nullptr;
  float* d_sdnn = nullptr;
  double* d_R = nullptr;
  double* d_wtab = nullptr;

  // job queues: [pass] -> batched order (length-descending, split by length class) and per-patch ranges
  struct Queue {
    Job* d = nullptr;
    int n = 0;
    std::vector<std::pair<int, int>> classes;   // (begin, Lmax) ranges of the batched order, end implied
    std::vector<int> class_end;
    Job* dpp = nullptr;                          // per-patch order
    std::vector<int> pbeg, pend, plmax;
    std::vector<Job> h;                          // host copy of the batched order
  };
  Queue q_cart1, q_cart2, q_gen1, q_gen2, q_filt1, q_filt2;
  int* d_fix = nullptr;
  int nfix = 0;
  // the y fluxes of the affine patches' points, written by the q1 pass for the q2 pass, and
  // the points on affine q2 lines that no affine q1 line visits (their y flux comes from
  // k_flux_y_points)
  double* d_Fy = nullptr;
  int* d_fyfix = nullptr;
  int nfyfix = 0;
  GFix* d_gfix = nullptr;
  int ngfix = 0;
  int* d_fcopy1 = nullptr;
  int nfcopy1 = 0;
  int* d_fcopy2 = nullptr;
  int nfcopy2 = 0;
  BcPt* d_bc = nullptr;
  int nbc = 0;
  // host copies of the point lists (restricted to the owned patches by fc_shard)
  std::vector<Recv> h_recv;
  std::vector<BcPt> h_bc;
  std::vector<WallPt> h_walls;
  std::vector<int> h_fix, h_fcopy1, h_fcopy2, h_cdst, h_cptr, h_csrc, h_fyfix;
  std::vector<GFix> h_gfix;
  // sharded execution (fc_shard): this rank of nranks, patch owners, the caller's transport
  int nranks = 1, rank = 0;
  std::vector<int> owner;
  fc_comm_fn comm = nullptr;
  void* comm_user = nullptr;
  uint8_t* d_owned = nullptr;
  struct XPlan {  // one kind of exchange: records per peer, in peer order
    std::vector<long long> scount, rcount;  // doubles per peer
    int nsend = 0, nrecv = 0;
    double* d_sbuf = nullptr;
    double* d_rbuf = nullptr;
  };
  XPlan xp_fringe, xp_visc;
  Recv* d_xsend = nullptr;   // fringe records this rank interpolates for others
  int* d_xsend_dst = nullptr;  // their receivers (other ranks' points): the adjoint's arrivals
  int* d_xrecv = nullptr;    // receivers of this rank filled from others
  int* d_vsend = nullptr;    // window-sum entries this rank sends
  int* d_vrecv = nullptr;    // window-sum entries this rank receives
  bool sharded() const { return nranks > 1; }
  bool comm_failed = false;
  double* d_dtmin = nullptr;
  double* d_ehost = nullptr;  // device copy of the state of fc_rk_step_host

  // free stream (fc_params.freestream) and the parameter adjoint of its Dirichlet points
  bool has_fs = false;
  FsJac fsj{};
  double* d_bcacc = nullptr;  // [nbc][2] per-record sums of one adjoint step
  double* d_part = nullptr;   // [SENS_BLOCKS][2] partial sums of fc_initial_sensitivity
  double* cur_acc = nullptr;  // d_bcacc while an adjoint step accumulates dparam, else null
  WallPt* d_walls = nullptr;  // no-slip adiabatic wall points (of the owned patches, when sharded)
  int nwalls = 0;
  bool any_walls = false;  // the workload has adiabatic walls (the same on every rank)
  Recv* d_recv = nullptr;  // receivers interpolated from 3 x 3 donor stencils
  int nrecv = 0;
  PtCopy* d_rcopy = nullptr;  // receivers that copy a coincident donor point
  int nrcopy = 0;
  Recv* d_recv_all = nullptr;  // every receiver (the exchange transpose zeroes them)
  int nrecv_all = 0;
  int* d_cross_dst = nullptr;
  int* d_cross_ptr = nullptr;
  int* d_cross_src = nullptr;
  int ncross = 0;
  double* d_den = nullptr;

  // workspaces
  double *d_B1 = nullptr, *d_B2 = nullptr, *d_B3 = nullptr, *d_R1 = nullptr, *d_G = nullptr;
  double *d_phi = nullptr, *d_S = nullptr, *d_muhat = nullptr, *d_num = nullptr, *d_tmp = nullptr, *d_mu = nullptr;
  double* d_dt = nullptr;
  unsigned long long* d_pmax = nullptr;
  unsigned long long* d_skip_lines = nullptr;
  double* d_skip_flops = nullptr;
  int* d_flag = nullptr;

  // discrete adjoint: exchange transpose as a CSR over donor points, stage states, accumulators
  int* d_dptr = nullptr;
  int* d_dsrc = nullptr;
  int* d_drecv = nullptr;
  double* d_dw = nullptr;
  int ndon = 0;
  double* d_U[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double *d_A0 = nullptr, *d_A14 = nullptr, *d_A2 = nullptr, *d_A3 = nullptr, *d_PSa = nullptr, *d_PSb = nullptr;
  double *d_FX = nullptr, *d_FY = nullptr;  // adjoint with the filter: state before / after it
  bool adj_ready = false;
  // wall ring for the drag functional
  int* d_wall = nullptr;
  int wall_patch = -1;  // the patch that carries the wall ring
  double* d_wallw = nullptr;
  double* d_wallc = nullptr;
  int nwall = 0;

  // kernel timing instrumentation (events around each launch group)
  bool prof = false;
  struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
    int launches;
  };
  std::vector<ProfRec> prec;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  std::vector<std::string> pnames;
  std::vector<double> pms;
  std::vector<int> pcount;

  cudaEvent_t ev() {
    if (evused == evpool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      evpool.push_back(e);
    }
    return evpool[evused++];
  }

  // graph cache
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};
  int gflags = -1;
  uint64_t glaunches = 0;
  cudaStream_t gstream = nullptr;

  // concurrency inside a pass (length classes) and between the affine and curvilinear
  // chains of a stage: side streams and fork / join events, created on first use
  static constexpr int NSIDE = 3;
  cudaStream_t side[NSIDE] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork_ev[2] = {nullptr, nullptr};
  cudaEvent_t join_ev[NSIDE] = {nullptr, nullptr, nullptr};
  bool side_ready = false;
  bool concurrent = true;
  bool ensure_side() {
    if (side_ready) return true;
    for (int k = 0; k < NSIDE; ++k)
      if (cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&join_ev[k], cudaEventDisableTiming) != cudaSuccess)
        return false;
    for (int k = 0; k < 2; ++k)
      if (cudaEventCreateWithFlags(&fork_ev[k], cudaEventDisableTiming) != cudaSuccess) return false;
    side_ready = true;
    return true;
  }

  ~fc_ctx() {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (int k = 0; k < NSIDE; ++k) {
      if (side[k]) cudaStreamDestroy(side[k]);
      if (join_ev[k]) cudaEventDestroy(join_ev[k]);
    }
    for (int k = 0; k < 2; ++k)
      if (fork_ev[k]) cudaEventDestroy(fork_ev[k]);
    for (cudaEvent_t e : evpool) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
  }

  template <class T>
  bool alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
      err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
      *p = nullptr;
      return false;
    }
    allocs.push_back(*p);
    return true;
  }
  template <class T>
  bool upload(T** p, const std::vector<T>& v) {
    if (!alloc(p, v.size())) return false;
    if (v.empty()) return true;
    cudaError_t e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      err = std::string("cudaMemcpy failed: ") + cudaGetErrorString(e);
      return false;
    }
    return true;
  }
};

namespace {

fc_status fail(fc_ctx* c, fc_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

fc_status cuda_check(fc_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, FC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return FC_OK;
}

// cuda_check, plus the status of the communication callbacks of a sharded call
fc_status comm_check(fc_ctx* c, const char* where) {
  if (c->comm_failed) {
    c->comm_failed = false;
    return fail(c, FC_ERR_CUDA, std::string(where) + ": the communication callback failed");
  }
  return cuda_check(c, where);
}

// ---------------------------------------------------------------- geometry (Sec. 3)
void grid_coords(HPatch& h) {
  const fc_patch_desc& d = h.d;
  h.x.resize((size_t)h.n1 * h.n2);
  h.y.resize(h.x.size());
  if (d.kind == FC_PATCH_GRID) {
    std::copy(d.x, d.x + h.x.size(), h.x.begin());
    std::copy(d.y, d.y + h.y.size(), h.y.begin());
  } else
  for (int j = 0; j < h.n2; ++j)
    for (int i = 0; i < h.n1; ++i) {
      const size_t k = (size_t)j * h.n1 + i;
      if (d.kind == FC_PATCH_AFFINE) {
        h.x[k] = d.geom[0] + (d.geom[1] - d.geom[0]) * i / (h.n1 - 1);
        h.y[k] = d.geom[2] + (d.geom[3] - d.geom[2]) * j / (h.n2 - 1);
      } else {
        const double th = 2.0 * PI * i / h.n1;
        const double r = d.geom[2] + (d.geom[3] - d.geom[2]) * j / (h.n2 - 1);
        h.x[k] = d.geom[0] + r * std::cos(th);
        h.y[k] = d.geom[1] + r * std::sin(th);
      }
    }
  h.bx0 = *std::min_element(h.x.begin(), h.x.end());
  h.bx1 = *std::max_element(h.x.begin(), h.x.end());
  h.by0 = *std::min_element(h.y.begin(), h.y.end());
  h.by1 = *std::max_element(h.y.begin(), h.y.end());
}

// GRID patches: the grid point nearest to (x, y) (ties: the smallest flat index), by
// rings of buckets around the query's bucket; -1 if (x, y) is more than one bucket
// outside the patch's bounding box
long long grid_nearest(const HPatch& h, double x, double y) {
  if (x < h.bx0 - h.hcell || x > h.bx1 + h.hcell || y < h.by0 - h.hcell || y > h.by1 + h.hcell) return -1;
  const int cx = std::min(std::max((int)std::floor((x - h.bx0) / h.hcell), 0), h.hnx - 1);
  const int cy = std::min(std::max((int)std::floor((y - h.by0) / h.hcell), 0), h.hny - 1);
  long long best = -1;
  double bd = 0;
  for (int r = 0; r <= std::max(h.hnx, h.hny); ++r) {
    for (int by = cy - r; by <= cy + r; ++by) {
      if (by < 0 || by >= h.hny) continue;
      for (int bx = cx - r; bx <= cx + r; ++bx) {
        if (bx < 0 || bx >= h.hnx) continue;
        if (std::max(std::abs(bx - cx), std::abs(by - cy)) != r) continue;
        const int b = by * h.hnx + bx;
        for (int q = h.hstart[b]; q < h.hstart[b + 1]; ++q) {
          const long long k = h.hidx[q];
          const double dx = h.x[k] - x, dy = h.y[k] - y, dd = dx * dx + dy * dy;
          if (best < 0 || dd < bd || (dd == bd && k < best)) {
            best = k;
            bd = dd;
          }
        }
      }
    }
    // every point of a bucket in ring r + 1 or beyond is at least r buckets away
    if (best >= 0 && bd < (r * h.hcell) * (r * h.hcell)) break;
  }
  return best;
}

// GRID patches: fractional indices of (x, y) by Newton's method on the 3 x 3 quadratic
// (Lagrange) interpolant of the grid around a stencil centre, started at the nearest
// grid point, which is also the first centre (clamped to [1, n - 2] along a
// non-periodic direction). A direction's centre moves to rnd(s) (clamped) only when the
// estimate is more than 0.75 from it: Newton cannot cycle between two neighbouring
// stencils across a half-integer. At most 30 steps, stopping after a step with
// |ds1| + |ds2| < 1e-11 (quadratic convergence leaves an error at rounding level).
// Returns false (and indices far outside the grid) when there is no nearby point or
// the iteration breaks down.
bool grid_inverse(const HPatch& h, double x, double y, double& s1, double& s2) {
  s1 = s2 = -1e9;
  const long long k0 = grid_nearest(h, x, y);
  if (k0 < 0) return false;
  double a1 = (double)(k0 % h.n1), a2 = (double)(k0 / h.n1);
  auto centre1 = [&](double a) {
    const long long c = rnd_half_up(a);
    return h.periodic1 ? c : std::min<long long>(std::max<long long>(c, 1), h.n1 - 2);
  };
  auto centre2 = [&](double a) { return std::min<long long>(std::max<long long>(rnd_half_up(a), 1), h.n2 - 2); };
  long long c1 = centre1(a1), c2 = centre2(a2);
  for (int it = 0; it < 30; ++it) {
    if (std::fabs(a1 - (double)c1) > 0.75) c1 = centre1(a1);
    if (std::fabs(a2 - (double)c2) > 0.75) c2 = centre2(a2);
    const double t1 = a1 - (double)c1, t2 = a2 - (double)c2;
    const double L[3] = {0.5 * t1 * (t1 - 1.0), 1.0 - t1 * t1, 0.5 * t1 * (t1 + 1.0)};
    const double dL[3] = {t1 - 0.5, -2.0 * t1, t1 + 0.5};
    const double M[3] = {0.5 * t2 * (t2 - 1.0), 1.0 - t2 * t2, 0.5 * t2 * (t2 + 1.0)};
    const double dM[3] = {t2 - 0.5, -2.0 * t2, t2 + 0.5};
    double X = 0, Y = 0, Xa = 0, Xb = 0, Ya = 0, Yb = 0;
    for (int b = 0; b < 3; ++b) {
      const long long jj = c2 + b - 1;
      for (int a = 0; a < 3; ++a) {
        long long ii = c1 + a - 1;
        if (h.periodic1) ii = ((ii % h.n1) + h.n1) % h.n1;
        const size_t k = (size_t)jj * h.n1 + (size_t)ii;
        const double w = L[a] * M[b], wa = dL[a] * M[b], wb = L[a] * dM[b];
        X += w * h.x[k];
        Y += w * h.y[k];
        Xa += wa * h.x[k];
        Xb += wb * h.x[k];
        Ya += wa * h.y[k];
        Yb += wb * h.y[k];
      }
    }
    const double rx = X - x, ry = Y - y, det = Xa * Yb - Xb * Ya;
    if (!(std::fabs(det) > 0.0)) return false;
    const double d1 = -(Yb * rx - Xb * ry) / det, d2 = -(-Ya * rx + Xa * ry) / det;
    a1 += d1;
    a2 += d2;
    if (!(std::fabs(a1) < 1e12 && std::fabs(a2) < 1e12)) return false;
    if (std::fabs(d1) + std::fabs(d2) < 1e-11) {
      s1 = h.periodic1 ? pymod(a1, (double)h.n1) : a1;
      s2 = a2;
      return true;
    }
  }
  return false;
}

// fractional grid indices of a physical point (inverse of the patch map)
inline void frac_index(const HPatch& h, double x, double y, double& s1, double& s2) {
  const fc_patch_desc& d = h.d;
  if (d.kind == FC_PATCH_GRID) {
    grid_inverse(h, x, y, s1, s2);
    return;
  }
  if (d.kind == FC_PATCH_AFFINE) {
    s1 = (x - d.geom[0]) / (d.geom[1] - d.geom[0]) * (h.n1 - 1);
    s2 = (y - d.geom[2]) / (d.geom[3] - d.geom[2]) * (h.n2 - 1);
  } else {
    const double th = pymod(std::atan2(y - d.geom[1], x - d.geom[0]), 2.0 * PI);
    const double r = std::hypot(x - d.geom[0], y - d.geom[1]);
    s1 = th / (2.0 * PI) * h.n1;
    s2 = (r - d.geom[2]) / (d.geom[3] - d.geom[2]) * (h.n2 - 1);
  }
}

inline void nearest(const HPatch& h, double s1, double s2, int& z1, int& z2) {
  long long a = rnd_half_up(s1), b = rnd_half_up(s2);
  if (h.periodic1) {
    a %= h.n1;
    if (a < 0) a += h.n1;
  } else {
    a = std::min<long long>(std::max<long long>(a, 0), h.n1 - 1);
  }
  b = std::min<long long>(std::max<long long>(b, 0), h.n2 - 1);
  z1 = (int)a;
  z2 = (int)b;
}

inline bool contains(const HPatch& h, double s1, double s2) {
  if (!(s2 >= -CONTAIN_TOL && s2 <= h.n2 - 1 + CONTAIN_TOL)) return false;
  if (!h.periodic1 && !(s1 >= -CONTAIN_TOL && s1 <= h.n1 - 1 + CONTAIN_TOL)) return false;
  int z1, z2;
  nearest(h, s1, s2, z1, z2);
  return !h.blank[(size_t)z2 * h.n1 + z1];
}

void build_patch(HPatch& h, const fc_params& prm) {
  const fc_patch_desc& d = h.d;
  h.n1 = d.n1;
  h.n2 = d.n2;
  h.periodic1 = d.kind == FC_PATCH_OGRID ||
                (d.kind == FC_PATCH_GRID && d.side[0] == FC_SIDE_PERIODIC && d.side[1] == FC_SIDE_PERIODIC);
  h.h1 = h.periodic1 ? 1.0 / h.n1 : 1.0 / (h.n1 - 1);
  h.h2 = 1.0 / (h.n2 - 1);
  grid_coords(h);
  if (d.kind == FC_PATCH_GRID) {
    // spacings: largest / smallest distance between index-adjacent points (periodic: wrapped)
    const size_t N = (size_t)h.n1 * h.n2;
    if (d.metrics)
      h.jm.assign(d.metrics, d.metrics + 4 * N);
    else
      h.jm.assign(4 * N, 0.0);  // computed on the device from the points after the upload
    double mx = 0.0, mn = 1e300;
    for (int j = 0; j < h.n2; ++j)
      for (int i = 0; i < h.n1; ++i) {
        const size_t k = (size_t)j * h.n1 + i;
        if (i + 1 < h.n1 || h.periodic1) {
          const size_t q = (size_t)j * h.n1 + (i + 1) % h.n1;
          const double dd = std::hypot(h.x[q] - h.x[k], h.y[q] - h.y[k]);
          mx = std::max(mx, dd);
          mn = std::min(mn, dd);
        }
        if (j + 1 < h.n2) {
          const size_t q = k + h.n1;
          const double dd = std::hypot(h.x[q] - h.x[k], h.y[q] - h.y[k]);
          mx = std::max(mx, dd);
          mn = std::min(mn, dd);
        }
      }
    h.hhat = mx;
    h.htil = mn;
    // bucket grid for nearest-point queries (bucket size: the largest spacing)
    h.hcell = std::max(mx, 1e-300);
    // at most about 4 buckets per point (a grid whose bounding box is large against its
    // spacings gets coarser buckets; the search result does not depend on their size)
    while ((h.bx1 - h.bx0) / h.hcell * ((h.by1 - h.by0) / h.hcell) > 4.0 * (double)N + 1024.0) h.hcell *= 2.0;
    h.hnx = std::max(1, (int)std::ceil((h.bx1 - h.bx0) / h.hcell) + 1);
    h.hny = std::max(1, (int)std::ceil((h.by1 - h.by0) / h.hcell) + 1);
    std::vector<int> cnt((size_t)h.hnx * h.hny + 1, 0), bk(N);
    for (size_t k = 0; k < N; ++k) {
      const int bx = std::min((int)std::floor((h.x[k] - h.bx0) / h.hcell), h.hnx - 1);
      const int by = std::min((int)std::floor((h.y[k] - h.by0) / h.hcell), h.hny - 1);
      bk[k] = by * h.hnx + bx;
      cnt[bk[k] + 1]++;
    }
    for (size_t b = 1; b < cnt.size(); ++b) cnt[b] += cnt[b - 1];
    h.hstart = cnt;
    h.hidx.assign(N, 0);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (size_t k = 0; k < N; ++k) h.hidx[fill[bk[k]]++] = (int)k;
  } else if (d.kind == FC_PATCH_AFFINE) {
    const double hx = (d.geom[1] - d.geom[0]) / (h.n1 - 1), hy = (d.geom[3] - d.geom[2]) / (h.n2 - 1);
    h.hhat = std::max(hx, hy);
    h.htil = std::min(hx, hy);
  } else {
    const double dr = (d.geom[3] - d.geom[2]) / (h.n2 - 1);
    const double ch = 2.0 * std::sin(PI / h.n1);
    h.hhat = std::max(dr, d.geom[3] * ch);
    h.htil = std::min(dr, d.geom[2] * ch);
  }
  const size_t N = (size_t)h.n1 * h.n2;
  h.blank.assign(N, 0);
  if (d.kind != FC_PATCH_OGRID && d.hole[2] > 0) {
    const double R2 = d.hole[2] * d.hole[2];
    for (size_t k = 0; k < N; ++k) {
      const double dx = h.x[k] - d.hole[0], dy = h.y[k] - d.hole[1];
      h.blank[k] = (dx * dx + dy * dy) < R2;
    }
  }
  // internal-boundary points: points of internal sides, and non-blank points next to a blanked one
  auto idx = [&](int i, int j) { return (size_t)j * h.n1 + i; };
  std::vector<int> dep(N, prm.depth_cap);
  std::vector<size_t> frontier;
  for (int j = 0; j < h.n2; ++j)
    for (int i = 0; i < h.n1; ++i) {
      const size_t k = idx(i, j);
      if (h.blank[k]) continue;
      bool ib = (i == 0 && d.side[0] == FC_SIDE_INTERNAL) || (i == h.n1 - 1 && d.side[1] == FC_SIDE_INTERNAL) ||
                (j == 0 && d.side[2] == FC_SIDE_INTERNAL) || (j == h.n2 - 1 && d.side[3] == FC_SIDE_INTERNAL);
      for (int b = -1; b <= 1 && !ib; ++b)
        for (int a = -1; a <= 1 && !ib; ++a) {
          int ii = i + a, jj = j + b;
          if (jj < 0 || jj >= h.n2) continue;
          if (h.periodic1)
            ii = (ii + h.n1) % h.n1;
          else if (ii < 0 || ii >= h.n1)
            continue;
          if (h.blank[idx(ii, jj)]) ib = true;
        }
      if (ib) {
        dep[k] = 0;
        frontier.push_back(k);
      }
    }
  // multi-source breadth-first search with 8-neighbour steps = max-index-norm distance (eq. fringe_region)
  for (int lev = 1; lev < prm.depth_cap && !frontier.empty(); ++lev) {
    std::vector<size_t> next;
    for (size_t k : frontier) {
      const int j = (int)(k / h.n1), i = (int)(k % h.n1);
      for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
          int ii = i + a, jj = j + b;
          if (jj < 0 || jj >= h.n2) continue;
          if (h.periodic1)
            ii = (ii + h.n1) % h.n1;
          else if (ii < 0 || ii >= h.n1)
            continue;
          const size_t q = idx(ii, jj);
          if (dep[q] > lev) {
            dep[q] = lev;
            next.push_back(q);
          }
        }
    }
    frontier.swap(next);
  }
  for (size_t k = 0; k < N; ++k)
    if (h.blank[k]) dep[k] = 0;
  h.depth = dep;
  h.recv.assign(N, 0);
  h.gen.assign(N, 0);
  for (size_t k = 0; k < N; ++k) {
    if (h.blank[k]) continue;
    h.recv[k] = dep[k] < prm.n_f;
    h.gen[k] = dep[k] >= prm.n_v;
  }
  // segments: maximal runs of non-blank points along grid lines
  h.seg1.clear();
  h.seg2.clear();
  for (int j = 0; j < h.n2; ++j) {
    if (h.periodic1) {
      h.seg1.push_back({j, 0, h.n1, true});
      continue;
    }
    int a = -1;
    for (int i = 0; i <= h.n1; ++i) {
      const bool on = i < h.n1 && !h.blank[idx(i, j)];
      if (on && a < 0) a = i;
      if (!on && a >= 0) {
        h.seg1.push_back({j, a, i - a, false});
        a = -1;
      }
    }
  }
  for (int i = 0; i < h.n1; ++i) {
    int a = -1;
    for (int j = 0; j <= h.n2; ++j) {
      const bool on = j < h.n2 && !h.blank[idx(i, j)];
      if (on && a < 0) a = j;
      if (!on && a >= 0) {
        h.seg2.push_back({i, a, j - a, false});
        a = -1;
      }
    }
  }
  h.nodiff = h.blank;
  for (const Seg& s : h.seg1)
    if (!s.periodic && s.n < 2 * prm.d)
      for (int t = 0; t < s.n; ++t) h.nodiff[idx(s.a + t, s.line)] = 1;
  for (const Seg& s : h.seg2)
    if (s.n < 2 * prm.d)
      for (int t = 0; t < s.n; ++t) h.nodiff[idx(s.line, s.a + t)] = 1;
}

// ---------------------------------------------------------------- FFT plans and continuation tables
// FP64 operations of a radix-R butterfly in the line engine (complex adds, the folded
// constant multiplies of the small DFTs)
int butterfly_ops(int R) { return R == 2 ? 4 : R == 4 ? 16 : R == 8 ? 52 : R == 3 ? 14 : R == 5 ? 36 : 66; }

// Cost of one in-place transform of two packed sequences with the given stage radices,
// counted in warp lane-slots: the FP64 pipe spends the same time on a warp instruction
// whatever the number of active lanes (measured), so a stage with 2 L / R butterflies
// costs ceil(2 L / R / 32) x 32 butterflies of R, and as many times R - 1 twiddle
// products on every stage but the last. (Charging each stage extra operations for its
// shared-memory round trip made the chosen plans slower on the Mach-25 workload, so the
// count is FP64 operations only.)
long long lane_cost(int L, const std::vector<int>& order) {
  long long c = 0;
  for (size_t s = 0; s < order.size(); ++s) {
    const int R = order[s];
    const long long slots = (long long)((2 * (L / R) + 31) / 32) * 32;
    c += slots * butterfly_ops(R);
    if (s + 1 < order.size()) c += slots * 4 * (R - 1);
  }
  return c;
}

// Stage radices of a continued length L: among the factorisations of its 7-smooth part
// into 8, 7, 5, 4, 3, 2, ordered with the power-of-two radices first, the one with the
// smallest lane_cost (ties: the first found); larger prime factors follow as generic
// stages. Power-of-two butterflies first: their sums and differences of samples half a
// span apart cancel a line's large mean exactly (the weighted sums of the odd radices
// do not), which keeps the transform of large-mean data (Mach-25 fluxes) accurate; an
// unrestricted order was 3x less accurate on 1080-point lines for 3% less work.
std::vector<std::vector<int>> plan_orders(int L, int k);
std::vector<int> factorize(int L) { return plan_orders(L, 1)[0]; }

// The k stage orders of smallest lane_cost (stable: equal costs keep the enumeration
// order, so the first is the cost model's choice): the candidates of the autotuner.
std::vector<std::vector<int>> plan_orders(int L, int k) {
  int m = L;
  for (int p : {2, 3, 5, 7})
    while (m % p == 0) m /= p;
  const int smooth = L / m;
  std::vector<int> rest;
  for (int p = 11; m > 1; p += 2)
    while (m % p == 0) {
      rest.push_back(p);
      m /= p;
    }
  std::vector<std::pair<long long, std::vector<int>>> all;
  std::vector<int> cur;
  const int radices[6] = {8, 7, 5, 4, 3, 2};
  // multisets in non-increasing radix order, then the distinct orders of each
  std::function<void(int, int)> rec = [&](int left, int from) {
    if (left == 1) {
      std::vector<int> p2, odd;
      for (int r : cur) (r == 2 || r == 4 || r == 8 ? p2 : odd).push_back(r);
      std::sort(p2.begin(), p2.end());
      do {
        std::sort(odd.begin(), odd.end());
        do {
          std::vector<int> perm = p2;
          perm.insert(perm.end(), odd.begin(), odd.end());
          all.push_back({lane_cost(L, perm), perm});
        } while (std::next_permutation(odd.begin(), odd.end()));
      } while (std::next_permutation(p2.begin(), p2.end()));
      return;
    }
    for (int k = from; k < 6; ++k)
      if (left % radices[k] == 0) {
        cur.push_back(radices[k]);
        rec(left / radices[k], k);
        cur.pop_back();
      }
  };
  rec(smooth, 0);
  std::stable_sort(all.begin(), all.end(),
                   [](const std::pair<long long, std::vector<int>>& a, const std::pair<long long, std::vector<int>>& b) {
                     return a.first < b.first;
                   });
  std::vector<std::vector<int>> out;
  for (size_t i = 0; i < all.size() && (int)out.size() < std::max(k, 1); ++i) {
    std::vector<int> o = all[i].second;
    o.insert(o.end(), rest.begin(), rest.end());
    out.push_back(o);
  }
  if (out.empty()) out.push_back(rest);  // L = 1 or a product of large primes only
  return out;
}

bool smooth7(int n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Estimated FP64 operations of one in-place transform of length L: L factored greedily
// into 8s, 4s, 2s, 3s, 5s, 7s (the order of the plans), L/R butterflies of radix R per
// stage at B(R) operations (B = 4, 16, 52 for R = 2, 4, 8; 14, 36, 66 for R = 3, 5, 7)
// and 4 operations per twiddled element, (R - 1) L / R of them, on every stage but the
// last. -1 when L has a prime factor above 7.
long long fft_cost(int L) {
  std::vector<int> f;
  int m = L;
  for (int r : {8, 4, 2, 3, 5, 7})
    while (m % r == 0) {
      f.push_back(r);
      m /= r;
    }
  if (m != 1) return -1;
  long long cost = 0;
  for (size_t s = 0; s < f.size(); ++s) {
    const int R = f[s];
    const int B = R == 2 ? 4 : R == 4 ? 16 : R == 8 ? 52 : R == 3 ? 14 : R == 5 ? 36 : 66;
    cost += (long long)(L / R) * B;
    if (s + 1 < f.size()) cost += 4LL * (L / R) * (R - 1);
  }
  return cost;
}

// Weights of the adiabatic wall temperature: theta_w = sum_{j=1}^{d-1} w[j-1] theta_j is the
// value at 0 of the polynomial p of degree d-1 with p'(0) = 0 and p(j) = theta_j,
// j = 1..d-1 (unit spacing along the wall-normal grid line; the Neumann FC end data).
// Solves for the coefficients (a_0, a_2, .., a_{d-1}) in long double; w = first row of
// the inverse.
std::vector<double> adiabatic_weights(int d) {
  const int m = d - 1;
  std::vector<long double> A((size_t)m * m), Inv((size_t)m * m, 0.0L);
  for (int j = 1; j <= m; ++j)
    for (int c = 0; c < m; ++c) {
      const int k = c == 0 ? 0 : c + 1;  // powers 0, 2, 3, .., d-1
      long double v = 1.0L;
      for (int q = 0; q < k; ++q) v *= (long double)j;
      A[(size_t)(j - 1) * m + c] = v;
    }
  for (int i = 0; i < m; ++i) Inv[(size_t)i * m + i] = 1.0L;
  for (int col = 0; col < m; ++col) {  // Gauss-Jordan with partial pivoting
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * m + col]) > std::fabs(A[(size_t)piv * m + col])) piv = r;
    for (int q = 0; q < m; ++q) {
      std::swap(A[(size_t)col * m + q], A[(size_t)piv * m + q]);
      std::swap(Inv[(size_t)col * m + q], Inv[(size_t)piv * m + q]);
    }
    const long double dv = A[(size_t)col * m + col];
    for (int q = 0; q < m; ++q) {
      A[(size_t)col * m + q] /= dv;
      Inv[(size_t)col * m + q] /= dv;
    }
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      const long double f = A[(size_t)r * m + col];
      for (int q = 0; q < m; ++q) {
        A[(size_t)r * m + q] -= f * A[(size_t)col * m + q];
        Inv[(size_t)r * m + q] -= f * Inv[(size_t)col * m + q];
      }
    }
  }
  std::vector<double> w(m);
  for (int j = 0; j < m; ++j) w[j] = (double)Inv[j];  // row 0: coefficient a_0 = p(0)
  return w;
}

// Continuation length C of a non-periodic line of N points (the paper leaves C free):
//   policy 0: C0 on every line;
//   policy 1: the smallest C >= C0 with N + C 7-smooth;
//   policy 2: the C in [C0, Cmax] whose continued length has the smallest fft_cost
//             (ties to the smaller C); policy 1 if none is 7-smooth.
int choose_continuation(int N, const fc_params& prm, int Cmax) {
  if (prm.c_policy == 0) return prm.C0;
  if (prm.c_policy == 2) {
    int best = -1;
    long long best_cost = 0;
    for (int C = prm.C0; C <= Cmax; ++C) {
      const long long k = fft_cost(N + C);
      if (k >= 0 && (best < 0 || k < best_cost)) {
        best = C;
        best_cost = k;
      }
    }
    if (best >= 0) return best;
  }
  int C = prm.C0;
  while (!smooth7(N + C)) ++C;
  return C;
}

}  // namespace

// ---------------------------------------------------------------- context build
namespace {

struct Builder {
  fc_ctx* c;
  std::map<int, int> plan_of_L;
  std::vector<Plan> plans;
  std::vector<double2> tw;
  std::vector<double> rp;
  std::vector<int> ip;
  std::map<int, int> fcm_of_C;

  std::vector<std::vector<Plan>> cands;  // per plan: stage orders for the autotuner, [0] = plans[i]

  // slot -> mode table of an in-place transform with p's stage order, appended to the int pool:
  // slot p = sum_s d_s L/(R_0..R_s) holds mode k = sum_s d_s R_0..R_{s-1}
  void rev_table(Plan& p) {
    const int L = p.L;
    p.rev = (int)ip.size();
    for (int slot = 0; slot < L; ++slot) {
      int rem = slot, k = 0, w = 1, span = L;
      for (int st = 0; st < p.nst; ++st) {
        span /= p.rad[st];
        const int dgt = rem / span;
        rem -= dgt * span;
        k += dgt * w;
        w *= p.rad[st];
      }
      ip.push_back(k);
    }
  }

  // the FMA-form records of p (fc_tables.h): inverse, then forward with the filter table
  void fma_tables(Plan& p) {
    fma_inverse_records(p, tw);
    const std::vector<int> rev(ip.begin() + p.rev, ip.begin() + p.rev + p.L);
    const std::vector<double> sig(rp.begin() + p.sig, rp.begin() + p.sig + p.L);
    fma_forward_records(p, tw, rp, rev.data(), sig.data());
  }

  int plan(int L) {
    auto it = plan_of_L.find(L);
    if (it != plan_of_L.end()) return it->second;
    Plan p{};
    p.L = L;
    const std::vector<std::vector<int>> orders = plan_orders(L, AUTOTUNE_PLANS);
    const std::vector<int>& f = orders[0];  // a length below 2^24 has at most MAXST prime factors
    p.nst = (int)f.size();
    for (int s = 0; s < p.nst; ++s) p.rad[s] = f[s];
    p.tw = (int)tw.size();
    for (int e = 0; e < L; ++e) {
      const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)e / (long double)L;
      double2 w;
      w.x = (double)cosl(ang);
      w.y = (double)sinl(ang);
      tw.push_back(w);
    }
    rev_table(p);
    p.sig = (int)rp.size();
    const fc_params& prm = c->prm;
    for (int t = 0; t < L; ++t) {
      long double k = (2 * t <= L) ? t : t - L;
      if (2 * t == L) k = L / 2.0L;
      const long double z = 2.0L * k / (long double)L;
      rp.push_back((double)(expl(-(long double)prm.alpha_f * powl(z, prm.p_f)) / (long double)L));
    }
    fma_tables(p);
    plans.push_back(p);
    std::vector<Plan> alt{p};
    for (size_t o = 1; o < orders.size(); ++o) {
      if ((int)orders[o].size() > MAXST) continue;
      Plan q = p;
      q.nst = (int)orders[o].size();
      for (int s = 0; s < q.nst; ++s) q.rad[s] = orders[o][s];
      rev_table(q);
      fma_tables(q);
      alt.push_back(q);
    }
    cands.push_back(alt);
    plan_of_L[L] = (int)plans.size() - 1;
    return (int)plans.size() - 1;
  }

  // combined continuation matrices ML = A_l Q^T, MR = A_r Q^T for C points
  int fcm(int C) {
    auto it = fcm_of_C.find(C);
    if (it != fcm_of_C.end()) return it->second;
    const int d = c->d;
    const double* base = c->fctab.data() + 3;
    for (int cc = c->Cmin; cc < C; ++cc) base += d * d + 2 * cc * d;
    const double* Q = base;
    const double* AL = Q + d * d;
    const double* AR = AL + C * d;
    const int off = (int)rp.size();
    // ML = A_l Q^T and MR = A_r Q^T (rows k, columns i), then uL = ML 1, vL = ML tau_l,
    // uR = MR 1, vR = MR tau_r with tau_l = i, tau_r = i - (d - 1) (detrended evaluation)
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
    fcm_of_C[C] = off;
    return off;
  }

  int choose_C(int N) { return choose_continuation(N, c->prm, c->Cmax); }
};

void make_queue(fc_ctx* c, fc_ctx::Queue& q, std::vector<Job>& jobs, const std::vector<Plan>& plans, int npatch,
                bool& ok) {
  // per-patch order: stable by patch
  std::vector<Job> pp = jobs;
  std::stable_sort(pp.begin(), pp.end(), [](const Job& a, const Job& b) { return a.patch < b.patch; });
  q.pbeg.assign(npatch, 0);
  q.pend.assign(npatch, 0);
  q.plmax.assign(npatch, 0);
  for (int k = 0; k < (int)pp.size(); ++k) {
    const int p = pp[k].patch;
    if (q.pend[p] == 0) q.pbeg[p] = k;
    q.pend[p] = k + 1;
    q.plmax[p] = std::max(q.plmax[p], plans[pp[k].plan].L);
  }
  // batched order: longest continued length first, split in power-of-two length classes
  std::stable_sort(jobs.begin(), jobs.end(),
                   [&](const Job& a, const Job& b) { return plans[a.plan].L > plans[b.plan].L; });
  q.n = (int)jobs.size();
  q.classes.clear();
  q.class_end.clear();
  int k = 0;
  while (k < q.n) {
    const int Lmax = plans[jobs[k].plan].L;
    int cls = 1;
    while (cls < Lmax) cls <<= 1;
    int e = k;
    while (e < q.n && plans[jobs[e].plan].L > cls / 2) ++e;
    q.classes.push_back({k, Lmax});
    q.class_end.push_back(e);
    k = e;
  }
  ok = ok && c->upload(&q.d, jobs) && c->upload(&q.dpp, pp);
  q.h = jobs;
}

}  // namespace

// ---------------------------------------------------------------- API
extern "C" {

fc_status fc_init_patches(fc_ctx** out, const fc_patch_desc* patches, int npatch, const fc_params* prm, void* stream) {
  if (!out || !patches || npatch <= 0 || !prm) return FC_ERR_INVALID;
  *out = nullptr;
  fc_ctx* c = new fc_ctx();
  c->prm = *prm;
  if (!prm->fc_tables || prm->fc_tables_len < 3) {
    fprintf(stderr, "fc_init_patches: missing FC tables\n");
    delete c;
    return FC_ERR_INVALID;
  }
  c->fctab.assign(prm->fc_tables, prm->fc_tables + prm->fc_tables_len);
  c->d = (int)c->fctab[0];
  c->Cmin = (int)c->fctab[1];
  c->Cmax = (int)c->fctab[2];
  auto bad = [&](const std::string& m) {
    fprintf(stderr, "fc_init_patches: %s\n", m.c_str());
    delete c;
    return FC_ERR_INVALID;
  };
  if (c->d != prm->d) return bad("table order d differs from params.d");
  {
    size_t need = 3;
    for (int C = c->Cmin; C <= c->Cmax; ++C) need += (size_t)c->d * c->d + 2 * (size_t)C * c->d;
    if (need != (size_t)prm->fc_tables_len) return bad("FC table length mismatch");
  }
  if (!prm->sdnn_w || prm->sdnn_len != SDNN_H * 7 + SDNN_H + SDNN_H * SDNN_H + SDNN_H + 4 * SDNN_H + 4)
    return bad("SDNN weights missing or of the wrong size");
  if (prm->win_r < 1 || prm->win_r > 32 || prm->n_f < 1 || prm->n_v < 1 || prm->depth_cap < 2) return bad("bad params");
  if (prm->wall_form != 0 && prm->wall_form != 1) return bad("wall_form must be 0 or 1");
  c->sdnn.assign(prm->sdnn_w, prm->sdnn_w + prm->sdnn_len);
  if (prm->freestream[0] > 0.0) {  // d e_fs / d(M, alpha) at fixed rho and p (eq. mach_flow_ic)
    const double rho = prm->freestream[0], u = prm->freestream[1], v = prm->freestream[2];
    const double pr = prm->freestream[3];
    if (!(pr > 0.0) || !std::isfinite(u) || !std::isfinite(v)) return bad("bad free stream");
    const double a = std::sqrt(prm->gamma * pr / rho), M = std::hypot(u, v) / a, al = std::atan2(v, u);
    const double ca = std::cos(al), sa = std::sin(al);
    const double dM[4] = {0.0, rho * a * ca, rho * a * sa, rho * a * a * M};
    const double dA[4] = {0.0, -rho * a * M * sa, rho * a * M * ca, 0.0};
    for (int k = 0; k < 4; ++k) {
      c->fsj.dM[k] = dM[k];
      c->fsj.dA[k] = dA[k];
    }
    c->has_fs = true;
  }
  cudaStream_t st = (cudaStream_t)stream;
  (void)st;

  // ---- host geometry
  c->hp.resize(npatch);
  long long off = 0, goff = 0;
  for (int p = 0; p < npatch; ++p) {
    HPatch& h = c->hp[p];
    h.d = patches[p];
    if (h.d.n1 < 2 || h.d.n2 < 2 ||
        (h.d.kind != FC_PATCH_AFFINE && h.d.kind != FC_PATCH_OGRID && h.d.kind != FC_PATCH_GRID))
      return bad("bad patch descriptor " + std::to_string(p));
    if (h.d.kind == FC_PATCH_GRID) {
      if (!h.d.x || !h.d.y || h.d.n1 < 3 || h.d.n2 < 3)
        return bad("GRID patch " + std::to_string(p) + " needs x, y and at least 3 x 3 points");
      const bool per1 = h.d.side[0] == FC_SIDE_PERIODIC;
      if (!h.d.metrics && ((!per1 && h.d.n1 < 2 * prm->d) || h.d.n2 < 2 * prm->d))
        return bad("GRID patch " + std::to_string(p) + " without metrics needs 2d points along every non-periodic line");
      for (int s = 0; s < 4; ++s)
        if (h.d.side[s] == FC_SIDE_SLIPWALL || (h.d.side[s] == FC_SIDE_PERIODIC && s >= 2))
          return bad("GRID patch " + std::to_string(p) + ": unsupported side type");
      if ((h.d.side[0] == FC_SIDE_PERIODIC) != (h.d.side[1] == FC_SIDE_PERIODIC))
        return bad("GRID patch " + std::to_string(p) + ": q1 is periodic on both sides or neither");
    }
    build_patch(h, *prm);
    h.off = off;
    off += (long long)h.n1 * h.n2;
    if (h.d.kind != FC_PATCH_AFFINE) {
      h.gbase = goff;
      goff += (long long)h.n1 * h.n2;
    }
  }
  c->P = off;
  c->Pg = goff;
  if (c->P >= (1LL << 31)) return bad("more than 2^31 points");
  c->active = 0;
  for (auto& h : c->hp)
    for (auto b : h.blank) c->active += !b;

  // ---- exchange: donors, stencils, weights (Sec. 3.4.1)
  std::vector<Recv> recv;
  {
    static const int OFFS[5] = {0, -1, 1, -2, 2};
    std::vector<std::pair<int, int>> cands;
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) cands.push_back({a, b});
    std::stable_sort(cands.begin(), cands.end(), [](const std::pair<int, int>& u, const std::pair<int, int>& v) {
      const int su = std::abs(OFFS[u.first]) + std::abs(OFFS[u.second]);
      const int sv = std::abs(OFFS[v.first]) + std::abs(OFFS[v.second]);
      if (su != sv) return su < sv;
      if (u.first != v.first) return u.first < v.first;
      return u.second < v.second;
    });
    long long missing = 0;
    for (int p = 0; p < npatch; ++p) {
      const HPatch& h = c->hp[p];
      std::vector<int> near;
      for (int q = 0; q < npatch; ++q) {
        const HPatch& g = c->hp[q];
        if (q != p && !(h.bx1 < g.bx0 || g.bx1 < h.bx0 || h.by1 < g.by0 || g.by1 < h.by0)) near.push_back(q);
      }
      for (int j = 0; j < h.n2; ++j)
        for (int i = 0; i < h.n1; ++i) {
          const size_t k = (size_t)j * h.n1 + i;
          if (!h.recv[k]) continue;
          const double x = h.x[k], y = h.y[k];
          int best = -1, bdep = -1, ba1 = 0, ba2 = 0;
          double bt1 = 0, bt2 = 0;
          for (int q : near) {
            const HPatch& g = c->hp[q];
            double s1, s2;
            frac_index(g, x, y, s1, s2);
            if (!contains(g, s1, s2)) continue;
            const long long c1 = rnd_half_up(s1), c2 = rnd_half_up(s2);
            bool found = false;
            long long a1 = 0, a2 = 0;
            for (auto& cd : cands) {
              const long long b1 = c1 - 1 + OFFS[cd.first], b2 = c2 - 1 + OFFS[cd.second];
              if (b2 < 0 || b2 > g.n2 - 3) continue;
              if (!g.periodic1 && (b1 < 0 || b1 > g.n1 - 3)) continue;
              bool ok = true;
              for (int m2 = 0; m2 < 3 && ok; ++m2)
                for (int m1 = 0; m1 < 3 && ok; ++m1) {
                  long long i1 = b1 + m1;
                  if (g.periodic1) i1 = ((i1 % g.n1) + g.n1) % g.n1;
                  const size_t kk = (size_t)(b2 + m2) * g.n1 + i1;
                  if (g.blank[kk] || g.recv[kk]) ok = false;
                }
              if (ok) {
                a1 = b1;
                a2 = b2;
                found = true;
                break;
              }
            }
            if (!found) continue;
            int z1, z2;
            nearest(g, s1, s2, z1, z2);
            const int dp = g.depth[(size_t)z2 * g.n1 + z1];
            if (dp > bdep) {
              bdep = dp;
              best = q;
              ba1 = (int)a1;
              ba2 = (int)a2;
              bt1 = g.periodic1 ? pymod(s1 - a1 + 0.5 * g.n1, (double)g.n1) - 0.5 * g.n1 : s1 - a1;
              bt2 = s2 - a2;
            }
          }
          if (best < 0) {
            ++missing;
            continue;
          }
          const HPatch& g = c->hp[best];
          Recv r{};
          r.dst = (int)(h.off + (long long)k);
          for (int m2 = 0; m2 < 3; ++m2)
            for (int m1 = 0; m1 < 3; ++m1) {
              long long i1 = ba1 + m1;
              if (g.periodic1) i1 = ((i1 % g.n1) + g.n1) % g.n1;
              r.src[3 * m2 + m1] = (int)(g.off + (long long)(ba2 + m2) * g.n1 + i1);
            }
          auto lag = [](double t, double* w) {
            w[0] = 0.5 * (t - 1.0) * (t - 2.0);
            w[1] = t * (2.0 - t);
            w[2] = 0.5 * t * (t - 1.0);
          };
          // a receiver that coincides with a donor grid point (shared overlap points of the
          // sub-patches of one patch, Sec. 3.4.2) takes that point's value: offsets within
          // rounding of an integer are that integer (unit weights, an exact copy)
          if (std::fabs(bt1 - std::nearbyint(bt1)) < SNAP_IDX) bt1 = std::nearbyint(bt1);
          if (std::fabs(bt2 - std::nearbyint(bt2)) < SNAP_IDX) bt2 = std::nearbyint(bt2);
          lag(bt1, r.w1);
          lag(bt2, r.w2);
          recv.push_back(r);
        }
    }
    if (missing) {
      c->err = std::to_string(missing) + " receiver points have no valid donor (donor-receiver condition)";
      fprintf(stderr, "fc_init_patches: %s\n", c->err.c_str());
      delete c;
      return FC_ERR_DONOR;
    }
  }
  // short segments must consist of receivers only
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    for (size_t k = 0; k < h.nodiff.size(); ++k)
      if (h.nodiff[k] && !h.blank[k] && !h.recv[k]) {
        c->err = "patch " + std::to_string(p) + " has a line too short for FC containing non-receiver points";
        fprintf(stderr, "fc_init_patches: %s\n", c->err.c_str());
        delete c;
        return FC_ERR_OVERLAP;
      }
  }

  // ---- boundary overwrite lists (Sec. 4.2): slip then Dirichlet; Dirichlet wins at corners
  std::vector<BcPt> bcs;
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    std::map<size_t, BcPt> m;
    auto side_pts = [&](int s, std::vector<size_t>& v) {
      v.clear();
      if (s < 2) {
        const int i = s == 0 ? 0 : h.n1 - 1;
        for (int j = 0; j < h.n2; ++j) v.push_back((size_t)j * h.n1 + i);
      } else {
        const int j = s == 2 ? 0 : h.n2 - 1;
        for (int i = 0; i < h.n1; ++i) v.push_back((size_t)j * h.n1 + i);
      }
    };
    std::vector<size_t> pts;
    for (int s = 0; s < 4; ++s) {
      if (h.d.side[s] != FC_SIDE_SLIPWALL) continue;
      side_pts(s, pts);
      for (size_t k : pts) {
        if (h.blank[k]) continue;
        BcPt& b = m[k];
        b.idx = (int)(h.off + (long long)k);
        if (h.d.kind == FC_PATCH_AFFINE) {
          b.mode |= (s < 2) ? 1 : 2;
        } else {
          const double dx = h.x[k] - h.d.geom[0], dy = h.y[k] - h.d.geom[1];
          const double r = std::hypot(dx, dy);
          b.mode |= 4;
          b.nx = dx / r;
          b.ny = dy / r;
        }
      }
    }
    for (int s = 0; s < 4; ++s) {
      if (h.d.side[s] != FC_SIDE_DIRICHLET) continue;
      side_pts(s, pts);
      // a bc of density 0 holds the free stream; a bc equal to it is a free-stream side too
      bool fs = h.d.bc[s][0] == 0.0;
      if (fs && !c->has_fs) return bad("a Dirichlet side holds the free stream (bc density 0) but none is set");
      const double* q = fs ? prm->freestream : h.d.bc[s];
      if (c->has_fs && !fs) fs = q[0] == prm->freestream[0] && q[1] == prm->freestream[1] &&
                                 q[2] == prm->freestream[2] && q[3] == prm->freestream[3];
      const double rho = q[0], u = q[1], v = q[2], pr = q[3];
      const double val[4] = {rho, rho * u, rho * v, pr / (prm->gamma - 1.0) + 0.5 * rho * (u * u + v * v)};
      for (size_t k : pts) {
        if (h.blank[k]) continue;
        BcPt& b = m[k];
        b.idx = (int)(h.off + (long long)k);
        b.mode = (b.mode & ~16) | 8 | (fs ? 16 : 0);
        for (int cc = 0; cc < 4; ++cc) b.val[cc] = val[cc];
      }
    }
    for (auto& kv : m) bcs.push_back(kv.second);
  }
  // ---- no-slip adiabatic wall points (Sec. 4.2, Remark adiabatic): applied after the overwrites above
  std::vector<WallPt> walls;
  {
    const std::vector<double> aw = adiabatic_weights(prm->d);
    for (int p = 0; p < npatch; ++p) {
      const HPatch& h = c->hp[p];
      for (int s = 0; s < 4; ++s) {
        if (h.d.side[s] != FC_SIDE_ADIABATIC) continue;
        if (h.periodic1 && s < 2) return bad("a wall of a patch periodic in q1 must be a q2 side");
        const int nline = s < 2 ? h.n1 : h.n2;
        if (nline < prm->d + 1) return bad("a wall-normal grid line is shorter than d + 1 points");
        const int step = s == 0 ? 1 : s == 1 ? -1 : s == 2 ? h.n1 : -h.n1;
        const int cnt = s < 2 ? h.n2 : h.n1;
        for (int t = 0; t < cnt; ++t) {
          const size_t k = s < 2 ? (size_t)t * h.n1 + (s == 0 ? 0 : h.n1 - 1) : (size_t)(s == 2 ? 0 : h.n2 - 1) * h.n1 + t;
          if (h.blank[k]) continue;
          WallPt wp;
          std::memset(&wp, 0, sizeof(wp));
          wp.idx = (int)(h.off + (long long)k);
          wp.step = step;
          wp.nw = prm->d - 1;
          for (int j = 0; j < wp.nw; ++j) wp.w[j] = aw[j];
          walls.push_back(wp);
        }
      }
    }
  }

  // ---- per-point flags and viscosity windows
  std::vector<uint32_t> info((size_t)c->P);
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    std::vector<uint8_t> w1((size_t)h.n1 * h.n2, 7), w2(w1.size(), 7);
    for (const Seg& s : h.seg1) {
      if (!s.periodic && s.n < 7) continue;
      for (int t = 0; t < s.n; ++t) {
        const int i = s.a + t;
        const int start = s.periodic ? i - 3 : std::min(std::max(i - 3, s.a), s.a + s.n - 7);
        w1[(size_t)s.line * h.n1 + i] = (uint8_t)(i - start);
      }
    }
    for (const Seg& s : h.seg2) {
      if (s.n < 7) continue;
      for (int t = 0; t < s.n; ++t) {
        const int j = s.a + t;
        const int start = std::min(std::max(j - 3, s.a), s.a + s.n - 7);
        w2[(size_t)j * h.n1 + s.line] = (uint8_t)(j - start);
      }
    }
    for (size_t k = 0; k < w1.size(); ++k) {
      uint32_t f = ((uint32_t)p << PT_PATCH_SHIFT) | ((uint32_t)w1[k] << PT_W1_SHIFT) | ((uint32_t)w2[k] << PT_W2_SHIFT);
      if (h.blank[k]) f |= PT_BLANK;
      if (h.nodiff[k]) f |= PT_NODIFF;
      if (h.gen[k]) f |= PT_GEN;
      info[(size_t)h.off + k] = f;
    }
  }

  // ---- line jobs
  Builder B{c};
  std::vector<Job> jc1, jc2, jg1, jg2, jf1, jf2;
  std::vector<uint8_t> cov2((size_t)c->P, 0), fcov1((size_t)c->P, 0), fcov2((size_t)c->P, 0);
  std::vector<GFix> gfix;
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    const bool aff = h.d.kind == FC_PATCH_AFFINE;
    const double sx = aff ? (h.n1 - 1) / (h.d.geom[1] - h.d.geom[0]) : 1.0 / h.h1;
    const double sy = aff ? (h.n2 - 1) / (h.d.geom[3] - h.d.geom[2]) : 1.0 / h.h2;
    for (const Seg& s : h.seg1) {
      if (!s.periodic && s.n < 2 * prm->d) continue;
      Job J{};
      J.base = h.off + (long long)s.line * h.n1 + s.a;
      J.stride = 1;
      J.n = s.n;
      J.patch = p;
      J.scale = sx;
      if (s.periodic) {
        J.C = 0;
        J.fcm = -1;
        J.plan = B.plan(s.n);
      } else {
        J.C = B.choose_C(s.n);
        if (J.C < c->Cmin || J.C > c->Cmax) return bad("continuation length outside the FC tables");
        J.fcm = B.fcm(J.C);
        J.plan = B.plan(s.n + J.C);
      }
      J.gbase = aff ? -1 : h.gbase + (long long)s.line * h.n1 + s.a;
      (aff ? jc1 : jg1).push_back(J);
      jf1.push_back(J);
      for (int t = 0; t < s.n; ++t) fcov1[(size_t)J.base + t] = 1;
    }
    for (const Seg& s : h.seg2) {
      if (s.n < 2 * prm->d) continue;
      Job J{};
      J.base = h.off + (long long)s.a * h.n1 + s.line;
      J.stride = h.n1;
      J.n = s.n;
      J.patch = p;
      J.scale = sy;
      J.C = B.choose_C(s.n);
      if (J.C < c->Cmin || J.C > c->Cmax) return bad("continuation length outside the FC tables");
      J.fcm = B.fcm(J.C);
      J.plan = B.plan(s.n + J.C);
      J.gbase = aff ? -1 : h.gbase + (long long)s.a * h.n1 + s.line;
      (aff ? jc2 : jg2).push_back(J);
      jf2.push_back(J);
      for (int t = 0; t < s.n; ++t) {
        cov2[(size_t)J.base + (size_t)t * h.n1] = 1;
        fcov2[(size_t)J.base + (size_t)t * h.n1] = 1;
      }
    }
    if (!aff) {
      // curvilinear patches: pass C (q1 lines) finishes a point; points that only one
      // direction's passes reach are completed by the GFix kernels
      const long long N = (long long)h.n1 * h.n2;
      std::vector<uint8_t> l1((size_t)N, 0), l2((size_t)N, 0);
      for (const Seg& s : h.seg1)
        if (s.periodic || s.n >= 2 * prm->d)
          for (int t = 0; t < s.n; ++t) l1[(size_t)s.line * h.n1 + s.a + t] = 1;
      for (const Seg& s : h.seg2)
        if (s.n >= 2 * prm->d)
          for (int t = 0; t < s.n; ++t) l2[(size_t)(s.a + t) * h.n1 + s.line] = 1;
      for (long long k = 0; k < N; ++k) {
        cov2[(size_t)(h.off + k)] = l1[k];
        if (l1[k] != l2[k]) gfix.push_back(GFix{(int)(h.off + k), (int)(h.gbase + k), l2[k] ? 1 : 2, 0});
      }
    }
  }
  // GRID patches given without metrics: FC derivatives of x and y along the full grid
  // lines (the same continuation rule as the data lines), assembled after the upload
  std::vector<Job> mj1, mj2;
  std::vector<GFix> mpts;
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    if (h.d.kind != FC_PATCH_GRID || h.d.metrics) continue;
    for (int j = 0; j < h.n2; ++j) {
      Job J{};
      J.base = h.off + (long long)j * h.n1;
      J.stride = 1;
      J.n = h.n1;
      J.patch = p;
      J.scale = 1.0 / h.h1;
      J.gbase = -1;
      if (h.periodic1) {
        J.C = 0;
        J.fcm = -1;
        J.plan = B.plan(h.n1);
      } else {
        J.C = B.choose_C(h.n1);
        if (J.C < c->Cmin || J.C > c->Cmax) return bad("continuation length outside the FC tables");
        J.fcm = B.fcm(J.C);
        J.plan = B.plan(h.n1 + J.C);
      }
      mj1.push_back(J);
    }
    for (int i = 0; i < h.n1; ++i) {
      Job J{};
      J.base = h.off + i;
      J.stride = h.n1;
      J.n = h.n2;
      J.patch = p;
      J.scale = 1.0 / h.h2;
      J.gbase = -1;
      J.C = B.choose_C(h.n2);
      if (J.C < c->Cmin || J.C > c->Cmax) return bad("continuation length outside the FC tables");
      J.fcm = B.fcm(J.C);
      J.plan = B.plan(h.n2 + J.C);
      mj2.push_back(J);
    }
    for (long long k = 0; k < (long long)h.n1 * h.n2; ++k)
      mpts.push_back(GFix{(int)(h.off + k), (int)(h.gbase + k), 0, 0});
  }
  std::vector<int> fix, fc1, fc2, fyfix;
  {
    std::vector<uint8_t> cov1c((size_t)c->P, 0);
    for (const Job& J : jc1)
      for (int t = 0; t < J.n; ++t) cov1c[(size_t)(J.base + (long long)t * J.stride)] = 1;
    for (const Job& J : jc2)
      for (int t = 0; t < J.n; ++t) {
        const long long k = J.base + (long long)t * J.stride;
        if (!cov1c[(size_t)k]) fyfix.push_back((int)k);
      }
  }
  for (long long k = 0; k < c->P; ++k) {
    if (!cov2[k]) fix.push_back((int)k);
    if (!(info[k] & PT_BLANK)) {
      if (!fcov1[k]) fc1.push_back((int)k);
      if (!fcov2[k]) fc2.push_back((int)k);
    }
  }

  // ---- viscosity windows, cross-patch nearest points (eqs. W, multipatch_W, zeta)
  std::vector<double> wtab(2 * prm->win_r - 1);
  for (int a = -(prm->win_r - 1); a <= prm->win_r - 1; ++a) {
    const long double t = std::fabs((long double)a);
    const long double cc = cosl(3.14159265358979323846264338327950288L * t / (2.0L * prm->win_r));
    wtab[a + prm->win_r - 1] = (double)(cc * cc);
  }
  std::vector<int> cdst, cptr{0}, csrc;
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    std::vector<int> near;
    for (int q = 0; q < npatch; ++q) {
      const HPatch& g = c->hp[q];
      if (q != p && !(h.bx1 < g.bx0 || g.bx1 < h.bx0 || h.by1 < g.by0 || g.by1 < h.by0)) near.push_back(q);
    }
    if (near.empty()) continue;
    for (size_t k = 0; k < h.x.size(); ++k) {
      if (h.blank[k]) continue;
      const double x = h.x[k], y = h.y[k];
      bool any = false;
      for (int q : near) {
        const HPatch& g = c->hp[q];
        if (x < g.bx0 - 1e-12 || x > g.bx1 + 1e-12 || y < g.by0 - 1e-12 || y > g.by1 + 1e-12) continue;
        double s1, s2;
        frac_index(g, x, y, s1, s2);
        if (!contains(g, s1, s2)) continue;
        int z1, z2;
        nearest(g, s1, s2, z1, z2);
        csrc.push_back((int)(g.off + (long long)z2 * g.n1 + z1));
        any = true;
      }
      if (any) {
        cdst.push_back((int)(h.off + (long long)k));
        cptr.push_back((int)csrc.size());
      }
    }
  }

  // ---- curvilinear metrics J = dq/dx (Sec. 3.3), layout [4][Pg]: J1x, J1y, J2x, J2y
  std::vector<double> Jm((size_t)4 * std::max<long long>(c->Pg, 1), 0.0);
  for (const HPatch& h : c->hp) {
    if (h.d.kind == FC_PATCH_GRID) {
      const long long N = (long long)h.n1 * h.n2;
      for (int m = 0; m < 4; ++m)
        for (long long k = 0; k < N; ++k) Jm[(size_t)(h.gbase + k) + (size_t)m * c->Pg] = h.jm[(size_t)m * N + k];
      continue;
    }
    if (h.d.kind != FC_PATCH_OGRID) continue;
    const double r0 = h.d.geom[2], r1 = h.d.geom[3];
    for (long long k = 0; k < (long long)h.n1 * h.n2; ++k) {
      const double dx = h.x[k] - h.d.geom[0], dy = h.y[k] - h.d.geom[1];
      const double r = std::hypot(dx, dy);
      const double cs = dx / r, sn = dy / r;
      const size_t g = (size_t)(h.gbase + k);
      Jm[g] = -sn / (2.0 * PI * r);
      Jm[g + c->Pg] = cs / (2.0 * PI * r);
      Jm[g + 2 * c->Pg] = cs / (r1 - r0);
      Jm[g + 3 * c->Pg] = sn / (r1 - r0);
    }
  }

  // ---- exchange transpose: for every donor point, the receivers it feeds and the weights
  std::vector<int> dptr{0}, dsrc, drecv;
  std::vector<double> dw;
  {
    std::vector<std::pair<int, std::pair<int, double>>> ent;
    ent.reserve(recv.size() * 9);
    for (const Recv& r : recv)
      for (int m2 = 0; m2 < 3; ++m2)
        for (int m1 = 0; m1 < 3; ++m1) ent.push_back({r.src[3 * m2 + m1], {r.dst, r.w1[m1] * r.w2[m2]}});
    std::stable_sort(ent.begin(), ent.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (size_t k = 0; k < ent.size(); ++k) {
      if (k == 0 || ent[k].first != ent[k - 1].first) {
        if (k) dptr.push_back((int)drecv.size());
        dsrc.push_back(ent[k].first);
      }
      drecv.push_back(ent[k].second.first);
      dw.push_back(ent[k].second.second);
    }
    if (!ent.empty()) dptr.push_back((int)drecv.size());
  }
  // ---- wall ring of the first curvilinear patch with a wall at q2 = 0 (drag functional)
  std::vector<int> wall;
  std::vector<double> wallw, wallc;
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    if (h.d.kind != FC_PATCH_OGRID || (h.d.side[2] != FC_SIDE_SLIPWALL && h.d.side[2] != FC_SIDE_ADIABATIC)) continue;
    c->wall_patch = p;
    for (int i = 0; i < h.n1; ++i) {
      const double dx = h.x[i] - h.d.geom[0], dy = h.y[i] - h.d.geom[1];
      wall.push_back((int)(h.off + i));
      wallc.push_back(dx / std::hypot(dx, dy));
      wallw.push_back(h.d.geom[2] * 2.0 * PI / h.n1);
    }
    break;
  }

  // ---- upload
  bool ok = true;
  make_queue(c, c->q_cart1, jc1, B.plans, npatch, ok);
  make_queue(c, c->q_cart2, jc2, B.plans, npatch, ok);
  make_queue(c, c->q_gen1, jg1, B.plans, npatch, ok);
  make_queue(c, c->q_gen2, jg2, B.plans, npatch, ok);
  make_queue(c, c->q_filt1, jf1, B.plans, npatch, ok);
  make_queue(c, c->q_filt2, jf2, B.plans, npatch, ok);
  std::vector<PatchDev> pdev(npatch);
  bool any_pform = false;
  for (int p = 0; p < npatch; ++p) {
    const HPatch& h = c->hp[p];
    bool wall = false;
    for (int sd = 0; sd < 4; ++sd) wall = wall || h.d.side[sd] == FC_SIDE_ADIABATIC;
    const int pform = prm->wall_form == 1 && wall ? 1 : 0;
    if (pform && h.d.kind == FC_PATCH_AFFINE)
      return bad("the product-rule wall form needs adiabatic walls on OGRID or GRID patches");
    any_pform = any_pform || pform;
    pdev[p] = PatchDev{h.off, h.gbase, h.n1, h.n2, h.d.kind, h.periodic1 ? 1 : 0, h.hhat, h.htil, pform, 0};
  }
  const std::vector<double> Rv(prm->R, prm->R + 4);
  for (const Plan& pl : B.plans)
    for (int st = 0; st < pl.nst; ++st)
      if (pl.rad[st] > MAX_GENERIC_RADIX) return bad("a continued line length has a prime factor above 128");
  std::vector<Recv> rinterp;
  std::vector<PtCopy> rcopy;
  split_exchange(recv, rinterp, rcopy);
  ok = ok && c->upload(&c->d_plans, B.plans) && c->upload(&c->d_tw, B.tw) && c->upload(&c->d_rp, B.rp) &&
       c->upload(&c->d_ip, B.ip) &&
       c->upload(&c->d_info, info) && c->upload(&c->d_patches, pdev) && c->upload(&c->d_J, Jm) &&
       c->upload(&c->d_sdnn, c->sdnn) && c->upload(&c->d_R, Rv) && c->upload(&c->d_wtab, wtab) &&
       c->upload(&c->d_fix, fix) && c->upload(&c->d_fyfix, fyfix) && c->upload(&c->d_gfix, gfix) &&
       c->upload(&c->d_fcopy1, fc1) && c->upload(&c->d_fcopy2, fc2) &&
       c->upload(&c->d_bc, bcs) && c->upload(&c->d_walls, walls) && c->upload(&c->d_recv, rinterp) &&
       c->upload(&c->d_rcopy, rcopy) && c->upload(&c->d_recv_all, recv) && c->upload(&c->d_cross_dst, cdst) &&
       c->upload(&c->d_cross_ptr, cptr) && c->upload(&c->d_cross_src, csrc) && c->upload(&c->d_dptr, dptr) &&
       c->upload(&c->d_dsrc, dsrc) && c->upload(&c->d_drecv, drecv) && c->upload(&c->d_dw, dw) &&
       c->upload(&c->d_wall, wall) && c->upload(&c->d_wallw, wallw) && c->upload(&c->d_wallc, wallc);
  c->plans_h = B.plans;
  c->plan_cands = B.cands;
  c->h_recv = recv;
  c->h_bc = bcs;
  c->h_walls = walls;
  c->h_fix = fix;
  c->h_fyfix = fyfix;
  c->h_gfix = gfix;
  c->h_fcopy1 = fc1;
  c->h_fcopy2 = fc2;
  c->h_cdst = cdst;
  c->h_cptr = cptr;
  c->h_csrc = csrc;
  c->ndon = (int)dsrc.size();
  c->nwall = (int)wall.size();
  c->nfix = (int)fix.size();
  c->nfyfix = (int)fyfix.size();
  c->ngfix = (int)gfix.size();
  c->nfcopy1 = (int)fc1.size();
  c->nfcopy2 = (int)fc2.size();
  c->nbc = (int)bcs.size();
  c->nwalls = (int)walls.size();
  c->any_walls = !walls.empty();
  c->nrecv = (int)rinterp.size();
  c->nrcopy = (int)rcopy.size();
  c->nrecv_all = (int)recv.size();
  c->ncross = (int)cdst.size();
  const size_t P = (size_t)c->P, Pg = (size_t)std::max<long long>(c->Pg, 1);
  ok = ok && c->alloc(&c->d_B1, 4 * P) && c->alloc(&c->d_B2, 4 * P) && c->alloc(&c->d_B3, 4 * P) &&
       c->alloc(&c->d_R1, 4 * P) && c->alloc(&c->d_G, 16 * Pg) && c->alloc(&c->d_phi, P) && c->alloc(&c->d_S, P) &&
       c->alloc(&c->d_muhat, P) && c->alloc(&c->d_num, P) && c->alloc(&c->d_tmp, P) && c->alloc(&c->d_mu, P) &&
       c->alloc(&c->d_den, P) && c->alloc(&c->d_dt, 1) && c->alloc(&c->d_pmax, 2 * (size_t)npatch) &&
       c->alloc(&c->d_flag, 1) && c->alloc(&c->d_skip_lines, 2) && c->alloc(&c->d_skip_flops, 2) &&
       (jc2.empty() || c->alloc(&c->d_Fy, 4 * P));
  if (!ok) {
    fprintf(stderr, "fc_init_patches: %s\n", c->err.c_str());
    delete c;
    return FC_ERR_OOM;
  }
  cudaMemset(c->d_flag, 0, sizeof(int));
  cudaMemset(c->d_skip_lines, 0, 2 * sizeof(unsigned long long));
  cudaMemset(c->d_skip_flops, 0, 2 * sizeof(double));
  DevTables& T = c->T;
  T.skip_lines = c->d_skip_lines;
  T.skip_flops = c->d_skip_flops;
  T.tw = c->d_tw;
  T.rp = c->d_rp;
  T.ip = c->d_ip;
  T.plans = c->d_plans;
  T.info = c->d_info;
  T.patches = c->d_patches;
  T.npatch = npatch;
  T.P = c->P;
  T.Pg = std::max<long long>(c->Pg, 1);
  T.gamma = prm->gamma;
  T.d = prm->d;
  T.any_pform = any_pform ? 1 : 0;
  set_kernel_attributes();
  if (!mpts.empty()) {  // metrics of GRID patches given by their points only
    std::vector<double> xy(2 * (size_t)c->P, 0.0);
    for (const HPatch& h : c->hp)
      if (h.d.kind == FC_PATCH_GRID && !h.d.metrics)
        for (size_t k = 0; k < h.x.size(); ++k) {
          xy[(size_t)h.off + k] = h.x[k];
          xy[(size_t)c->P + (size_t)h.off + k] = h.y[k];
        }
    Job *d_mj1 = nullptr, *d_mj2 = nullptr;
    GFix* d_mp = nullptr;
    int* d_bad = nullptr;
    int Lm1 = 1, Lm2 = 1;
    for (const Job& J : mj1) Lm1 = std::max(Lm1, B.plans[J.plan].L);
    for (const Job& J : mj2) Lm2 = std::max(Lm2, B.plans[J.plan].L);
    if (!(c->upload(&d_mj1, mj1) && c->upload(&d_mj2, mj2) && c->upload(&d_mp, mpts) && c->alloc(&d_bad, 1)))
      return bad("device allocation failed (GRID metrics)");
    cudaMemset(c->d_B1, 0, sizeof(double) * 4 * (size_t)c->P);
    cudaMemcpy(c->d_B1, xy.data(), xy.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemset(d_bad, 0, sizeof(int));
    launch_deriv_lines(c->T, d_mj1, (int)mj1.size(), Lm1, c->d_B1, c->d_B2, nullptr);
    launch_deriv_lines(c->T, d_mj2, (int)mj2.size(), Lm2, c->d_B1, c->d_B3, nullptr);
    launch_grid_metrics(d_mp, (int)mpts.size(), c->d_B2, c->d_B3, c->P, c->d_J, c->T.Pg, d_bad, nullptr);
    int nbad = 0;
    if (cudaMemcpy(&nbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bad(std::string("GRID metrics: ") + cudaGetErrorString(cudaGetLastError()));
    if (nbad) return bad("a GRID patch has a singular or non-finite Jacobian (metrics from its points)");
  }
  {  // FCSDNN_CONCURRENT=0 runs every batched pass on the caller's stream alone (A/B timing)
    const char* v = getenv("FCSDNN_CONCURRENT");
    c->concurrent = !(v && v[0] == '0');
    // side streams and events now, not during a later graph capture
    if (c->concurrent && !c->ensure_side()) return bad("could not create the side streams");
  }

  // normaliser of eq. (multipatch_W_norm): window sums of the generation indicator, own + other patches
  {
    std::vector<double> ind((size_t)c->P), ones((size_t)c->P, 1.0);
    for (size_t k = 0; k < info.size(); ++k) ind[k] = (info[k] & PT_GEN) ? 1.0 : 0.0;
    // the generation indicator goes through mu^'s buffer, the unit divisor through phi's
    cudaMemcpy(c->d_muhat, ind.data(), ind.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_phi, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice);
    launch_window_rows(T, c->d_muhat, c->d_tmp, c->d_wtab, prm->win_r, 0);
    launch_window_cols(T, c->d_tmp, c->d_num, c->d_wtab, prm->win_r, 0);
    launch_mu_final(T, c->d_num, c->d_phi, c->d_cross_dst, c->d_cross_ptr, c->d_cross_src, c->ncross, c->d_den, 0);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      fprintf(stderr, "fc_init_patches: %s\n", cudaGetErrorString(e));
      delete c;
      return FC_ERR_CUDA;
    }
  }
  *out = c;
  return FC_OK;
}

size_t fc_state_size(const fc_ctx* c) { return c ? (size_t)c->P : 0; }
size_t fc_active_points(const fc_ctx* c) { return c ? (size_t)c->active : 0; }
fc_status fc_patch_offset(const fc_ctx* c, int patch, size_t* off) {
  if (!c || !off || patch < 0 || patch >= (int)c->hp.size()) return FC_ERR_INVALID;
  *off = (size_t)c->hp[patch].off;
  return FC_OK;
}
uint64_t fc_launch_count(const fc_ctx* c) { return c ? c->launches : 0; }
const char* fc_last_error(const fc_ctx* c) { return c ? c->err.c_str() : "null context"; }
void fc_destroy(fc_ctx* c) { delete c; }

}  // extern "C"

// ---------------------------------------------------------------- orchestration
namespace {

// brackets a launch group with events when instrumentation is on
struct Prof {
  fc_ctx* c;
  cudaStream_t st;
  const char* name;
  cudaEvent_t a = nullptr;
  uint64_t l0;
  Prof(fc_ctx* c_, cudaStream_t s, const char* n) : c(c_), st(s), name(n), l0(c_->launches) {
    if (c->prof) {
      a = c->ev();
      cudaEventRecord(a, st);
    }
  }
  ~Prof() {
    if (a) {
      cudaEvent_t b = c->ev();
      cudaEventRecord(b, st);
      c->prec.push_back({name, a, b, (int)(c->launches - l0)});
    }
  }
};

// run one pass over a queue, batched (one launch per length class) or one launch per patch.
// Batched: the length classes of a pass touch disjoint lines, so classes after the first
// run on side streams forked from st and joined back into it (their tails overlap;
// inside a CUDA graph they become parallel branches). first_side: the first side
// stream this pass may use (a chain already running on a side stream keeps it). While
// the per-pass profile is on, passes run one after another so that each pass's time is
// its own.
template <class F>
void run_queue(fc_ctx* c, const fc_ctx::Queue& q, bool per_patch, cudaStream_t st, const char* name, F&& launch,
               int first_side = 1) {
  if (q.n == 0) return;
  Prof pr(c, st, name);
  if (!per_patch) {
    const int ncls = (int)q.classes.size();
    const int nside = fc_ctx::NSIDE - first_side;
    const bool fork = c->concurrent && !c->prof && ncls > 1 && nside > 0 && c->ensure_side();
    if (fork) cudaEventRecord(c->fork_ev[0], st);
    for (int k = 0; k < ncls; ++k) {
      const int b = q.classes[k].first, e = q.class_end[k];
      cudaStream_t s = st;
      if (fork && k > 0) {
        s = c->side[first_side + (k - 1) % nside];
        if (k - 1 < nside) cudaStreamWaitEvent(s, c->fork_ev[0], 0);
      }
      launch(q.d + b, e - b, q.classes[k].second, s);
      c->launches++;
    }
    if (fork)
      for (int k = 0; k < std::min(ncls - 1, nside); ++k) {
        cudaEventRecord(c->join_ev[first_side + k], c->side[first_side + k]);
        cudaStreamWaitEvent(st, c->join_ev[first_side + k], 0);
      }
  } else {
    for (size_t p = 0; p < q.pbeg.size(); ++p) {
      const int n = q.pend[p] - q.pbeg[p];
      if (n <= 0) continue;
      launch(q.dpp + q.pbeg[p], n, q.plmax[p], st);
      c->launches++;
    }
  }
}

void stage(fc_ctx* c, const StageCoef& sc, const double* mu, bool per_patch, cudaStream_t st) {
  const DevTables& T = c->T;
  const double* e = sc.Ucur;
  // the curvilinear chain (passes A, B, C) and the affine chain (q1, q2) touch different
  // patches: batched, the curvilinear chain runs on its own side stream
  const bool overlap =
      !per_patch && c->concurrent && !c->prof && c->q_gen1.n > 0 && c->q_cart1.n > 0 && c->ensure_side();
  cudaStream_t sg = st;
  int gside = 1;
  if (overlap) {
    cudaEventRecord(c->fork_ev[1], st);
    cudaStreamWaitEvent(c->side[0], c->fork_ev[1], 0);
    sg = c->side[0];
    gside = fc_ctx::NSIDE;  // no class forks inside the curvilinear chain
  }
  run_queue(c, c->q_gen1, per_patch, sg, "gen_A",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_gen_A(T, j, n, L, e, c->d_G, s); }, gside);
  if (c->ngfix) {
    launch_gen_fix(T, c->d_gfix, c->ngfix, e, mu, c->d_J, c->d_G, sg);
    c->launches++;
  }
  if (c->nfyfix) {
    launch_flux_y_points(T, c->d_fyfix, c->nfyfix, e, c->d_Fy, st);
    c->launches++;
  }
  run_queue(c, c->q_cart1, per_patch, st, "cart_q1", [&](const Job* j, int n, int L, cudaStream_t s) {
    launch_cart_q1(T, j, n, L, e, mu, c->d_R1, c->d_Fy, s);
  });
  run_queue(c, c->q_gen2, per_patch, sg, "gen_B",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_gen_B(T, j, n, L, e, mu, c->d_J, c->d_G, s); },
            gside);
  run_queue(c, c->q_cart2, per_patch, st, "cart_q2",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_cart_q2(T, j, n, L, mu, c->d_R1, c->d_Fy, sc, s); });
  run_queue(c, c->q_gen1, per_patch, sg, "gen_C",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_gen_C(T, j, n, L, c->d_J, c->d_G, sc, s); },
            gside);
  if (overlap) {
    cudaEventRecord(c->join_ev[0], c->side[0]);
    cudaStreamWaitEvent(st, c->join_ev[0], 0);
  }
  if (c->nfix) {
    Prof pr(c, st, "rk_fixup");
    launch_rk_fixup(T, c->d_fix, c->nfix, sc, st);
    c->launches++;
  }
}

void project(fc_ctx* c, double* e, cudaStream_t st) {
  Prof pr(c, st, "bc_exchange");
  if (c->nbc) {
    launch_bc(c->d_bc, c->nbc, e, c->P, st);
    c->launches++;
  }
  if (c->nwalls) {
    launch_bc_wall(c->d_walls, c->nwalls, e, c->P, c->prm.gamma, st);
    c->launches++;
  }
  if (c->nrecv) {
    launch_exchange(c->d_recv, c->nrecv, e, c->P, st);
    c->launches++;
  }
  if (c->nrcopy) {
    launch_copy_points(c->d_rcopy, c->nrcopy, e, c->P, st);
    c->launches++;
  }
  if (c->sharded()) {  // fringe values interpolated on the donors' ranks
    fc_ctx::XPlan& x = c->xp_fringe;
    launch_xpack(c->d_xsend, x.nsend, e, c->P, x.d_sbuf, st);
    if (c->comm(c->comm_user, FC_COMM_EXCHANGE, x.d_sbuf, x.scount.data(), x.d_rbuf, x.rcount.data(), st) != 0)
      c->comm_failed = true;
    launch_xunpack(c->d_xrecv, x.nrecv, x.d_rbuf, e, c->P, st);
    c->launches += (x.nsend > 0) + (x.nrecv > 0);
  }
}

void viscosity(fc_ctx* c, const double* e, double* mu, int32_t* tau, cudaStream_t st) {
  Prof pr(c, st, "viscosity");
  const DevTables& T = c->T;
  launch_visc_point(T, e, c->d_phi, c->d_S, st);
  launch_visc_muhat(T, c->d_phi, c->d_S, c->d_sdnn, c->d_R, c->d_muhat, tau, st);
  launch_window_rows(T, c->d_muhat, c->d_tmp, c->d_wtab, c->prm.win_r, st);
  launch_window_cols(T, c->d_tmp, c->d_num, c->d_wtab, c->prm.win_r, st);
  if (c->sharded()) {  // window sums of other ranks' patches that the cross-patch sums read
    fc_ctx::XPlan& x = c->xp_visc;
    launch_gather(c->d_vsend, x.nsend, c->d_num, x.d_sbuf, st);
    if (c->comm(c->comm_user, FC_COMM_EXCHANGE, x.d_sbuf, x.scount.data(), x.d_rbuf, x.rcount.data(), st) != 0)
      c->comm_failed = true;
    launch_scatter(c->d_vrecv, x.nrecv, x.d_rbuf, c->d_num, st);
    c->launches += (x.nsend > 0) + (x.nrecv > 0);
  }
  launch_mu_final(T, c->d_num, c->d_den, c->d_cross_dst, c->d_cross_ptr, c->d_cross_src, c->ncross, mu, st);
  c->launches += 5 + (c->ncross > 0);
}

void filter(fc_ctx* c, double* e, bool per_patch, cudaStream_t st) {
  const DevTables& T = c->T;
  double* F = c->d_B3;
  run_queue(c, c->q_filt1, per_patch, st, "filter_q1",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_filter_q1(T, j, n, L, e, F, s); });
  if (c->nfcopy1) {
    launch_filter_copy_q1(T, c->d_fcopy1, c->nfcopy1, e, F, st);
    c->launches++;
  }
  run_queue(c, c->q_filt2, per_patch, st, "filter_q2",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_filter_q2(T, j, n, L, F, e, s); });
  if (c->nfcopy2) {
    launch_filter_copy_q2(T, c->d_fcopy2, c->nfcopy2, F, e, st);
    c->launches++;
  }
}

// transpose of filter() linearised at its input state pre (filt: its output): lam -> out;
// MF is scratch; blanked points pass lam through
void filterT(fc_ctx* c, const double* lam, const double* pre, const double* filt, double* MF, double* out,
             cudaStream_t st) {
  const DevTables& T = c->T;
  cudaMemcpyAsync(out, lam, sizeof(double) * 4 * (size_t)c->P, cudaMemcpyDeviceToDevice, st);
  run_queue(c, c->q_filt2, false, st, "filterT_q2",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_filterT_q2(T, j, n, L, lam, filt, MF, s); });
  if (c->nfcopy2) {
    launch_filterT_copy2(T, c->d_fcopy2, c->nfcopy2, lam, filt, MF, st);
    c->launches++;
  }
  run_queue(c, c->q_filt1, false, st, "filterT_q1",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_filterT_q1(T, j, n, L, MF, pre, out, s); });
  if (c->nfcopy1) {
    launch_filterT_copy1(T, c->d_fcopy1, c->nfcopy1, MF, pre, out, st);
    c->launches++;
  }
}

void timestep(fc_ctx* c, const double* e, const double* mu, double* dt, cudaStream_t st) {
  Prof pr(c, st, "timestep");
  launch_dt(c->T, e, mu, c->d_pmax, c->prm.cfl, dt, st);
  c->launches += 2;
  if (c->sharded()) {
    const long long one[1] = {1};
    if (c->comm(c->comm_user, FC_COMM_MIN, dt, one, c->d_dtmin, one, st) != 0) c->comm_failed = true;
    cudaMemcpyAsync(dt, c->d_dtmin, sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
}

void rk_body(fc_ctx* c, double* e, double* dt, double* mu, int flags, cudaStream_t st) {
  const bool pp = (flags & FC_STEP_PER_PATCH) != 0;
  project(c, e, st);
  if (!(flags & FC_STEP_FROZEN_MU)) viscosity(c, e, mu, nullptr, st);
  if (flags & FC_STEP_FILTER) {
    filter(c, e, pp, st);
    project(c, e, st);
  }
  if (!(flags & FC_STEP_FIXED_DT)) timestep(c, e, mu, dt, st);
  StageCoef s{};
  s.dt = dt;
  // stage 1: u1 = u0 + b1 dt L(u0)
  s.U0 = e; s.Ucur = e; s.Uaux = nullptr; s.out = c->d_B1; s.out2 = nullptr;
  s.c0 = 0.0; s.c1 = 1.0; s.c2 = 0.0; s.cb = B1;
  stage(c, s, mu, pp, st);
  project(c, c->d_B1, st);
  // stage 2
  s.Ucur = c->d_B1; s.out = c->d_B2; s.c0 = A20; s.c1 = A21; s.cb = B2;
  stage(c, s, mu, pp, st);
  project(c, c->d_B2, st);
  // stage 3
  s.Ucur = c->d_B2; s.out = c->d_B3; s.c0 = A30; s.c1 = A32; s.cb = B3;
  stage(c, s, mu, pp, st);
  project(c, c->d_B3, st);
  // stage 4: u4 = a40 u0 + a43 u3 + b4 dt L(u3); acc = a52 u2 + a53 u3 + b53 dt L(u3) (in place over u2)
  s.Ucur = c->d_B3; s.Uaux = c->d_B2; s.out = c->d_B1; s.out2 = c->d_B2;
  s.c0 = A40; s.c1 = A43; s.c2 = 0.0; s.cb = B4; s.d1 = A53; s.d2 = A52; s.db = B53;
  stage(c, s, mu, pp, st);
  project(c, c->d_B1, st);
  // stage 5: u5 = acc + a54 u4 + b54 dt L(u4)
  s.U0 = nullptr; s.Ucur = c->d_B1; s.Uaux = c->d_B2; s.out = e; s.out2 = nullptr;
  s.c0 = 0.0; s.c1 = A54; s.c2 = 1.0; s.cb = B54;
  stage(c, s, mu, pp, st);
  project(c, e, st);
}

// transpose of project(); u: the state project() was applied to (used by the adiabatic walls)
void projectT(fc_ctx* c, double* lam, double* gbc, const double* u, cudaStream_t st) {
  Prof pr(c, st, "bc_exchange_T");
  if (c->sharded()) {  // the exchange reversed: receivers' adjoint back to the donors' ranks
    fc_ctx::XPlan& x = c->xp_fringe;
    launch_xgather(c->d_xrecv, x.nrecv, lam, c->P, x.d_rbuf, st);
    if (c->comm(c->comm_user, FC_COMM_EXCHANGE, x.d_rbuf, x.rcount.data(), x.d_sbuf, x.scount.data(), st) != 0)
      c->comm_failed = true;
    launch_xunpack(c->d_xsend_dst, x.nsend, x.d_sbuf, lam, c->P, st);
    c->launches += (x.nsend > 0) + (x.nrecv > 0);
  }
  launch_exchange_T(c->d_dptr, c->d_dsrc, c->d_drecv, c->d_dw, c->ndon, c->d_recv_all, c->nrecv_all, lam, c->P, st);
  launch_bc_wall_T(c->d_walls, c->nwalls, u, lam, c->P, c->prm.gamma, st);
  launch_bc_T(c->d_bc, c->nbc, lam, gbc, c->cur_acc, c->fsj, c->P, st);
  c->launches += (c->ndon > 0) + (c->nrecv_all > 0) + (c->nwalls > 0) + (c->nbc > 0);
}

// acc += dt L'(u)^T psi
void adj_stage(fc_ctx* c, const double* u, const double* mu, const double* psi, double* acc, const double* dt,
               cudaStream_t st) {
  const DevTables& T = c->T;
  cudaMemsetAsync(c->d_R1, 0, sizeof(double) * 4 * (size_t)c->P, st);
  run_queue(c, c->q_gen1, false, st, "adj_gen_A",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_adj_gen_A(T, j, n, L, c->d_J, u, psi, c->d_G, s); });
  if (c->ngfix) {
    launch_adj_gen_fixA(T, c->d_gfix, c->ngfix, c->d_J, u, mu, psi, c->d_G, st);
    c->launches++;
  }
  run_queue(c, c->q_cart1, false, st, "adj_cart_q1",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_adj_cart(T, j, n, L, 0, u, mu, psi, c->d_R1, acc, dt, s); });
  run_queue(c, c->q_gen2, false, st, "adj_gen_B",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_adj_gen_B(T, j, n, L, c->d_J, u, mu, psi, c->d_G, s); });
  if (c->ngfix) {
    launch_adj_gen_fixB(T, c->d_gfix, c->ngfix, c->d_G, c->d_R1, st);
    c->launches++;
  }
  run_queue(c, c->q_cart2, false, st, "adj_cart_q2",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_adj_cart(T, j, n, L, 1, u, mu, psi, c->d_R1, acc, dt, s); });
  run_queue(c, c->q_gen1, false, st, "adj_gen_C",
            [&](const Job* j, int n, int L, cudaStream_t s) { launch_adj_gen_C(T, j, n, L, u, c->d_G, acc, dt, s); });
  if (c->nfix) {
    launch_adj_fixup(c->d_fix, c->nfix, c->d_R1, acc, c->P, dt, st);
    c->launches++;
  }
}

void axpby(fc_ctx* c, double a, const double* x, double b, double* y, cudaStream_t st) {
  launch_axpby(4 * c->P, a, x, b, y, st);
  c->launches++;
}

}  // namespace

extern "C" {

fc_status fc_rhs(fc_ctx* c, const double* e, double* rhs, const double* mu, void* stream) {
  if (!c || !e || !rhs) return FC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (!mu) {
    viscosity(c, e, c->d_mu, nullptr, st);
    mu = c->d_mu;
  }
  StageCoef s{};
  s.Ucur = e;
  s.out = rhs;
  s.rhs_only = 1;
  s.dt = c->d_dt;
  stage(c, s, mu, false, st);
  return comm_check(c, "fc_rhs");
}

fc_status fc_viscosity(fc_ctx* c, const double* e, double* mu, int32_t* tau, void* stream) {
  if (!c || !e || !mu) return FC_ERR_INVALID;
  viscosity(c, e, mu, tau, (cudaStream_t)stream);
  return comm_check(c, "fc_viscosity");
}

fc_status fc_filter(fc_ctx* c, double* e, void* stream) {
  if (!c || !e) return FC_ERR_INVALID;
  filter(c, e, false, (cudaStream_t)stream);
  return cuda_check(c, "fc_filter");
}

fc_status fc_project(fc_ctx* c, double* e, void* stream) {
  if (!c || !e) return FC_ERR_INVALID;
  project(c, e, (cudaStream_t)stream);
  return comm_check(c, "fc_project");
}

fc_status fc_timestep(fc_ctx* c, const double* e, const double* mu, double* dt, void* stream) {
  if (!c || !e || !mu || !dt) return FC_ERR_INVALID;
  timestep(c, e, mu, dt, (cudaStream_t)stream);
  return comm_check(c, "fc_timestep");
}

fc_status fc_rk_step(fc_ctx* c, double* e, double* dt, double* mu, int flags, void* stream) {
  if (!c || !e) return FC_ERR_INVALID;
  if ((flags & FC_STEP_FROZEN_MU) && !mu) return fail(c, FC_ERR_INVALID, "FROZEN_MU needs mu");
  if ((flags & FC_STEP_FIXED_DT) && !dt) return fail(c, FC_ERR_INVALID, "FIXED_DT needs dt");
  cudaStream_t st = (cudaStream_t)stream;
  if (!mu) mu = c->d_mu;
  if (!dt) dt = c->d_dt;
  if (c->sharded() && (flags & (FC_STEP_GRAPH | FC_STEP_PER_PATCH)))
    return fail(c, FC_ERR_UNIMPLEMENTED, "graph and per-patch steps are not available while sharded");
  if (!(flags & FC_STEP_GRAPH)) {
    rk_body(c, e, dt, mu, flags, st);
    return comm_check(c, "fc_rk_step");
  }
  // graph mode: capture the step once per (buffers, flags, stream) and replay it
  const int gf = flags & ~FC_STEP_GRAPH;
  const bool hit = c->gexec && c->gflags == gf && c->gkey[0] == e && c->gkey[1] == dt && c->gkey[2] == mu &&
                   c->gstream == st;
  if (!hit) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    if (st == nullptr) return fail(c, FC_ERR_INVALID, "graph mode needs a non-default stream");
    cudaGraph_t g;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail(c, FC_ERR_CUDA, "stream capture failed to begin");
    const uint64_t l0 = c->launches;
    const bool prof = c->prof;
    c->prof = false;
    rk_body(c, e, dt, mu, gf, st);
    c->prof = prof;
    if (cudaStreamEndCapture(st, &g) != cudaSuccess) return cuda_check(c, "graph capture");
    cudaError_t er = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (er != cudaSuccess) return fail(c, FC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(er));
    c->gkey[0] = e;
    c->gkey[1] = dt;
    c->gkey[2] = mu;
    c->gflags = gf;
    c->gstream = st;
    c->glaunches = c->launches - l0;  // kernels per replay
    c->launches = l0;
  }
  if (cudaGraphLaunch(c->gexec, st) != cudaSuccess) return cuda_check(c, "graph launch");
  c->launches += c->glaunches;
  return cuda_check(c, "fc_rk_step");
}

fc_status fc_rk_step_host(fc_ctx* c, double* e_host, double* dt, double* mu, int flags, void* stream) {
  if (!c || !e_host) return FC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * 4 * (size_t)c->P;
  if (!c->d_ehost && !c->alloc(&c->d_ehost, 4 * (size_t)c->P)) return fail(c, FC_ERR_OOM, c->err);
  if (cudaMemcpyAsync(c->d_ehost, e_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return cuda_check(c, "fc_rk_step_host (upload)");
  const fc_status s = fc_rk_step(c, c->d_ehost, dt, mu, flags, stream);
  if (s != FC_OK) return s;
  if (cudaMemcpyAsync(e_host, c->d_ehost, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cuda_check(c, "fc_rk_step_host (read-back)");
  return FC_OK;
}

fc_status fc_autotune(fc_ctx* c, int flags, double* report, void* stream) {
  if (!c) return FC_ERR_INVALID;
  if (c->sharded()) return fail(c, FC_ERR_UNIMPLEMENTED, "fc_autotune is not available while sharded");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "fc_autotune");
  double rep[6] = {0, 0, 0, 0, 0, 0};
  // synthetic inputs in the stage scratch: smooth-in-index waves, viscous everywhere (both rounds run)
  double* e = c->d_B1;
  const long long P = c->P;
  for (int k = 0; k < 4; ++k) launch_fill_wave(e + k * P, P, 1.0 + k, 0.25, 0.37 + 0.11 * k, st);
  launch_fill_wave(c->d_mu, P, 1e-3, 0.0, 0.0, st);
  cudaEvent_t ea, eb;
  cudaEventCreate(&ea);
  cudaEventCreate(&eb);
  constexpr int MAXT = 16384, MINT = 2048, REPS = 3;
  if (!c->d_tune_jobs && !c->alloc(&c->d_tune_jobs, MAXT)) return fail(c, FC_ERR_OOM, c->err);
  Job* d_tj = c->d_tune_jobs;
  auto time_q1 = [&](const Job* jobs, int n, int Lmax) {
    launch_cart_q1(c->T, jobs, n, Lmax, e, c->d_mu, c->d_R1, c->d_Fy, st);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < REPS; ++r) {
      cudaEventRecord(ea, st);
      launch_cart_q1(c->T, jobs, n, Lmax, e, c->d_mu, c->d_R1, c->d_Fy, st);
      cudaEventRecord(eb, st);
      cudaEventSynchronize(eb);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ea, eb);
      best = std::min(best, ms);
    }
    return (double)best;
  };
  // R1 of the first timed line, 4 components (strided copy)
  auto sample = [&](const Job& J, std::vector<double>& out) {
    out.assign(4 * (size_t)J.n, 0.0);
    for (int k = 0; k < 4; ++k)
      cudaMemcpy2DAsync(out.data() + (size_t)k * J.n, sizeof(double), c->d_R1 + k * P + J.base,
                        (size_t)J.stride * sizeof(double), sizeof(double), J.n, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
  };
  fc_status status = FC_OK;
  // (1) stage order of each continued length, timed on that length's lines
  if (flags & FC_TUNE_PLANS) {
    const fc_ctx::Queue* qs[6] = {&c->q_cart1, &c->q_cart2, &c->q_gen1, &c->q_gen2, &c->q_filt1, &c->q_filt2};
    for (size_t pi = 0; pi < c->plans_h.size() && status == FC_OK; ++pi) {
      const std::vector<Plan>& cand = c->plan_cands[pi];
      if (cand.size() < 2) continue;
      std::vector<Job> base;
      for (const fc_ctx::Queue* q : qs) {
        for (const Job& J : q->h)
          if (J.plan == (int)pi) base.push_back(J);
        if (!base.empty()) break;  // the first pass with lines of this length
      }
      if (base.empty()) continue;
      std::vector<Job> tj;
      while ((int)tj.size() < MINT)
        for (const Job& J : base) {
          if ((int)tj.size() >= MAXT) break;
          tj.push_back(J);
        }
      // copies on `stream` itself: it may be a non-blocking stream, unordered with the legacy one
      cudaMemcpyAsync(d_tj, tj.data(), tj.size() * sizeof(Job), cudaMemcpyHostToDevice, st);
      const int L = c->plans_h[pi].L;
      std::vector<double> ref, got;
      double t0 = 0, tb = 0;
      int best = 0;
      for (size_t k = 0; k < cand.size(); ++k) {
        cudaMemcpyAsync(c->d_plans + pi, &cand[k], sizeof(Plan), cudaMemcpyHostToDevice, st);
        const double t = time_q1(d_tj, (int)tj.size(), L);
        sample(tj[0], k == 0 ? ref : got);
        if (k == 0) {
          t0 = tb = t;
          continue;
        }
        double dmax = 0, rmax = 0;
        for (size_t q = 0; q < ref.size(); ++q) {
          dmax = std::max(dmax, std::fabs(got[q] - ref[q]));
          rmax = std::max(rmax, std::fabs(ref[q]));
        }
        const bool agrees = std::isfinite(dmax) && dmax <= 1e-10 * std::max(rmax, 1e-300);
        if (agrees && t < 0.99 * tb) {
          tb = t;
          best = (int)k;
        }
      }
      c->plans_h[pi] = cand[best];
      cudaMemcpyAsync(c->d_plans + pi, &cand[best], sizeof(Plan), cudaMemcpyHostToDevice, st);
      rep[0] += 1;
      rep[1] += best != 0;
      rep[4] += t0;
      rep[5] += tb;
      if (cudaGetLastError() != cudaSuccess) status = cuda_check(c, "fc_autotune (plans)");
    }
  }
  // (2) warps per CTA of each length class, timed on the class's q1 and q2 lines
  if ((flags & FC_TUNE_WARPS) && status == FC_OK) {
    std::map<int, std::vector<std::pair<const fc_ctx::Queue*, int>>> byclass;  // class -> (queue, class slot)
    for (const fc_ctx::Queue* q : {&c->q_cart1, &c->q_cart2})
      for (size_t k = 0; k < q->classes.size(); ++k) byclass[length_class(q->classes[k].second)].push_back({q, (int)k});
    for (auto& kv : byclass) {
      const int cls = kv.first;
      int Lcap = 1;
      for (auto& qk : kv.second) Lcap = std::max(Lcap, qk.first->classes[qk.second].second);
      auto total = [&]() {
        double t = 0;
        for (auto& qk : kv.second) {
          const fc_ctx::Queue* q = qk.first;
          const int b = q->classes[qk.second].first, en = q->class_end[qk.second];
          t += time_q1(q->d + b, en - b, q->classes[qk.second].second);
        }
        return t;
      };
      c->T.lw[cls] = 0;
      const int wdef = line_warps(c->T, Lcap);
      const double t0 = total();
      double tb = t0;
      int best = 0;
      for (int w : {1, 2, 4, 8}) {
        if (w > line_warps_max(Lcap)) break;
        c->T.lw[cls] = w;
        const double t = total();
        if (t < 0.99 * tb) {
          tb = t;
          best = w;
        }
      }
      c->T.lw[cls] = best;
      rep[2] += 1;
      rep[3] += best != 0 && best != wdef;
      rep[4] += t0;
      rep[5] += tb;
    }
    if (cudaGetLastError() != cudaSuccess) status = cuda_check(c, "fc_autotune (warps)");
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  c->gflags = -1;  // launch shapes and plans changed: the next graph step captures again
  for (int k = 0; k < 6; ++k) c->tune_report[k] = rep[k];
  if (report)
    for (int k = 0; k < 6; ++k) report[k] = rep[k];
  if (status != FC_OK) return status;
  return cuda_check(c, "fc_autotune");
}

fc_status fc_drag(fc_ctx* c, const double* e, double* J, double* dJde, void* stream) {
  if (!c || !e || !J) return FC_ERR_INVALID;
  if (c->nwall == 0) return fail(c, FC_ERR_INVALID, "no curvilinear patch with a slip wall");
  cudaStream_t st = (cudaStream_t)stream;
  if (dJde) cudaMemsetAsync(dJde, 0, sizeof(double) * 4 * (size_t)c->P, st);
  // sharded: the rank that owns the wall ring's patch evaluates J; the others report 0
  const bool mine = !c->sharded() || c->owner[c->wall_patch] == c->rank;
  launch_drag(c->d_wall, c->d_wallw, c->d_wallc, mine ? c->nwall : 0, e, c->P, c->prm.gamma, J, dJde, st);
  c->launches++;
  return cuda_check(c, "fc_drag");
}

fc_status fc_sync_status(fc_ctx* c, const double* e, int check_state, void* stream) {
  if (!c) return FC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (check_state && e) {
    launch_check_state(c->T, e, c->d_flag, st);
    c->launches++;
  }
  int flag = 0;
  if (cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cuda_check(c, "fc_sync_status");
  if (flag) {
    cudaMemsetAsync(c->d_flag, 0, sizeof(int), st);
    return fail(c, (fc_status)flag, flag == FC_ERR_NONFINITE ? "non-finite or non-physical state" : "device timeout");
  }
  return FC_OK;
}

fc_status fc_profile_enable(fc_ctx* c, int enable) {
  if (!c) return FC_ERR_INVALID;
  c->prof = enable != 0;
  return FC_OK;
}

int fc_profile_read(fc_ctx* c) {
  if (!c) return -1;
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  for (const auto& r : c->prec) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    size_t k = 0;
    while (k < c->pnames.size() && c->pnames[k] != r.name) ++k;
    if (k == c->pnames.size()) {
      c->pnames.push_back(r.name);
      c->pms.push_back(0.0);
      c->pcount.push_back(0);
    }
    c->pms[k] += ms;
    c->pcount[k] += r.launches;
  }
  c->prec.clear();
  c->evused = 0;
  return (int)c->pnames.size();
}

fc_status fc_profile_get(const fc_ctx* c, int k, const char** name, double* ms, int* launches) {
  if (!c || k < 0 || k >= (int)c->pnames.size() || !name || !ms || !launches) return FC_ERR_INVALID;
  *name = c->pnames[k].c_str();
  *ms = c->pms[k];
  *launches = c->pcount[k];
  return FC_OK;
}

fc_status fc_profile_reset(fc_ctx* c) {
  if (!c) return FC_ERR_INVALID;
  c->pnames.clear();
  c->pms.clear();
  c->pcount.clear();
  c->prec.clear();
  c->evused = 0;
  return FC_OK;
}

// Algorithmic FP64 work of one launch of a line pass, by the conventional counts:
// 5 L log2 L flops per complex FFT of length L (two real lines per transform, one
// forward and one inverse per derivative), 4dC flops per continued real line
// (2d-term matvec per continuation point), 2 flops per complex mode for the
// multiplier, and the pointwise flux / viscous-flux / stage-combination work.
// Bytes: the compulsory HBM traffic of the pass (8 B per double read or written once).
fc_status fc_pass_stats(const fc_ctx* c, const char* pass, double* flops, double* bytes, long long* lines,
                        long long* points) {
  if (!c || !pass || !flops || !bytes || !lines || !points) return FC_ERR_INVALID;
  const fc_ctx::Queue* q = nullptr;
  int rounds = 2;              // derivative rounds per line
  double pw = 0.0, bw = 0.0;   // pointwise flops and bytes per point
  const std::string n(pass);
  if (n == "cart_q1") {
    q = &c->q_cart1;
    pw = 25.0;    // primitives once, x and y fluxes
    bw = 104.0;   // read e (32) and mu (8), write R1 (32) and the y fluxes (32)
  } else if (n == "cart_q2") {
    q = &c->q_cart2;
    pw = 37.0;    // L assembly and stage combination (the y fluxes come from the q1 pass)
    bw = 200.0;   // read the y fluxes, e, mu, R1, one more stage operand; write the stage output(s)
  } else if (n == "filter_q1" || n == "filter_q2") {
    q = n == "filter_q1" ? &c->q_filt1 : &c->q_filt2;
    rounds = 1;
    pw = 12.0;
    bw = 64.0;
  } else {
    return FC_ERR_INVALID;
  }
  // job lengths are not kept on the host after upload: recompute them from the patches
  double F = 0, Bt = 0;
  long long nl = 0, np = 0;
  auto add_line = [&](int nn, int L, int C) {
    F += rounds * (2.0 * 2.0 * 5.0 * L * std::log2((double)L) + 4.0 * 4.0 * c->d * C + 2.0 * 2.0 * 2.0 * L) + pw * nn;
    Bt += bw * nn;
    nl++;
    np += nn;
  };
  for (const HPatch& h : c->hp) {
    const bool aff = h.d.kind == FC_PATCH_AFFINE;
    const bool want1 = (n == "cart_q1" && aff) || n == "filter_q1";
    const bool want2 = (n == "cart_q2" && aff) || n == "filter_q2";
    if (want1)
      for (const Seg& s : h.seg1) {
        if (!s.periodic && s.n < 2 * c->prm.d) continue;
        const int C = s.periodic ? 0 : choose_continuation(s.n, c->prm, c->Cmax);
        add_line(s.n, s.n + C, C);
      }
    if (want2)
      for (const Seg& s : h.seg2) {
        if (s.n < 2 * c->prm.d) continue;
        const int C = choose_continuation(s.n, c->prm, c->Cmax);
        add_line(s.n, s.n + C, C);
      }
  }
  (void)q;
  *flops = F;
  *bytes = Bt;
  *lines = nl;
  *points = np;
  return FC_OK;
}

fc_status fc_line_stats(fc_ctx* c, long long* lines_q1, long long* lines_q2, double* flops_q1, double* flops_q2,
                        int reset) {
  if (!c) return FC_ERR_INVALID;
  unsigned long long l[2] = {0, 0};
  double f[2] = {0, 0};
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(l, c->d_skip_lines, sizeof(l), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(f, c->d_skip_flops, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check(c, "fc_line_stats");
  if (lines_q1) *lines_q1 = (long long)l[0];
  if (lines_q2) *lines_q2 = (long long)l[1];
  if (flops_q1) *flops_q1 = f[0];
  if (flops_q2) *flops_q2 = f[1];
  if (reset) {
    cudaMemset(c->d_skip_lines, 0, sizeof(l));
    cudaMemset(c->d_skip_flops, 0, sizeof(f));
  }
  return FC_OK;
}

fc_status fc_adjoint_step(fc_ctx* c, const double* e_n, const double* mu, const double* dt, const double* lam_np1,
                          double* lam_n, double* gbc, double* dparam, int flags, void* stream) {
  if (!c || !e_n || !mu || !dt || !lam_np1 || !lam_n) return FC_ERR_INVALID;
  if (dparam && !c->has_fs) return fail(c, FC_ERR_INVALID, "dparam needs fc_params.freestream");
  cudaStream_t st = (cudaStream_t)stream;
  if (dparam && !c->d_bcacc && c->nbc > 0) {
    if (!c->alloc(&c->d_bcacc, 2 * (size_t)c->nbc)) return FC_ERR_OOM;
    if (cudaMemsetAsync(c->d_bcacc, 0, sizeof(double) * 2 * (size_t)c->nbc, st) != cudaSuccess)
      return cuda_check(c, "fc_adjoint_step");
  }
  struct AccScope {  // the boundary transposes of this step feed dparam
    fc_ctx* c;
    AccScope(fc_ctx* c_, bool on) : c(c_) { c->cur_acc = on ? c->d_bcacc : nullptr; }
    ~AccScope() { c->cur_acc = nullptr; }
  } acc_scope(c, dparam != nullptr);
  auto finish = [&]() {
    if (dparam) {
      launch_pair_reduce(c->d_bcacc, c->nbc, dparam, st);
      c->launches += c->nbc > 0;
    }
    return comm_check(c, "fc_adjoint_step");
  };
  if (!c->adj_ready) {
    const size_t n4 = 4 * (size_t)c->P;
    bool ok = true;
    for (int k = 0; k < 5; ++k) ok = ok && c->alloc(&c->d_U[k], n4);
    ok = ok && c->alloc(&c->d_A0, n4) && c->alloc(&c->d_A14, n4) && c->alloc(&c->d_A2, n4) &&
         c->alloc(&c->d_A3, n4) && c->alloc(&c->d_PSa, n4) && c->alloc(&c->d_PSb, n4);
    if (!ok) return FC_ERR_OOM;
    c->adj_ready = true;
  }
  const bool filt = (flags & FC_STEP_FILTER) != 0;
  const size_t bytes4 = sizeof(double) * 4 * (size_t)c->P;
  if (filt && !c->d_FX) {
    if (!(c->alloc(&c->d_FX, 4 * (size_t)c->P) && c->alloc(&c->d_FY, 4 * (size_t)c->P))) return FC_ERR_OOM;
  }
  double** U = c->d_U;
  // forward recompute of the stage states u_0..u_4 (mu, dt frozen); with the filter,
  // u_0 = P(F(P(e_n))) and the states before (FX) and after (FY) F are kept
  cudaMemcpyAsync(U[0], e_n, bytes4, cudaMemcpyDeviceToDevice, st);
  project(c, U[0], st);
  if (filt) {
    cudaMemcpyAsync(c->d_FX, U[0], bytes4, cudaMemcpyDeviceToDevice, st);
    filter(c, U[0], false, st);
    cudaMemcpyAsync(c->d_FY, U[0], bytes4, cudaMemcpyDeviceToDevice, st);
    project(c, U[0], st);
  }
  StageCoef s{};
  s.dt = dt;
  s.U0 = U[0];
  const double c0[4] = {0.0, A20, A30, A40}, c1[4] = {1.0, A21, A32, A43}, cb[4] = {B1, B2, B3, B4};
  double *A0 = c->d_A0, *A14 = c->d_A14, *A2 = c->d_A2, *A3 = c->d_A3, *PSa = c->d_PSa, *PSb = c->d_PSb;
  for (int i = 0; i < 4; ++i) {
    s.Ucur = U[i];
    s.out = U[i + 1];
    s.c0 = c0[i];
    s.c1 = c1[i];
    s.cb = cb[i];
    if (i == 3 && c->any_walls) {  // acc = a52 u2 + a53 u3 + b53 dt L(u3) for u5 below
      s.Uaux = U[2];
      s.out2 = PSb;
      s.d1 = A53;
      s.d2 = A52;
      s.db = B53;
    }
    stage(c, s, mu, false, st);
    project(c, U[i + 1], st);
  }
  // the adiabatic walls' transpose at the last projection needs u5 = e_{n+1} (in A3 until
  // the reverse sweep first writes A3)
  if (c->any_walls) {
    StageCoef s5{};
    s5.dt = dt;
    s5.Ucur = U[4];
    s5.Uaux = PSb;
    s5.out = A3;
    s5.c1 = A54;
    s5.c2 = 1.0;
    s5.cb = B54;
    stage(c, s5, mu, false, st);
    project(c, A3, st);
  }
  // reverse sweep (Shu-Osher coefficients, see the forward stages)
  axpby(c, 1.0, lam_np1, 0.0, A14, st);
  projectT(c, A14, gbc, A3, st);  // lam_v5
  axpby(c, A53, A14, 0.0, A3, st);
  axpby(c, B53, A14, 0.0, PSb, st);
  axpby(c, A52, A14, 0.0, A2, st);
  axpby(c, B54, A14, 0.0, PSa, st);
  axpby(c, A54, A14, 0.0, A14, st);  // lam_u4 (without its L' term)
  adj_stage(c, U[4], mu, PSa, A14, dt, st);
  projectT(c, A14, gbc, U[4], st);  // lam_v4
  axpby(c, A40, A14, 0.0, A0, st);
  axpby(c, A43, A14, 1.0, A3, st);
  axpby(c, B4, A14, 1.0, PSb, st);
  adj_stage(c, U[3], mu, PSb, A3, dt, st);
  projectT(c, A3, gbc, U[3], st);  // lam_v3
  axpby(c, A30, A3, 1.0, A0, st);
  axpby(c, A32, A3, 1.0, A2, st);
  axpby(c, B3, A3, 0.0, PSa, st);
  adj_stage(c, U[2], mu, PSa, A2, dt, st);
  projectT(c, A2, gbc, U[2], st);  // lam_v2
  axpby(c, A20, A2, 1.0, A0, st);
  axpby(c, A21, A2, 0.0, A14, st);
  axpby(c, B2, A2, 0.0, PSb, st);
  adj_stage(c, U[1], mu, PSb, A14, dt, st);
  projectT(c, A14, gbc, U[1], st);  // lam_v1
  axpby(c, 1.0, A14, 1.0, A0, st);
  axpby(c, B1, A14, 0.0, PSa, st);
  adj_stage(c, U[0], mu, PSa, A0, dt, st);
  projectT(c, A0, gbc, U[0], st);
  if (filt) {  // transposes of F and of the projection before it
    filterT(c, A0, c->d_FX, c->d_FY, PSb, PSa, st);
    projectT(c, PSa, gbc, c->d_FX, st);
    cudaMemcpyAsync(lam_n, PSa, bytes4, cudaMemcpyDeviceToDevice, st);
    return finish();
  }
  cudaMemcpyAsync(lam_n, A0, bytes4, cudaMemcpyDeviceToDevice, st);
  return finish();
}

// ---------------------------------------------------------------- sharded execution

fc_status fc_partition(const fc_patch_desc* patches, int npatch, int nranks, int* owner) {
  if (!patches || npatch <= 0 || nranks < 1 || !owner) return FC_ERR_INVALID;
  // active points and centre of every patch
  std::vector<double> w(npatch), cx(npatch), cy(npatch);
  for (int p = 0; p < npatch; ++p) {
    const fc_patch_desc& d = patches[p];
    if (d.n1 < 1 || d.n2 < 1) return FC_ERR_INVALID;
    const long long N = (long long)d.n1 * d.n2;
    double sx = 0.0, sy = 0.0;
    long long act = 0;
    const bool hole = d.kind != FC_PATCH_OGRID && d.hole[2] > 0.0;
    for (int j = 0; j < d.n2; ++j)
      for (int i = 0; i < d.n1; ++i) {
        double x, y;
        if (d.kind == FC_PATCH_AFFINE) {
          x = d.geom[0] + (d.geom[1] - d.geom[0]) * (d.n1 > 1 ? (double)i / (d.n1 - 1) : 0.0);
          y = d.geom[2] + (d.geom[3] - d.geom[2]) * (d.n2 > 1 ? (double)j / (d.n2 - 1) : 0.0);
        } else if (d.kind == FC_PATCH_OGRID) {
          const double r = d.geom[2] + (d.geom[3] - d.geom[2]) * (d.n2 > 1 ? (double)j / (d.n2 - 1) : 0.0);
          const double th = 2.0 * PI * i / d.n1;
          x = d.geom[0] + r * std::cos(th);
          y = d.geom[1] + r * std::sin(th);
        } else {
          if (!d.x || !d.y) return FC_ERR_INVALID;
          x = d.x[(size_t)j * d.n1 + i];
          y = d.y[(size_t)j * d.n1 + i];
        }
        sx += x;
        sy += y;
        if (!hole || std::hypot(x - d.hole[0], y - d.hole[1]) >= d.hole[2]) ++act;
      }
    w[p] = (double)act;
    cx[p] = sx / (double)N;
    cy[p] = sy / (double)N;
  }
  // Morton order of the centres on a 2^16 x 2^16 grid over their bounding box
  double x0 = *std::min_element(cx.begin(), cx.end()), x1 = *std::max_element(cx.begin(), cx.end());
  double y0 = *std::min_element(cy.begin(), cy.end()), y1 = *std::max_element(cy.begin(), cy.end());
  const double span = std::max(std::max(x1 - x0, y1 - y0), 1e-300);
  auto spread = [](uint64_t v) {  // bits of v at even positions
    v &= 0xFFFF;
    v = (v | (v << 8)) & 0x00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0Full;
    v = (v | (v << 2)) & 0x33333333ull;
    v = (v | (v << 1)) & 0x55555555ull;
    return v;
  };
  std::vector<std::pair<uint64_t, int>> key(npatch);
  for (int p = 0; p < npatch; ++p) {
    const uint64_t qx = (uint64_t)std::min(65535.0, std::floor((cx[p] - x0) / span * 65535.0));
    const uint64_t qy = (uint64_t)std::min(65535.0, std::floor((cy[p] - y0) / span * 65535.0));
    key[p] = {spread(qx) | (spread(qy) << 1), p};
  }
  std::sort(key.begin(), key.end());
  // contiguous runs of about total / nranks along the curve
  double total = 0.0;
  for (double v : w) total += v;
  std::vector<int> first(nranks + 1, npatch);  // run r = order positions [first[r], first[r+1])
  first[0] = 0;
  {
    double cum = 0.0;
    int r = 1;
    for (int k = 0; k < npatch && r < nranks; ++k) {
      const double wk = w[key[k].second];
      while (r < nranks && cum + 0.5 * wk > total * r / nranks) first[r++] = k;
      cum += wk;
    }
    while (r < nranks) first[r++] = npatch;
  }
  // move boundaries by single patches while that lowers the larger neighbouring load
  std::vector<double> pre(npatch + 1, 0.0);  // weights along the curve, prefix sums
  for (int k = 0; k < npatch; ++k) pre[k + 1] = pre[k] + w[key[k].second];
  auto load = [&](int r) { return pre[first[r + 1]] - pre[first[r]]; };
  for (int pass = 0; pass < 4 * npatch; ++pass) {
    bool moved = false;
    for (int r = 1; r < nranks; ++r) {
      const double a = load(r - 1), b = load(r);
      const double cur = std::max(a, b);
      if (first[r] > first[r - 1] + 1) {  // left run gives its last patch
        const double v = w[key[first[r] - 1].second];
        if (std::max(a - v, b + v) < cur) {
          --first[r];
          moved = true;
          continue;
        }
      }
      if (first[r] + 1 < first[r + 1]) {  // right run gives its first patch
        const double v = w[key[first[r]].second];
        if (std::max(a + v, b - v) < cur) {
          ++first[r];
          moved = true;
        }
      }
    }
    if (!moved) break;
  }
  for (int r = 0; r < nranks; ++r)
    for (int k = first[r]; k < first[r + 1]; ++k) owner[key[k].second] = r;
  return FC_OK;
}

fc_status fc_shard(fc_ctx* c, int nranks, int rank, const int* owner, fc_comm_fn comm, void* user) {
  if (!c || nranks < 1 || rank < 0 || rank >= nranks || !owner) return FC_ERR_INVALID;
  if (c->nranks != 1 || !c->owner.empty()) return fail(c, FC_ERR_INVALID, "fc_shard: the context is sharded already");
  if (nranks > 1 && !comm) return fail(c, FC_ERR_INVALID, "fc_shard: a communication callback is needed");
  const int npatch = (int)c->hp.size();
  for (int p = 0; p < npatch; ++p)
    if (owner[p] < 0 || owner[p] >= nranks) return fail(c, FC_ERR_INVALID, "fc_shard: owner out of range");
  std::vector<int> own(owner, owner + npatch);
  std::vector<long long> offs(npatch + 1, 0);
  for (int p = 0; p < npatch; ++p) offs[p + 1] = c->hp[p].off + (long long)c->hp[p].n1 * c->hp[p].n2;
  auto patch_of = [&](long long idx) {
    return (int)(std::upper_bound(offs.begin() + 1, offs.end(), idx) - offs.begin() - 1);
  };
  auto mine = [&](long long idx) { return own[patch_of(idx)] == rank; };
  bool ok = true;
  // line queues of the owned patches
  for (fc_ctx::Queue* q : {&c->q_cart1, &c->q_cart2, &c->q_gen1, &c->q_gen2, &c->q_filt1, &c->q_filt2}) {
    std::vector<Job> jobs;
    for (const Job& J : q->h)
      if (own[J.patch] == rank) jobs.push_back(J);
    make_queue(c, *q, jobs, c->plans_h, npatch, ok);
  }
  // point lists of the owned patches
  std::vector<BcPt> bc;
  for (const BcPt& b : c->h_bc)
    if (mine(b.idx)) bc.push_back(b);
  std::vector<WallPt> walls;
  for (const WallPt& wp : c->h_walls)
    if (mine(wp.idx)) walls.push_back(wp);
  std::vector<int> fix, fc1, fc2, fyfix;
  for (int k : c->h_fix)
    if (mine(k)) fix.push_back(k);
  for (int k : c->h_fyfix)
    if (mine(k)) fyfix.push_back(k);
  for (int k : c->h_fcopy1)
    if (mine(k)) fc1.push_back(k);
  for (int k : c->h_fcopy2)
    if (mine(k)) fc2.push_back(k);
  std::vector<GFix> gfix;
  for (const GFix& g : c->h_gfix)
    if (mine(g.p)) gfix.push_back(g);
  // fringe receivers: local ones, and per peer the ones this rank interpolates for it and
  // the ones it receives, both in the order of the unsharded receiver list
  std::vector<Recv> loc, xsend;
  std::vector<int> xrecv;
  c->xp_fringe.scount.assign(nranks, 0);
  c->xp_fringe.rcount.assign(nranks, 0);
  for (int q = 0; q < nranks; ++q)
    for (const Recv& r : c->h_recv) {
      const int pd = own[patch_of(r.dst)], ps = own[patch_of(r.src[0])];
      if (q == rank && pd == rank && ps == rank) loc.push_back(r);
      if (q != rank && ps == rank && pd == q) {
        xsend.push_back(r);
        c->xp_fringe.scount[q] += 4;
      }
      if (q != rank && pd == rank && ps == q) {
        xrecv.push_back(r.dst);
        c->xp_fringe.rcount[q] += 4;
      }
    }
  // cross-patch blending: the owned points' entries, and the window sums of other ranks'
  // points they read (per peer, sorted, unique); the same rule on the peers' entries gives
  // what this rank sends
  std::vector<int> cdst, cptr{0}, csrc;
  std::vector<std::vector<int>> need(nranks), give(nranks);
  for (size_t i = 0; i < c->h_cdst.size(); ++i) {
    const int pd = own[patch_of(c->h_cdst[i])];
    if (pd == rank) cdst.push_back(c->h_cdst[i]);
    for (int k = c->h_cptr[i]; k < c->h_cptr[i + 1]; ++k) {
      const int src = c->h_csrc[k], ps = own[patch_of(src)];
      if (pd == rank) csrc.push_back(src);
      if (pd == rank && ps != rank) need[ps].push_back(src);
      if (pd != rank && ps == rank) give[pd].push_back(src);
    }
    if (pd == rank) cptr.push_back((int)csrc.size());
  }
  std::vector<int> vsend, vrecv;
  c->xp_visc.scount.assign(nranks, 0);
  c->xp_visc.rcount.assign(nranks, 0);
  for (int q = 0; q < nranks; ++q) {
    for (std::vector<int>* v : {&need[q], &give[q]}) {
      std::sort(v->begin(), v->end());
      v->erase(std::unique(v->begin(), v->end()), v->end());
    }
    vrecv.insert(vrecv.end(), need[q].begin(), need[q].end());
    vsend.insert(vsend.end(), give[q].begin(), give[q].end());
    c->xp_visc.rcount[q] = (long long)need[q].size();
    c->xp_visc.scount[q] = (long long)give[q].size();
  }
  std::vector<uint8_t> mask(npatch);
  for (int p = 0; p < npatch; ++p) mask[p] = own[p] == rank ? 1 : 0;
  std::vector<Recv> loc_interp;
  std::vector<PtCopy> loc_copy;
  split_exchange(loc, loc_interp, loc_copy);
  std::vector<int> xsend_dst;
  for (const Recv& r : xsend) xsend_dst.push_back(r.dst);
  ok = ok && c->upload(&c->d_bc, bc) && c->upload(&c->d_walls, walls) && c->upload(&c->d_fix, fix) &&
       c->upload(&c->d_fyfix, fyfix) && c->upload(&c->d_fcopy1, fc1) && c->upload(&c->d_fcopy2, fc2) && c->upload(&c->d_gfix, gfix) &&
       c->upload(&c->d_recv, loc_interp) && c->upload(&c->d_rcopy, loc_copy) && c->upload(&c->d_xsend, xsend) &&
       c->upload(&c->d_xsend_dst, xsend_dst) &&
       c->upload(&c->d_xrecv, xrecv) &&
       c->upload(&c->d_cross_dst, cdst) && c->upload(&c->d_cross_ptr, cptr) && c->upload(&c->d_cross_src, csrc) &&
       c->upload(&c->d_vsend, vsend) && c->upload(&c->d_vrecv, vrecv) && c->upload(&c->d_owned, mask) &&
       c->alloc(&c->xp_fringe.d_sbuf, 4 * xsend.size()) && c->alloc(&c->xp_fringe.d_rbuf, 4 * xrecv.size()) &&
       c->alloc(&c->xp_visc.d_sbuf, vsend.size()) && c->alloc(&c->xp_visc.d_rbuf, vrecv.size()) &&
       c->alloc(&c->d_dtmin, 1);
  if (!ok) return fail(c, FC_ERR_OOM, c->err);
  c->nbc = (int)bc.size();
  c->nwalls = (int)walls.size();
  c->nfix = (int)fix.size();
  c->nfyfix = (int)fyfix.size();
  c->nfcopy1 = (int)fc1.size();
  c->nfcopy2 = (int)fc2.size();
  c->ngfix = (int)gfix.size();
  c->nrecv = (int)loc_interp.size();
  c->nrcopy = (int)loc_copy.size();
  c->ncross = (int)cdst.size();
  c->xp_fringe.nsend = (int)xsend.size();
  c->xp_fringe.nrecv = (int)xrecv.size();
  c->xp_visc.nsend = (int)vsend.size();
  c->xp_visc.nrecv = (int)vrecv.size();
  c->owner = own;
  c->nranks = nranks;
  c->rank = rank;
  c->comm = comm;
  c->comm_user = user;
  c->T.owned = c->d_owned;
  if (c->gexec) {  // a captured step of the whole workload is stale now
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->gflags = -1;
  return cuda_check(c, "fc_shard");
}

fc_status fc_shard_counts(const fc_ctx* c, int which, int peer, long long* send, long long* recv) {
  if (!c || !send || !recv || which < 0 || which > 1 || peer < 0 || peer >= c->nranks || c->owner.empty())
    return FC_ERR_INVALID;
  const fc_ctx::XPlan& x = which == 0 ? c->xp_fringe : c->xp_visc;
  *send = x.scount[peer];
  *recv = x.rcount[peer];
  return FC_OK;
}

fc_status fc_initial_sensitivity(fc_ctx* c, const double* e0, const double* lam0, double* drho, double* dparam,
                                 void* stream) {
  if (!c || !e0 || !lam0) return FC_ERR_INVALID;
  if (dparam && !c->has_fs) return fail(c, FC_ERR_INVALID, "dparam needs fc_params.freestream");
  if (!drho && !dparam) return FC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (dparam && !c->d_part) {
    if (!c->alloc(&c->d_part, 2 * (size_t)SENS_BLOCKS)) return FC_ERR_OOM;
  }
  launch_init_sens(c->d_info, c->d_owned, c->P, e0, lam0, drho, dparam ? c->d_part : nullptr, c->fsj, st);
  c->launches++;
  if (dparam) {
    launch_pair_reduce(c->d_part, SENS_BLOCKS, dparam, st);
    c->launches++;
  }
  return cuda_check(c, "fc_initial_sensitivity");
}

}  // extern "C"
