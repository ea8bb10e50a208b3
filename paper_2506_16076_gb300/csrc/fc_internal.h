// Internal structures shared by the host runtime (fc_host.cpp) and the kernels (fc_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fcsdnn.h"

namespace fcx {

constexpr int MAXST = 24;       // max FFT stages per plan
constexpr int MAXW = 8;         // max warps per CTA in the line kernels
constexpr int LINE_WARPS_DEFAULT = 1;  // default warps per CTA in the line kernels
constexpr size_t SMEM_CAP = 200 * 1024;  // dynamic shared memory budget per CTA
constexpr int SDNN_H = 16;      // hidden width of the stand-in classifier
constexpr int MAX_GENERIC_RADIX = 128;  // largest prime factor of a continued length
constexpr int CONT_TMP = 32;    // complex scratch per warp after the line buffer (detrended end data, d <= 8)
constexpr int NCLASS = 24;      // length classes of the line queues: ceil(log2 Lmax)

// Per-point flag word.
enum : uint32_t {
  PT_BLANK = 1u,      // blanked (inside a hole): never updated, mu = 0
  PT_NODIFF = 2u,     // on a line segment too short for FC in some direction: L = 0
  PT_GEN = 4u,        // viscosity-generation point (depth >= n_v)
  PT_W1_SHIFT = 3,    // 3 bits: 7-point window start offset along q1 (0..6) or 7 = none
  PT_W2_SHIFT = 6,    // 3 bits: same along q2
  PT_PATCH_SHIFT = 9  // remaining bits: patch index
};
__host__ __device__ inline int pt_patch(uint32_t f) { return (int)(f >> PT_PATCH_SHIFT); }
__host__ __device__ inline int pt_w1(uint32_t f) { return (int)((f >> PT_W1_SHIFT) & 7u); }
__host__ __device__ inline int pt_w2(uint32_t f) { return (int)((f >> PT_W2_SHIFT) & 7u); }

// FFT plan of one length L (mixed-radix Stockham, natural order in and out).
struct Plan {
  int L;
  int nst;
  int rad[MAXST];
  int tw;     // offset of the L-entry forward twiddle table exp(-2 pi i e / L) in the twiddle pool
  int sig;    // offset of the L-entry filter table sigma(2k/L)/L in the real pool (-1: none)
  int rev;    // offset of the L-entry slot -> mode table of the in-place transforms in the int pool
  // FMA-form butterfly records and scale tables (fc_tables.h): offsets in the twiddle pool
  // of the inverse (fmd) and forward (fmf) records; bit st of fmsc: forward stage st
  // multiplies its inputs by the L pending factors that follow psc in the real pool;
  // per-slot derivative (dmul) and filter (sigp, -1: none) factors in the real pool; bit
  // st of fmod: forward stage st (odd radix, span 1) folds its inputs' factors into the
  // butterfly through per-butterfly records among the forward records
  int fmd, fmf, fmsc, psc, dmul, sigp, fmod;
};

// One line segment processed by one warp.
struct Job {
  long long base;   // flat index of the first point
  int stride;       // 1 (q1 line) or n1 (q2 line)
  int n;            // points on the segment
  int plan;         // plan index (L = n + C, or n when periodic)
  int fcm;          // offset of the combined continuation matrices in the real pool (-1: periodic)
  int C;            // continuation points (0 when periodic)
  int patch;
  long long gbase;  // index of the first point in the curvilinear scratch (-1: affine patch)
  double scale;     // multiplier of the per-index derivative: 1/h (affine: per unit x or y)
};

struct PatchDev {
  long long off;    // first flat index
  long long gbase;  // first index in the curvilinear scratch (-1 for affine)
  int n1, n2, kind, periodic1;
  double hhat, htil;
  int pform;        // 1: the product-rule form of the operator (adiabatic wall patch, fc_params.wall_form)
  int pad;
};

// Receiver of the inter-patch exchange: 3x3 donor stencil, iterated quadratic weights.
struct Recv {
  int dst;
  int src[9];       // donor flat indices, row-major over (m2, m1)
  double w1[3], w2[3];
};

// Receiver that coincides with a donor grid point (sub-patches of one patch share their
// overlap points, Sec. 3.4.2): the exchange copies the value.
struct PtCopy {
  int dst, src;
};

// Boundary overwrite of one point.
struct BcPt {
  int idx;
  int mode;         // bit0: zero rho u, bit1: zero rho v, bit2: remove normal (nx, ny), bit3: Dirichlet,
                    // bit4: the Dirichlet state is the free stream (its adjoint feeds dJ/d(M, alpha))
  double nx, ny;
  double val[4];    // Dirichlet conserved state
};

// No-slip adiabatic wall point: momenta set to 0, E = rho theta_w / (gamma - 1) with
// theta_w = sum_j w[j] theta(e at idx + (j + 1) step), j < nw (the inward grid line).
struct WallPt {
  int idx;
  int step;  // state-index step to the next point inward along the wall-normal grid line
  int nw;    // d - 1
  double w[7];
};

// Curvilinear point that only one direction's line passes reach (hole-cut or short
// segments): mode 1 = on a long q2 segment only, mode 2 = on a long q1 segment only.
struct GFix {
  int p;     // flat state index
  int g;     // index into the curvilinear scratch / metrics
  int mode;
  int pad;
};

// Runge-Kutta stage combination applied in the last pass of a stage:
//   out  = c0 U0 + c1 Ucur + c2 Uaux + cb dt L
//   out2 = d2 Uaux + d1 Ucur + db dt L        (only when out2 != nullptr)
//   rhs_only: out = L
struct StageCoef {
  const double* U0;
  const double* Ucur;
  const double* Uaux;
  double* out;
  double* out2;
  double c0, c1, c2, cb, d1, d2, db;
  const double* dt;
  int rhs_only;
};

struct DevTables {
  const double2* tw;        // twiddle pool
  const double* rp;         // real pool (continuation matrices, filter tables)
  const int* ip;            // int pool (slot -> mode tables)
  const Plan* plans;
  const uint32_t* info;     // per-point flags
  const PatchDev* patches;
  int npatch;
  long long P;              // points (component stride of the state)
  long long Pg;             // points of curvilinear patches (component stride of the scratch)
  double gamma;
  int d;
  // lines whose gradient round was skipped because mu == 0 on the whole line (H = f(e)
  // exactly there), and the algorithmic flops of the skipped rounds: [q1, q2] each
  unsigned long long* skip_lines;
  double* skip_flops;
  // warps per CTA of the line kernels per length class ceil(log2 Lmax) (0: the default);
  // set by the autotuner
  int lw[NCLASS];
  // sharded execution: 1 for the patches this rank owns (null: all patches are owned)
  const uint8_t* owned;
  // 1 when some patch uses the product-rule wall form (fc_params.wall_form)
  int any_pform;
};

// ---- launch wrappers (fc_kernels.cu) ----
// Fy (nullable): the y fluxes of the affine points, written by the q1 pass (and by
// launch_flux_y_points where no q1 line passes) and read by the q2 pass instead of
// recomputing them from the state; null: the q2 pass computes them
void launch_cart_q1(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, const double* mu,
                    double* R1, double* Fy, cudaStream_t st);
void launch_cart_q2(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* mu, const double* R1,
                    const double* Fy, const StageCoef& sc, cudaStream_t st);
void launch_flux_y_points(const DevTables& T, const int* idx, int n, const double* e, double* Fy, cudaStream_t st);
void launch_gen_A(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, double* G, cudaStream_t st);
void launch_gen_B(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, const double* mu,
                  const double* J, double* G, cudaStream_t st);
void launch_gen_C(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* J, double* G,
                  const StageCoef& sc, cudaStream_t st);
void launch_rk_fixup(const DevTables& T, const int* idx, int n, const StageCoef& sc, cudaStream_t st);
void launch_gen_fix(const DevTables& T, const GFix* f, int n, const double* e, const double* mu, const double* J,
                    double* G, cudaStream_t st);
void launch_adj_gen_fixA(const DevTables& T, const GFix* f, int n, const double* J, const double* u,
                         const double* mu, const double* psi, double* G, cudaStream_t st);
void launch_adj_gen_fixB(const DevTables& T, const GFix* f, int n, const double* G, double* R1, cudaStream_t st);
void launch_bc(const BcPt* bc, int n, double* e, long long P, cudaStream_t st);
void launch_bc_wall(const WallPt* w, int n, double* e, long long P, double gamma, cudaStream_t st);
void launch_bc_wall_T(const WallPt* w, int n, const double* u, double* lam, long long P, double gamma,
                      cudaStream_t st);
void launch_filterT_q2(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* lam, const double* ef,
                       double* MF, cudaStream_t st);
void launch_filterT_q1(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* MF, const double* e,
                       double* out, cudaStream_t st);
void launch_filterT_copy2(const DevTables& T, const int* idx, int n, const double* lam, const double* ef, double* MF,
                          cudaStream_t st);
void launch_filterT_copy1(const DevTables& T, const int* idx, int n, const double* MF, const double* e, double* out,
                          cudaStream_t st);
void launch_exchange(const Recv* r, int n, double* e, long long P, cudaStream_t st);
void launch_copy_points(const PtCopy* c, int n, double* e, long long P, cudaStream_t st);
// sharded exchange: buf[4 i + c] = the interpolated value of record i (as launch_exchange
// would write it), and its scatter e[dst[i] + c P] = buf[4 i + c]
void launch_xpack(const Recv* r, int n, const double* e, long long P, double* buf, cudaStream_t st);
void launch_xunpack(const int* dst, int n, const double* buf, double* e, long long P, cudaStream_t st);
// buf[i] = src[idx[i]] and dst[idx[i]] = buf[i]
void launch_gather(const int* idx, int n, const double* src, double* buf, cudaStream_t st);
// buf[4 i + c] = e[dst[i] + c P] (the adjoint's reversed fringe exchange)
void launch_xgather(const int* dst, int n, const double* e, long long P, double* buf, cudaStream_t st);
void launch_scatter(const int* idx, int n, const double* buf, double* dst, cudaStream_t st);
void launch_filter_q1(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, double* F, cudaStream_t st);
void launch_filter_q2(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* F, double* e, cudaStream_t st);
void launch_filter_copy_q1(const DevTables& T, const int* idx, int n, const double* e, double* F, cudaStream_t st);
void launch_filter_copy_q2(const DevTables& T, const int* idx, int n, const double* F, double* e, cudaStream_t st);
void launch_visc_point(const DevTables& T, const double* e, double* phi, double* S, cudaStream_t st);
void launch_visc_muhat(const DevTables& T, const double* phi, const double* S, const float* w, const double* R,
                       double* muhat, int32_t* tau, cudaStream_t st);
void launch_window_rows(const DevTables& T, const double* in, double* out, const double* wtab, int r, cudaStream_t st);
void launch_window_cols(const DevTables& T, const double* in, double* out, const double* wtab, int r, cudaStream_t st);
void launch_mu_final(const DevTables& T, const double* num, const double* den, const int* cross_dst,
                     const int* cross_ptr, const int* cross_src, int ncross, double* mu, cudaStream_t st);
void launch_dt(const DevTables& T, const double* e, const double* mu, unsigned long long* pmax, double cfl,
               double* dt, cudaStream_t st);
void launch_check_state(const DevTables& T, const double* e, int* flag, cudaStream_t st);
void launch_adj_cart(const DevTables& T, const Job* jobs, int njobs, int Lmax, int dir, const double* u,
                     const double* mu, const double* psi, double* R1, double* acc, const double* dt, cudaStream_t st);
void launch_adj_gen_A(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* J, const double* u,
                      const double* psi, double* G, cudaStream_t st);
void launch_adj_gen_B(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* J, const double* u,
                      const double* mu, const double* psi, double* G, cudaStream_t st);
void launch_adj_gen_C(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* u, const double* G,
                      double* acc, const double* dt, cudaStream_t st);
void launch_adj_fixup(const int* idx, int n, const double* R1, double* acc, long long P, const double* dt,
                      cudaStream_t st);
void launch_exchange_T(const int* dptr, const int* dsrc, const int* drecv, const double* dw, int nd, const Recv* r,
                       int nr, double* lam, long long P, cudaStream_t st);
// d e_fs / dM and d e_fs / dalpha of the conserved free stream at fixed density and pressure
struct FsJac {
  double dM[4], dA[4];
};
// acc (nullable, [n][2]): per boundary record, += its Dirichlet adjoint . (dM, dA) on free-stream points
void launch_bc_T(const BcPt* bc, int n, double* lam, double* gbc, double* acc, FsJac fj, long long P,
                 cudaStream_t st);
// out[0..1] += the sums over i < n of acc[2 i], acc[2 i + 1] in a fixed order; acc is zeroed
void launch_pair_reduce(double* acc, int n, double* out, cudaStream_t st);
constexpr int SENS_BLOCKS = 1024;
// drho (nullable) = lam0 . d e / d rho at fixed u, v, p; part (nullable, [SENS_BLOCKS][2]): per-block
// sums of lam0 . (dM, dA) over non-blanked points (of the owned patches, owned non-null)
void launch_init_sens(const uint32_t* info, const uint8_t* owned, long long P, const double* e0, const double* lam0,
                      double* drho, double* part, FsJac fj, cudaStream_t st);
void launch_drag(const int* wall, const double* w, const double* nx, int n, const double* e, long long P, double gam,
                 double* J, double* dJde, cudaStream_t st);
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t st);
int length_class(int Lmax);
size_t line_smem_bytes(const DevTables& T, int Lmax);
int line_warps(const DevTables& T, int Lmax);
int line_warps_max(int Lmax);
void launch_deriv_lines(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* src, double* dst,
                        cudaStream_t st);
void launch_grid_metrics(const GFix* pts, int n, const double* D1, const double* D2, long long P, double* Jm,
                         long long Pg, int* bad, cudaStream_t st);
void launch_fill_wave(double* p, long long n, double a, double b, double w, cudaStream_t st);
void set_kernel_attributes();

}  // namespace fcx
