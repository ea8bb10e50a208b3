// Device kernels of the multi-patch FC-SDNN operator (sm_103a, FP64).
//
// Line kernels: one warp per grid-line segment, shared-memory mixed-radix Stockham
// FFTs of the FC-Gram continued line (Sec. 2.2), fused with the Euler flux, the
// artificial-viscosity flux and the SSPRK stage combination (Sec. 2.1, 2.3, 4.1).
// The path is bound by the FP64 pipe (2 FP64 lanes/clk/SM on GB300), so the kernels
// minimise FP64 instructions: packed real pairs per complex FFT, radix 2/3/4/5/7/8
// butterflies with table twiddles, continuation as a 2d-term matvec.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "fc_internal.h"
#include "fc_line.cuh"

namespace fcx {

// Register budget of the line kernels: by default the compiler may use up to 255
// registers per thread for a 256-thread CTA; FC_LINE_MAXNREG (a build flag) caps it
// instead, trading a few spills for more resident warps per SM.
#ifdef FC_LINE_MAXNREG
#define LINE_KERNEL_BOUNDS __maxnreg__(FC_LINE_MAXNREG)
#else
#define LINE_KERNEL_BOUNDS __launch_bounds__(MAXW * 32)
#endif

// Warps per CTA of the line kernels. Each warp owns one line at a time and the warps of
// a CTA never synchronise with each other, so small CTAs let the block scheduler hand a
// freed warp slot the next line at once (lines differ in length and in the number of
// derivative rounds); FCSDNN_LINE_WARPS (1..8) overrides the default for launch-shape
// sweeps. Shared memory per warp: 2 Lmax complex values (two packed sequences,
// transformed in place) plus the continuation's end data.
static int line_warps_cap() {
  static int cap = [] {
    const char* v = getenv("FCSDNN_LINE_WARPS");
    const int c = v ? atoi(v) : LINE_WARPS_DEFAULT;
    return c < 1 ? 1 : (c > MAXW ? MAXW : c);
  }();
  return cap;
}
int length_class(int Lmax) {
  int k = 0;
  while (k + 1 < NCLASS && (1 << k) < Lmax) ++k;
  return k;
}
// most warps whose line buffers fit the shared-memory budget (at most MAXW)
int line_warps_max(int Lmax) {
  const size_t per = (size_t)(2 * Lmax + CONT_TMP) * sizeof(double2);
  const int w = (int)(SMEM_CAP / per);
  return w < 1 ? 1 : (w > MAXW ? MAXW : w);
}
// warps per CTA: the class's tuned value, else FCSDNN_LINE_WARPS / the default, within the budget
int line_warps(const DevTables& T, int Lmax) {
  const int tuned = T.lw[length_class(Lmax)];
  const int want = tuned > 0 ? tuned : line_warps_cap();
  const int w = line_warps_max(Lmax);
  return want < w ? want : w;
}
size_t line_smem_bytes(const DevTables& T, int Lmax) {
  return (size_t)line_warps(T, Lmax) * (2 * Lmax + CONT_TMP) * sizeof(double2);
}

__device__ __forceinline__ void flux_xy(double r, double mx, double my, double E, double gam, double* fx, double* fy) {
  const double ir = 1.0 / r;
  const double u = mx * ir, v = my * ir;
  const double p = (gam - 1.0) * (E - 0.5 * (mx * u + my * v));
  fx[0] = mx;
  fx[1] = fma(mx, u, p);
  fx[2] = mx * v;
  fx[3] = u * (E + p);
  fy[0] = my;
  fy[1] = my * u;
  fy[2] = fma(my, v, p);
  fy[3] = v * (E + p);
}

__device__ __forceinline__ void flux_x(double r, double mx, double my, double E, double gam, double* f) {
  const double ir = 1.0 / r;
  const double u = mx * ir, v = my * ir;
  const double p = (gam - 1.0) * (E - 0.5 * (mx * u + my * v));
  f[0] = mx;
  f[1] = fma(mx, u, p);
  f[2] = mx * v;
  f[3] = u * (E + p);
}
__device__ __forceinline__ void flux_y(double r, double mx, double my, double E, double gam, double* f) {
  const double ir = 1.0 / r;
  const double u = mx * ir, v = my * ir;
  const double p = (gam - 1.0) * (E - 0.5 * (mx * u + my * v));
  f[0] = my;
  f[1] = my * u;
  f[2] = fma(my, v, p);
  f[3] = v * (E + p);
}

// ---- product-rule form on adiabatic wall patches (Remark adiabatic)
// Derivatives along one direction of e = (rho, rho u, rho v, E) and of p from those of
// Q = (rho, rho u, rho v, theta): dp = theta drho + rho dtheta (eq. p_T),
// dE = dp / (gamma - 1) + u d(rho u) + v d(rho v) - (u^2 + v^2) / 2 drho (eq. perfect_gas_T).
__device__ __forceinline__ void product_rule(const double* Q, const double* DQ, double gm1, double* De, double& Dp) {
  const double ir = 1.0 / Q[0];
  const double u = Q[1] * ir, v = Q[2] * ir;
  Dp = fma(Q[3], DQ[0], Q[0] * DQ[3]);
  De[0] = DQ[0];
  De[1] = DQ[1];
  De[2] = DQ[2];
  De[3] = fma(-0.5 * fma(u, u, v * v), DQ[0], fma(u, DQ[1], fma(v, DQ[2], Dp / gm1)));
}

// div f(e) (eq. euler 2d equation) by the sum and product rules from the x and y derivatives
// of e (ex, ey) and p (px, py); theta = p / rho; du = (d(rho u) - u drho) / rho
__device__ __forceinline__ void conv_div_product(const double* e, double th, const double* ex, double px,
                                                 const double* ey, double py, double* out) {
  const double ir = 1.0 / e[0];
  const double u = e[1] * ir, v = e[2] * ir, p = e[0] * th;
  const double ux = (ex[1] - u * ex[0]) * ir, vy = (ey[2] - v * ey[0]) * ir;
  out[0] = ex[1] + ey[2];
  out[1] = fma(u, ex[1], fma(e[1], ux, px)) + fma(v, ey[1], e[1] * vy);
  out[2] = fma(u, ex[2], e[2] * ux) + fma(v, ey[2], fma(e[2], vy, py));
  out[3] = fma(e[3] + p, ux + vy, fma(u, ex[3] + px, v * (ey[3] + py)));
}

// theta = p / rho (eq. p_T)
__device__ __forceinline__ double theta_of(double r, double mx, double my, double E, double gam) {
  const Prim q = primitives(r, mx, my, E, gam);
  return q.p / r;
}

// Load 4 state components of a line into two packed complex sequences.
__device__ __forceinline__ void load4(double2* A, int L, const Job& J, const double* __restrict__ src, long long cs,
                                      int lane) {
  for (int t = lane; t < J.n; t += 32) {
    const long long p = J.base + (long long)t * J.stride;
    A[t] = cpx(src[p], src[p + cs]);
    A[L + t] = cpx(src[p + 2 * cs], src[p + 3 * cs]);
  }
}

// The same with theta in place of E (the product-rule form's differentiated quantities).
__device__ __forceinline__ void load4_theta(double2* A, int L, const Job& J, const double* __restrict__ e,
                                            long long cs, double gam, int lane) {
  for (int t = lane; t < J.n; t += 32) {
    const long long p = J.base + (long long)t * J.stride;
    const double r = e[p], mx = e[p + cs], my = e[p + 2 * cs];
    A[t] = cpx(r, mx);
    A[L + t] = cpx(my, theta_of(r, mx, my, e[p + 3 * cs], gam));
  }
}

// In place on the two sequences in A (continued first if the line is not periodic):
// forward transform, derivative multiplier, inverse transform (eq. fc_der).
__device__ __forceinline__ void deriv2(double2* A, int Lmax, const Job& J, const Plan& P, const DevTables& T,
                                       int lane) {
  if (J.fcm >= 0) {
    FC_SYNC();
    continue_lines(A, P.L, J.n, J.C, T.d, T.rp + J.fcm, 2, lane, 32, A + 2 * Lmax);
  }
  FC_SYNC();
  fft_forward_mul<MUL_DERIV>(A, P, 2, T.tw, T.rp, J.scale * TWO_PI / ((double)P.L * (double)P.L), lane, 32);
  fft_inplace<true>(A, P, 2, T.tw, T.rp, lane, 32);
}

// true on every lane when mu != 0 somewhere on the line (warp vote)
__device__ __forceinline__ bool line_viscous(const Job& J, const double* __restrict__ mu, int lane) {
  bool v = false;
  for (int t = lane; t < J.n; t += 32) v |= (mu[J.base + (long long)t * J.stride] != 0.0);
  return __any_sync(0xffffffffu, v);
}

// record a skipped gradient round: one line, its algorithmic flops (2 packed transforms
// forward and inverse, continuation of 4 components, multiplier)
__device__ __forceinline__ void count_skip(const DevTables& T, int dir, const Job& J, int L, int lane) {
  if (lane == 0 && T.skip_lines) {
    atomicAdd(T.skip_lines + dir, 1ull);
    const double f = 4.0 * 5.0 * L * log2((double)L) + 16.0 * T.d * J.C + 8.0 * L;
    atomicAdd(T.skip_flops + dir, f);
  }
}

__device__ __forceinline__ void stage_write(const StageCoef& sc, long long p, long long cs, const double* L4) {
  if (sc.rhs_only) {
#pragma unroll
    for (int c = 0; c < 4; ++c) sc.out[p + c * cs] = L4[c];
    return;
  }
  const double dt = *sc.dt;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const long long q = p + c * cs;
    const double cur = sc.Ucur[q];
    double v = sc.c1 * cur;
    double aux = 0.0;
    if (sc.c0 != 0.0) v = fma(sc.c0, sc.U0[q], v);
    if (sc.Uaux) aux = sc.Uaux[q];
    if (sc.c2 != 0.0) v = fma(sc.c2, aux, v);
    v = fma(sc.cb * dt, L4[c], v);
    if (sc.out2) sc.out2[q] = fma(sc.db * dt, L4[c], fma(sc.d2, aux, sc.d1 * cur));
    sc.out[q] = v;
  }
}

// ---------------------------------------------------------------- affine patches, q1 lines
// d/dx of e -> H_x = f_x(e) - mu d/dx e -> R1 = d/dx H_x  (J11 folded into J.scale = 1/hx)
// Fy (nullable): the y fluxes of the line's points, from the same primitives, for the q2 pass
__global__ void LINE_KERNEL_BOUNDS k_cart_q1(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                        const double* __restrict__ e, const double* __restrict__ mu,
                                                        double* __restrict__ R1, double* __restrict__ Fy) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    const bool visc = line_viscous(J, mu, lane);
    if (visc) {
      load4(A, L, J, e, cs, lane);
      deriv2(A, Lmax, J, P, T, lane);
    } else {
      count_skip(T, 0, J, L, lane);
    }
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      double f[4];
      if (Fy) {
        double fy[4];
        flux_xy(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma, f, fy);
#pragma unroll
        for (int c = 0; c < 4; ++c) Fy[p + c * cs] = fy[c];
      } else {
        flux_x(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma, f);
      }
      if (visc) {
        const double m = mu[p];
        const double2 g0 = A[t], g1 = A[L + t];
        A[t] = cpx(fma(-m, g0.x, f[0]), fma(-m, g0.y, f[1]));
        A[L + t] = cpx(fma(-m, g1.x, f[2]), fma(-m, g1.y, f[3]));
      } else {
        A[t] = cpx(f[0], f[1]);
        A[L + t] = cpx(f[2], f[3]);
      }
    }
    deriv2(A, Lmax, J, P, T, lane);
    double2* Z = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const double2 a = Z[t], b = Z[L + t];
      R1[p] = a.x;
      R1[p + cs] = a.y;
      R1[p + 2 * cs] = b.x;
      R1[p + 3 * cs] = b.y;
    }
    FC_SYNC();
  }
}

// ---------------------------------------------------------------- affine patches, q2 lines
// d/dy of e -> H_y -> R2 = d/dy H_y; L = -(R1 + R2) (0 on PT_NODIFF points); stage combination.
// Fy (nullable): the y fluxes written by the q1 pass, read instead of computed
__device__ __forceinline__ void q2_line(const DevTables& T, const Job& J, const Plan& P, double2* A, int Lmax,
                                        const double* __restrict__ mu, const double* __restrict__ R1,
                                        const double* __restrict__ Fy, const StageCoef& sc, int lane) {
  const long long cs = T.P;
  const double* e = sc.Ucur;
  const int L = P.L;
  const bool visc = line_viscous(J, mu, lane);
  if (visc) {
    load4(A, L, J, e, cs, lane);
    deriv2(A, Lmax, J, P, T, lane);
  } else {
    count_skip(T, 1, J, L, lane);
  }
  for (int t = lane; t < J.n; t += 32) {
    const long long p = J.base + (long long)t * J.stride;
    double f[4];
    if (Fy) {
#pragma unroll
      for (int c = 0; c < 4; ++c) f[c] = Fy[p + c * cs];
    } else {
      flux_y(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma, f);
    }
    if (visc) {
      const double m = mu[p];
      const double2 g0 = A[t], g1 = A[L + t];
      A[t] = cpx(fma(-m, g0.x, f[0]), fma(-m, g0.y, f[1]));
      A[L + t] = cpx(fma(-m, g1.x, f[2]), fma(-m, g1.y, f[3]));
    } else {
      A[t] = cpx(f[0], f[1]);
      A[L + t] = cpx(f[2], f[3]);
    }
  }
  deriv2(A, Lmax, J, P, T, lane);
  for (int t = lane; t < J.n; t += 32) {
    const long long p = J.base + (long long)t * J.stride;
    const double2 a = A[t], b = A[L + t];
    double L4[4];
    if (T.info[p] & PT_NODIFF) {
      L4[0] = L4[1] = L4[2] = L4[3] = 0.0;
    } else {
      L4[0] = -(R1[p] + a.x);
      L4[1] = -(R1[p + cs] + a.y);
      L4[2] = -(R1[p + 2 * cs] + b.x);
      L4[3] = -(R1[p + 3 * cs] + b.y);
    }
    stage_write(sc, p, cs, L4);
  }
}

// one warp per line
__global__ void LINE_KERNEL_BOUNDS k_cart_q2(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                        const double* __restrict__ mu, const double* __restrict__ R1,
                                                        const double* __restrict__ Fy, StageCoef sc) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    q2_line(T, J, T.plans[J.plan], A, Lmax, mu, R1, Fy, sc, lane);
    FC_SYNC();
  }
}

// ---------------------------------------------------------------- affine patches, q2 lines, tiled
// A CTA of TW warps takes TW consecutive jobs of the queue. When they are TW adjacent
// columns of one patch with the same segment (the common case), the CTA reads their
// points row by row (TW consecutive doubles per row: whole 32-byte sectors) into the
// warps' line buffers, and writes the stage result the same way; in between each warp
// transforms its own column. Other job sets run one line per warp as in k_cart_q2.
// Registers are held to 5 resident CTAs per SM (measured a little faster than 4 CTAs
// with more registers and no spills).
constexpr int TW = 4;
__host__ __device__ inline int tiled_stride(int Lmax) {
  const int b = 2 * Lmax + CONT_TMP;
  return b + ((2 - b % 8) + 8) % 8;  // = 2 (mod 8): conflict-free row-by-column smem access
}
__global__ void __launch_bounds__(TW * 32, 5) k_cart_q2_tiled(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                            int Lmax, const double* __restrict__ mu,
                                                            const double* __restrict__ R1,
                                                            const double* __restrict__ Fy, StageCoef sc) {
  extern __shared__ double2 sm[];
  __shared__ int vflag[TW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sA = tiled_stride(Lmax);
  double2* A = sm + warp * sA;
  const long long cs = T.P;
  const double* e = sc.Ucur;
  for (int g0 = blockIdx.x * TW; g0 < njobs; g0 += gridDim.x * TW) {
    const int nc = min(TW, njobs - g0);
    const Job J0 = jobs[g0];
    bool tiled = true;
    for (int c = 1; c < nc; ++c) {
      const Job Jc = jobs[g0 + c];
      tiled = tiled && Jc.base == J0.base + c && Jc.stride == J0.stride && Jc.n == J0.n && Jc.plan == J0.plan &&
              Jc.fcm == J0.fcm && Jc.C == J0.C && Jc.scale == J0.scale;
    }
    if (!tiled) {
      if (warp < nc) {
        const Job J = jobs[g0 + warp];
        q2_line(T, J, T.plans[J.plan], A, Lmax, mu, R1, Fy, sc, lane);
      }
      __syncthreads();
      continue;
    }
    const Plan P = T.plans[J0.plan];
    const int L = P.L, n = J0.n, st = J0.stride;
    if (threadIdx.x < TW) vflag[threadIdx.x] = 0;
    __syncthreads();
    // rows of the TW columns: the y fluxes (Fy) or e into the line buffers, viscosity
    // vote per column
    const double* src = Fy ? Fy : e;
    for (int k = threadIdx.x; k < n * TW; k += TW * 32) {
      const int r = k / TW, c = k % TW;
      if (c < nc) {
        const long long p = J0.base + c + (long long)r * st;
        if (mu[p] != 0.0) vflag[c] = 1;
        double2* Ac = sm + c * sA;
        Ac[r] = cpx(src[p], src[p + cs]);
        Ac[L + r] = cpx(src[p + 2 * cs], src[p + 3 * cs]);
      }
    }
    __syncthreads();
    if (warp < nc) {
      const Job J = jobs[g0 + warp];
      const bool visc = vflag[warp] != 0;
      if (visc) {  // gradient of e first (e of this column again if the rows held Fy)
        if (Fy) {
          FC_SYNC();
          load4(A, L, J, e, cs, lane);
        }
        deriv2(A, Lmax, J, P, T, lane);
        for (int t = lane; t < n; t += 32) {
          const long long p = J.base + (long long)t * st;
          double f[4];
          if (Fy) {
#pragma unroll
            for (int c = 0; c < 4; ++c) f[c] = Fy[p + c * cs];
          } else {
            flux_y(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma, f);
          }
          const double m = mu[p];
          const double2 g0v = A[t], g1v = A[L + t];
          A[t] = cpx(fma(-m, g0v.x, f[0]), fma(-m, g0v.y, f[1]));
          A[L + t] = cpx(fma(-m, g1v.x, f[2]), fma(-m, g1v.y, f[3]));
        }
      } else {
        count_skip(T, 1, J, L, lane);
        if (!Fy) {
          for (int t = lane; t < n; t += 32) {
            const double2 a = A[t], b = A[L + t];
            double f[4];
            flux_y(a.x, a.y, b.x, b.y, T.gamma, f);
            A[t] = cpx(f[0], f[1]);
            A[L + t] = cpx(f[2], f[3]);
          }
        }
      }
      deriv2(A, Lmax, J, P, T, lane);
    }
    __syncthreads();
    // rows again: stage combination of the TW columns
    for (int k = threadIdx.x; k < n * TW; k += TW * 32) {
      const int r = k / TW, c = k % TW;
      if (c < nc) {
        const long long p = J0.base + c + (long long)r * st;
        const double2* Ac = sm + c * sA;
        const double2 a = Ac[r], b = Ac[L + r];
        double L4[4];
        if (T.info[p] & PT_NODIFF) {
          L4[0] = L4[1] = L4[2] = L4[3] = 0.0;
        } else {
          L4[0] = -(R1[p] + a.x);
          L4[1] = -(R1[p + cs] + a.y);
          L4[2] = -(R1[p + 2 * cs] + b.x);
          L4[3] = -(R1[p + 3 * cs] + b.y);
        }
        stage_write(sc, p, cs, L4);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- curvilinear patches
// scratch G (component stride Pg): slot 0 = D1e then R1, slot 1 = H_x, slot 2 = H_y, slot 3 = R2
__device__ __forceinline__ double* gslot(double* G, long long Pg, int slot, int c) { return G + (4 * slot + c) * Pg; }
__device__ __forceinline__ const double* gslot(const double* G, long long Pg, int slot, int c) {
  return G + (4 * slot + c) * Pg;
}

// pass A: D1e = d/dq1 e (product-rule form: d/dq1 of (rho, rho u, rho v, theta))
__global__ void LINE_KERNEL_BOUNDS k_gen_A(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                      const double* __restrict__ e, double* __restrict__ G) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    if (T.patches[J.patch].pform)
      load4_theta(A, P.L, J, e, T.P, T.gamma, lane);
    else
      load4(A, P.L, J, e, T.P, lane);
    deriv2(A, Lmax, J, P, T, lane);
    double2* X = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      gslot(G, T.Pg, 0, 0)[g] = X[t].x;
      gslot(G, T.Pg, 0, 1)[g] = X[t].y;
      gslot(G, T.Pg, 0, 2)[g] = X[P.L + t].x;
      gslot(G, T.Pg, 0, 3)[g] = X[P.L + t].y;
    }
    FC_SYNC();
  }
}

// pass B: D2e; grad_x e = J1x D1 + J2x D2, grad_y e = J1y D1 + J2y D2; H_x, H_y;
// R2 = J2x d/dq2 H_x + J2y d/dq2 H_y.
// Product-rule form (adiabatic wall patches, Remark adiabatic): D1, D2 of (rho, rho u,
// rho v, theta); grad e and grad p by the product rules; H = -mu grad e (viscous flux
// only); R2 = div f(e) (from the product rules) + J2x d/dq2 H_x + J2y d/dq2 H_y.
__global__ void LINE_KERNEL_BOUNDS k_gen_B(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                      const double* __restrict__ e, const double* __restrict__ mu,
                                                      const double* __restrict__ Jm, double* __restrict__ G) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P, Pg = T.Pg;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    const bool pf = T.patches[J.patch].pform != 0;
    if (pf)
      load4_theta(A, L, J, e, cs, T.gamma, lane);
    else
      load4(A, L, J, e, cs, lane);
    deriv2(A, Lmax, J, P, T, lane);
    double2* X = A;
    double2* Y = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const long long g = J.gbase + (long long)t * J.stride;
      const double j1x = Jm[g], j1y = Jm[g + Pg], j2x = Jm[g + 2 * Pg], j2y = Jm[g + 3 * Pg];
      const double d2[4] = {X[t].x, X[t].y, X[L + t].x, X[L + t].y};
      const double m = mu[p];
      double hx[4], hy[4];
      if (pf) {
        const double e4[4] = {e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs]};
        const double th = theta_of(e4[0], e4[1], e4[2], e4[3], T.gamma);
        const double Q[4] = {e4[0], e4[1], e4[2], th};
        double qx[4], qy[4], ex[4], ey[4], px, py, div[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double d1 = gslot(G, Pg, 0, c)[g];
          qx[c] = fma(j1x, d1, j2x * d2[c]);
          qy[c] = fma(j1y, d1, j2y * d2[c]);
        }
        product_rule(Q, qx, T.gamma - 1.0, ex, px);
        product_rule(Q, qy, T.gamma - 1.0, ey, py);
        conv_div_product(e4, th, ex, px, ey, py, div);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          hx[c] = -m * ex[c];
          hy[c] = -m * ey[c];
          gslot(G, Pg, 1, c)[g] = hx[c];
          gslot(G, Pg, 2, c)[g] = hy[c];
          gslot(G, Pg, 3, c)[g] = div[c];
        }
      } else {
        double fx[4], fy[4];
        flux_xy(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma, fx, fy);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double d1 = gslot(G, Pg, 0, c)[g];
          const double gx = fma(j1x, d1, j2x * d2[c]);
          const double gy = fma(j1y, d1, j2y * d2[c]);
          hx[c] = fma(-m, gx, fx[c]);
          hy[c] = fma(-m, gy, fy[c]);
          gslot(G, Pg, 1, c)[g] = hx[c];
          gslot(G, Pg, 2, c)[g] = hy[c];
        }
      }
      Y[t] = cpx(hx[0], hx[1]);
      Y[L + t] = cpx(hx[2], hx[3]);
    }
    deriv2(A, Lmax, J, P, T, lane);
    double2* Z = A;
    double2* W = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      const double j2x = Jm[g + 2 * Pg];
      if (pf) {
        double* r = gslot(G, Pg, 3, 0);
        r[g] = fma(j2x, Z[t].x, r[g]);
        r = gslot(G, Pg, 3, 1);
        r[g] = fma(j2x, Z[t].y, r[g]);
        r = gslot(G, Pg, 3, 2);
        r[g] = fma(j2x, Z[L + t].x, r[g]);
        r = gslot(G, Pg, 3, 3);
        r[g] = fma(j2x, Z[L + t].y, r[g]);
      } else {
        gslot(G, Pg, 3, 0)[g] = j2x * Z[t].x;
        gslot(G, Pg, 3, 1)[g] = j2x * Z[t].y;
        gslot(G, Pg, 3, 2)[g] = j2x * Z[L + t].x;
        gslot(G, Pg, 3, 3)[g] = j2x * Z[L + t].y;
      }
      W[t] = cpx(gslot(G, Pg, 2, 0)[g], gslot(G, Pg, 2, 1)[g]);
      W[L + t] = cpx(gslot(G, Pg, 2, 2)[g], gslot(G, Pg, 2, 3)[g]);
    }
    deriv2(A, Lmax, J, P, T, lane);
    double2* V = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      const double j2y = Jm[g + 3 * Pg];
      double* r = gslot(G, Pg, 3, 0);
      r[g] = fma(j2y, V[t].x, r[g]);
      r = gslot(G, Pg, 3, 1);
      r[g] = fma(j2y, V[t].y, r[g]);
      r = gslot(G, Pg, 3, 2);
      r[g] = fma(j2y, V[L + t].x, r[g]);
      r = gslot(G, Pg, 3, 3);
      r[g] = fma(j2y, V[L + t].y, r[g]);
    }
    FC_SYNC();
  }
}

// pass C: R1 = J1x d/dq1 H_x + J1y d/dq1 H_y; L = -(R1 + R2); stage combination
__global__ void LINE_KERNEL_BOUNDS k_gen_C(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                      const double* __restrict__ Jm, double* __restrict__ G,
                                                      StageCoef sc) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P, Pg = T.Pg;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      A[t] = cpx(gslot(G, Pg, 1, 0)[g], gslot(G, Pg, 1, 1)[g]);
      A[L + t] = cpx(gslot(G, Pg, 1, 2)[g], gslot(G, Pg, 1, 3)[g]);
    }
    deriv2(A, Lmax, J, P, T, lane);
    double2* X = A;
    double2* Y = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      const double j1x = Jm[g];
      gslot(G, Pg, 0, 0)[g] = j1x * X[t].x;
      gslot(G, Pg, 0, 1)[g] = j1x * X[t].y;
      gslot(G, Pg, 0, 2)[g] = j1x * X[L + t].x;
      gslot(G, Pg, 0, 3)[g] = j1x * X[L + t].y;
      Y[t] = cpx(gslot(G, Pg, 2, 0)[g], gslot(G, Pg, 2, 1)[g]);
      Y[L + t] = cpx(gslot(G, Pg, 2, 2)[g], gslot(G, Pg, 2, 3)[g]);
    }
    deriv2(A, Lmax, J, P, T, lane);
    double2* Z = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const long long g = J.gbase + (long long)t * J.stride;
      const double j1y = Jm[g + Pg];
      const double d[4] = {Z[t].x, Z[t].y, Z[L + t].x, Z[L + t].y};
      double L4[4];
      const bool nod = (T.info[p] & PT_NODIFF) != 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double r1 = fma(j1y, d[c], gslot(G, Pg, 0, c)[g]);
        L4[c] = nod ? 0.0 : -(r1 + gslot(G, Pg, 3, c)[g]);
      }
      stage_write(sc, p, cs, L4);
    }
    FC_SYNC();
  }
}

// after pass A, at points that only one direction's passes reach (the derivative along
// the other direction is 0 there, as on every point off a long segment):
// mode 1 (no long q1 segment): D1e = 0 before pass B reads it;
// mode 2 (no long q2 segment): H_x, H_y with D2e = 0, which pass C differentiates along q1
__global__ void k_gen_fix(DevTables T, const GFix* __restrict__ f, int n, const double* __restrict__ e,
                          const double* __restrict__ mu, const double* __restrict__ Jm, double* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GFix q = f[i];
  const long long Pg = T.Pg, cs = T.P, g = q.g, p = q.p;
  if (q.mode == 1) {
#pragma unroll
    for (int c = 0; c < 4; ++c) gslot(G, Pg, 0, c)[g] = 0.0;
    return;
  }
  const double m = mu[p], j1x = Jm[g], j1y = Jm[g + Pg];
  if (T.patches[pt_patch(T.info[p])].pform) {
    // product-rule form: the viscous flux alone, grad E from the product rule (the point's
    // own L is 0, so its convective divergence is not needed)
    const double th = theta_of(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma);
    const double Q[4] = {e[p], e[p + cs], e[p + 2 * cs], th};
    double qx[4], qy[4], ex[4], ey[4], px, py;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double d1 = gslot(G, Pg, 0, c)[g];
      qx[c] = fma(j1x, d1, 0.0);
      qy[c] = fma(j1y, d1, 0.0);
    }
    product_rule(Q, qx, T.gamma - 1.0, ex, px);
    product_rule(Q, qy, T.gamma - 1.0, ey, py);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      gslot(G, Pg, 1, c)[g] = -m * ex[c];
      gslot(G, Pg, 2, c)[g] = -m * ey[c];
    }
    return;
  }
  double fx[4], fy[4];
  flux_xy(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma, fx, fy);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double d1 = gslot(G, Pg, 0, c)[g];
    gslot(G, Pg, 1, c)[g] = fma(-m, fma(j1x, d1, 0.0), fx[c]);
    gslot(G, Pg, 2, c)[g] = fma(-m, fma(j1y, d1, 0.0), fy[c]);
  }
}

// FC derivatives of the 4 components of src along each job's line into dst (the
// Jacobian of GRID patches given by their points: src = (x, y, 0, 0))
__global__ void LINE_KERNEL_BOUNDS k_deriv_lines(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                 const double* __restrict__ src, double* __restrict__ dst) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    load4(A, L, J, src, cs, lane);
    deriv2(A, Lmax, J, P, T, lane);
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      dst[p] = A[t].x;
      dst[p + cs] = A[t].y;
      dst[p + 2 * cs] = A[L + t].x;
      dst[p + 3 * cs] = A[L + t].y;
    }
    FC_SYNC();
  }
}

// metrics dq/dx = inverse of [[x_q1, x_q2], [y_q1, y_q2]] (D1 = (x_q1, y_q1), D2 = (x_q2, y_q2),
// component stride P); a singular or non-finite Jacobian is counted in *bad
__global__ void k_grid_metrics(const GFix* __restrict__ pts, int n, const double* __restrict__ D1,
                               const double* __restrict__ D2, long long P, double* __restrict__ Jm, long long Pg,
                               int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = pts[i].p, g = pts[i].g;
  const double xa = D1[p], ya = D1[p + P], xb = D2[p], yb = D2[p + P];
  const double det = __dsub_rn(__dmul_rn(xa, yb), __dmul_rn(xb, ya));
  if (!(fabs(det) > 0.0) || !isfinite(det)) {
    atomicAdd(bad, 1);
    Jm[g] = Jm[g + Pg] = Jm[g + 2 * Pg] = Jm[g + 3 * Pg] = 0.0;
    return;
  }
  Jm[g] = __ddiv_rn(yb, det);
  Jm[g + Pg] = __ddiv_rn(-xb, det);
  Jm[g + 2 * Pg] = __ddiv_rn(-ya, det);
  Jm[g + 3 * Pg] = __ddiv_rn(xa, det);
}

// points no final line pass covers (blanked points, short segments): L = 0
__global__ void k_rk_fixup(DevTables T, const int* __restrict__ idx, int n, StageCoef sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double L4[4] = {0.0, 0.0, 0.0, 0.0};
  stage_write(sc, idx[i], T.P, L4);
}

// ---------------------------------------------------------------- boundary overwrite (Sec. 4.2)
// y fluxes of listed affine points that no q1 line visits (read by the q2 pass)
__global__ void k_flux_y_points(DevTables T, const int* __restrict__ idx, int n, const double* __restrict__ e,
                                double* __restrict__ Fy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = idx[i], cs = T.P;
  double f[4];
  flux_y(e[p], e[p + cs], e[p + 2 * cs], e[p + 3 * cs], T.gamma, f);
#pragma unroll
  for (int c = 0; c < 4; ++c) Fy[p + c * cs] = f[c];
}

__global__ void k_bc(const BcPt* __restrict__ bc, int n, double* __restrict__ e, long long P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BcPt b = bc[i];
  const long long p = b.idx;
  if (b.mode & 1) e[p + P] = 0.0;
  if (b.mode & 2) e[p + 2 * P] = 0.0;
  if (b.mode & 4) {
    const double mx = e[p + P], my = e[p + 2 * P];
    const double mn = mx * b.nx + my * b.ny;
    e[p + P] = mx - mn * b.nx;
    e[p + 2 * P] = my - mn * b.ny;
  }
  if (b.mode & 8) {
#pragma unroll
    for (int c = 0; c < 4; ++c) e[p + c * P] = b.val[c];
  }
}

// no-slip adiabatic wall (Sec. 4.2, Remark adiabatic): zero momenta; the wall temperature
// from the inward temperatures with zero normal derivative; E = rho theta_w / (gamma - 1)
__global__ void k_bc_wall(const WallPt* __restrict__ wp, int n, double* __restrict__ e, long long P, double gam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const WallPt w = wp[i];
  double th = 0.0;
  for (int j = 0; j < w.nw; ++j) {
    const long long q = w.idx + (long long)(j + 1) * w.step;
    const double r = e[q], mx = e[q + P], my = e[q + 2 * P], E = e[q + 3 * P];
    const double tj = (gam - 1.0) * (E - 0.5 * (mx * mx + my * my) / r) / r;
    th = fma(w.w[j], tj, th);
  }
  const long long p = w.idx;
  e[p + P] = 0.0;
  e[p + 2 * P] = 0.0;
  e[p + 3 * P] = e[p] * th / (gam - 1.0);
}

// ---------------------------------------------------------------- inter-patch exchange (Sec. 3.4.1)
// iterated 1-D quadratic interpolation: along q1 in each of the 3 stencil rows, then along q2
// iterated quadratic interpolation of one component from the 3 x 3 donor stencil
__device__ __forceinline__ double interp33(const Recv& R, const double* __restrict__ ec) {
  double acc = 0.0;
#pragma unroll
  for (int m2 = 0; m2 < 3; ++m2) {
    double row = 0.0;
#pragma unroll
    for (int m1 = 0; m1 < 3; ++m1) row = fma(R.w1[m1], ec[R.src[3 * m2 + m1]], row);
    acc = fma(R.w2[m2], row, acc);
  }
  return acc;
}
__global__ void k_exchange(const Recv* __restrict__ r, int n, double* __restrict__ e, long long P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Recv R = r[i];
#pragma unroll
  for (int c = 0; c < 4; ++c) e[R.dst + c * P] = interp33(R, e + c * P);
}
// intra-patch exchange: receivers that coincide with a donor point take its value
__global__ void k_copy_points(const PtCopy* __restrict__ cp, int n, double* __restrict__ e, long long P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const PtCopy c = cp[i];
#pragma unroll
  for (int k = 0; k < 4; ++k) e[c.dst + k * P] = e[c.src + k * P];
}
// sharded exchange: the values a rank owes to others, and their scatter on arrival
__global__ void k_xpack(const Recv* __restrict__ r, int n, const double* __restrict__ e, long long P,
                        double* __restrict__ buf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Recv R = r[i];
#pragma unroll
  for (int c = 0; c < 4; ++c) buf[4 * (long long)i + c] = interp33(R, e + c * P);
}
__global__ void k_xunpack(const int* __restrict__ dst, int n, const double* __restrict__ buf, double* __restrict__ e,
                          long long P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int c = 0; c < 4; ++c) e[dst[i] + c * P] = buf[4 * (long long)i + c];
}
__global__ void k_xgather(const int* __restrict__ dst, int n, const double* __restrict__ e, long long P,
                          double* __restrict__ buf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int c = 0; c < 4; ++c) buf[4 * (long long)i + c] = e[dst[i] + c * P];
}
__global__ void k_gather(const int* __restrict__ idx, int n, const double* __restrict__ src, double* __restrict__ buf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) buf[i] = src[idx[i]];
}
__global__ void k_scatter(const int* __restrict__ idx, int n, const double* __restrict__ buf, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = buf[i];
}

// ---------------------------------------------------------------- per-step filter (Sec. 4.3.1)
__device__ __forceinline__ double energy_of(double r, double mx, double my, double th, double gam) {
  return r * th / (gam - 1.0) + 0.5 * (mx * mx + my * my) / r;
}

__device__ __forceinline__ void filter2(double2* A, int Lmax, const Job& J, const Plan& P, const DevTables& T,
                                        int lane) {
  if (J.fcm >= 0) {
    FC_SYNC();
    continue_lines(A, P.L, J.n, J.C, T.d, T.rp + J.fcm, 2, lane, 32, A + 2 * Lmax);
  }
  FC_SYNC();
  fft_forward_mul<MUL_FILTER>(A, P, 2, T.tw, T.rp, 0.0, lane, 32);
  fft_inplace<true>(A, P, 2, T.tw, T.rp, lane, 32);
}

__global__ void LINE_KERNEL_BOUNDS k_filter_q1(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                          int Lmax, const double* __restrict__ e,
                                                          double* __restrict__ F) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const double r = e[p], mx = e[p + cs], my = e[p + 2 * cs];
      A[t] = cpx(r, mx);
      A[L + t] = cpx(my, theta_of(r, mx, my, e[p + 3 * cs], T.gamma));
    }
    filter2(A, Lmax, J, P, T, lane);
    double2* X = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      F[p] = X[t].x;
      F[p + cs] = X[t].y;
      F[p + 2 * cs] = X[L + t].x;
      F[p + 3 * cs] = X[L + t].y;
    }
    FC_SYNC();
  }
}

__global__ void LINE_KERNEL_BOUNDS k_filter_q2(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                          int Lmax, const double* __restrict__ F,
                                                          double* __restrict__ e) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    load4(A, L, J, F, cs, lane);
    filter2(A, Lmax, J, P, T, lane);
    double2* X = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const double r = X[t].x, mx = X[t].y, my = X[L + t].x, th = X[L + t].y;
      e[p] = r;
      e[p + cs] = mx;
      e[p + 2 * cs] = my;
      e[p + 3 * cs] = energy_of(r, mx, my, th, T.gamma);
    }
    FC_SYNC();
  }
}

__global__ void k_filter_copy_q1(DevTables T, const int* __restrict__ idx, int n, const double* __restrict__ e,
                                 double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = idx[i], cs = T.P;
  const double r = e[p], mx = e[p + cs], my = e[p + 2 * cs];
  F[p] = r;
  F[p + cs] = mx;
  F[p + 2 * cs] = my;
  F[p + 3 * cs] = theta_of(r, mx, my, e[p + 3 * cs], T.gamma);
}

__global__ void k_filter_copy_q2(DevTables T, const int* __restrict__ idx, int n, const double* __restrict__ F,
                                 double* __restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = idx[i], cs = T.P;
  const double r = F[p], mx = F[p + cs], my = F[p + 2 * cs];
  e[p] = r;
  e[p + cs] = mx;
  e[p + 2 * cs] = my;
  e[p + 3 * cs] = energy_of(r, mx, my, F[p + 3 * cs], T.gamma);
}

// ---------------------------------------------------------------- viscosity (Sec. 5)
// Proxy Phi (local Mach number) and MWSB S = |u| + |v| + a, evaluated with explicitly
// rounded operations in a fixed order (no contraction), so the classifier input is
// reproducible.
__global__ void k_visc_point(DevTables T, const double* __restrict__ e, double* __restrict__ phi,
                             double* __restrict__ S) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= T.P) return;
  if (T.info[p] & PT_BLANK) {
    phi[p] = 0.0;
    S[p] = 0.0;
    return;
  }
  const long long cs = T.P;
  const double gam = T.gamma;
  const double rho = e[p];
  const double u = __ddiv_rn(e[p + cs], rho);
  const double v = __ddiv_rn(e[p + 2 * cs], rho);
  const double s2 = __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v));
  const double ke = __dmul_rn(__dmul_rn(0.5, rho), s2);
  const double pr = __dmul_rn(__dsub_rn(gam, 1.0), __dsub_rn(e[p + 3 * cs], ke));
  phi[p] = __dmul_rn(__dsqrt_rn(s2), __dsqrt_rn(__ddiv_rn(rho, __dmul_rn(gam, pr))));
  S[p] = __dadd_rn(__dadd_rn(fabs(u), fabs(v)), __dsqrt_rn(__ddiv_rn(__dmul_rn(gam, pr), rho)));
}

__device__ __forceinline__ int classify7(const double* w, const float* __restrict__ W) {
  double lo = w[0], hi = w[0], am = fabs(w[0]);
#pragma unroll
  for (int k = 1; k < 7; ++k) {
    lo = fmin(lo, w[k]);
    hi = fmax(hi, w[k]);
    am = fmax(am, fabs(w[k]));
  }
  const double rg = __dsub_rn(hi, lo);
  if (rg < __dmul_rn(1e-6, fmax(1.0, am))) return 4;
  float x[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) x[k] = __double2float_rn(__ddiv_rn(__dsub_rn(w[k], lo), rg));
  const float* W1 = W;
  const float* b1 = W1 + SDNN_H * 7;
  const float* W2 = b1 + SDNN_H;
  const float* b2 = W2 + SDNN_H * SDNN_H;
  const float* W3 = b2 + SDNN_H;
  const float* b3 = W3 + 4 * SDNN_H;
  float h1[SDNN_H], h2[SDNN_H];
#pragma unroll
  for (int o = 0; o < SDNN_H; ++o) {
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < 7; ++k) a = fmaf(W1[o * 7 + k], x[k], a);
    h1[o] = fmaxf(a + b1[o], 0.f);
  }
#pragma unroll
  for (int o = 0; o < SDNN_H; ++o) {
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < SDNN_H; ++k) a = fmaf(W2[o * SDNN_H + k], h1[k], a);
    h2[o] = fmaxf(a + b2[o], 0.f);
  }
  int best = 0;
  float bv = -INFINITY;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < SDNN_H; ++k) a = fmaf(W3[o * SDNN_H + k], h2[k], a);
    a += b3[o];
    if (a > bv) {
      bv = a;
      best = o;
    }
  }
  return best + 1;
}

// mu^ = R(tau~) max_{7x7} S h^ on generating points, 0 elsewhere (eq. V2D_unscaled)
__global__ void k_visc_muhat(DevTables T, const double* __restrict__ phi, const double* __restrict__ S,
                             const float* __restrict__ W, const double* __restrict__ Rw, double* __restrict__ muhat,
                             int32_t* __restrict__ tau) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= T.P) return;
  const uint32_t f = T.info[p];
  if (!(f & PT_GEN)) {
    muhat[p] = 0.0;
    if (tau) tau[p] = 0;
    return;
  }
  const PatchDev pd = T.patches[pt_patch(f)];
  const long long loc = p - pd.off;
  const int j = (int)(loc / pd.n1), i = (int)(loc - (long long)j * pd.n1);
  int t1 = 4, t2 = 4;
  double w[7];
  const int o1 = pt_w1(f), o2 = pt_w2(f);
  if (o1 != 7) {
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      int ii = i - o1 + k;
      if (pd.periodic1) ii = (ii + pd.n1) % pd.n1;
      w[k] = phi[pd.off + (long long)j * pd.n1 + ii];
    }
    t1 = classify7(w, W);
  }
  if (o2 != 7) {
#pragma unroll
    for (int k = 0; k < 7; ++k) w[k] = phi[pd.off + (long long)(j - o2 + k) * pd.n1 + i];
    t2 = classify7(w, W);
  }
  const int tc = min(t1, t2);
  // 7x7 maximum of S (clipped to the grid, wrapped along a periodic q1); S >= 0, so the
  // IEEE bit patterns order like the values and the maximum runs on integer compares
  long long mb = 0;
  for (int b = -3; b <= 3; ++b) {
    const int jj = j + b;
    if (jj < 0 || jj >= pd.n2) continue;
    for (int a = -3; a <= 3; ++a) {
      int ii = i + a;
      if (pd.periodic1) {
        ii = (ii + pd.n1) % pd.n1;
      } else if (ii < 0 || ii >= pd.n1) {
        continue;
      }
      const long long bits = __double_as_longlong(S[pd.off + (long long)jj * pd.n1 + ii]);
      mb = bits > mb ? bits : mb;
    }
  }
  muhat[p] = __dmul_rn(__dmul_rn(Rw[tc - 1], __longlong_as_double(mb)), pd.hhat);
  if (tau) tau[p] = tc;
}

// separable window sums of eq. (Lambda): rows (q1) then columns (q2), zero outside, wrapped if periodic
__global__ void k_window_rows(DevTables T, const double* __restrict__ in, double* __restrict__ out,
                              const double* __restrict__ wtab, int r) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= T.P) return;
  const PatchDev pd = T.patches[pt_patch(T.info[p])];
  const long long loc = p - pd.off;
  const int j = (int)(loc / pd.n1), i = (int)(loc - (long long)j * pd.n1);
  const double* row = in + pd.off + (long long)j * pd.n1;
  double acc = 0.0;
  for (int a = -(r - 1); a <= r - 1; ++a) {
    int ii = i + a;
    if (pd.periodic1) {
      ii = (ii + pd.n1) % pd.n1;
    } else if (ii < 0 || ii >= pd.n1) {
      continue;
    }
    acc = fma(wtab[a + r - 1], row[ii], acc);
  }
  out[p] = acc;
}

__global__ void k_window_cols(DevTables T, const double* __restrict__ in, double* __restrict__ out,
                              const double* __restrict__ wtab, int r) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= T.P) return;
  const PatchDev pd = T.patches[pt_patch(T.info[p])];
  const long long loc = p - pd.off;
  const int j = (int)(loc / pd.n1), i = (int)(loc - (long long)j * pd.n1);
  double acc = 0.0;
  for (int b = -(r - 1); b <= r - 1; ++b) {
    const int jj = j + b;
    if (jj < 0 || jj >= pd.n2) continue;
    acc = fma(wtab[b + r - 1], in[pd.off + (long long)jj * pd.n1 + i], acc);
  }
  out[p] = acc;
}

// mu = (own window sum + window sums of the other patches at their nearest points) / normaliser
__global__ void k_mu_own(DevTables T, const double* __restrict__ num, const double* __restrict__ den,
                         double* __restrict__ mu) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= T.P) return;
  const double d = den[p];
  mu[p] = ((T.info[p] & PT_BLANK) || !(d > 0.0)) ? 0.0 : num[p] / d;
}
__global__ void k_mu_cross(const double* __restrict__ num, const double* __restrict__ den, const int* __restrict__ dst,
                           const int* __restrict__ ptr, const int* __restrict__ src, int n, double* __restrict__ mu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = dst[i];
  double s = num[p];
  for (int k = ptr[i]; k < ptr[i + 1]; ++k) s += num[src[k]];
  const double d = den[p];
  mu[p] = d > 0.0 ? s / d : 0.0;
}

// ---------------------------------------------------------------- time step, eq. (CFL)
__global__ void k_dt_reduce(DevTables T, const double* __restrict__ e, const double* __restrict__ mu,
                            unsigned long long* __restrict__ pmax) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int patch = -1;
  unsigned long long bs = 0, bm = 0;
  if (p < T.P) {
    const uint32_t f = T.info[p];
    if (!(f & PT_BLANK) && (!T.owned || T.owned[pt_patch(f)])) {
      patch = pt_patch(f);
      const long long cs = T.P;
      const double gam = T.gamma;
      const double rho = e[p];
      const double u = __ddiv_rn(e[p + cs], rho);
      const double v = __ddiv_rn(e[p + 2 * cs], rho);
      const double s2 = __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v));
      const double pr = __dmul_rn(__dsub_rn(gam, 1.0), __dsub_rn(e[p + 3 * cs], __dmul_rn(__dmul_rn(0.5, rho), s2)));
      const double Sv = __dadd_rn(__dadd_rn(fabs(u), fabs(v)), __dsqrt_rn(__ddiv_rn(__dmul_rn(gam, pr), rho)));
      bs = (unsigned long long)__double_as_longlong(Sv);
      bm = (unsigned long long)__double_as_longlong(mu[p]);
      if (!(Sv >= 0.0)) bs = 0x7FF8000000000000ull;  // NaN: poison the patch maximum
    }
  }
  const unsigned mask = __activemask();
  const int p0 = __shfl_sync(mask, patch, 0);
  if (__all_sync(mask, patch == p0) && p0 >= 0) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long s2 = __shfl_down_sync(mask, bs, o);
      const unsigned long long m2 = __shfl_down_sync(mask, bm, o);
      bs = s2 > bs ? s2 : bs;
      bm = m2 > bm ? m2 : bm;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(pmax + 2 * p0, bs);
      atomicMax(pmax + 2 * p0 + 1, bm);
    }
  } else if (patch >= 0) {
    atomicMax(pmax + 2 * patch, bs);
    atomicMax(pmax + 2 * patch + 1, bm);
  }
}

__global__ void k_dt_final(DevTables T, const unsigned long long* __restrict__ pmax, double cfl, double* dt) {
  __shared__ double red[256];
  double best = INFINITY;
  for (int q = threadIdx.x; q < T.npatch; q += blockDim.x) {
    if (T.owned && !T.owned[q]) continue;
    const double Sm = __longlong_as_double((long long)pmax[2 * q]);
    const double Mm = __longlong_as_double((long long)pmax[2 * q + 1]);
    const double h = T.patches[q].htil;
    const double v = __ddiv_rn(cfl, __dadd_rn(__ddiv_rn(Sm, h), __ddiv_rn(Mm, __dmul_rn(h, h))));
    best = (v < best || v != v) ? v : best;
  }
  red[threadIdx.x] = best;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = red[threadIdx.x + s];
      if (o < red[threadIdx.x] || o != o) red[threadIdx.x] = o;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *dt = __ddiv_rn(red[0], 3.141592653589793);
}

// non-finite / non-physical state detector: raises *flag, never traps
__global__ void k_check_state(DevTables T, const double* __restrict__ e, int* flag) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= T.P) return;
  if (T.info[p] & PT_BLANK) return;
  if (T.owned && !T.owned[pt_patch(T.info[p])]) return;
  const long long cs = T.P;
  const double r = e[p], mx = e[p + cs], my = e[p + 2 * cs], E = e[p + 3 * cs];
  const Prim q = primitives(r, mx, my, E, T.gamma);
  const bool ok = isfinite(r) && isfinite(mx) && isfinite(my) && isfinite(E) && r > 0.0 && q.p > 0.0;
  if (!ok) atomicExch(flag, (int)FC_ERR_NONFINITE);
}

// ---------------------------------------------------------------- discrete adjoint (mu, dt frozen)
// Transposed line operator of the two packed sequences in A (data in [0, n)):
// extend^T o M o zero padding with M = -spectral derivative (the transposed FC
// derivative, FILT false) or the spectral filter (FILT true: real and even in k, so
// symmetric); extend^T folds the C continuation entries back onto the first and last d
// points with ML^T and MR^T.
template <bool FILT>
__device__ __forceinline__ double2* line2T(double2* A, const Job& J, const Plan& P, const DevTables& T, int lane) {
  const int L = P.L, n = J.n, C = J.C, d = T.d;
  for (int idx = lane; idx < 2 * C; idx += 32) {
    const int s = idx / C, k = idx - s * C;
    A[s * L + n + k] = cpx(0.0, 0.0);
  }
  FC_SYNC();
  fft_inplace<false>(A, P, 2, T.tw, T.rp, lane, 32);
  if (FILT)
    mul_filter_slot(A, L, 2, T.rp + P.sigp, lane, 32);
  else
    mul_deriv_slot(A, L, 2, -J.scale * TWO_PI / ((double)L * (double)L), T.rp + P.dmul, lane, 32);
  FC_SYNC();
  fft_inplace<true>(A, P, 2, T.tw, T.rp, lane, 32);
  double2* X = A;
  if (J.fcm >= 0) {
    const double* ML = T.rp + J.fcm;
    const double* MR = ML + C * d;
    double2 acc = cpx(0.0, 0.0);
    int dst = -1;
    if (lane < 4 * d) {  // 2 sequences x (d left + d right) end points
      const int s = lane / (2 * d), q = lane - s * 2 * d;
      const bool left = q < d;
      const int j = left ? q : q - d;
      const double* M = left ? ML : MR;
      const double2* ext = X + s * L + n;
      for (int k = 0; k < C; ++k) {
        const double m = M[k * d + j];
        acc.x = fma(m, ext[k].x, acc.x);
        acc.y = fma(m, ext[k].y, acc.y);
      }
      dst = s * L + (left ? j : n - d + j);
    }
    FC_SYNC();
    if (dst >= 0) X[dst] = cadd(X[dst], acc);
    FC_SYNC();
  }
  return X;
}

// ---- transpose of the product-rule wall form's pointwise map (Remark adiabatic)
// Forward-mode dual number: value and derivative along one input direction.
struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, fma(a.v, b.d, a.d * b.v)}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual inv(Dual a) {
  const double r = 1.0 / a.v;
  return {r, -a.d * r * r};
}

// The pointwise map of the product-rule form at one point: from the state u and the x and
// y derivatives gx, gy of Q = (rho, rho u, rho v, theta) to out = (div f(e), H_x, H_y),
// H = -mu grad e, with grad p = theta grad rho + rho grad theta (eq. p_T) and
// grad E = grad p / (gamma - 1) + u grad(rho u) + v grad(rho v) - (u^2 + v^2) / 2 grad rho
// (eq. perfect_gas_T); written once for the dual numbers of its transpose.
__device__ __forceinline__ void wall_point(const Dual* u, const Dual* gx, const Dual* gy, double mu, double gam,
                                           Dual* out) {
  const Dual ir = inv(u[0]);
  const Dual U = u[1] * ir, V = u[2] * ir;
  const Dual p = (gam - 1.0) * (u[3] - 0.5 * (u[1] * U + u[2] * V));
  const Dual th = p * ir;
  const Dual k = 0.5 * (U * U + V * V);
  Dual e[2][4], pd[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const Dual* g = i ? gy : gx;
    pd[i] = th * g[0] + u[0] * g[3];
    e[i][0] = g[0];
    e[i][1] = g[1];
    e[i][2] = g[2];
    e[i][3] = (1.0 / (gam - 1.0)) * pd[i] + U * g[1] + V * g[2] - k * g[0];
  }
  const Dual ux = (e[0][1] - U * e[0][0]) * ir, vy = (e[1][2] - V * e[1][0]) * ir;
  out[0] = e[0][1] + e[1][2];
  out[1] = U * e[0][1] + u[1] * ux + pd[0] + V * e[1][1] + u[1] * vy;
  out[2] = U * e[0][2] + u[2] * ux + V * e[1][2] + u[2] * vy + pd[1];
  out[3] = (u[3] + p) * (ux + vy) + U * (e[0][3] + pd[0]) + V * (e[1][3] + pd[1]);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    out[4 + c] = (-mu) * e[0][c];
    out[8 + c] = (-mu) * e[1][c];
  }
}

// Transpose of the pointwise map's Jacobian at (u, gx, gy) applied to the output adjoints
// wbar (12): the adjoints of the 12 inputs, one forward-mode evaluation per input.
__device__ __forceinline__ void wall_point_T(const double* u, const double* gx, const double* gy, double mu, double gam,
                                             const double* wbar, double* ubar, double* gxbar, double* gybar) {
#pragma unroll 1
  for (int j = 0; j < 12; ++j) {
    Dual a[4], bx[4], by[4], out[12];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      a[c] = {u[c], j == c ? 1.0 : 0.0};
      bx[c] = {gx[c], j == 4 + c ? 1.0 : 0.0};
      by[c] = {gy[c], j == 8 + c ? 1.0 : 0.0};
    }
    wall_point(a, bx, by, mu, gam, out);
    double s = 0.0;
#pragma unroll
    for (int o = 0; o < 12; ++o) s = fma(wbar[o], out[o].d, s);
    if (j < 4)
      ubar[j] = s;
    else if (j < 8)
      gxbar[j - 4] = s;
    else
      gybar[j - 8] = s;
  }
}

// adjoint pass B of the product-rule form at one point: in: D_2 Q at *a, *b (packed), D_1 Q in slot 3, eta in slots 0
// and 1; out: partial = ubar (slot 2), g1 = -(J1x gxbar + J1y gybar) (slot 3) and
// g2 = -(J2x gxbar + J2y gybar) packed into *a, *b for its q2 transpose
__device__ __forceinline__ void adj_wall_point_B(const DevTables& T, long long p, long long g, const double* Jm,
                                              const double* u, const double* mu, const double* psi, double* G,
                                              double2* a, double2* b) {
  const long long cs = T.P, Pg = T.Pg;
  const double j1x = Jm[g], j1y = Jm[g + Pg], j2x = Jm[g + 2 * Pg], j2y = Jm[g + 3 * Pg];
  const double d2[4] = {a->x, a->y, b->x, b->y};
  const bool nod = (T.info[p] & PT_NODIFF) != 0;
  double u4[4], gx[4], gy[4], wbar[12], ub[4], gxb[4], gyb[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double d1 = gslot(G, Pg, 3, c)[g];
    u4[c] = u[p + c * cs];
    gx[c] = fma(j1x, d1, j2x * d2[c]);
    gy[c] = fma(j1y, d1, j2y * d2[c]);
    wbar[c] = nod ? 0.0 : -psi[p + c * cs];
    wbar[4 + c] = gslot(G, Pg, 0, c)[g];
    wbar[8 + c] = gslot(G, Pg, 1, c)[g];
  }
  wall_point_T(u4, gx, gy, mu[p], T.gamma, wbar, ub, gxb, gyb);
  double g2[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    gslot(G, Pg, 2, c)[g] = ub[c];
    gslot(G, Pg, 3, c)[g] = -fma(j1x, gxb[c], j1y * gyb[c]);
    g2[c] = -fma(j2x, gxb[c], j2y * gyb[c]);
  }
  *a = cpx(g2[0], g2[1]);
  *b = cpx(g2[2], g2[3]);
}

// (dQ/du)^T a for Q = (rho, rho u, rho v, theta), theta = (gamma - 1) (E / rho - |rho u|^2 / (2 rho^2))
__device__ __forceinline__ void thetaT_add(const double* u, double gam, const double* a, double* out) {
  const double ir = 1.0 / u[0], g1 = gam - 1.0;
  const double m2 = fma(u[1], u[1], u[2] * u[2]);
  out[0] += a[0] + a[3] * g1 * ir * ir * (m2 * ir - u[3]);
  out[1] += a[1] - a[3] * g1 * u[1] * ir * ir;
  out[2] += a[2] - a[3] * g1 * u[2] * ir * ir;
  out[3] += a[3] * g1 * ir;
}

// A^T eta for the x (dir 0) or y (dir 1) flux Jacobian at state e (eq. euler 2d equation)
__device__ __forceinline__ void fluxT(int dir, double r, double mx, double my, double E, double gam, const double* eta,
                                      double* out) {
  const double ir = 1.0 / r;
  const double u = mx * ir, v = my * ir;
  const double g1 = gam - 1.0;
  const double q2 = u * u + v * v;
  const double p = g1 * (E - 0.5 * r * q2);
  const double H = (E + p) * ir;
  const double pr = 0.5 * g1 * q2, pm = -g1 * u, pn = -g1 * v, pE = g1;
  if (dir == 0) {
    // rows c = 0..3 of A_x, columns j: out_j = sum_c A[c][j] eta_c
    out[0] = (-u * u + pr) * eta[1] + (-u * v) * eta[2] + (-u * H + u * pr) * eta[3];
    out[1] = eta[0] + (2.0 * u + pm) * eta[1] + v * eta[2] + (H + u * pm) * eta[3];
    out[2] = pn * eta[1] + u * eta[2] + u * pn * eta[3];
    out[3] = pE * eta[1] + u * (1.0 + pE) * eta[3];
  } else {
    out[0] = (-u * v) * eta[1] + (-v * v + pr) * eta[2] + (-v * H + v * pr) * eta[3];
    out[1] = v * eta[1] + pm * eta[2] + v * pm * eta[3];
    out[2] = eta[0] + u * eta[1] + (2.0 * v + pn) * eta[2] + (H + v * pn) * eta[3];
    out[3] = pE * eta[2] + v * (1.0 + pE) * eta[3];
  }
}

__device__ __forceinline__ void load4_masked(double2* A, int L, const Job& J, const DevTables& T,
                                             const double* __restrict__ src, int lane) {
  const long long cs = T.P;
  for (int t = lane; t < J.n; t += 32) {
    const long long p = J.base + (long long)t * J.stride;
    if (T.info[p] & PT_NODIFF) {
      A[t] = cpx(0.0, 0.0);
      A[L + t] = cpx(0.0, 0.0);
    } else {
      A[t] = cpx(src[p], src[p + cs]);
      A[L + t] = cpx(src[p + 2 * cs], src[p + 3 * cs]);
    }
  }
}

// affine patches, pass 1 (q1 lines): R1 = A_x^T eta_x - D_x^T(mu eta_x), eta_x = -D_x^T (N psi)
// pass 2 (q2 lines): acc += dt (R1 + A_y^T eta_y - D_y^T(mu eta_y))
__global__ void LINE_KERNEL_BOUNDS k_adj_cart(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                         int Lmax, int dir, const double* __restrict__ u,
                                                         const double* __restrict__ mu, const double* __restrict__ psi,
                                                         double* __restrict__ R1, double* __restrict__ acc,
                                                         const double* __restrict__ dtp) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    load4_masked(A, L, J, T, psi, lane);
    double2* X = line2T<false>(A, J, P, T, lane);
    double2* Y = A;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const double eta[4] = {-X[t].x, -X[t].y, -X[L + t].x, -X[L + t].y};
      double r[4];
      fluxT(dir, u[p], u[p + cs], u[p + 2 * cs], u[p + 3 * cs], T.gamma, eta, r);
      const double m = mu[p];
      if (dir == 0) {
        R1[p] = r[0];
        R1[p + cs] = r[1];
        R1[p + 2 * cs] = r[2];
        R1[p + 3 * cs] = r[3];
      } else {
        // R1 + A_y^T eta_y so far, kept in the stage buffer until the last transform
        R1[p] += r[0];
        R1[p + cs] += r[1];
        R1[p + 2 * cs] += r[2];
        R1[p + 3 * cs] += r[3];
      }
      Y[t] = cpx(m * eta[0], m * eta[1]);
      Y[L + t] = cpx(m * eta[2], m * eta[3]);
    }
    double2* Z = line2T<false>(A, J, P, T, lane);
    const double dt = dir ? *dtp : 0.0;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const double z[4] = {Z[t].x, Z[t].y, Z[L + t].x, Z[L + t].y};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double v = R1[p + c * cs] - z[c];
        if (dir == 0)
          R1[p + c * cs] = v;
        else
          acc[p + c * cs] = fma(dt, v, acc[p + c * cs]);
      }
    }
    FC_SYNC();
  }
}

// curvilinear patches. scratch G slots: 0 = S1x then eta_x, 1 = S1y, 2 = partial, 3 = g1
// (product-rule wall form: 3 = D_1 Q, the forward q1 derivative of Q = (rho, rho u, rho v,
// theta) at the stage state, until pass B replaces it by g1)
// pass A (q1): S1x = D_1^T(J1x N psi), S1y = D_1^T(J1y N psi)
__global__ void LINE_KERNEL_BOUNDS k_adj_gen_A(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                          int Lmax, const double* __restrict__ Jm,
                                                          const double* __restrict__ u,
                                                          const double* __restrict__ psi, double* __restrict__ G) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P, Pg = T.Pg;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    for (int which = 0; which < 2; ++which) {
      for (int t = lane; t < J.n; t += 32) {
        const long long p = J.base + (long long)t * J.stride;
        const long long g = J.gbase + (long long)t * J.stride;
        const double w = (T.info[p] & PT_NODIFF) ? 0.0 : Jm[g + which * Pg];
        A[t] = cpx(w * psi[p], w * psi[p + cs]);
        A[L + t] = cpx(w * psi[p + 2 * cs], w * psi[p + 3 * cs]);
      }
      double2* X = line2T<false>(A, J, P, T, lane);
      for (int t = lane; t < J.n; t += 32) {
        const long long g = J.gbase + (long long)t * J.stride;
        gslot(G, Pg, which, 0)[g] = X[t].x;
        gslot(G, Pg, which, 1)[g] = X[t].y;
        gslot(G, Pg, which, 2)[g] = X[L + t].x;
        gslot(G, Pg, which, 3)[g] = X[L + t].y;
      }
      FC_SYNC();
    }
    if (T.patches[J.patch].pform) {
      load4_theta(A, L, J, u, cs, T.gamma, lane);
      deriv2(A, Lmax, J, P, T, lane);
      for (int t = lane; t < J.n; t += 32) {
        const long long g = J.gbase + (long long)t * J.stride;
        gslot(G, Pg, 3, 0)[g] = A[t].x;
        gslot(G, Pg, 3, 1)[g] = A[t].y;
        gslot(G, Pg, 3, 2)[g] = A[L + t].x;
        gslot(G, Pg, 3, 3)[g] = A[L + t].y;
      }
      FC_SYNC();
    }
  }
}

// pass B (q2): eta_x = -(S1x + D_2^T(J2x N psi)), eta_y = -(S1y + D_2^T(J2y N psi));
// partial = A_x^T eta_x + A_y^T eta_y - D_2^T(mu (J2x eta_x + J2y eta_y)); g1 = mu (J1x eta_x + J1y eta_y)
// adjoint pass B, first part (q2 lines): eta_x = -(S1x + D_2^T(J2x N psi)),
// eta_y = -(S1y + D_2^T(J2y N psi)) into slots 0 and 1
__device__ __forceinline__ void adj_eta_q2(double2* A, int L, const Job& J, const Plan& P, const DevTables& T,
                                           const double* __restrict__ Jm, const double* __restrict__ psi,
                                           double* __restrict__ G, int lane) {
  const long long cs = T.P, Pg = T.Pg;
  for (int which = 0; which < 2; ++which) {
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const long long g = J.gbase + (long long)t * J.stride;
      const double w = (T.info[p] & PT_NODIFF) ? 0.0 : Jm[g + (2 + which) * Pg];
      A[t] = cpx(w * psi[p], w * psi[p + cs]);
      A[L + t] = cpx(w * psi[p + 2 * cs], w * psi[p + 3 * cs]);
    }
    double2* X = line2T<false>(A, J, P, T, lane);
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      const double x[4] = {X[t].x, X[t].y, X[L + t].x, X[L + t].y};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double* s = gslot(G, Pg, which, c);
        s[g] = -(s[g] + x[c]);  // eta_x (which 0) or eta_y (which 1)
      }
    }
    FC_SYNC();
  }
}

__global__ void LINE_KERNEL_BOUNDS k_adj_gen_B(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                          int Lmax, const double* __restrict__ Jm,
                                                          const double* __restrict__ u, const double* __restrict__ mu,
                                                          const double* __restrict__ psi, double* __restrict__ G) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P, Pg = T.Pg;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    if (T.patches[J.patch].pform) continue;  // k_adj_gen_B_wall
    adj_eta_q2(A, L, J, P, T, Jm, psi, G, lane);
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const long long g = J.gbase + (long long)t * J.stride;
      double ex[4], ey[4], ax[4], ay[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        ex[c] = gslot(G, Pg, 0, c)[g];
        ey[c] = gslot(G, Pg, 1, c)[g];
      }
      fluxT(0, u[p], u[p + cs], u[p + 2 * cs], u[p + 3 * cs], T.gamma, ex, ax);
      fluxT(1, u[p], u[p + cs], u[p + 2 * cs], u[p + 3 * cs], T.gamma, ey, ay);
      const double m = mu[p];
      const double j1x = Jm[g], j1y = Jm[g + Pg], j2x = Jm[g + 2 * Pg], j2y = Jm[g + 3 * Pg];
      double g2[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        gslot(G, Pg, 2, c)[g] = ax[c] + ay[c];
        gslot(G, Pg, 3, c)[g] = m * fma(j1x, ex[c], j1y * ey[c]);
        g2[c] = m * fma(j2x, ex[c], j2y * ey[c]);
      }
      A[t] = cpx(g2[0], g2[1]);
      A[L + t] = cpx(g2[2], g2[3]);
    }
    double2* Z = line2T<false>(A, J, P, T, lane);
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      const double z[4] = {Z[t].x, Z[t].y, Z[L + t].x, Z[L + t].y};
#pragma unroll
      for (int c = 0; c < 4; ++c) gslot(G, Pg, 2, c)[g] -= z[c];
    }
    FC_SYNC();
  }
}

// adjoint pass B of the product-rule wall form (Remark adiabatic; its jobs only): eta as in
// k_adj_gen_B, then the pointwise map's transpose at the forward derivatives of Q
// (partial = ubar, g1 = -(J1x gxbar + J1y gybar), g2 = -(J2x gxbar + J2y gybar)) and
// partial -= (dQ/du)^T D_2^T(g2)
__global__ void LINE_KERNEL_BOUNDS k_adj_gen_B_wall(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                               int Lmax, const double* __restrict__ Jm,
                                                               const double* __restrict__ u,
                                                               const double* __restrict__ mu,
                                                               const double* __restrict__ psi,
                                                               double* __restrict__ G) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P, Pg = T.Pg;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    if (!T.patches[J.patch].pform) continue;
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    adj_eta_q2(A, L, J, P, T, Jm, psi, G, lane);
    // product-rule wall form: the pointwise map's transpose at the forward derivatives
    // of Q; partial = ubar, g1 = -(J1x gxbar + J1y gybar), g2 = -(J2x gxbar + J2y gybar)
    load4_theta(A, L, J, u, cs, T.gamma, lane);
    deriv2(A, Lmax, J, P, T, lane);
    for (int t = lane; t < J.n; t += 32)
      adj_wall_point_B(T, J.base + (long long)t * J.stride, J.gbase + (long long)t * J.stride, Jm, u, mu, psi, G,
                       A + t, A + L + t);
    double2* Z = line2T<false>(A, J, P, T, lane);
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const long long g = J.gbase + (long long)t * J.stride;
      const double z[4] = {-Z[t].x, -Z[t].y, -Z[L + t].x, -Z[L + t].y};
      const double u4[4] = {u[p], u[p + cs], u[p + 2 * cs], u[p + 3 * cs]};
      double part[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) part[c] = gslot(G, Pg, 2, c)[g];
      thetaT_add(u4, T.gamma, z, part);
#pragma unroll
      for (int c = 0; c < 4; ++c) gslot(G, Pg, 2, c)[g] = part[c];
    }
    FC_SYNC();
  }
}

// pass C (q1): acc += dt (partial - D_1^T(g1))
// (product-rule wall form: acc += dt (partial - (dQ/du)^T D_1^T(g1)))
__global__ void LINE_KERNEL_BOUNDS k_adj_gen_C(DevTables T, const Job* __restrict__ jobs, int njobs,
                                                          int Lmax, const double* __restrict__ u,
                                                          const double* __restrict__ G,
                                                          double* __restrict__ acc, const double* __restrict__ dtp) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P, Pg = T.Pg;
  const double dt = *dtp;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    for (int t = lane; t < J.n; t += 32) {
      const long long g = J.gbase + (long long)t * J.stride;
      A[t] = cpx(gslot(G, Pg, 3, 0)[g], gslot(G, Pg, 3, 1)[g]);
      A[L + t] = cpx(gslot(G, Pg, 3, 2)[g], gslot(G, Pg, 3, 3)[g]);
    }
    double2* X = line2T<false>(A, J, P, T, lane);
    const bool pf = T.patches[J.patch].pform != 0;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const long long g = J.gbase + (long long)t * J.stride;
      double x[4] = {X[t].x, X[t].y, X[L + t].x, X[L + t].y};
      if (pf) {
        const double u4[4] = {u[p], u[p + cs], u[p + 2 * cs], u[p + 3 * cs]};
        double y[4] = {0.0, 0.0, 0.0, 0.0};
        thetaT_add(u4, T.gamma, x, y);
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = y[c];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[p + c * cs] = fma(dt, gslot(G, Pg, 2, c)[g] - x[c], acc[p + c * cs]);
    }
    FC_SYNC();
  }
}

// transposes of k_gen_fix, after adjoint pass A:
// mode 1 (no long q1 segment): S1x = S1y = 0 before pass B completes eta there;
// mode 2 (no long q2 segment): eta = -S1, partial = A_x^T eta_x + A_y^T eta_y and
// g1 = mu (J1x eta_x + J1y eta_y), which pass C finishes along q1
__global__ void k_adj_gen_fixA(DevTables T, const GFix* __restrict__ f, int n, const double* __restrict__ Jm,
                               const double* __restrict__ u, const double* __restrict__ mu,
                               const double* __restrict__ psi, double* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GFix q = f[i];
  const long long Pg = T.Pg, cs = T.P, g = q.g, p = q.p;
  const bool pf = T.patches[pt_patch(T.info[p])].pform != 0;
  if (q.mode == 1) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      gslot(G, Pg, 0, c)[g] = 0.0;
      gslot(G, Pg, 1, c)[g] = 0.0;
      if (pf) gslot(G, Pg, 3, c)[g] = 0.0;  // D_1 Q = 0 off the long q1 segments
    }
    return;
  }
  if (pf) {  // product-rule wall form with D_2 Q = 0
    const double j1x = Jm[g], j1y = Jm[g + Pg];
    const bool nod = (T.info[p] & PT_NODIFF) != 0;
    double u4[4], gx[4], gy[4], wbar[12], ub[4], gxb[4], gyb[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double d1 = gslot(G, Pg, 3, c)[g];
      u4[c] = u[p + c * cs];
      gx[c] = fma(j1x, d1, 0.0);
      gy[c] = fma(j1y, d1, 0.0);
      wbar[c] = nod ? 0.0 : -psi[p + c * cs];
      wbar[4 + c] = -gslot(G, Pg, 0, c)[g];
      wbar[8 + c] = -gslot(G, Pg, 1, c)[g];
      gslot(G, Pg, 0, c)[g] = wbar[4 + c];
      gslot(G, Pg, 1, c)[g] = wbar[8 + c];
    }
    wall_point_T(u4, gx, gy, mu[p], T.gamma, wbar, ub, gxb, gyb);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      gslot(G, Pg, 2, c)[g] = ub[c];
      gslot(G, Pg, 3, c)[g] = -fma(j1x, gxb[c], j1y * gyb[c]);
    }
    return;
  }
  double ex[4], ey[4], ax[4], ay[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    ex[c] = -gslot(G, Pg, 0, c)[g];
    ey[c] = -gslot(G, Pg, 1, c)[g];
    gslot(G, Pg, 0, c)[g] = ex[c];
    gslot(G, Pg, 1, c)[g] = ey[c];
  }
  fluxT(0, u[p], u[p + cs], u[p + 2 * cs], u[p + 3 * cs], T.gamma, ex, ax);
  fluxT(1, u[p], u[p + cs], u[p + 2 * cs], u[p + 3 * cs], T.gamma, ey, ay);
  const double m = mu[p], j1x = Jm[g], j1y = Jm[g + Pg];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    gslot(G, Pg, 2, c)[g] = ax[c] + ay[c];
    gslot(G, Pg, 3, c)[g] = m * fma(j1x, ex[c], j1y * ey[c]);
  }
}

// after adjoint pass B, mode 1: no pass C finishes the point, so its partial goes to R1
// (zeroed at the start of the stage), which the fixup adds to acc
__global__ void k_adj_gen_fixB(DevTables T, const GFix* __restrict__ f, int n, const double* __restrict__ G,
                               double* __restrict__ R1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GFix q = f[i];
  if (q.mode != 1) return;
  const long long Pg = T.Pg, cs = T.P;
#pragma unroll
  for (int c = 0; c < 4; ++c) R1[q.p + c * cs] = gslot(G, Pg, 2, c)[q.g];
}

// points no column pass finishes: acc += dt R1 (R1 is zero where no row pass wrote it)
__global__ void k_adj_fixup(const int* __restrict__ idx, int n, const double* __restrict__ R1, double* __restrict__ acc,
                            long long P, const double* __restrict__ dtp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dt = *dtp;
  const long long p = idx[i];
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[p + c * P] = fma(dt, R1[p + c * P], acc[p + c * P]);
}

// exchange transpose: every donor gathers w * adjoint of the receivers it feeds (CSR by donor),
// then the receivers are zeroed (they do not depend on their own previous value)
__global__ void k_exchange_T(const int* __restrict__ dptr, const int* __restrict__ dsrc, const int* __restrict__ drecv,
                             const double* __restrict__ dw, int nd, double* __restrict__ lam, long long P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const long long s = dsrc[i];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double a = lam[s + c * P];
    for (int k = dptr[i]; k < dptr[i + 1]; ++k) a = fma(dw[k], lam[drecv[k] + c * P], a);
    lam[s + c * P] = a;
  }
}
__global__ void k_zero_points(const Recv* __restrict__ r, int n, double* __restrict__ lam, long long P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = r[i].dst;
#pragma unroll
  for (int c = 0; c < 4; ++c) lam[p + c * P] = 0.0;
}
// boundary transpose: Dirichlet points hand their adjoint to gbc and are zeroed; slip walls
// zero (affine) or project out (curvilinear) the wall-normal momentum adjoint
// (acc: the free-stream points' adjoint dotted with d e_fs / d(M, alpha), per record, in call order)
__global__ void k_bc_T(const BcPt* __restrict__ bc, int n, double* __restrict__ lam, double* __restrict__ gbc,
                       double* __restrict__ acc, FsJac fj, long long P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BcPt b = bc[i];
  const long long p = b.idx;
  if (b.mode & 8) {
    double sm = 0.0, sa = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double l = lam[p + c * P];
      if (gbc) gbc[p + c * P] += l;
      sm = fma(l, fj.dM[c], sm);
      sa = fma(l, fj.dA[c], sa);
      lam[p + c * P] = 0.0;
    }
    if (acc && (b.mode & 16)) {
      acc[2 * i] += sm;
      acc[2 * i + 1] += sa;
    }
    return;
  }
  if (b.mode & 1) lam[p + P] = 0.0;
  if (b.mode & 2) lam[p + 2 * P] = 0.0;
  if (b.mode & 4) {
    const double mx = lam[p + P], my = lam[p + 2 * P];
    const double mn = mx * b.nx + my * b.ny;
    lam[p + P] = mx - mn * b.nx;
    lam[p + 2 * P] = my - mn * b.ny;
  }
}
// out[0..1] += the pair sums of acc over n records, in a fixed order (one block of 512
// threads: strided partial sums, then a fixed tree); acc is zeroed for the next step
__global__ void __launch_bounds__(512) k_pair_reduce(double* __restrict__ acc, int n, double* __restrict__ out) {
  __shared__ double s0[512], s1[512];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = t; i < n; i += 512) {
    a += acc[2 * i];
    b += acc[2 * i + 1];
    acc[2 * i] = 0.0;
    acc[2 * i + 1] = 0.0;
  }
  s0[t] = a;
  s1[t] = b;
  __syncthreads();
  for (int h = 256; h > 0; h >>= 1) {
    if (t < h) {
      s0[t] += s0[t + h];
      s1[t] += s1[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    out[0] += s0[0];
    out[1] += s1[0];
  }
}
// sensitivities to the initial data: drho = lam . d e / d rho at fixed u, v, p
// (lam_rho + lam_mx u + lam_my v + lam_E |u|^2 / 2), and per-block sums of lam . (dM, dA)
// over non-blanked points (grid-stride in a fixed order, fixed tree per block)
__global__ void __launch_bounds__(256) k_init_sens(const uint32_t* __restrict__ info,
                                                   const uint8_t* __restrict__ owned, long long P,
                                                   const double* __restrict__ e, const double* __restrict__ lam,
                                                   double* __restrict__ drho, double* __restrict__ part, FsJac fj) {
  __shared__ double s0[256], s1[256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (long long p = (long long)blockIdx.x * 256 + t; p < P; p += (long long)gridDim.x * 256) {
    const bool blank = (info[p] & PT_BLANK) != 0 || (owned && !owned[pt_patch(info[p])]);
    const double l0 = lam[p], l1 = lam[p + P], l2 = lam[p + 2 * P], l3 = lam[p + 3 * P];
    if (drho) {
      double r = 0.0;
      if (!blank) {
        const double rho = e[p], u = e[p + P] / rho, v = e[p + 2 * P] / rho;
        r = l0 + l1 * u + l2 * v + l3 * (0.5 * (u * u + v * v));
      }
      drho[p] = r;
    }
    if (!blank) {
      a += l0 * fj.dM[0] + l1 * fj.dM[1] + l2 * fj.dM[2] + l3 * fj.dM[3];
      b += l0 * fj.dA[0] + l1 * fj.dA[1] + l2 * fj.dA[2] + l3 * fj.dA[3];
    }
  }
  if (!part) return;
  s0[t] = a;
  s1[t] = b;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (t < h) {
      s0[t] += s0[t + h];
      s1[t] += s1[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    part[2 * blockIdx.x] = s0[0];
    part[2 * blockIdx.x + 1] = s1[0];
  }
}
// ---- transpose of the linearised per-step filter (Sec. 4.3.1) -----------------------------
// forward: Q = (rho, rho u, rho v, theta(e)) filtered along q1 lines (into F), then along q2
// lines, and E rebuilt from the filtered Q (eq. perfect_gas_T)
__device__ __forceinline__ void rebuild_T(const double* __restrict__ lam, const double* __restrict__ ef, long long p,
                                          long long cs, double gam, double* o) {
  const double r = ef[p], m = ef[p + cs], nn = ef[p + 2 * cs];
  const double th = theta_of(r, m, nn, ef[p + 3 * cs], gam);
  const double g1 = gam - 1.0, lE = lam[p + 3 * cs], ir = 1.0 / r;
  o[0] = lam[p] + lE * (th / g1 - 0.5 * (m * m + nn * nn) * ir * ir);
  o[1] = lam[p + cs] + lE * m * ir;
  o[2] = lam[p + 2 * cs] + lE * nn * ir;
  o[3] = lE * r / g1;
}
__device__ __forceinline__ void theta_T(const double* q, const double* __restrict__ e, long long p, long long cs,
                                        double gam, double* o) {
  const double r = e[p], m = e[p + cs], nn = e[p + 2 * cs], E = e[p + 3 * cs];
  const double g1 = gam - 1.0, lt = q[3], ir = 1.0 / r, ir2 = ir * ir;
  o[0] = q[0] + lt * g1 * (-E * ir2 + (m * m + nn * nn) * ir2 * ir);
  o[1] = q[1] + lt * (-g1 * m * ir2);
  o[2] = q[2] + lt * (-g1 * nn * ir2);
  o[3] = lt * g1 * ir;
}

// q2 lines: lam (adjoint of the filtered state), ef (the filter output) -> MF
__global__ void LINE_KERNEL_BOUNDS k_filterT_q2(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                const double* __restrict__ lam, const double* __restrict__ ef,
                                                double* __restrict__ MF) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      double o[4];
      rebuild_T(lam, ef, p, cs, T.gamma, o);
      A[t] = cpx(o[0], o[1]);
      A[L + t] = cpx(o[2], o[3]);
    }
    FC_SYNC();
    double2* X = line2T<true>(A, J, P, T, lane);
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      MF[p] = X[t].x;
      MF[p + cs] = X[t].y;
      MF[p + 2 * cs] = X[L + t].x;
      MF[p + 3 * cs] = X[L + t].y;
    }
    FC_SYNC();
  }
}
// q1 lines: MF, e (the state the filter was applied to) -> out (adjoint of that state)
__global__ void LINE_KERNEL_BOUNDS k_filterT_q1(DevTables T, const Job* __restrict__ jobs, int njobs, int Lmax,
                                                const double* __restrict__ MF, const double* __restrict__ e,
                                                double* __restrict__ out) {
  extern __shared__ double2 sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double2* A = sm + warp * (2 * Lmax + CONT_TMP);
  const long long cs = T.P;
  for (int ji = blockIdx.x * nw + warp; ji < njobs; ji += gridDim.x * nw) {
    const Job J = jobs[ji];
    const Plan P = T.plans[J.plan];
    const int L = P.L;
    load4(A, L, J, MF, cs, lane);
    FC_SYNC();
    double2* X = line2T<true>(A, J, P, T, lane);
    for (int t = lane; t < J.n; t += 32) {
      const long long p = J.base + (long long)t * J.stride;
      const double q[4] = {X[t].x, X[t].y, X[L + t].x, X[L + t].y};
      double o[4];
      theta_T(q, e, p, cs, T.gamma, o);
      out[p] = o[0];
      out[p + cs] = o[1];
      out[p + 2 * cs] = o[2];
      out[p + 3 * cs] = o[3];
    }
    FC_SYNC();
  }
}
// points that no filtered line covers (identity filter there)
__global__ void k_filterT_copy2(DevTables T, const int* __restrict__ idx, int n, const double* __restrict__ lam,
                                const double* __restrict__ ef, double* __restrict__ MF) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = idx[i], cs = T.P;
  double o[4];
  rebuild_T(lam, ef, p, cs, T.gamma, o);
  for (int c = 0; c < 4; ++c) MF[p + c * cs] = o[c];
}
__global__ void k_filterT_copy1(DevTables T, const int* __restrict__ idx, int n, const double* __restrict__ MF,
                                const double* __restrict__ e, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long p = idx[i], cs = T.P;
  const double q[4] = {MF[p], MF[p + cs], MF[p + 2 * cs], MF[p + 3 * cs]};
  double o[4];
  theta_T(q, e, p, cs, T.gamma, o);
  for (int c = 0; c < 4; ++c) out[p + c * cs] = o[c];
}

// transpose of the linearised adiabatic wall condition at the state u it was applied to
// (u's wall density and inward points are unchanged by it): the wall momenta and energy
// adjoints are cleared and lam_E,w is passed to rho_w and, through theta, to the inward points
__global__ void k_bc_wall_T(const WallPt* __restrict__ wp, int n, const double* __restrict__ u,
                            double* __restrict__ lam, long long P, double gam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const WallPt w = wp[i];
  const long long p = w.idx;
  const double g1 = gam - 1.0;
  const double lE = lam[p + 3 * P];
  const double rw = u[p];
  double th = 0.0;
  for (int j = 0; j < w.nw; ++j) {
    const long long q = w.idx + (long long)(j + 1) * w.step;
    const double r = u[q], mx = u[q + P], my = u[q + 2 * P], E = u[q + 3 * P];
    th = fma(w.w[j], g1 * (E - 0.5 * (mx * mx + my * my) / r) / r, th);
    const double g = lE * rw / g1 * w.w[j];
    const double ir = 1.0 / r, ir2 = ir * ir;
    atomicAdd(lam + q, g * g1 * (-E * ir2 + (mx * mx + my * my) * ir2 * ir));
    atomicAdd(lam + q + P, g * (-g1 * mx * ir2));
    atomicAdd(lam + q + 2 * P, g * (-g1 * my * ir2));
    atomicAdd(lam + q + 3 * P, g * (g1 * ir));
  }
  lam[p + P] = 0.0;
  lam[p + 2 * P] = 0.0;
  lam[p + 3 * P] = 0.0;
  atomicAdd(lam + p, lE * th / g1);
}

// y = a x + b y over n doubles (b == 0: y = a x)
__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

// ---------------------------------------------------------------- wall drag functional
// J = sum_i w_i n_x,i p_i over the wall ring (periodic trapezoid of the wall-pressure integral);
// dJde (optional): its gradient at the wall points, zero elsewhere (caller zeroes it)
__global__ void k_drag(const int* __restrict__ wall, const double* __restrict__ w, const double* __restrict__ nx, int n,
                       const double* __restrict__ e, long long P, double gam, double* J, double* dJde) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const long long p = wall[i];
    const double r = e[p], mx = e[p + P], my = e[p + 2 * P], E = e[p + 3 * P];
    const double u = mx / r, v = my / r;
    const double g1 = gam - 1.0;
    const double pr = g1 * (E - 0.5 * r * (u * u + v * v));
    const double wn = w[i] * nx[i];
    acc += wn * pr;
    if (dJde) {
      dJde[p] = wn * 0.5 * g1 * (u * u + v * v);
      dJde[p + P] = -wn * g1 * u;
      dJde[p + 2 * P] = -wn * g1 * v;
      dJde[p + 3 * P] = wn * g1;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = red[0];
}

// ---------------------------------------------------------------- launch wrappers
static inline int grid_lines(const DevTables& T, int njobs, int Lmax) {
  const int w = line_warps(T, Lmax);
  int g = (njobs + w - 1) / w;
  return g < 1 ? 1 : g;
}
#define LINE_CFG(njobs, Lmax) grid_lines(T, njobs, Lmax), line_warps(T, Lmax) * 32, line_smem_bytes(T, Lmax), st
static inline unsigned grid_pts(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_cart_q1(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, const double* mu,
                    double* R1, double* Fy, cudaStream_t st) {
  if (njobs <= 0) return;
  k_cart_q1<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, e, mu, R1, Fy);
}
void launch_cart_q2(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* mu, const double* R1,
                    const double* Fy, const StageCoef& sc, cudaStream_t st) {
  if (njobs <= 0) return;
  const size_t smem = (size_t)TW * tiled_stride(Lmax) * sizeof(double2);
  if (smem <= SMEM_CAP)
    k_cart_q2_tiled<<<(njobs + TW - 1) / TW, TW * 32, smem, st>>>(T, jobs, njobs, Lmax, mu, R1, Fy, sc);
  else
    k_cart_q2<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, mu, R1, Fy, sc);
}
void launch_flux_y_points(const DevTables& T, const int* idx, int n, const double* e, double* Fy, cudaStream_t st) {
  if (n <= 0) return;
  k_flux_y_points<<<grid_pts(n, 256), 256, 0, st>>>(T, idx, n, e, Fy);
}
void launch_gen_A(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, double* G,
                  cudaStream_t st) {
  if (njobs <= 0) return;
  k_gen_A<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, e, G);
}
void launch_gen_B(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, const double* mu,
                  const double* J, double* G, cudaStream_t st) {
  if (njobs <= 0) return;
  k_gen_B<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, e, mu, J, G);
}
void launch_gen_C(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* J, double* G,
                  const StageCoef& sc, cudaStream_t st) {
  if (njobs <= 0) return;
  k_gen_C<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, J, G, sc);
}
void launch_rk_fixup(const DevTables& T, const int* idx, int n, const StageCoef& sc, cudaStream_t st) {
  if (n <= 0) return;
  k_rk_fixup<<<grid_pts(n, 256), 256, 0, st>>>(T, idx, n, sc);
}
void launch_filterT_q2(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* lam, const double* ef,
                       double* MF, cudaStream_t st) {
  if (njobs <= 0) return;
  k_filterT_q2<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, lam, ef, MF);
}
void launch_filterT_q1(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* MF, const double* e,
                       double* out, cudaStream_t st) {
  if (njobs <= 0) return;
  k_filterT_q1<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, MF, e, out);
}
void launch_filterT_copy2(const DevTables& T, const int* idx, int n, const double* lam, const double* ef, double* MF,
                          cudaStream_t st) {
  if (n <= 0) return;
  k_filterT_copy2<<<grid_pts(n, 256), 256, 0, st>>>(T, idx, n, lam, ef, MF);
}
void launch_filterT_copy1(const DevTables& T, const int* idx, int n, const double* MF, const double* e, double* out,
                          cudaStream_t st) {
  if (n <= 0) return;
  k_filterT_copy1<<<grid_pts(n, 256), 256, 0, st>>>(T, idx, n, MF, e, out);
}
void launch_bc_wall_T(const WallPt* w, int n, const double* u, double* lam, long long P, double gamma,
                      cudaStream_t st) {
  if (n <= 0) return;
  k_bc_wall_T<<<grid_pts(n, 128), 128, 0, st>>>(w, n, u, lam, P, gamma);
}
void launch_bc_wall(const WallPt* w, int n, double* e, long long P, double gamma, cudaStream_t st) {
  if (n <= 0) return;
  k_bc_wall<<<grid_pts(n, 128), 128, 0, st>>>(w, n, e, P, gamma);
}
void launch_bc(const BcPt* bc, int n, double* e, long long P, cudaStream_t st) {
  if (n <= 0) return;
  k_bc<<<grid_pts(n, 256), 256, 0, st>>>(bc, n, e, P);
}
void launch_exchange(const Recv* r, int n, double* e, long long P, cudaStream_t st) {
  if (n <= 0) return;
  k_exchange<<<grid_pts(n, 256), 256, 0, st>>>(r, n, e, P);
}
void launch_filter_q1(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* e, double* F,
                      cudaStream_t st) {
  if (njobs <= 0) return;
  k_filter_q1<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, e, F);
}
void launch_filter_q2(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* F, double* e,
                      cudaStream_t st) {
  if (njobs <= 0) return;
  k_filter_q2<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, F, e);
}
void launch_filter_copy_q1(const DevTables& T, const int* idx, int n, const double* e, double* F, cudaStream_t st) {
  if (n <= 0) return;
  k_filter_copy_q1<<<grid_pts(n, 256), 256, 0, st>>>(T, idx, n, e, F);
}
void launch_filter_copy_q2(const DevTables& T, const int* idx, int n, const double* F, double* e, cudaStream_t st) {
  if (n <= 0) return;
  k_filter_copy_q2<<<grid_pts(n, 256), 256, 0, st>>>(T, idx, n, F, e);
}
void launch_visc_point(const DevTables& T, const double* e, double* phi, double* S, cudaStream_t st) {
  k_visc_point<<<grid_pts(T.P, 256), 256, 0, st>>>(T, e, phi, S);
}
void launch_visc_muhat(const DevTables& T, const double* phi, const double* S, const float* w, const double* R,
                       double* muhat, int32_t* tau, cudaStream_t st) {
  k_visc_muhat<<<grid_pts(T.P, 128), 128, 0, st>>>(T, phi, S, w, R, muhat, tau);
}
void launch_window_rows(const DevTables& T, const double* in, double* out, const double* wtab, int r,
                        cudaStream_t st) {
  k_window_rows<<<grid_pts(T.P, 256), 256, 0, st>>>(T, in, out, wtab, r);
}
void launch_window_cols(const DevTables& T, const double* in, double* out, const double* wtab, int r,
                        cudaStream_t st) {
  k_window_cols<<<grid_pts(T.P, 256), 256, 0, st>>>(T, in, out, wtab, r);
}
void launch_mu_final(const DevTables& T, const double* num, const double* den, const int* cross_dst,
                     const int* cross_ptr, const int* cross_src, int ncross, double* mu, cudaStream_t st) {
  k_mu_own<<<grid_pts(T.P, 256), 256, 0, st>>>(T, num, den, mu);
  if (ncross > 0) k_mu_cross<<<grid_pts(ncross, 256), 256, 0, st>>>(num, den, cross_dst, cross_ptr, cross_src, ncross, mu);
}
void launch_dt(const DevTables& T, const double* e, const double* mu, unsigned long long* pmax, double cfl, double* dt,
               cudaStream_t st) {
  cudaMemsetAsync(pmax, 0, sizeof(unsigned long long) * 2 * T.npatch, st);
  k_dt_reduce<<<grid_pts(T.P, 256), 256, 0, st>>>(T, e, mu, pmax);
  k_dt_final<<<1, 256, 0, st>>>(T, pmax, cfl, dt);
}

void launch_adj_cart(const DevTables& T, const Job* jobs, int njobs, int Lmax, int dir, const double* u,
                     const double* mu, const double* psi, double* R1, double* acc, const double* dt, cudaStream_t st) {
  if (njobs <= 0) return;
  k_adj_cart<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, dir, u, mu, psi, R1, acc, dt);
}
void launch_adj_gen_A(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* J, const double* u,
                      const double* psi, double* G, cudaStream_t st) {
  if (njobs <= 0) return;
  k_adj_gen_A<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, J, u, psi, G);
}
void launch_adj_gen_B(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* J, const double* u,
                      const double* mu, const double* psi, double* G, cudaStream_t st) {
  if (njobs <= 0) return;
  k_adj_gen_B<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, J, u, mu, psi, G);
  if (T.any_pform) k_adj_gen_B_wall<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, J, u, mu, psi, G);
}
void launch_adj_gen_C(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* u, const double* G,
                      double* acc, const double* dt, cudaStream_t st) {
  if (njobs <= 0) return;
  k_adj_gen_C<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, u, G, acc, dt);
}
void launch_gen_fix(const DevTables& T, const GFix* f, int n, const double* e, const double* mu, const double* J,
                    double* G, cudaStream_t st) {
  if (n <= 0) return;
  k_gen_fix<<<grid_pts(n, 256), 256, 0, st>>>(T, f, n, e, mu, J, G);
}
void launch_adj_gen_fixA(const DevTables& T, const GFix* f, int n, const double* J, const double* u,
                         const double* mu, const double* psi, double* G, cudaStream_t st) {
  if (n <= 0) return;
  k_adj_gen_fixA<<<grid_pts(n, 256), 256, 0, st>>>(T, f, n, J, u, mu, psi, G);
}
void launch_adj_gen_fixB(const DevTables& T, const GFix* f, int n, const double* G, double* R1, cudaStream_t st) {
  if (n <= 0) return;
  k_adj_gen_fixB<<<grid_pts(n, 256), 256, 0, st>>>(T, f, n, G, R1);
}
void launch_adj_fixup(const int* idx, int n, const double* R1, double* acc, long long P, const double* dt,
                      cudaStream_t st) {
  if (n <= 0) return;
  k_adj_fixup<<<grid_pts(n, 256), 256, 0, st>>>(idx, n, R1, acc, P, dt);
}
void launch_exchange_T(const int* dptr, const int* dsrc, const int* drecv, const double* dw, int nd, const Recv* r,
                       int nr, double* lam, long long P, cudaStream_t st) {
  if (nd > 0) k_exchange_T<<<grid_pts(nd, 256), 256, 0, st>>>(dptr, dsrc, drecv, dw, nd, lam, P);
  if (nr > 0) k_zero_points<<<grid_pts(nr, 256), 256, 0, st>>>(r, nr, lam, P);
}
void launch_bc_T(const BcPt* bc, int n, double* lam, double* gbc, double* acc, FsJac fj, long long P,
                 cudaStream_t st) {
  if (n <= 0) return;
  k_bc_T<<<grid_pts(n, 256), 256, 0, st>>>(bc, n, lam, gbc, acc, fj, P);
}
void launch_copy_points(const PtCopy* c, int n, double* e, long long P, cudaStream_t st) {
  if (n > 0) k_copy_points<<<grid_pts(n, 256), 256, 0, st>>>(c, n, e, P);
}
void launch_xpack(const Recv* r, int n, const double* e, long long P, double* buf, cudaStream_t st) {
  if (n > 0) k_xpack<<<grid_pts(n, 128), 128, 0, st>>>(r, n, e, P, buf);
}
void launch_xunpack(const int* dst, int n, const double* buf, double* e, long long P, cudaStream_t st) {
  if (n > 0) k_xunpack<<<grid_pts(n, 256), 256, 0, st>>>(dst, n, buf, e, P);
}
void launch_xgather(const int* dst, int n, const double* e, long long P, double* buf, cudaStream_t st) {
  if (n > 0) k_xgather<<<grid_pts(n, 256), 256, 0, st>>>(dst, n, e, P, buf);
}
void launch_gather(const int* idx, int n, const double* src, double* buf, cudaStream_t st) {
  if (n > 0) k_gather<<<grid_pts(n, 256), 256, 0, st>>>(idx, n, src, buf);
}
void launch_scatter(const int* idx, int n, const double* buf, double* dst, cudaStream_t st) {
  if (n > 0) k_scatter<<<grid_pts(n, 256), 256, 0, st>>>(idx, n, buf, dst);
}
void launch_pair_reduce(double* acc, int n, double* out, cudaStream_t st) {
  if (n <= 0) return;
  k_pair_reduce<<<1, 512, 0, st>>>(acc, n, out);
}
void launch_init_sens(const uint32_t* info, const uint8_t* owned, long long P, const double* e0, const double* lam0,
                      double* drho, double* part, FsJac fj, cudaStream_t st) {
  k_init_sens<<<SENS_BLOCKS, 256, 0, st>>>(info, owned, P, e0, lam0, drho, part, fj);
}
// p[i] = a + b sin(w i): synthetic inputs of the autotuner
void launch_deriv_lines(const DevTables& T, const Job* jobs, int njobs, int Lmax, const double* src, double* dst,
                        cudaStream_t st) {
  if (njobs <= 0) return;
  k_deriv_lines<<<LINE_CFG(njobs, Lmax)>>>(T, jobs, njobs, Lmax, src, dst);
}
void launch_grid_metrics(const GFix* pts, int n, const double* D1, const double* D2, long long P, double* Jm,
                         long long Pg, int* bad, cudaStream_t st) {
  if (n <= 0) return;
  k_grid_metrics<<<grid_pts(n, 256), 256, 0, st>>>(pts, n, D1, D2, P, Jm, Pg, bad);
}

__global__ void k_fill_wave(double* __restrict__ p, long long n, double a, double b, double w) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = a + b * sin(w * (double)(i % 100003));
}
void launch_fill_wave(double* p, long long n, double a, double b, double w, cudaStream_t st) {
  if (n <= 0) return;
  k_fill_wave<<<grid_pts(n, 256), 256, 0, st>>>(p, n, a, b, w);
}
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t st) {
  k_axpby<<<grid_pts(n, 256), 256, 0, st>>>(n, a, x, b, y);
}

void launch_drag(const int* wall, const double* w, const double* nx, int n, const double* e, long long P, double gam,
                 double* J, double* dJde, cudaStream_t st) {
  k_drag<<<1, 256, 0, st>>>(wall, w, nx, n, e, P, gam, J, dJde);
}

void set_kernel_attributes() {
  const int cap = (int)SMEM_CAP;
  cudaFuncSetAttribute(k_cart_q1, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_cart_q2, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_cart_q2_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_gen_A, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_gen_B, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_gen_C, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_filter_q1, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_filter_q2, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_adj_cart, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_adj_gen_A, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_adj_gen_B, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_adj_gen_B_wall, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_adj_gen_C, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_filterT_q1, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_filterT_q2, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(k_deriv_lines, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}
void launch_check_state(const DevTables& T, const double* e, int* flag, cudaStream_t st) {
  k_check_state<<<grid_pts(T.P, 256), 256, 0, st>>>(T, e, flag);
}

}  // namespace fcx
