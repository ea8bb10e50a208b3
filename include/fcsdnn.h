/*
 * fcsdnn.h -- C ABI of the GB300 multi-patch FC-SDNN spatial operator.
 *
 * The library evaluates, on one GPU in FP64, the spatial operator of the
 * multi-patch FC-SDNN scheme of Bruno & Leibovici ("General-domain FC-based
 * shock-dynamics solver I", arXiv 2506.16076) and advances it in time:
 *   - FC-Gram continued spectral derivatives along every grid line
 *     (Sec. 2.2, eqs. continuation and fc_der),
 *   - 2-D Euler fluxes and the artificial-viscosity divergence in the
 *     curvilinear form (Sec. 2.1, 2.3, 3.3, eq. general_curvilinear),
 *   - SDNN-driven viscosity with the smoothing-blending operator (Sec. 5),
 *   - inter-patch interpolation and boundary overwrite (Sec. 3.4, 4.2),
 *   - the per-step spectral filter, the CFL time step and SSPRK-4 (Sec. 4, Alg. 1).
 *
 * Conventions
 *   State layout: structure of arrays e[4][P] in FP64 (rho, rho u, rho v, E),
 *   P = fc_state_size(); patch k occupies points [off_k, off_k + n1*n2) in
 *   row-major (n2, n1) order, q1 fastest; off_k from fc_patch_offset().
 *   Pointers named *_dev are device pointers owned by the caller, 16-byte
 *   aligned. Host pointers (descriptors, tables, weights) are read during the
 *   call only. Every call that takes a stream is asynchronous on that stream
 *   (a cudaStream_t passed as void*, NULL = legacy default stream); device-side
 *   errors (non-finite state, bounded-wait timeout) are raised into a device
 *   flag that fc_sync_status() reads back. No call throws; every call returns
 *   an fc_status and fc_last_error() describes the last failure of a context.
 */
#ifndef FCSDNN_H
#define FCSDNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fc_ctx fc_ctx;

typedef enum {
  FC_OK = 0,
  FC_ERR_INVALID = 1,       /* bad argument or descriptor */
  FC_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  FC_ERR_DONOR = 3,         /* donor-receiver condition violated (Sec. 3.4, Remark overlap_cond) */
  FC_ERR_OVERLAP = 4,       /* a line too short for FC has points that are not receivers */
  FC_ERR_NONFINITE = 5,     /* NaN/Inf or non-positive density/pressure detected on the device */
  FC_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  FC_ERR_UNIMPLEMENTED = 7,
  FC_ERR_OOM = 8            /* device allocation failed */
} fc_status;

/* patch kinds (Sec. 3.1): affine box (C/I-type), annulus around an obstacle with a periodic
 * angle, and a general curvilinear grid given point by point (S-type patches along any
 * smooth boundary) */
enum { FC_PATCH_AFFINE = 0, FC_PATCH_OGRID = 1, FC_PATCH_GRID = 2 };
/* side types, side order (q1=0, q1=1, q2=0, q2=1) (Sec. 3.4 internal/external sides, Sec. 4.2).
 * SLIPWALL: the wall-normal momentum is set to 0 at every stage.
 * ADIABATIC: no-slip adiabatic wall (Sec. 4.2, Remarks adiabatic_th and adiabatic): both
 *   momenta are set to 0 and the wall temperature is the value at the wall of the
 *   degree d-1 polynomial through the temperatures of the d-1 next points inward with
 *   zero normal derivative at the wall (the Neumann FC end data); E follows from it. */
enum {
  FC_SIDE_INTERNAL = 0,
  FC_SIDE_DIRICHLET = 1,
  FC_SIDE_SLIPWALL = 2,
  FC_SIDE_OUTFLOW = 3,
  FC_SIDE_PERIODIC = 4,
  FC_SIDE_ADIABATIC = 5
};

/* One patch (Sec. 3.1-3.2). AFFINE: geom = (x0, x1, y0, y1), q1 -> x, q2 -> y.
 * OGRID: geom = (xc, yc, r0, r1), q1 -> angle (periodic, n1 points), q2 -> radius.
 * bc[s] = primitive (rho, u, v, p) imposed on side s when it is DIRICHLET.
 * hole = (xc, yc, R): points of AFFINE and GRID patches with distance < R are blanked
 * (R <= 0: none; OGRID patches ignore it). */
typedef struct {
  int kind;
  int n1, n2;
  double geom[4];
  int side[4];
  double bc[4][4];
  double hole[3];
  /* GRID only (NULL otherwise; host arrays, read during fc_init_patches): the physical
   * coordinates x, y of the grid points (n2 x n1, row-major, q1 fastest) and the metrics
   * dq/dx as [4][n2 x n1] = (dq1/dx, dq1/dy, dq2/dx, dq2/dy) for the parameters
   * q1 = i / (n1 - 1) (q1 = i / n1 when sides 0 and 1 are PERIODIC) and q2 = j / (n2 - 1)
   * (Sec. 3.3). metrics NULL: computed on the device at init by inverting the Jacobian
   * d(x, y)/d(q1, q2) from FC derivatives of x and y along the full grid lines (Fourier
   * along a periodic q1; at least 2d points per non-periodic line; FC_ERR_INVALID if the
   * Jacobian is singular anywhere). Other patches locate points of a GRID patch by
   * Newton's method on its 3 x 3 quadratic interpolant, started at the nearest grid
   * point. GRID sides may be INTERNAL, DIRICHLET, OUTFLOW, ADIABATIC or PERIODIC (q1
   * only); geom is unused. */
  const double *x, *y, *metrics;
} fc_patch_desc;

/* Method parameters. Defaults of the paper: gamma 1.4 (Sec. 2.1), alpha_f 10,
 * p_f 14 (Sec. 4.3.1), CFL 0.5 (Sec. 6), n_f 5, n_v 9 (Sec. 3.4), window
 * w_{0,9} (win_r 9, Sec. 5.2), 7x7 localisation (loc 7), R = (1.5,1,0.5,0) (Sec. 5.1).
 * fc_tables: host array, [0]=d, [1]=Cmin, [2]=Cmax, then for C = Cmin..Cmax the
 *   blocks Q (d x d), A_l (C x d), A_r (C x d), row-major (eq. continuation).
 * c_policy (the paper leaves C free, Sec. 2.2): 0: C = C0 on every line; 1: smallest
 *   C >= C0 with N + C 7-smooth; 2: the C in [C0, Cmax] whose continued length N + C
 *   has the smallest estimated transform cost: N + C factored greedily into 8, 4, 2,
 *   3, 5, 7, cost = sum over stages of (L/R) B(R) with B = 4, 16, 52, 14, 36, 66 for
 *   R = 2, 4, 8, 3, 5, 7, plus 4 (L/R)(R-1) on every stage but the last; ties to the
 *   smaller C; falls back to policy 1 when no N + C in range is 7-smooth.
 * sdnn_w: host FP32 weights of the 7-16-16-4 classifier: W1[16][7], b1[16],
 *   W2[16][16], b2[16], W3[4][16], b3[4] (sdnn_len = 420).
 * depth_cap: cap of the index distance used to rank donors. */
typedef struct {
  int d, C0, c_policy;
  double gamma, alpha_f;
  int p_f;
  double cfl;
  int n_f, n_v, win_r, loc;
  double R[4];
  int depth_cap;
  const double *fc_tables;
  int fc_tables_len;
  const float *sdnn_w;
  int sdnn_len;
  /* Free stream (rho, u, v, p) of the problem (Sec. 7, eq. mach_flow_ic), or rho <= 0 for
   * none. It drives the Dirichlet data: a DIRICHLET side whose bc density is 0 holds the
   * free stream. Dirichlet points that hold it (that way, or through a bc equal to it) are
   * the free-stream points whose adjoint fc_adjoint_step turns into dJ/dM and dJ/dalpha,
   * M = |(u, v)| / a the Mach number and alpha = atan2(v, u) the angle of attack, at fixed
   * density and pressure (sound speed a = sqrt(gamma p / rho)). */
  double freestream[4];
  /* Operator on patches with an ADIABATIC side (Remark adiabatic). 0: the flux form used on
   * every other patch (FC derivatives of the flux components). 1: the product-rule form:
   * rho, rho u, rho v and the temperature theta = p / rho are FC-differentiated (theta in
   * place of E; along the wall-normal lines its continuation is the Neumann expansion,
   * the wall overwrite having put the Neumann end data's value at the wall), the x and y
   * derivatives of p = rho theta (eq. p_T) and E (eq. perfect_gas_T) follow from them by
   * the sum and product rules, the convective divergence div f(e) is formed from these
   * derivatives by the same rules, and the viscous fluxes mu grad e, with grad E from the
   * product rule, are FC-differentiated as elsewhere. Patches without an adiabatic side
   * keep the flux form. With 1, an AFFINE patch with an ADIABATIC side is FC_ERR_INVALID
   * at init; fc_adjoint_step transposes whichever form each patch uses. Other values:
   * FC_ERR_INVALID. */
  int wall_form;
} fc_params;

/* fc_rk_step flags */
enum {
  FC_STEP_FILTER = 1,      /* apply the per-step spectral filter (Sec. 4.3.1) */
  FC_STEP_FROZEN_MU = 2,   /* use mu_dev as given instead of computing it (Sec. 5) */
  FC_STEP_PER_PATCH = 4,   /* one launch per patch and pass (baseline schedule) */
  FC_STEP_FIXED_DT = 8,    /* use *dt_dev as the step instead of eq. CFL */
  FC_STEP_GRAPH = 16       /* capture the step once and replay it as a CUDA graph */
};

/* Build a context: patch grids, metrics, fringes, donors and interpolation
 * weights (Sec. 3, Alg. 1 line 2), FFT plans per continued length, viscosity
 * windows and normalisers (eq. multipatch_W_norm). Checks the donor-receiver
 * condition (FC_ERR_DONOR). Allocates all device workspaces. */
fc_status fc_init_patches(fc_ctx **out, const fc_patch_desc *patches, int npatch, const fc_params *prm, void *stream);

/* Number of points P (state has 4*P doubles) and per-patch offsets. */
size_t fc_state_size(const fc_ctx *ctx);
fc_status fc_patch_offset(const fc_ctx *ctx, int patch, size_t *offset);
/* Number of non-blanked points (the points that receive an update). */
size_t fc_active_points(const fc_ctx *ctx);

/* rhs_dev = L[e_dev] (eq. semi-discrete) with viscosity mu_dev (P doubles);
 * mu_dev NULL: mu is computed from e_dev (Sec. 5). L = 0 on blanked points
 * and on lines too short for FC. */
fc_status fc_rhs(fc_ctx *ctx, const double *e_dev, double *rhs_dev, const double *mu_dev, void *stream);

/* mu_dev = Lambda[mu^[e_dev]] (eqs. V2D_unscaled, Lambda, viscosity);
 * tau_dev (nullable, P int32): the smoothness class on generating points, 0 elsewhere. */
fc_status fc_viscosity(fc_ctx *ctx, const double *e_dev, double *mu_dev, int32_t *tau_dev, void *stream);

/* In-place per-step filter of rho, rho u, rho v, theta with E rebuilt (Sec. 4.3.1). */
fc_status fc_filter(fc_ctx *ctx, double *e_dev, void *stream);

/* In-place boundary overwrite followed by the inter-patch exchange (Sec. 4.2, Sec. 3.4.1). */
fc_status fc_project(fc_ctx *ctx, double *e_dev, void *stream);

/* *dt_dev = eq. (CFL) for state e_dev and viscosity mu_dev (device scalar). */
fc_status fc_timestep(fc_ctx *ctx, const double *e_dev, const double *mu_dev, double *dt_dev, void *stream);

/* One time step of Algorithm 1 in place on e_dev: project, viscosity (unless
 * FROZEN_MU), filter (if FILTER), project, dt (unless FIXED_DT; written to
 * *dt_dev), then five SSPRK-4 stages, each followed by the boundary overwrite
 * and the exchange. mu_dev: P doubles, written (or read with FROZEN_MU).
 * Batched (no PER_PATCH), the length classes of a pass and the curvilinear chain of a
 * stage run on the context's own side streams, forked from and joined back into
 * `stream` with events; the call is ordered on `stream` like a single-stream one.
 * FCSDNN_CONCURRENT=0 in the environment at fc_init_patches keeps everything on
 * `stream`. */
fc_status fc_rk_step(fc_ctx *ctx, double *e_dev, double *dt_dev, double *mu_dev, int flags, void *stream);

/* fc_rk_step on a state held in host memory: e_host (4 P doubles, the layout above) is
 * copied to a device buffer the context owns (allocated on the first call), advanced by
 * one fc_rk_step (flags as there; FC_STEP_GRAPH captures the step on that buffer once),
 * and copied back; the call synchronises `stream` before it returns, so e_host holds the
 * new state then. dt_dev and mu_dev are device buffers as in fc_rk_step. Page-locked host
 * memory (cudaHostAlloc / cudaHostRegister, torch pin_memory) copies at the link's rate;
 * pageable memory works but copies slower. */
fc_status fc_rk_step_host(fc_ctx *ctx, double *e_host, double *dt_dev, double *mu_dev, int flags, void *stream);

/* fc_autotune flags */
enum { FC_TUNE_PLANS = 1, FC_TUNE_WARPS = 2 };
/* Measured schedule choice for this context's lines (no paper counterpart: the paper's
 * CPU code has no launch schedule). FC_TUNE_PLANS: for every continued length L, the
 * stage orders of the FFT with the smallest modelled cost (up to 4, power-of-two radices
 * first) are each timed on that length's own lines and the fastest kept (if at least 1%
 * faster than the model's choice and its output agrees with it to 1e-10 relative).
 * FC_TUNE_WARPS: for every power-of-two length class, 1, 2, 4 or 8 warps per CTA, timed
 * on the class's q1 and q2 lines. The choices change rounding only, never the method.
 * Synchronises `stream`, overwrites the context's scratch (stage buffers, R1, its
 * internal mu), invalidates a captured step graph (the next FC_STEP_GRAPH step captures
 * again) and allocates 1 MB of device memory on its first call. report (nullable, 6 host doubles):
 * lengths examined, lengths changed, classes examined, classes changed, and the summed
 * time (ms) of the timed line batches before and after. */
fc_status fc_autotune(fc_ctx *ctx, int flags, double *report, void *stream);

/* Discrete adjoint of one fc_rk_step with mu and dt frozen (the smoothness
 * classifier is not differentiable, so the viscosity of the forward step is held
 * fixed): lam_n_dev = (d e_{n+1} / d e_n)^T lam_np1_dev for the step that starts from
 * e_n_dev with viscosity mu_dev (P doubles) and step *dt_dev (device scalar). flags:
 * FC_STEP_FILTER when the forward step applied the per-step filter (Sec. 4.3.1); other
 * bits are ignored. The stage states are recomputed from e_n_dev. Transposes: FC
 * derivative (zero padding, negated spectral derivative, continuation folded back onto
 * the 2d end points), flux Jacobians, viscous term with mu fixed, inter-patch exchange
 * (donors gather the receivers' adjoint with the interpolation weights), boundary
 * overwrite, adiabatic walls (linearised at the stage state), and the filter
 * (linearised at the state it was applied to: theta and E rebuild Jacobians around
 * the line filters, whose transposes fold the continuation back like the derivative's).
 * gbc_dev (nullable, [4][P]) accumulates the adjoint that reaches the Dirichlet
 * points, i.e. the sensitivity of the step result to the imposed states.
 * dparam_dev (nullable, 2 device doubles) accumulates, in a fixed order, the part of
 * dJ/d(M, alpha) that enters through the free-stream Dirichlet states during this step:
 * the sum over the free-stream points of that adjoint times d e_fs / d(M, alpha)
 * (FC_ERR_INVALID when fc_params.freestream is not set). The first call allocates 11
 * state-sized device buffers, and 2 more with the filter. */
fc_status fc_adjoint_step(fc_ctx *ctx, const double *e_n_dev, const double *mu_dev, const double *dt_dev,
                          const double *lam_np1_dev, double *lam_n_dev, double *gbc_dev, double *dparam_dev,
                          int flags, void *stream);

/* Sensitivities to the initial data of a functional J whose gradient with respect to the
 * initial state e_0 is lam0_dev ([4][P], e.g. lam_n of the adjoint step of step 0):
 * drho_dev (nullable, P doubles) = dJ/drho_0 point by point at fixed velocity and
 *   pressure, i.e. lam0 . d e_0 / d rho = lam_rho + lam_mx u + lam_my v + lam_E |u|^2 / 2
 *   (0 on blanked points);
 * dparam_dev (nullable, 2 doubles) accumulates dJ/d(M, alpha) through e_0 when e_0 is the
 *   uniform free stream of fc_params.freestream on every non-blanked point (the sum over
 *   those points of lam0 . d e_fs / d(M, alpha); FC_ERR_INVALID without a free stream).
 * Both sums and all accumulations are in a fixed order: results are reproducible. */
fc_status fc_initial_sensitivity(fc_ctx *ctx, const double *e0_dev, const double *lam0_dev, double *drho_dev,
                                 double *dparam_dev, void *stream);

/* Wall-pressure drag functional J = sum over the wall ring of the first OGRID
 * patch with a slip or adiabatic wall of p n_x r0 dtheta (periodic trapezoid of the integral of
 * wall pressure times n_x, n the outward body normal); J_dev: device scalar.
 * dJde_dev (nullable, [4][P]): dJ/de, zero off the wall. */
fc_status fc_drag(fc_ctx *ctx, const double *e_dev, double *J_dev, double *dJde_dev, void *stream);

/* Reads the device error flag (synchronises the stream): FC_OK, FC_ERR_NONFINITE or FC_ERR_TIMEOUT.
 * check_state != 0 also scans e_dev (may be NULL otherwise) for NaN/Inf and rho, p <= 0. */
fc_status fc_sync_status(fc_ctx *ctx, const double *e_dev, int check_state, void *stream);

/* Number of kernel launches issued by this context so far (instrumentation). */
uint64_t fc_launch_count(const fc_ctx *ctx);

/* Kernel timing instrumentation. When enabled, every launch group of a call made
 * outside graph capture is bracketed by CUDA events on the call's stream.
 * fc_profile_read() synchronises the device, folds the recorded pairs into
 * per-group totals and returns the number of groups (-1 on error); fc_profile_get()
 * returns group k: its name (owned by the context), total milliseconds and launches.
 * While enabled, the batched passes run one after another on the call's stream (no
 * overlap of length classes or of the curvilinear and affine chains), so each group's
 * time is its own. */
fc_status fc_profile_enable(fc_ctx *ctx, int enable);
int fc_profile_read(fc_ctx *ctx);
fc_status fc_profile_get(const fc_ctx *ctx, int k, const char **name, double *ms, int *launches);
fc_status fc_profile_reset(fc_ctx *ctx);

/* Affine-patch line passes skip the gradient round of a line on which mu is zero at every
 * point (the viscous flux vanishes and H = f(e) exactly). Counts of skipped lines and of
 * the algorithmic flops of the skipped rounds since the last reset, per direction
 * (synchronises the device). */
fc_status fc_line_stats(fc_ctx *ctx, long long *lines_q1, long long *lines_q2, double *flops_q1, double *flops_q2,
                        int reset);

/* Algorithmic work of one launch of a line pass ("cart_q1", "cart_q2", "filter_q1",
 * "filter_q2"): FP64 flops by the conventional FFT count (5 L log2 L per complex
 * transform) plus continuation, multiplier and pointwise work; compulsory HBM
 * bytes; number of lines and points. Used to place a measured duration on the
 * FP64 and HBM rooflines. */
fc_status fc_pass_stats(const fc_ctx *ctx, const char *pass, double *flops, double *bytes, long long *lines,
                        long long *points);

/* ---- Sharded execution over several ranks (one GPU per rank) ----
 * The patches are the unit of work: a rank advances only the patches it owns, and the
 * operator couples patches only through the inter-patch exchange of every projection
 * (Sec. 3.4.1, Sec. 4.2), the cross-patch sums of the smoothing-blending operator of the
 * viscosity (Sec. 5.2) and the global minimum of the time step (eq. CFL): the
 * communication step of Algorithm 1. */

/* Host-only (no device needed): owner[p] in [0, nranks) for every patch. Patches are
 * ordered along the Morton (Z-order) curve of their centres, so that neighbours share a
 * rank, and the order is cut into nranks contiguous runs of about equal active (non-
 * blanked) point counts; a boundary then moves by single patches while that lowers the
 * larger of the two loads it separates. Deterministic. FC_ERR_INVALID for nranks < 1. */
fc_status fc_partition(const fc_patch_desc *patches, int npatch, int nranks, int *owner);

/* What a rank exchanges with the others, through a callback the caller supplies (NCCL,
 * gloo, or an in-process transport). op FC_COMM_EXCHANGE: send_dev holds, for every
 * rank q = 0..nranks-1 in order, send_counts[q] doubles owed to q (0 for this rank);
 * the callback fills recv_dev with recv_counts[q] doubles from every q, in the same
 * order, before any later work on `stream` (an all-to-all with these splits). op
 * FC_COMM_MIN: recv_dev[0] = the minimum over ranks of send_dev[0] (send_counts[0] = 1).
 * Buffers are device memory owned by the context. Return 0 on success; any other value
 * makes the calling function fail with FC_ERR_CUDA. */
enum { FC_COMM_EXCHANGE = 0, FC_COMM_MIN = 1 };
typedef int (*fc_comm_fn)(void *user, int op, const double *send_dev, const long long *send_counts, double *recv_dev,
                          const long long *recv_counts, void *stream);

/* Turn ctx (built on the whole workload, identically on every rank) into rank `rank` of
 * nranks with the patch owners `owner` (host array of npatch entries): from then on
 * fc_rk_step, fc_rhs, fc_project, fc_viscosity, fc_filter, fc_timestep and
 * fc_sync_status work on the owned patches only. State buffers keep the full layout;
 * entries of other ranks' patches are neither read nor written, except the fringe values
 * and window sums that arrive through `comm`. Per projection every rank packs the
 * interpolated fringe values (3 x 3 donor stencils) it owes to others, calls comm
 * (FC_COMM_EXCHANGE) and scatters what it receives; per viscosity evaluation the same
 * for the window sums of the cross-patch blending; per time step one FC_COMM_MIN. The
 * results equal the unsharded context's bit for bit (the same kernels on the same
 * values). fc_adjoint_step runs sharded too: its projections' transposes send each
 * receiver's adjoint back to the donors' rank (the exchange reversed), so lam_n on the
 * owned patches equals the unsharded one bit for bit; fc_drag evaluates J and dJ/de on
 * the rank that owns the wall ring's patch (J = 0 elsewhere), and the dparam sums of
 * fc_adjoint_step and fc_initial_sensitivity cover the owned patches: the caller adds J
 * and dparam over the ranks. Not available while sharded: FC_STEP_GRAPH and
 * FC_STEP_PER_PATCH steps and fc_autotune (FC_ERR_UNIMPLEMENTED). Once per context. */
fc_status fc_shard(fc_ctx *ctx, int nranks, int rank, const int *owner, fc_comm_fn comm, void *user);

/* Doubles this rank sends to / receives from `peer` in one FC_COMM_EXCHANGE of a
 * projection (which = 0) or of a viscosity evaluation (which = 1). */
fc_status fc_shard_counts(const fc_ctx *ctx, int which, int peer, long long *send, long long *recv);

/* FP64 throughput probes of the current device (instrumentation, no paper counterpart):
 * *dfma_gflops = FP64 FMA rate of independent chains on every SM, *dmma_gflops = rate of the
 * FP64 matrix instruction (m8n8k4), both in GFLOP/s (2 flops per multiply-add), timed with
 * CUDA events on `stream` (synchronised) after one warm-up round; about 0.1 s. Allocates
 * 8 bytes (stream-ordered) for a result sink. */
fc_status fc_probe_fp64(double *dfma_gflops, double *dmma_gflops, void *stream);

/* RHS of one stand-alone affine patch without any device allocation. For callers that
 * cannot allocate device memory: code under a host memory manager that owns all device
 * memory, plug-ins whose host forbids allocation, paths that must not allocate once set
 * up. (The paper has no counterpart: this is an interface of this library.)
 * rhs_dev = L[e_dev] on the box [box[0], box[1]] x [box[2], box[3]] (host array) with
 * n1 x n2 points (q1 fastest, state layout as above, P = n1 n2), viscosity mu_dev,
 * FC order d and C continuation points on every line; table: host array of the
 * d x d Q, C x d A_l and C x d A_r blocks (one C block of the fc_params tables), of
 * table_len = d d + 2 C d values (any other length: FC_ERR_INVALID).
 * No boundary condition is applied (as in fc_rhs). The scratch is one static device
 * array of 10.0 MB (9,990,656 bytes) held by every GPU that loads the library until exit; limits:
 * n1 n2 <= 262144, n + C <= 1024, C <= 128, d <= 8 (beyond them the call prints the
 * limits to stderr and returns FC_ERR_INVALID). All calls share the array and it keeps
 * the last call's contents: calls that overlap on the GPU (other streams, other host
 * threads) race. The first call on a device looks up the array's device address with
 * that device current; make that first call before any stream capture. The call
 * synchronises the stream once (table upload from host memory). */
fc_status fc_rhs_patch_noalloc(const double *e_dev, const double *mu_dev, double *rhs_dev, int n1, int n2,
                               const double *box, int d, int C, const double *table, int table_len, double gamma,
                               void *stream);

const char *fc_last_error(const fc_ctx *ctx);
void fc_destroy(fc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
