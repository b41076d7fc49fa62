/*
 * tt.h -- C ABI of the GB300 (sm_103a) tensor-train multigroup S_N transport step.
 *
 * The method is the tensor-train (TT) multigroup discrete-ordinates solver of
 * "Multigroup Thermal Radiation Transport with Tensor Trains" (arXiv 2602.00290):
 * the solution I_{k l p} = Z_k Theta_l Phi_p with a merged spatio-spectral core Z
 * (Sec. 3.1, Eq. tensor_decomp_mer), advanced by step-then-truncate (end of Sec. 3.1):
 * forward-Euler transport (upwind, Rusanov or central flux) as a sum of n rank-1 TT operators
 * (Appendix A, 'Value of n'), SVD-based rounding (Sec. 3.1 footnote), the
 * backward-Euler operator-split source of Eq. (discRTsource) at fixed material
 * temperature, and rounding again.
 *
 * Conventions for every call
 * --------------------------
 * - Every pointer inside tt_tensor / tt_problem is DEVICE memory owned by the caller
 *   unless stated otherwise.  The library never frees caller memory.
 * - All calls are asynchronous on the context's CUDA stream and return after enqueueing.
 *   Argument errors that the host can see are returned immediately.  Errors detected on
 *   the device (rank capacity exceeded, non-finite values) are latched in a device status
 *   word and returned by the next tt_sync().  No kernel traps; every device-side wait is
 *   bounded.
 * - TT layout: core j has shape (r_{j-1}, n_j, r_j) and is stored row-major as
 *   [rcap_{j-1} * n_j][rcap_j] in the tensor's dtype, i.e. element (a, i, b) lives at
 *   (a * n_j + i) * rcap_j + b.  r_0 = r_d = 1.  Live ranks are in device memory
 *   (rank[0..d], int32) and are read and written by the library, so a sequence of calls
 *   never needs the host to know them.  Entries outside the live ranks must be zero on
 *   input; the library keeps them zero on output.
 * - Core 0 is the merged spatio-spectral core Z with rows k = g + G*(ix + Nx*(iy + Ny*iz)).
 *   Supported topologies: d = 2 (planar slab: Z, mu core) and d = 3 (Z, polar core Theta,
 *   azimuthal core Phi).
 */
#ifndef TT_H
#define TT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_MAX_CORES 8

typedef enum {
  TT_OK = 0,
  TT_ERR_ARG = 1,          /* null pointer, bad enum, negative tolerance, ...            */
  TT_ERR_SHAPE = 2,        /* incompatible mode sizes or topology                         */
  TT_ERR_CAPACITY = 3,     /* a result rank would exceed the output rank capacity         */
  TT_ERR_CUDA = 4,         /* a CUDA runtime call failed                                  */
  TT_ERR_NONFINITE = 5,    /* NaN/Inf met in a norm or a singular value on the device     */
  TT_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                          */
  TT_ERR_UNSUPPORTED = 7,  /* valid request outside what this build implements            */
  TT_ERR_WORKSPACE = 8     /* the context workspace is too small for the request          */
} tt_status;

typedef enum { TT_F64 = 0, TT_F32 = 1 } tt_dtype;

/* Arithmetic of the rounding and contraction kernels.
 * TT_PREC_FP64  : every step in FP64.
 * TT_PREC_MIXED : bulk passes over the merged core in FP32 (FP32 storage of Z allowed),
 *                 small-core SVDs, the rank decisions, norms and the energy check in FP64.
 * TT_PREC_MIXED_3XTF32 : TT_PREC_MIXED with the dense contractions over the merged core on the
 *                 tensor cores (tcgen05 kind::tf32) in split precision: each FP32 operand is split
 *                 into its TF32 part and remainder and three products (hi hi, hi lo, lo hi) are
 *                 summed in the FP32 accumulator, FP32-level products.  Where a pass cannot take the
 *                 tensor-core kernel (FP64 storage of Z, rank capacities that are not multiples of
 *                 8, shared memory) it runs the TT_PREC_MIXED kernel. */
typedef enum { TT_PREC_FP64 = 0, TT_PREC_MIXED = 1, TT_PREC_MIXED_3XTF32 = 2 } tt_precision;

typedef enum { TT_QUAD_GAUSS_LEGENDRE_MU = 0, TT_QUAD_LATLONG_MIDPOINT = 1 } tt_quadrature;

/* Numerical flux of the transport operator (Appendix A, 'Value of n').
 * UPWIND: n = 2 d_X rank-1 terms, per axis the two one-sided differences times n_a 1[n_a >= 0]
 *   and n_a 1[n_a < 0].
 * RUSANOV: n = 2 d_X, per axis the central difference (I_{i+1} - I_{i-1})/2 times n_a and the
 *   isotropic diffusion term -(I_{i+1} - 2 I_i + I_{i-1})/2 (largest speed alpha = c).
 * CENTRAL: n = d_X, the Rusanov flux with wavespeed S+ = 0 (the pure central difference the
 *   Gaussian-diffusion test of Sec. 4.3 uses): per axis the central-difference term only.
 * RUSANOV and CENTRAL are read with vacuum ghost cells: a problem with an inflow face is
 * TT_ERR_UNSUPPORTED. */
typedef enum { TT_FLUX_UPWIND = 0, TT_FLUX_RUSANOV = 1, TT_FLUX_CENTRAL = 2 } tt_flux;

/* Tensor-train layout of the state (Sec. 3.1 and the split topologies of Sec. 5).
 * MERGED: the first core merges all spatial axes with the frequency groups, Z(x nu) (row
 *   k = g + G (ix + Nx (iy + Ny iz))), followed by the angular cores (Theta, Phi; mu for the slab).
 *   The only layout built.
 * MERGED_NUX_Y: [Z(nu x)][y][theta][phi], the y axis in a core of its own (d = 4).
 * SPLIT_X: [X][nu][theta][phi], the spatial core apart from the groups (d = 4).
 * tt_plan_create refuses the two d = 4 layouts with TT_ERR_UNSUPPORTED. */
typedef enum { TT_TOPO_MERGED = 0, TT_TOPO_MERGED_NUX_Y = 1, TT_TOPO_SPLIT_X = 2 } tt_topology;

typedef struct {
  int32_t d;                       /* number of cores, 2 or 3                               */
  int32_t n[TT_MAX_CORES];         /* mode sizes n_0..n_{d-1}                               */
  int32_t rcap[TT_MAX_CORES + 1];  /* rank capacities, rcap[0] = rcap[d] = 1                */
  int32_t *rank;                   /* device int32[d+1], live ranks                         */
  void *core[TT_MAX_CORES];        /* device, core j: [rcap_{j-1} * n_j][rcap_j]            */
  tt_dtype dtype;                  /* element type of every core                            */
} tt_tensor;

/* Raw physical problem (Sec. 2, Sec. 2.1, Sec. 4 preamble).  Units h = k_B = c = a = 1
 * unless c and a_rad say otherwise; x = nu / T in the Planck integrals. */
typedef struct {
  int32_t ndim_x;                  /* spatial axes d_X: 1 (slab, needs d = 2) or 2, 3 (d = 3) */
  int32_t nx, ny, nz;              /* cells per axis (1 for unused axes)                    */
  int32_t ngroup;                  /* G frequency groups                                    */
  int32_t quadrature;              /* tt_quadrature                                         */
  int32_t ntheta, nphi;            /* polar (or mu) nodes, azimuthal nodes (1 for the slab) */
  double dx, dy, dz;               /* cell sizes                                            */
  double c, dt, a_rad;             /* speed of light, time step, radiation constant         */
  const double *group_edges;       /* device double[G+1]: 0, log-spaced interior, +inf      */
  const double *temperature;       /* device double[N_X]: fixed material temperature        */
  const double *rho_kappa_a;       /* device double[N_X*G] per merged row                   */
  const double *rho_kappa_s;       /* device double[N_X*G] per merged row                   */
  double inflow_temperature[6];    /* faces x-,x+,y-,y+,z-,z+; < 0 means vacuum             */
  int32_t flux;                    /* tt_flux                                               */
  const double *rho_cv;            /* device double[N_X] volumetric heat capacity rho c_v, or
                                      NULL: the material temperature stays fixed.  Non-NULL
                                      couples it (Sec. 2.1, Eq. Tupdate): every tt_step solves
                                      the f(T^dagger) root per cell, uses epsilon(T^dagger) in
                                      the source update and advances T by total energy
                                      conservation with the rounded state's J^{m+1}.  The plan
                                      then carries the material state of ONE problem.      */
  int32_t topology;                /* tt_topology (TT_TOPO_MERGED)                          */
} tt_problem;

typedef struct tt_context tt_context;
/* Factor of the merged core in the first sweep of every rounding (tt_round, tt_step).
 * TT_ROUND_TSQR: Householder TSQR (the SVD-based rounding of Sec. 3.1; the default).
 * TT_ROUND_GRAM: Gram-based (Sec. 3.1 lists it among the solver's rounding methods): the FP64 Gram
 * matrix G = A^T A of the merged core's unfolding (virtual transport sum included) and a square
 * root R of G (R^T R = G, diagonally pivoted Cholesky) replace the TSQR's R; the rest of the
 * rounding is unchanged.  Forming G squares the condition number (the paper's caution):
 * singular values below about 1e-8 |X| are not resolved, so use it at tolerances above that.
 * TT_ROUND_RANDOMIZED: randomized (Sec. 3.1 lists it too): the merged core's first unfolding is
 * sketched as Y = A (B0 omega) with the caller's sketch omega (tt_context_set_sketch), Q from a
 * Householder TSQR of Y's l columns, and C = Q^T A (FP64 accumulation) replaces the TSQR's R;
 * the SVD-based truncation follows at the same tolerance.  With l >= the rank of the unfolding
 * this is the SVD rounding; otherwise it keeps the directions the sketch captured. */
typedef enum { TT_ROUND_TSQR = 0, TT_ROUND_GRAM = 1, TT_ROUND_RANDOMIZED = 2 } tt_rounding;

typedef struct tt_plan tt_plan;

/* Status text for a tt_status value (static storage, never NULL). */
const char *tt_status_string(tt_status s);

/* Create a context bound to CUDA device `device` and stream `cuda_stream` (a cudaStream_t,
 * NULL = legacy default stream).  `workspace_bytes` > 0 pre-allocates that much device
 * workspace; 0 lets the library size it on first use (outside any stream capture).
 * The context owns its workspace and its device status word. */
tt_status tt_context_create(tt_context **ctx, int device, void *cuda_stream, size_t workspace_bytes);
tt_status tt_context_destroy(tt_context *ctx);

/* Opt-in instrumentation of a context (off by default).  While timing is enabled, every
 * later call records CUDA events on the context stream around its hot kernels, grouped as
 * TT_TIMER_* categories.  Launch counts are always collected. */
typedef enum {
  TT_TIMER_TSQR_LEAF = 0,   /* leaf pass of the tall-skinny QR over the merged core (the
                               transport sum in tt_step, the tensor itself in tt_round)    */
  TT_TIMER_TSQR_MERGE = 1,  /* merge tree of the R factors                                 */
  TT_TIMER_SMALL = 2,       /* small-core sweep (QRs, Jacobi SVDs, rank decisions)         */
  TT_TIMER_UPDATE = 3,      /* update pass Z_new = Z_sum W (and the fused source step)     */
  TT_TIMER_OTHER = 4,       /* everything else (counted only)                              */
  TT_TIMER_TSQR_LEAF_SOURCE = 5, /* leaf pass over the source sum (second rounding of tt_step) */
  TT_TIMER_UPDATE_SOURCE = 6     /* update pass of the second rounding of tt_step (the source sum);
                                    TT_TIMER_UPDATE then times the first one alone              */
} tt_timer;
#define TT_TIMER_COUNT 7
tt_status tt_context_set_timing(tt_context *ctx, int enable);

/* Replay tt_step as a CUDA graph (enable != 0; default off).  With it on, the first tt_step for a
 * given key runs eagerly (so every kernel of the step is loaded and configured outside any
 * capture), the second captures the step's launch sequence, and later ones replay it; the key is
 * (the plan, by its creation, so that a
 * plan made at a destroyed plan's address is a new key; state pointers, rank capacities
 * and dtype; tol, rmax, precision, energy_dev; the context's workspace, rounding method, sketch
 * and TSQR kernel table) and replays that graph, on the context's stream, while the key stays
 * the same; a new key drops the old graph and captures again.  Device data (ranks, cores, plan
 * arrays) may change freely between replays: the host reads none of it.  The capture runs on a
 * private stream, so the context's stream may be the legacy default stream; tt_step called
 * while the context's stream is itself being captured runs eagerly (it then becomes part of
 * the caller's graph).  With kernel timing on (tt_context_set_timing), or when a step cannot be
 * captured, tt_step runs eagerly with the same results.  Launch counters count each replay's
 * kernels; tt_context_diagnostics reports replays, captures and refused captures.  Turning it
 * off releases the graph.  Errors: TT_ERR_ARG (ctx NULL). */
tt_status tt_context_set_graphs(tt_context *ctx, int enable);

/* Select the rounding method of the context (TT_ERR_ARG for an unknown method).  With
 * TT_ROUND_GRAM the TT_TIMER_TSQR_LEAF(_SOURCE) categories time the Gram pass instead; with
 * TT_ROUND_RANDOMIZED they time the TSQR of the sketch (the sketch itself is an update pass). */
tt_status tt_context_set_rounding(tt_context *ctx, tt_rounding method);

/* Sketch of randomized rounding: omega_dev (device, nang x ell row-major, FP64, caller-owned and
 * kept allocated while the context rounds with it; e.g. iid N(0,1)), nang = n_1 ... n_{d-1} of
 * the tensors rounded, 1 <= ell <= 64 (the target rank plus oversampling).  The same sketch is
 * used at every rounding; a call whose angular size differs from nang fails with TT_ERR_SHAPE. */
tt_status tt_context_set_sketch(tt_context *ctx, const double *omega_dev, int32_t nang, int32_t ell);

/* Kernels of the tall-skinny QR over the merged core (the first sweep of the rounding, Sec. 3.1
 * footnote), per pass shape: for passes of ncap columns at precision prec (TT_PREC_FP64: FP64
 * passes; TT_PREC_MIXED: FP32 passes):
 *   variant 0: one thread per column (the default; at most 256 threads, i.e. ncap <= 256);
 *   variant 1: four lanes per column, each holding a quarter of the rows of a block (4 ncap <= 1024);
 *   variant 2: FP32 only, one thread per column over 32-row blocks with registers held so that
 *              four CTAs share an SM (ncap <= 160);
 *   variant 3: FP32 only, blocked: 256-row blocks (a row per thread) held in tensor memory,
 *              32-column panels factored with block-wide reductions and their compact-WY block
 *              reflector applied to the trailing columns at once; one CTA per SM (ncap <= 224).
 * A variant that cannot take the shape runs variant 0.  The variant picks the leaf kernel; the
 * merge tree over the leaves' R factors runs four lanes per column in every variant when
 * 4 ncap <= 1024.  leaves = cap on the TSQR leaves: <= 0 gives the default wave (2 CTAs per SM for
 * FP64, 3 for FP32); larger caps are clamped to 6 per SM.  The choice changes the order of
 * rounding errors only.  ncap <= 0 clears every entry.  tt_context_get_tsqr reports what a pass
 * of ncap columns would run.  The paper has no counterpart: these are launch-shape choices. */
tt_status tt_context_set_tsqr(tt_context *ctx, tt_precision prec, int32_t ncap, int32_t variant, int32_t leaves);
tt_status tt_context_get_tsqr(const tt_context *ctx, tt_precision prec, int32_t ncap, int32_t *variant,
                              int32_t *leaves);

/* Launch geometry of the tall-skinny QR over the merged core (the first sweep of the rounding,
 * Sec. 3.1 footnote) for a pass of ncap columns and nrows rows at precision prec with TSQR
 * variant `variant` (as tt_context_set_tsqr; variants that cannot take the shape are reported as
 * the one that runs), max_leaves the leaf cap in force (<= 0: none), on a device with num_sms
 * SMs where per_sm leaf CTAs are resident at once (what the occupancy query reports for the leaf
 * kernel).  A host computation by the functions the launches use: it needs no GPU and touches
 * no device.  out[0..nout) (nout <= 12): [0] leaves, [1] rows per leaf (the last leaf takes the
 * ragged rest), [2] rows per block, [3] leaf threads per CTA, [4] leaf dynamic shared-memory
 * bytes, [5] merge threads per CTA, [6] merge dynamic shared-memory bytes, [7] merge levels,
 * [8] and [9] doubles of the two R-factor buffers the step's workspace holds (leaf output and
 * merge levels alternate between them), [10] the variant that runs, [11] rows of the second
 * factor a merge absorbs at a time.  TT_ERR_UNSUPPORTED for a
 * shape no kernel takes (too many columns, or per_sm < 1 for the row-split leaf).  The paper has
 * no counterpart: these are launch-shape choices. */
tt_status tt_tsqr_geometry(tt_precision prec, int32_t variant, int32_t ncap, int64_t nrows, int32_t num_sms,
                           int32_t per_sm, int32_t max_leaves, int64_t *out, int32_t nout);

/* Autotune the TSQR choice (tt_context_set_tsqr) of the two passes of tt_step for state I with
 * this plan, tolerance and precision: the transport-sum pass ((2 d_X + 1) rcap_1 + n_b columns)
 * and the source pass (rcap_1 + 1 columns).  Each candidate (variant x leaf cap, one pass at a
 * time, the other at its best so far) is timed with CUDA events over `steps` (1..64) tt_steps,
 * after one untimed step, on a device copy of I; I itself is not modified, and a coupled plan's
 * material temperature is restored afterwards.  The fastest entries are stored in the context.
 * Synchronous; allocates the copy with cudaMalloc, so never under stream capture (TT_ERR_ARG).
 * chosen[4] (host, nullable): variant and leaf cap of the transport pass, then of the source
 * pass; ms[2] (host, nullable): ms per step with the defaults and with the choice.  Only the
 * TSQR rounding has these passes (TT_ERR_UNSUPPORTED under another tt_rounding).  The paper has
 * no counterpart. */
tt_status tt_autotune(tt_context *ctx, const tt_plan *plan, const tt_tensor *I, double tol, int32_t rmax,
                      tt_precision prec, int32_t steps, int32_t *chosen, float *ms);

/* Synchronise the context stream and report, per tt_timer category, the summed kernel time
 * in milliseconds (ms[TT_TIMER_COUNT], nullable) and the number of kernel launches
 * (launches[TT_TIMER_COUNT], nullable) since the last reset; reset != 0 clears both. */
tt_status tt_context_counters(tt_context *ctx, double *ms, int64_t *launches, int reset);

/* Synchronise the context stream and copy iteration statistics since the last reset into
 * out[0..n) (n <= 6): [0] the largest number of Jacobi sweeps of one SVD, [1] the number of
 * Jacobi SVDs, [2] their total number of sweeps (device-side counts); [3] tt_step graph replays,
 * [4] graph captures, [5] captures that failed, after which the step ran eagerly (host-side
 * counts of tt_context_set_graphs).  reset != 0 clears them. */
tt_status tt_context_diagnostics(tt_context *ctx, int64_t *out, int n, int reset);

/* Limits of the bounded device-side iterations of a context, for tests of the failure paths (the
 * paper has no counterpart).  jacobi_sweeps > 0 caps the sweeps of every FP64 one-sided Jacobi
 * SVD (default 40): an SVD still rotating at the cap latches TT_ERR_TIMEOUT.  barrier_spins > 0
 * caps the spins of one wait at the grid-wide barrier of a cooperative kernel (default 2^24 spins
 * of about 64 ns each).  barrier_extra > 0 makes every such barrier wait for that many arrivals
 * beyond the grid, which never come, so every wait runs out: the kernel latches TT_ERR_TIMEOUT,
 * all its CTAs leave, and the context stays usable (the next cooperative launch starts a fresh
 * barrier).  0 restores a default.  Synchronous (one small host-to-device copy); a step graph
 * captured earlier reads the new limits when it replays. */
tt_status tt_context_set_limits(tt_context *ctx, int32_t jacobi_sweeps, int64_t barrier_spins,
                                int32_t barrier_extra);

/* Synchronise the context stream, then return and clear the latched device status. */
tt_status tt_sync(tt_context *ctx);

/* Workspace the context needs for tt_step / tt_round on tensors of capacity `x` with
 * problem `plan` (NULL for tt_round only). */
tt_status tt_workspace_query(tt_context *ctx, const tt_plan *plan, const tt_tensor *x,
                             tt_precision prec, size_t *bytes);

/* Build the per-step coefficients of a problem on the device: angular quadrature (Sec. 4
 * preamble: Gauss-Legendre mu for the slab, lat/long midpoint rule otherwise), group
 * emission epsilon_f(T) per merged row by Planck integrals (Eqs. Ttoeps1-2, evaluated with
 * polylogarithm-type series as at the end of Sec. 2.1), the backward-Euler coefficients
 * c*dt*rho*kappa of Eq. (discRTsource), inflow spectra and the angular factors of the 2 d_X
 * rank-1 transport operators (Appendix A).  The plan copies what it needs; the problem's
 * device arrays may be freed after the call returns and the stream has run. */
tt_status tt_plan_create(tt_context *ctx, const tt_problem *prob, tt_plan **plan);
tt_status tt_plan_destroy(tt_plan *plan);

/* Device arrays owned by the plan (valid until tt_plan_destroy), for inspection:
 * which = 0: emission per row (N_Z), 1: solid-angle weights (N_theta*N_phi),
 *         2: mu nodes (N_theta), 3: phi nodes (N_phi), 4: c*dt*rho*kappa_a per row,
 *         5: c*dt*rho*kappa_s per row, 6: inflow spectra [6][G] (0 for vacuum faces),
 *         7: material temperature per cell (N_X; advanced by tt_step when coupled),
 *         8: T^dagger of the last coupled step per cell (N_X; TT_ERR_ARG when not coupled). */
tt_status tt_plan_array(const tt_plan *plan, int which, const double **ptr, int64_t *len);

/* y <- alpha * x + y by rank concatenation (TT addition, Sec. 3.1): ranks add.
 * x and y must have equal d and mode sizes.  If a summed rank exceeds y's capacity the
 * call leaves y unchanged and latches TT_ERR_CAPACITY. */
tt_status tt_axpy(tt_context *ctx, double alpha, const tt_tensor *x, tt_tensor *y);

/* *out_dev <- <x, y> (Frobenius inner product), FP64 accumulation, deterministic order: the
 * full contraction of two TTs among the basic TT operations the solver relies on (Sec. 3.1:
 * addition, integration, rounding), which gives the Frobenius norms behind the relative errors
 * of Sec. 5.4 (||x - y||^2 = <x,x> - 2<x,y> + <y,y>).  First core: W1 = Z_x^T Z_y (a reduction
 * over the merged rows), then the small cores.  x and y: equal d, mode sizes and dtype (else
 * TT_ERR_SHAPE).  out_dev is a device double owned by the caller, written asynchronously on the
 * context's stream. */
tt_status tt_dot(tt_context *ctx, const tt_tensor *x, const tt_tensor *y, double *out_dev);

/* In-place SVD-based rounding (Sec. 3.1 footnote; Oseledets 2011): left-to-right QR
 * orthogonalisation, then right-to-left truncated SVD with delta = rel_tol*||x||/sqrt(d-1);
 * each bond keeps the smallest rank whose discarded tail is <= delta, capped at rmax
 * (rel_tol = 0 keeps the full rank of every unfolding).  rmax must not exceed x's rank
 * capacities.  A zero tensor rounds to ranks 1 with zero cores. */
tt_status tt_round(tt_context *ctx, tt_tensor *x, double rel_tol, int32_t rmax, tt_precision prec);

/* out <- the unrounded forward-Euler upwind transport update of `in` (Appendix A: the sum
 * of the solution, its n = 2 d_X rank-1 operator images and the Dirichlet inflow tensor),
 * materialised with ranks (n+1) r + n_b where n_b counts operators whose upwind face has
 * inflow.  out must have the same d and mode sizes and enough capacity, else
 * TT_ERR_CAPACITY is latched and out is left unchanged. */
tt_status tt_apply_transport(tt_context *ctx, const tt_plan *plan, const tt_tensor *in, tt_tensor *out);

/* One time step in place (end of Sec. 3.1): transport, round, source (Eq. discRTsource at
 * fixed T), round, all on the device without materialising the transport sum.  Under
 * TT_ROUND_TSQR the QR passes over the merged core take at most 256 columns:
 * (2 d_X + 1) rcap_1 + n_b <= 256 (n_b inflow faces), else TT_ERR_UNSUPPORTED before the state
 * is touched (tt_round: rcap_1 <= 256).
 * energy_dev (nullable, device double[4]) receives the radiation energy before and after
 * the step, the energy of the post-transport tensor, and the absorption-emission exchange
 * (4 pi / c) sum dV c dt rho kappa_a (eps - J^{m+1}). */
tt_status tt_step(tt_context *ctx, const tt_plan *plan, tt_tensor *I, double tol, int32_t rmax,
                  tt_precision prec, double *energy_dev);

/* Internal delta-ranks of the merged core (Sec. 5.2): r1 (frequency-leading) and r1x
 * (space-leading) of reshape(Z, [N_nu, N_X r]) and reshape(Z, [N_X, N_nu r]) at relative tolerance
 * delta_rel (the delta-SVD of Sec. 5.4: smallest rank whose discarded singular values have a
 * Frobenius norm <= delta_rel |Z|).  x must be a rounded state (angular cores right-orthonormal,
 * as tt_round and tt_step leave them), so that the local errors are global ones.  Synchronous:
 * ranks[2] (host) receives r1, r1x; sigma_nu / sigma_x (host, nullable) receive up to nsigma_*
 * singular values, decreasing.  The singular values come from FP64 Gram matrices (N_nu x N_nu and
 * N_nu rcap x N_nu rcap, at most 4096) and Jacobi eigen-solves, so values below about 1e-8 of the
 * largest are not resolved.  TT_ERR_UNSUPPORTED beyond 4096.  The status latched on the device
 * during the call is returned (and cleared): TT_ERR_TIMEOUT when a Jacobi solve reached its sweep
 * cap, with the ranks of its last sweep still written. */
tt_status tt_internal_ranks(tt_context *ctx, const tt_plan *plan, const tt_tensor *x, double delta_rel,
                            int32_t *ranks, double *sigma_nu, int64_t nsigma_nu, double *sigma_x, int64_t nsigma_x);

/* ---- Batched stepping of independent problems (many plans and states, one CUDA graph) ----
 * Each problem's step is the tt_step of the paper's step-then-truncate scheme (Sec. 2.1 source
 * update, Sec. 3.1 rounding, Appendix A transport); the batching itself has no counterpart in
 * the paper.  A batch steps nprob independent problems together: plans[i] with state states[i] (descriptor
 * copied; the cores stay owned by the caller and must stay allocated until tt_batch_destroy),
 * tolerance tol[i] and rank cap rmax[i], all at precision prec.  Each problem runs exactly the
 * launch sequence of tt_step on its own device control block and workspace region (sized once
 * here by dry runs and allocated as one buffer); problems are spread over nstreams streams
 * (<= 0: 128), largest first onto the least-loaded stream, so that the latency-bound small-core
 * phases of different problems overlap.  The cooperative Jacobi of the FP64 path runs as a
 * single CTA per problem inside a batch (concurrent problems never wait on one another).
 * Same argument checks as tt_step (TT_ERR_ARG, TT_ERR_SHAPE, TT_ERR_CAPACITY). */
typedef struct tt_batch tt_batch;
tt_status tt_batch_create(tt_context *ctx, int32_t nprob, const tt_plan *const *plans, const tt_tensor *states,
                          const double *tol, const int32_t *rmax, tt_precision prec, int32_t nstreams,
                          tt_batch **out);
/* Advance every problem of the batch by nsteps time steps, asynchronously on the context stream.
 * The first batched step runs eagerly (every kernel loaded and configured outside any capture),
 * the next one is captured as a CUDA graph (so neither may be made under an outer stream
 * capture), and every later step is a replay of that graph.  Device-detected errors are
 * latched per problem and reported by tt_batch_sync. */
tt_status tt_batch_step(tt_batch *b, int32_t nsteps);
/* Synchronise the context stream; status_out[nprob] (nullable) receives each problem's latched
 * status; returns the first non-OK one. */
tt_status tt_batch_sync(tt_batch *b, int32_t *status_out);
/* Kernel launches in one captured batched step (-1 before the graph is captured), total
 * workspace bytes, streams used.  Each pointer is nullable. */
tt_status tt_batch_info(const tt_batch *b, int64_t *launches_per_step, size_t *workspace_bytes, int32_t *nstreams);
tt_status tt_batch_destroy(tt_batch *b);

/* *out_dev <- <x, y> like tt_dot, for callers that cannot allocate device memory: programs
 * that reserve a fixed device-memory budget up front and may not grow it, and code that must
 * not block while it runs (a real-time loop, a host callback), where cudaMalloc/cudaFree can
 * synchronise the device.  The paper has no counterpart; this is a deployment variant of
 * tt_dot.  It takes a stream of the CURRENT device instead of a context and allocates
 * nothing: its scratch is one file-scope device array of 4 MiB (2^19 doubles) per device,
 * held from the first call on that device until the process exits.  The first call on a
 * device (in each CUDA context) looks up the array's device address; that look-up loads this part
 * of the library on the device, which may block and reserves the array there, so make that first
 * call before any stream capture on the device and outside any region that must not allocate or
 * block (e.g. one warm-up call at start-up).  If the row chunking cannot fit in the 4 MiB (rank capacities with
 * rcap_1(x)*rcap_1(y)*3 + (rcap_1(x)+rcap_1(y))*n_1*n_2 beyond 2^19 doubles) the call returns
 * TT_ERR_WORKSPACE and launches nothing.  Every call writes all the scratch it reads, so no
 * clearing is needed between calls, but all calls on a device share the one array: calls
 * that overlap on the GPU (several streams, or several host threads) race and give wrong
 * results.  Same arguments, layout and errors as tt_dot otherwise. */
tt_status tt_dot_noalloc(void *cuda_stream, const tt_tensor *x, const tt_tensor *y, double *out_dev);

/* D <- A B^T on the tensor cores (tcgen05, kind::tf32 with FP32 accumulation): A (M x K), B (N x K)
 * and D (M x N), row-major FP32 device arrays owned by the caller, on stream cuda_stream of the
 * current device.  passes = 3: split TF32 (each operand x = hi + lo, hi = x rounded to TF32, and
 * hi_a hi_b + hi_a lo_b + lo_a hi_b summed in FP32: products to about 2^-22 relative); passes = 1:
 * plain TF32 (about 2^-11).  N a multiple of 16 with 16 <= N <= 256; M, K >= 1.  status_dev
 * (nullable device int32) latches TT_ERR_TIMEOUT if a bounded wait for the tensor cores runs out.
 * The paper has no counterpart: this is the product the mixed path's tensor-core kernels use, as a
 * plain call, so that its arithmetic can be checked against an FP64 product. */
tt_status tt_tc_gemm(void *cuda_stream, int64_t M, int32_t N, int32_t K, const float *A, const float *B, float *D,
                     int32_t passes, int32_t *status_dev);

/* Peak probe of one arithmetic pipe, timed with CUDA events on cuda_stream (synchronous):
 * kind 0 = FP64 FMA, 1 = FP32 FMA (8 independent chains per thread, every SM full), 2 = the
 * tensor pipe in kind::tf32 (one CTA per SM issuing `iters` MMAs of 128 x 256 x 8 on operands
 * resident in shared memory).  *flops receives the flops counted (2 per FMA), *ms the time.  The
 * paper has no counterpart: these are the measured denominators of the roofline fractions. */
tt_status tt_peak_probe(void *cuda_stream, int32_t kind, int64_t iters, double *flops, float *ms);

/* Radiation energy density per merged row, E_f = (4 pi / c) J_f (Sec. 2), into the
 * device array out_dev[N_Z]. */
tt_status tt_energy_density(tt_context *ctx, const tt_plan *plan, const tt_tensor *x, double *out_dev);

#ifdef __cplusplus
}
#endif
#endif /* TT_H */
