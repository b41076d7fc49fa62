// Host orchestration of the time step and of the TT primitives on the device.  No host
// synchronisation happens inside any of these calls: ranks and truncation decisions stay in
// device memory (tensor rank arrays and the context control block).
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "bigpass.cuh"
#include "gram.cuh"
#include "rand.cuh"
#include "small.cuh"
#include "step.cuh"
#include "tc_update.cuh"
#include "tsqr_blk.cuh"
#include "tsqr_rs.cuh"
#include "tune.cuh"

namespace ttk {
namespace {

constexpr double kPi = 3.14159265358979323846;
// rows per update tile: FP32 tiles of 64 rows (two output rows per thread), FP64 of 32
template <typename T>
struct UpdTM {
  static constexpr int value = sizeof(T) == 8 ? 32 : 64;
};
// rows per TSQR block over the merged core: FP64 registers hold 32 rows per column, FP32 64
template <typename T>
struct BigBR {
  static constexpr int value = sizeof(T) == 8 ? 32 : 64;
};
// leaves of the TSQR over the merged core per SM: FP64 R factors fill ~103 KB of shared memory
// (two CTAs per SM), FP32 ones ~52 KB (three CTAs per SM, register-limited, hide the
// reflector latency)
template <typename T>
struct BigLeaves {
  static constexpr int per_sm = sizeof(T) == 8 ? 2 : 3;
};

// u = W vJ (R x k times k): J* of the rounded transport update is A u row by row.
__global__ void k_wvj(int R, int k, const double* __restrict__ W, const double* __restrict__ vJ,
                      double* __restrict__ u) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= R) return;
  double s = 0.0;
  for (int j = 0; j < k; ++j) s += W[(size_t)c * k + j] * vJ[j];
  u[c] = s;
}

// J*[k] = sum_c A[k][c] u[c] over the (virtual) sum's live columns, one warp per row (FP64).
template <class Src>
__global__ void k_jstar(Src src, LivePattern lp, long nrows, const double* __restrict__ u,
                        double* __restrict__ jstar) {
  const int ncap = lp.ncap();
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long k = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); k < nrows; k += warps) {
    double s = 0.0;
    for (int c = lane; c < ncap; c += 32)
      if (lp.live(c, r)) s += src.load(src.col(c), k) * u[c];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) jstar[k] = s;
  }
}

// B0 of the transport sum: block t = 0 is the right part of the state, block t = 1..nterm is
// the same right part scaled by the operator's angular factors f1_t(l) f2_t(p), and each
// inflow column carries the factors alone (Appendix A: rank-1 operators and the rank-1
// Dirichlet tensor).
__global__ void k_b0_transport(int rcap, int nterm, int nbc, int n1, int n2, const double* __restrict__ Bbase,
                               const double* __restrict__ fac1, const double* __restrict__ fac2,
                               const int* __restrict__ bc_term_dev, double* __restrict__ B0) {
  const int nang = n1 * n2;
  const int R = (nterm + 1) * rcap + nbc;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)R * nang;
       idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / nang);
    const int i = (int)(idx - (long)c * nang);
    const int l = i / n2, p = i - (i / n2) * n2;
    const int t = c / rcap;
    double v;
    if (t == 0) {
      v = Bbase[(size_t)c * nang + i];
    } else if (t <= nterm) {
      const int q = c - t * rcap;
      v = fac1[(t - 1) * n1 + l] * fac2[(t - 1) * n2 + p] * Bbase[(size_t)q * nang + i];
    } else {
      const int tt = bc_term_dev[c - (nterm + 1) * rcap];
      v = fac1[tt * n1 + l] * fac2[tt * n2 + p];
    }
    B0[idx] = v;
  }
}

// B0 of the source sum [diag(1/(1+a+s)) Z_new, g]: the new right part, then a row of ones
// (the isotropic rank-1 term).
__global__ void k_b0_source(int rcap, int nang, const double* __restrict__ Bnew, double* __restrict__ B0) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)(rcap + 1) * nang;
       idx += (long)gridDim.x * blockDim.x)
    B0[idx] = (idx < (long)rcap * nang) ? Bnew[idx] : 1.0;
}

template <typename S>
__global__ void k_commit(int d, int n1, int n2, int K1, int K2, const double* __restrict__ c1,
                         const double* __restrict__ c2, S* __restrict__ core1, S* __restrict__ core2,
                         const DevCtrl* ctrl, int* rank) {
  const long tot1 = (long)K1 * n1 * (d == 3 ? K2 : 1);
  const long tot2 = (d == 3) ? (long)K2 * n2 : 0;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot1 + tot2;
       idx += (long)gridDim.x * blockDim.x) {
    if (idx < tot1)
      core1[idx] = (S)c1[idx];
    else
      core2[idx - tot1] = (S)c2[idx - tot1];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    rank[1] = ctrl->k[0];
    if (d == 3) rank[2] = ctrl->k[1];
  }
}

__global__ void k_save_ranks(DevCtrl* ctrl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctrl->k[2] = ctrl->k[0];
    ctrl->k[3] = ctrl->k[1];
  }
}

// per-CTA partial sums of Z[k,:] . v (mean intensity J per row summed)
template <typename S>
__global__ void k_rowdot_partials(long nrows, int ld, int ncol, const S* __restrict__ Z, const double* __restrict__ v,
                                  double* __restrict__ partials, double* __restrict__ per_row, double row_scale) {
  __shared__ double red[33];
  double s = 0.0;
  const long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k < nrows) {
    double j = 0.0;
    for (int q = 0; q < ncol; ++q) j += (double)Z[k * ld + q] * v[q];
    s = j;
    if (per_row) per_row[k] = row_scale * j;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0 && partials) partials[blockIdx.x] = s;
}

__global__ void k_energy_pack(const double* __restrict__ e_before, const double* __restrict__ e1,
                              const double* __restrict__ e2, double scale, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    out[0] = e_before ? scale * e_before[0] : 0.0;
    out[1] = scale * e2[0];
    out[2] = scale * e1[0];
    out[3] = scale * e1[1];
  }
}

}  // namespace

template <typename S>
static void fill_stencil(SrcStencil<S>& src, const tt_plan* p, const S* Z, int rcap1) {
  src.Z = Z;
  src.ldz = rcap1;
  src.rcap = rcap1;
  src.nterm = p->nterm;
  src.G = p->G;
  for (int a = 0; a < 3; ++a) {
    src.ext[a] = p->ext[a];
    src.stride[a] = p->stride[a];
  }
  for (int t = 0; t < kMaxTerms; ++t) {
    src.lam[t] = (t < p->nterm) ? p->lam[p->term_axis[t]] : 0.0;
    src.axis[t] = (t < p->nterm) ? p->term_axis[t] : 0;
    src.w[t] = (t < p->nterm) ? p->term_w[t] : 1;
    src.bc_term[t] = (t < p->nbc) ? p->bc_term[t] : 0;
  }
  src.bcval = p->bcval;
  src.nax = p->ndim;
}

// Launches the persistent update pass; *grid_out (if given) receives the number of CTAs, i.e.
// of energy partial pairs written.
template <class Src>
struct StencilOf {
  static constexpr bool value = false;
};
template <typename S>
struct StencilOf<SrcStencil<S>> {
  static constexpr bool value = true;
};

// FP32 passes over the stencil sum run from staged row blocks with combined weights
// (k_update_blk) when the rows can be staged (16-byte granules) and the tile fits; returns
// TT_ERR_UNSUPPORTED (nothing launched) otherwise.
template <class Epi, typename S>
static tt_status launch_update_blk(cudaStream_t s, int num_sms, const SrcStencil<S>& src, LivePattern lp,
                                   long nrows, const double* W, int kcap, const Epi& epi, double* partials,
                                   long* grid_out, int cat) {
  constexpr int TM = UpdTM<float>::value;
  if (((size_t)src.ldz * sizeof(S)) % 16 != 0 || ((size_t)src.Z % 16) != 0 || src.nax < 1 || src.rcap != lp.rcap)
    return TT_ERR_UNSUPPORTED;
  const size_t smem = update_blk_smem_bytes<TM, S>(src, update_kpad<Epi>(kcap), lp.nextra);
  if (smem > 227 * 1024) return TT_ERR_UNSUPPORTED;
  auto kern = k_update_blk<TM, S, Epi>;
  if (const tt_status a = smem_optin(kern, smem); a != TT_OK) return a;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem) != cudaSuccess || occ < 1) occ = 1;
  const long ntiles = (nrows + TM - 1) / TM;
  long grid = (long)num_sms * occ;
  if (grid > ntiles) grid = ntiles > 0 ? ntiles : 1;
  if (grid_out) *grid_out = grid;
  TimerScope scope(cat, s);
  kern<<<(unsigned)grid, 256, smem, s>>>(src, lp, nrows, W, kcap, epi, partials); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// The update pass of a rounding: the tensor-core kernel (ctx->tensor_cores, FP32 storage of the
// stencil source) where it takes the pass, else the FP32 kernel over staged row blocks, else the
// generic kernel.
template <typename T, class Src, class Epi>
static tt_status launch_update(const tt_context* ctx, cudaStream_t s, int num_sms, const Src& src, LivePattern lp,
                               long nrows, const double* W, int kcap, const Epi& epi, double* partials,
                               long* grid_out, int cat = kUpdate) {
  constexpr int TM = UpdTM<T>::value;
  if constexpr (sizeof(T) == 4 && std::is_same<Src, SrcStencil<float>>::value) {
    if (ctx->tensor_cores && update_tc_fits(src, lp, nrows, kcap, ctx->smem_optin))
      return launch_update_tc(s, num_sms, src, lp, nrows, W, kcap, epi, partials, grid_out, cat);
  }
  if constexpr (sizeof(T) == 4 && StencilOf<Src>::value) {
    const tt_status bst = launch_update_blk(s, num_sms, src, lp, nrows, W, kcap, epi, partials, grid_out, cat);
    if (bst != TT_ERR_UNSUPPORTED) return bst;
  }
  // Staging the stencil rows takes shared memory: keep it when it costs no resident CTA or
  // still leaves two per SM.
  Src src2 = src;
  set_staged(src2, 1);
  size_t stage = update_stage_bytes(src2, TM);
  if (stage > 0) {
    const size_t s1 = update_smem_bytes<T, TM, Src, Epi>(lp.ncap(), kcap, stage);
    const size_t s0 = update_smem_bytes<T, TM, Src, Epi>(lp.ncap(), kcap, 0);
    const int o1 = (int)((228 * 1024) / (s1 + 1024)), o0 = (int)((228 * 1024) / (s0 + 1024));
    if (s1 > 227 * 1024 || (o1 < o0 && o1 < 2)) {
      set_staged(src2, 0);
      stage = 0;
    }
  }
  const size_t smem = update_smem_bytes<T, TM, Src, Epi>(lp.ncap(), kcap, stage);
  if (smem > 227 * 1024) return TT_ERR_UNSUPPORTED;
  const long grid = update_grid<T, TM, Src, Epi>(num_sms, lp.ncap(), kcap, nrows, stage);
  if (grid < 1) return TT_ERR_CUDA;
  if (grid_out) *grid_out = grid;
  TimerScope scope(cat, s);
  k_update<T, TM, Src, Epi><<<(unsigned)grid, 256, smem, s>>>(src2, lp, nrows, W, kcap, epi, partials); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// Cap on the TSQR leaves over the merged core: a full wave of resident CTAs, or the context's
// own cap (a batch gives each problem a share of the GPU in proportion to its rows).
template <typename T>
inline int leaf_cap(const tt_context* ctx) {
  const int full = BigLeaves<T>::per_sm * ctx->num_sms;
  return (ctx->tsqr_leaf_cap > 0 && ctx->tsqr_leaf_cap < full) ? ctx->tsqr_leaf_cap : full;
}

// TSQR kernels and leaf cap for an ncap-column pass (the context's tuned entry, if any).
template <typename T>
inline TsqrCfg tsqr_cfg(const tt_context* ctx, int ncap) {
  return resolve_tsqr(ctx, (int)sizeof(T), ncap, leaf_cap<T>(ctx));
}

// Leaves that any TSQR variant may launch over nrows rows (workspace bound): the 32-row blocks
// of the smallest variant.
template <typename T>
inline long tsqr_leaf_bound(int num_sms, int ncap, long nrows, int max_leaves) {
  return tsqr_max_leaves<T, 32>(num_sms, ncap, nrows, max_leaves);
}

template <typename T, class Src>
inline tt_status run_tsqr_cfg(const TsqrCfg& cfg, cudaStream_t s, int num_sms, const Src& src, LivePattern lp,
                              long nrows, double* ws_a, double* ws_b, double** Rfinal, int leaf_cat = kTsqrLeaf) {
  constexpr int BR = BigBR<T>::value;
  if (cfg.variant == kTsqrRowSplit)
    return run_tsqr_rs<T, BR, 4>(s, num_sms, src, lp, nrows, cfg.leaves, ws_a, ws_b, Rfinal, leaf_cat);
  if constexpr (sizeof(T) == 4) {
    if (cfg.variant == kTsqrColumnDense)
      return run_tsqr<T, 32, 160, 4>(s, num_sms, src, lp, nrows, cfg.leaves, ws_a, ws_b, Rfinal, leaf_cat);
    if (cfg.variant == kTsqrBlocked)
      return run_tsqr_blk(s, num_sms, src, lp, nrows, cfg.leaves, ws_a, ws_b, Rfinal, leaf_cat);
  }
  return run_tsqr<T, BR>(s, num_sms, src, lp, nrows, cfg.leaves, ws_a, ws_b, Rfinal, leaf_cat);
}

// Workspace carving shared by dry runs (size queries) and real runs.
struct RoundBufs {
  double* tsqr_a;
  double* tsqr_b;
  double* Bbase;
  double* B0;
  double* W;
  double* core1;
  double* core2;
  double* Bnew;
  double* vJ;
};

template <typename T>
static RoundBufs take_round_bufs(Bump& ws, int num_sms, int max_leaves, int d, int R, long nrows, int n1, int n2,
                                 int K1, int K2, int rcapin1) {
  RoundBufs b;
  const long L = tsqr_leaf_bound<T>(num_sms, R, nrows, max_leaves);
  b.tsqr_a = ws.take<double>((size_t)L * R * R);
  b.tsqr_b = ws.take<double>((size_t)((L + 1) / 2) * R * R);
  b.Bbase = ws.take<double>((size_t)rcapin1 * n1 * n2);
  b.B0 = ws.take<double>((size_t)R * n1 * n2);
  b.W = ws.take<double>((size_t)R * K1);
  b.core1 = ws.take<double>((size_t)K1 * n1 * (d == 3 ? K2 : 1));
  b.core2 = ws.take<double>((size_t)(d == 3 ? K2 * n2 : 1));
  b.Bnew = ws.take<double>((size_t)K1 * n1 * n2);
  b.vJ = ws.take<double>(K1);
  return b;
}

// Randomized factor RZ (R x R; rows >= l zero) of the source's columns A: Y = A (B0 omega) by the
// update pass, Householder TSQR of Y, Q = Y R_Y^{-1} in place, C = Q^T A by the cross product.
// Takes its workspace from `ws` in dry runs too (same order), launches nothing then.
template <typename S, typename T, class Src>
static tt_status randomized_factor(tt_context* ctx, cudaStream_t s, const Src& src, LivePattern lp, long N,
                                   const double* B0, int nang, Bump& ws, double** RZ_out, int timer_cat) {
  const int R = lp.ncap();
  if (!ctx->sketch) return TT_ERR_ARG;
  if (ctx->sketch_nang != nang) return TT_ERR_SHAPE;
  const int l = ctx->sketch_ell < R ? ctx->sketch_ell : R;
  double* Op = ws.take<double>((size_t)R * l);
  S* Y = ws.take<S>((size_t)N * l);
  const TsqrCfg ycfg = tsqr_cfg<T>(ctx, l);
  const long L = tsqr_leaf_bound<T>(ctx->num_sms, l, N, ycfg.leaves);
  double* ta = ws.take<double>((size_t)L * l * l);
  double* tb = ws.take<double>((size_t)((L + 1) / 2) * l * l);
  const int nbi = (l + 63) / 64, nbj = (R + 63) / 64;
  long nsplit = ((long)ctx->num_sms * 3 * 8 + nbi * nbj - 1) / (nbi * nbj);
  const long maxsplit = (N + kCrossTM - 1) / kCrossTM;
  if (nsplit > maxsplit) nsplit = maxsplit;
  if (nsplit < 1) nsplit = 1;
  long rps = (N + nsplit - 1) / nsplit;
  rps = ((rps + kCrossTM - 1) / kCrossTM) * kCrossTM;
  nsplit = (N + rps - 1) / rps;
  if (nsplit < 1) nsplit = 1;
  double* part = ws.take<double>((size_t)nsplit * nbi * nbj * 64 * 64);
  double* RZ = ws.take<double>((size_t)R * R);
  constexpr bool kCorrect = sizeof(T) == 4;  // FP32 TSQR of the sketch: project with Q's own Gram
  double* G = kCorrect ? ws.take<double>((size_t)l * l) : nullptr;
  double* partG = kCorrect ? ws.take<double>((size_t)nsplit * 64 * 64) : nullptr;
  *RZ_out = RZ;
  if (ws.dry) return TT_OK;
  small_gemm<double, double>(s, R, l, nang, B0, nang, 1, ctx->sketch, ctx->sketch_ell, 1, Op, l, nullptr, nullptr);
  tt_status st = launch_update<T>(ctx, s, ctx->num_sms, src, lp, N, Op, l, EpiPlain<S>{Y, l, &ctx->ctrl->status}, nullptr, nullptr);
  if (st != TT_OK) return st;
  double* RY = nullptr;
  st = run_tsqr_cfg<T>(ycfg, s, ctx->num_sms, SrcRows<S>{Y, l}, LivePattern{nullptr, l, 1, 0}, N, ta, tb, &RY,
                       timer_cat);
  if (st != TT_OK) return st;
  const long sb = (N + 127) / 128 < 4096 ? (N + 127) / 128 : 4096;
  k_rand_solve<<<(unsigned)sb, 128, sizeof(double) * (size_t)l * l, s>>>(
      N, l, RY, sizeof(S) == 4 ? (float*)Y : nullptr, sizeof(S) == 8 ? (double*)Y : nullptr); count_launch();
  k_cross_tiles<SrcRows<S>, Src><<<dim3((unsigned)nsplit, (unsigned)(nbi * nbj)), 256, 0, s>>>(
      SrcRows<S>{Y, l}, l, src, lp, N, rps, nbj, part); count_launch();
  k_cross_reduce<<<(unsigned)(((long)R * R + 255) / 256), 256, 0, s>>>(l, R, (int)nsplit, nbi, nbj, part, RZ);
  count_launch();
  if (kCorrect) {
    k_cross_tiles<SrcRows<S>, SrcRows<S>><<<dim3((unsigned)nsplit, 1u), 256, 0, s>>>(
        SrcRows<S>{Y, l}, l, SrcRows<S>{Y, l}, LivePattern{nullptr, l, 1, 0}, N, rps, 1, partG); count_launch();
    k_cross_reduce<<<(unsigned)(((long)l * l + 255) / 256), 256, 0, s>>>(l, l, (int)nsplit, 1, 1, partG, G);
    count_launch();
    k_rand_correct<<<1, 128, 0, s>>>(l, R, G, RZ); count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

template <typename S, typename T>
tt_status round_impl(tt_context* ctx, tt_tensor* x, double tol, int rmax, Bump& ws) {
  cudaStream_t s = ctx->stream;
  const int d = x->d;
  const long N = x->n[0];
  const int n1 = x->n[1], n2 = (d == 3) ? x->n[2] : 1;
  const int K1 = x->rcap[1], K2 = (d == 3) ? x->rcap[2] : 1;
  LivePattern lp{x->rank + 1, K1, 1, 0};
  const int R = lp.ncap();
  const TsqrCfg cfg = tsqr_cfg<T>(ctx, R);
  RoundBufs b = take_round_bufs<T>(ws, ctx->num_sms, cfg.leaves, d, R, N, n1, n2, K1, K2, K1);
  SmallJob job{};
  job.d = d;
  job.n1 = n1;
  job.n2 = n2;
  job.nrowsZ = N;
  job.lp = lp;
  job.r2_ptr = (d == 3) ? x->rank + 2 : nullptr;
  job.r2_nblk = 1;
  job.r2_nextra = 0;
  job.tol = tol;
  job.rmax = rmax;
  job.K1cap = K1;
  job.K2cap = K2;
  job.B0 = b.Bbase;
  job.domega = nullptr;
  job.W = b.W;
  job.core1 = b.core1;
  job.core2 = b.core2;
  job.Bnew = b.Bnew;
  job.vJ = b.vJ;
  job.ctrl = ctx->ctrl;
  job.coop_grid_max = ctx->coop_grid_max;
  job.mixed = (sizeof(T) == 4);
  double* domega_ones = ws.take<double>((size_t)n1 * n2);
  job.domega = domega_ones;
  double* RZ = nullptr;
  if (!ws.dry) {
    right_part<S>(s, d, K1, n1, K2, n2, (const S*)x->core[1], d == 3 ? (const S*)x->core[2] : nullptr, b.Bbase);
    cudaMemsetAsync(domega_ones, 0, sizeof(double) * (size_t)n1 * n2, s);
  }
  if (ctx->rounding == TT_ROUND_GRAM) {
    tt_status st = gram_factor(s, ctx->num_sms, SrcRows<S>{(const S*)x->core[0], K1}, lp, N, ws, ctx->ctrl,
                               ctx->coop_grid_max, &RZ);
    if (st != TT_OK) return st;
  } else if (ctx->rounding == TT_ROUND_RANDOMIZED) {
    tt_status st = randomized_factor<S, T>(ctx, s, SrcRows<S>{(const S*)x->core[0], K1}, lp, N, b.Bbase, n1 * n2, ws,
                                           &RZ, kTsqrLeaf);
    if (st != TT_OK) return st;
  } else if (!ws.dry) {
    tt_status st = run_tsqr_cfg<T>(cfg, s, ctx->num_sms, SrcRows<S>{(const S*)x->core[0], K1}, lp, N, b.tsqr_a,
                                   b.tsqr_b, &RZ);
    if (st != TT_OK) return st;
  }
  job.RZ = RZ;
  tt_status st = small_round(s, ctx->num_sms, job, ws);
  if (st != TT_OK || ws.dry) return st;
  st = launch_update<T>(ctx, s, ctx->num_sms, SrcRows<S>{(const S*)x->core[0], K1}, lp, N, b.W, K1,
                        EpiPlain<S>{(S*)x->core[0], K1, &ctx->ctrl->status}, nullptr, nullptr);
  if (st != TT_OK) return st;
  const long tot = (long)K1 * n1 * K2 + (long)K2 * n2;
  k_commit<S><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d, n1, n2, K1, K2, b.core1, b.core2,
                                                            (S*)x->core[1], d == 3 ? (S*)x->core[2] : nullptr,
                                                            ctx->ctrl, x->rank); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

template <typename S, typename T>
tt_status step_impl(tt_context* ctx, const tt_plan* p, tt_tensor* I, double tol, int rmax, double* energy,
                    Bump& ws) {
  cudaStream_t s = ctx->stream;
  const int d = I->d;
  const long N = I->n[0];
  const int n1 = p->n1, n2 = p->n2, nang = n1 * n2;
  const int K1 = I->rcap[1], K2 = (d == 3) ? I->rcap[2] : 1;
  // ---- first rounding: the transport sum, never materialised
  LivePattern lp1{I->rank + 1, K1, p->nterm + 1, p->nbc};
  const int R1 = lp1.ncap();
  const TsqrCfg cfg1 = tsqr_cfg<T>(ctx, R1);
  RoundBufs b1 = take_round_bufs<T>(ws, ctx->num_sms, cfg1.leaves, d, R1, N, n1, n2, K1, K2, K1);
  S* Zsrc = ws.take<S>((size_t)N * (K1 + 1));
  const long ngrid = (N + 31) / 32;  // bounds the persistent update grids (tiles of >= 32 rows)
  double* part1 = ws.take<double>((size_t)2 * ngrid);
  double* part2 = ws.take<double>((size_t)2 * ngrid);
  long ngrid1 = 0, ngrid2 = 0;
  double* part0 = ws.take<double>((size_t)((N + 255) / 256));
  double* sums = ws.take<double>(8);
  double* vJ0 = ws.take<double>(K1);
  SrcStencil<S> src1{};
  fill_stencil<S>(src1, p, (const S*)I->core[0], K1);
  SmallJob j1{};
  j1.d = d;
  j1.n1 = n1;
  j1.n2 = n2;
  j1.nrowsZ = N;
  j1.lp = lp1;
  j1.r2_ptr = (d == 3) ? I->rank + 2 : nullptr;
  j1.r2_nblk = p->nterm + 1;
  j1.r2_nextra = p->nbc;
  j1.tol = tol;
  j1.rmax = rmax;
  j1.K1cap = K1;
  j1.K2cap = K2;
  j1.B0 = b1.B0;
  j1.domega = p->domega;
  j1.W = b1.W;
  j1.core1 = b1.core1;
  j1.core2 = b1.core2;
  j1.Bnew = b1.Bnew;
  j1.vJ = b1.vJ;
  j1.ctrl = ctx->ctrl;
  j1.coop_grid_max = ctx->coop_grid_max;
  j1.mixed = (sizeof(T) == 4);
  double* RZ1 = nullptr;
  if (!ws.dry) {
    right_part<S>(s, d, K1, n1, K2, n2, (const S*)I->core[1], d == 3 ? (const S*)I->core[2] : nullptr, b1.Bbase);
    if (energy) {
      k_vj_host_launch(s, K1, nang, b1.Bbase, p->domega, vJ0);
      k_rowdot_partials<S><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, K1, K1, (const S*)I->core[0], vJ0, part0,
                                                                      nullptr, 0.0); count_launch();
      reduce_partials(s, part0, (N + 255) / 256, 1, sums, 1.0);
    }
    k_b0_transport<<<256, 256, 0, s>>>(K1, p->nterm, p->nbc, n1, n2, b1.Bbase, p->fac1, p->fac2, p->bc_term_dev,
                                       b1.B0); count_launch();
  }
  const bool gram = (ctx->rounding == TT_ROUND_GRAM);
  const bool rnd = (ctx->rounding == TT_ROUND_RANDOMIZED);
  if (gram) {
    tt_status st = gram_factor(s, ctx->num_sms, src1, lp1, N, ws, ctx->ctrl, ctx->coop_grid_max, &RZ1);
    if (st != TT_OK) return st;
  } else if (rnd) {
    tt_status st = randomized_factor<S, T>(ctx, s, src1, lp1, N, b1.B0, nang, ws, &RZ1, kTsqrLeaf);
    if (st != TT_OK) return st;
  } else if (!ws.dry) {
    tt_status st = run_tsqr_cfg<T>(cfg1, s, ctx->num_sms, src1, lp1, N, b1.tsqr_a, b1.tsqr_b, &RZ1);
    if (st != TT_OK) return st;
  }
  j1.RZ = RZ1;
  tt_status st = small_round(s, ctx->num_sms, j1, ws);
  if (st != TT_OK) return st;
  // ---- source step fused into the write of the rounded transport update
  LivePattern lp2{nullptr, K1, 1, 1};
  const TsqrCfg cfg2 = tsqr_cfg<T>(ctx, lp2.ncap());
  RoundBufs b2 = take_round_bufs<T>(ws, ctx->num_sms, cfg2.leaves, d, lp2.ncap(), N, n1, n2, K1, K2, K1);
  double *cpl_u = nullptr, *jstar = nullptr, *jnew = nullptr;
  if (p->coupled) {
    cpl_u = ws.take<double>(R1);
    jstar = ws.take<double>(N);
    jnew = ws.take<double>(N);
  }
  if (ws.dry) {
    SmallJob j2 = j1;
    j2.lp = lp2;
    if (gram) {
      double* RZ2 = nullptr;
      st = gram_factor(s, ctx->num_sms, SrcRows<S>{Zsrc, K1 + 1}, lp2, N, ws, ctx->ctrl, ctx->coop_grid_max, &RZ2);
      if (st != TT_OK) return st;
    } else if (rnd) {
      double* RZ2 = nullptr;
      st = randomized_factor<S, T>(ctx, s, SrcRows<S>{Zsrc, K1 + 1}, lp2, N, b2.B0, nang, ws, &RZ2, kTsqrLeafSrc);
      if (st != TT_OK) return st;
    }
    return small_round(s, ctx->num_sms, j2, ws);
  }
  if (p->coupled) {
    // material temperature (Sec. 2.1): T^dagger per cell from J* of the rounded transport
    // update, epsilon(T^dagger) into the plan before the source step reads it
    k_wvj<<<(R1 + 255) / 256, 256, 0, s>>>(R1, K1, b1.W, b1.vJ, cpl_u); count_launch();
    const long jb = (N + 7) / 8 < 4096 ? (N + 7) / 8 : 4096;
    k_jstar<<<(unsigned)jb, 256, 0, s>>>(src1, lp1, N, cpl_u, jstar); count_launch();
    st = coupled_t_dagger(s, const_cast<tt_plan*>(p), jstar);  // the plan holds the material state
    if (st != TT_OK) return st;
  }
  st = launch_update<T>(ctx, s, ctx->num_sms, src1, lp1, N, b1.W, K1,
                        EpiSource<S>{Zsrc, K1 + 1, b1.vJ, p->acoef, p->scoef, p->eps, &ctx->ctrl->status}, part1,
                        &ngrid1);
  if (st != TT_OK) return st;
  k_save_ranks<<<1, 32, 0, s>>>(ctx->ctrl); count_launch();
  lp2.r_ptr = &ctx->ctrl->k[2];
  // ---- second rounding: [D^-1 Z_new, g]
  k_b0_source<<<64, 256, 0, s>>>(K1, nang, b1.Bnew, b2.B0); count_launch();
  double* RZ2 = nullptr;
  if (gram)
    st = gram_factor(s, ctx->num_sms, SrcRows<S>{Zsrc, K1 + 1}, lp2, N, ws, ctx->ctrl, ctx->coop_grid_max, &RZ2,
                     kTsqrLeafSrc);
  else if (rnd)
    st = randomized_factor<S, T>(ctx, s, SrcRows<S>{Zsrc, K1 + 1}, lp2, N, b2.B0, nang, ws, &RZ2, kTsqrLeafSrc);
  else
    st = run_tsqr_cfg<T>(cfg2, s, ctx->num_sms, SrcRows<S>{Zsrc, K1 + 1}, lp2, N, b2.tsqr_a, b2.tsqr_b, &RZ2,
                         kTsqrLeafSrc);
  if (st != TT_OK) return st;
  SmallJob j2 = j1;
  j2.lp = lp2;
  j2.r2_ptr = (d == 3) ? &ctx->ctrl->k[3] : nullptr;
  j2.r2_nblk = 1;
  j2.r2_nextra = 1;
  j2.B0 = b2.B0;
  j2.RZ = RZ2;
  j2.W = b2.W;
  j2.core1 = b2.core1;
  j2.core2 = b2.core2;
  j2.Bnew = b2.Bnew;
  j2.vJ = b2.vJ;
  st = small_round(s, ctx->num_sms, j2, ws);
  if (st != TT_OK) return st;
  st = launch_update<T>(ctx, s, ctx->num_sms, SrcRows<S>{Zsrc, K1 + 1}, lp2, N, b2.W, K1,
                        EpiFinal<S>{(S*)I->core[0], K1, b2.vJ, jnew, &ctx->ctrl->status}, part2, &ngrid2,
                        kUpdateSrc);
  if (st != TT_OK) return st;
  if (p->coupled) {
    st = coupled_t_update(s, const_cast<tt_plan*>(p), jstar, jnew);
    if (st != TT_OK) return st;
  }
  const long tot = (long)K1 * n1 * K2 + (long)K2 * n2;
  k_commit<S><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d, n1, n2, K1, K2, b2.core1, b2.core2,
                                                            (S*)I->core[1], d == 3 ? (S*)I->core[2] : nullptr,
                                                            ctx->ctrl, I->rank); count_launch();
  if (energy) {
    reduce_partials(s, part1, ngrid1, 2, sums + 2, 1.0);
    reduce_partials(s, part2, ngrid2, 2, sums + 4, 1.0);
    k_energy_pack<<<1, 32, 0, s>>>(sums, sums + 2, sums + 4, 4.0 * kPi / p->c * p->dV, energy); count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

template tt_status round_impl<double, double>(tt_context*, tt_tensor*, double, int, Bump&);
template tt_status round_impl<float, double>(tt_context*, tt_tensor*, double, int, Bump&);
template tt_status round_impl<double, float>(tt_context*, tt_tensor*, double, int, Bump&);
template tt_status round_impl<float, float>(tt_context*, tt_tensor*, double, int, Bump&);
template tt_status step_impl<double, double>(tt_context*, const tt_plan*, tt_tensor*, double, int, double*, Bump&);
template tt_status step_impl<float, double>(tt_context*, const tt_plan*, tt_tensor*, double, int, double*, Bump&);
template tt_status step_impl<double, float>(tt_context*, const tt_plan*, tt_tensor*, double, int, double*, Bump&);
template tt_status step_impl<float, float>(tt_context*, const tt_plan*, tt_tensor*, double, int, double*, Bump&);

template <typename S>
tt_status energy_density_impl(tt_context* ctx, const tt_plan* p, const tt_tensor* x, double* out, Bump& ws) {
  cudaStream_t s = ctx->stream;
  const int d = x->d;
  const long N = x->n[0];
  const int n1 = x->n[1], n2 = (d == 3) ? x->n[2] : 1;
  const int K1 = x->rcap[1], K2 = (d == 3) ? x->rcap[2] : 1;
  double* Bb = ws.take<double>((size_t)K1 * n1 * n2);
  double* v = ws.take<double>(K1);
  if (ws.dry) return TT_OK;
  right_part<S>(s, d, K1, n1, K2, n2, (const S*)x->core[1], d == 3 ? (const S*)x->core[2] : nullptr, Bb);
  k_vj_host_launch(s, K1, n1 * n2, Bb, p->domega, v);
  k_rowdot_partials<S><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, K1, K1, (const S*)x->core[0], v, nullptr, out,
                                                                  4.0 * kPi / p->c); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}
template tt_status energy_density_impl<double>(tt_context*, const tt_plan*, const tt_tensor*, double*, Bump&);
template tt_status energy_density_impl<float>(tt_context*, const tt_plan*, const tt_tensor*, double*, Bump&);

}  // namespace ttk
