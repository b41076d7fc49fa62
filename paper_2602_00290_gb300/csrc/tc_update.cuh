// Update pass over the stencil sum on the tensor cores (mixed path, FP32 storage of the merged
// core): the GEMM of k_update_blk, Z_new = C W_0 + sum_a (D_L,a WL_a + D_H,a WH_a), as tcgen05
// kind::tf32 MMAs in split precision (3xTF32) with the FP32 accumulator in tensor memory.
//
// A tile is 128 rows.  The centre rows C and their lower and upper neighbours along every axis are
// staged by cp.async straight into the K-major core-matrix layout of the A operand (K = the
// stencil sum's width, (1 + 2 d_X) rcap), the neighbours are turned into the differences
// D_L = C - L and D_H = H - C in place, and every value is split into its TF32 part and the FP32
// remainder (itself rounded to TF32, so that the tensor core's truncation of its operands adds no
// bias).  The combined weights (formed once per CTA in FP64, as in k_update_blk) are the B operand,
// split the same way.  One thread issues three MMAs per K step of 8 (lo hi, hi lo, hi hi).  The
// hi hi products are spread over several accumulators in tensor memory, at most two K steps each,
// and the small products of all steps go to one more (update_tc_acc_plan), because the tensor
// core's FP32 accumulation is not rounded to nearest: its error, biased toward zero, grows with
// the MMAs summed into one accumulator.  Four warps read the accumulators back (a row per thread)
// and add them in FP32, the inflow columns are added per row, and the update epilogue (energy dot,
// source or final scaling, non-finite check) runs on the tile as for the other update kernels.
#pragma once
#include <type_traits>

#include "tc.cuh"
#include "update_blk.cuh"

namespace ttk {

constexpr int kTcRows = 128;     // rows per tile: the M of one MMA, one TMEM lane per row
constexpr int kTcThreads = 512;  // 16 warps: the tile phases are latency-bound at 8

// Output columns of the tensor-core update: kcap rounded up to a multiple of 16 (the MMA's N).
__host__ __device__ inline int update_tc_n(int kcap) { return (kcap + 15) & ~15; }
// Accumulators in tensor memory (N FP32 columns each, 512 columns in all): the hi x hi products of
// the K steps (of 8) go to nhh accumulators of at most `sph` steps each, the two small products
// of every step (lo x hi, hi x lo, about 2^-11 of the result) to one more.  The tensor core's FP32
// accumulation rounds toward zero, up to an ulp of the partial sum per MMA, so the bias of an
// accumulator grows with the MMAs summed into it; keeping the large products few per accumulator
// and the small ones apart holds that bias to about one ulp of the result (the accumulators are
// added in FP32 rounded to nearest).
struct TcAccPlan {
  int sph, nhh, nacc;
};
__host__ __device__ inline TcAccPlan update_tc_acc_plan(int K, int N) {
  const int ksteps = K / 8;
  int amax = 512 / N;  // N <= 256: at least 2
  if (amax < 2) amax = 2;
  const int hmax = amax - 1;
  TcAccPlan p;
  p.sph = (ksteps + hmax - 1) / hmax;
  if (p.sph < 1) p.sph = 1;
  p.nhh = (ksteps + p.sph - 1) / p.sph;
  p.nacc = p.nhh + 1;
  return p;
}

// Shared memory: A hi and lo [128][K] and B hi and lo [N][K] (FP32, K-major core matrices),
// inflow weights [nbc][N], row scalars [3][128] (FP64), vJ [N], row flags [2][128].  The output tile
// [128][N + 1] reuses A lo once the MMAs of a tile are done, the energy partials reuse A hi.
__host__ __device__ inline size_t update_tc_smem_bytes(int K, int N, int nbc) {
  size_t b = sizeof(float) * (2 * (size_t)kTcRows * K + 2 * (size_t)N * K + (size_t)nbc * N);
  b = (b + 7) & ~(size_t)7;
  return b + sizeof(double) * 3 * kTcRows + sizeof(float) * (size_t)N + sizeof(unsigned) * 2 * kTcRows;
}

// Row flags of k_update_blk (neighbour bits 2a and 2a + 1, the group in bits 8 and up) in 32-bit
// arithmetic: the host takes this kernel only for merged cores of fewer than 2^31 rows.
template <typename S>
__device__ __forceinline__ unsigned tc_row_flags(const SrcStencil<S>& src, unsigned k) {
  unsigned f = 0u;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const unsigned idx = (k / (unsigned)src.stride[a]) % (unsigned)src.ext[a];
    f |= (idx > 0u ? 1u : 0u) << (2 * a);
    f |= (idx + 1u < (unsigned)src.ext[a] ? 1u : 0u) << (2 * a + 1);
  }
  return f | ((k % (unsigned)src.G) << 8);
}

// NB row blocks (1 + 2 d_X) of RCAP columns each: K = NB RCAP, compile-time.  kTcThreads threads:
// all of them stage, split and run the epilogue; warps 0-3 read the accumulators (TMEM lanes =
// rows).
template <class Epi, int NB, int RCAP>
__global__ void __launch_bounds__(kTcThreads, 1) k_update_tc(SrcStencil<float> src, LivePattern lp, long nrows,
                                                      const double* __restrict__ W, int kcap, Epi epi,
                                                      double* __restrict__ partials) {
  extern __shared__ __align__(1024) unsigned char tcu_smem[];
  constexpr int K = NB * RCAP, GPR = RCAP / 4;
  static_assert(RCAP % 8 == 0, "whole MMA K steps per row block");
  const int nbc = lp.nextra;
  const int N = update_tc_n(kcap), ldo = N + 1;
  const TcAccPlan ap = update_tc_acc_plan(K, N);
  const int sph = ap.sph, nhh = ap.nhh, nacc = ap.nacc;
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  const int rq = r < RCAP ? r : RCAP;  // live columns of each Z block
  float* Ahi = reinterpret_cast<float*>(tcu_smem);
  float* Alo = Ahi + (size_t)kTcRows * K;
  float* Bhi = Alo + (size_t)kTcRows * K;
  float* Blo = Bhi + (size_t)N * K;
  float* Wbc = Blo + (size_t)N * K;  // [nbc][N]
  size_t off = sizeof(float) * (2 * (size_t)kTcRows * K + 2 * (size_t)N * K + (size_t)nbc * N);
  off = (off + 7) & ~(size_t)7;
  double* rowv = reinterpret_cast<double*>(tcu_smem + off);  // [3][128]
  float* vJs = reinterpret_cast<float*>(rowv + 3 * kTcRows);  // [N]
  unsigned* fl = reinterpret_cast<unsigned*>(vJs + N);        // [2][128]
  float* Os = Alo;                                            // [128][N + 1] after a tile's MMAs
  double* red = reinterpret_cast<double*>(Ahi);               // energy partials after the last tile
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* vJ = epi_vj(epi);
  const uint32_t ncols = tc::tmem_cols(nacc * N);
  if (warp == 0) {
    tc::tmem_alloc(&tbase, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&bar, 1);

  // combined weights B[n][k] for k = b RCAP + q (FP64 sums as in k_update_blk), split in TF32 parts
  for (int i = tid; i < N * K; i += blockDim.x) {
    const int n = i / K, kk = i - (i / K) * K;
    const int b = kk / RCAP, q = kk - (kk / RCAP) * RCAP;
    double sum = 0.0;
    if (n < kcap && q < rq) {
      if (b == 0) {
        sum = W[(size_t)q * kcap + n];
      } else {
        for (int t = 1; t <= src.nterm; ++t) {
          const int ax = src.axis[t - 1];
          if (b != 1 + 2 * ax && b != 2 + 2 * ax) continue;
          double cL, cH;
          blk_coefs(src, t, cL, cH);
          const double cf = (b == 1 + 2 * ax) ? cL : cH;
          if (cf != 0.0) sum += cf * W[(size_t)(t * RCAP + q) * kcap + n];
        }
      }
    }
    const float f = (float)sum, h = tc::tf32_hi(f);
    const uint32_t o = tc::kmajor_off(n, kk, K) >> 2;
    Bhi[o] = h;
    Blo[o] = tc::tf32_hi(f - h);
  }
  for (int i = tid; i < nbc * N; i += blockDim.x) {
    const int e = i / N, n = i - (i / N) * N;
    const int c = (src.nterm + 1) * RCAP + e;
    Wbc[i] = (n < kcap && lp.live(c, r)) ? (float)W[(size_t)c * kcap + n] : 0.0f;
  }
  for (int n = tid; n < N; n += blockDim.x) vJs[n] = (vJ && n < kcap) ? (float)vJ[n] : 0.0f;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint32_t idesc = tc::idesc_tf32(kTcRows, N);
  constexpr uint32_t lbo = 128, sbo = (uint32_t)(K / 4) * 128u;
  const long ntiles = (nrows + kTcRows - 1) / kTcRows;
  uint32_t phase = 0;
  bool ok = true;
  double e0t = 0.0, e1t = 0.0;
  // row flags of a tile into f (threads < 128)
  auto flags_of = [&](long row0, unsigned* f) {
    if (tid < kTcRows) f[tid] = (row0 + tid < nrows) ? tc_row_flags(src, (unsigned)(row0 + tid)) : 0u;
  };
  // every granule of a tile's row blocks in flight at once, into the A layout; rows outside the
  // core and neighbours the row does not have are zero-filled.  Eight consecutive threads take
  // one granule of eight consecutive rows (one 128-byte core matrix: no bank conflict), a warp
  // four granules of them (whole 32-byte sectors of every row it reads)
  auto stage = [&](long row0, const unsigned* f) {
    constexpr int per_block = kTcRows * GPR;
#pragma unroll 4
    for (int i = tid; i < NB * per_block; i += kTcThreads) {
      const int b = i / per_block, rem = i - b * per_block;
      const int r8 = rem >> 3, g = r8 % GPR, m = (r8 / GPR) * 8 + (rem & 7);
      long k = row0 + m;
      bool okr = k < nrows;
      if (b > 0) {
        const int ax = (b - 1) >> 1;
        const bool upper = ((b - 1) & 1) != 0;
        okr = okr && ((f[m] >> (2 * ax + (upper ? 1 : 0))) & 1u);
        k += upper ? src.stride[ax] : -src.stride[ax];
      }
      float* dst = Ahi + (tc::kmajor_off(m, b * RCAP + 4 * g, K) >> 2);
      const float* from = okr ? src.Z + k * RCAP + (size_t)4 * g : src.Z;
      cp_async16(dst, from, okr ? 16 : 0);
    }
    // the source step's per-row coefficients of the tile into L2 ahead of its epilogue
    if constexpr (std::is_same<Epi, EpiSource<float>>::value) {
      const long last = (row0 + kTcRows < nrows ? row0 + kTcRows : nrows) - 1;
      if (tid < 24) {
        const double* arr = tid < 8 ? epi.acoef : tid < 16 ? epi.scoef : epi.eps;
        const long k = row0 + (long)(tid & 7) * 16;
        if (k <= last) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(arr + k));
      }
    }
  };
  // Tile pipeline: a tile's rows are staged as soon as the previous tile's MMAs have read the A
  // buffer, so the copies overlap that tile's read-back and epilogue; row flags alternate
  // between two buffers (the read-back of one tile and the staging of the next use both).
  int fb = 0;
  if ((long)blockIdx.x < ntiles) {
    flags_of((long)blockIdx.x * kTcRows, fl);
    __syncthreads();
    stage((long)blockIdx.x * kTcRows, fl);
  }
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long row0 = tile * kTcRows;
    const unsigned* flc = fl + fb * kTcRows;
    cp_async_wait_all();
    __syncthreads();  // the tile's rows are in place, and the previous epilogue is done with A lo
    // neighbours to differences with the centre rows (L -> C - L, H -> H - C), then every value
    // to its TF32 part (A hi) and rounded remainder (A lo); a thread takes 4 consecutive K values
    // of a row (16-byte vectors; a warp's 32 rows fall on distinct banks)
    for (int i = tid; i < kTcRows * GPR; i += kTcThreads) {
      const int g = i / kTcRows, m = i - g * kTcRows;
      const uint32_t oc = tc::kmajor_off(m, 4 * g, K) >> 2;
      const float4 c = *reinterpret_cast<const float4*>(Ahi + oc);
#pragma unroll
      for (int b = 1; b < NB; ++b) {
        const uint32_t o = tc::kmajor_off(m, b * RCAP + 4 * g, K) >> 2;
        float4 v = *reinterpret_cast<const float4*>(Ahi + o);
        if (b & 1) {
          v = make_float4(c.x - v.x, c.y - v.y, c.z - v.z, c.w - v.w);
        } else {
          v = make_float4(v.x - c.x, v.y - c.y, v.z - c.z, v.w - c.w);
        }
        const float4 h = make_float4(tc::tf32_hi(v.x), tc::tf32_hi(v.y), tc::tf32_hi(v.z), tc::tf32_hi(v.w));
        *reinterpret_cast<float4*>(Ahi + o) = h;
        *reinterpret_cast<float4*>(Alo + o) = make_float4(tc::tf32_hi(v.x - h.x), tc::tf32_hi(v.y - h.y),
                                                          tc::tf32_hi(v.z - h.z), tc::tf32_hi(v.w - h.w));
      }
      const float4 h = make_float4(tc::tf32_hi(c.x), tc::tf32_hi(c.y), tc::tf32_hi(c.z), tc::tf32_hi(c.w));
      *reinterpret_cast<float4*>(Ahi + oc) = h;
      *reinterpret_cast<float4*>(Alo + oc) = make_float4(tc::tf32_hi(c.x - h.x), tc::tf32_hi(c.y - h.y),
                                                         tc::tf32_hi(c.z - h.z), tc::tf32_hi(c.w - h.w));
    }
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll 4
      for (int s = 0; s < K / 8; ++s) {
        const uint32_t so = 256u * (uint32_t)s;
        const uint64_t dah = tc::smem_desc(ah + so, lbo, sbo), dal = tc::smem_desc(al + so, lbo, sbo);
        const uint64_t dbh = tc::smem_desc(bh + so, lbo, sbo), dbl = tc::smem_desc(bl + so, lbo, sbo);
        const uint32_t dhh = tmem + (uint32_t)((s / sph) * N);  // this step's hi x hi accumulator
        const uint32_t dlo = tmem + (uint32_t)(nhh * N);        // the small products of every step
        tc::mma_tf32(dlo, dal, dbh, idesc, s ? 1u : 0u);
        tc::mma_tf32(dlo, dah, dbl, idesc, 1u);
        tc::mma_tf32(dhh, dah, dbh, idesc, (s % sph) ? 1u : 0u);
      }
      tc::mma_commit(&bar);
    }
    ok = __syncthreads_and(tc::mbar_wait(&bar, phase)) != 0;
    if (!ok) break;
    phase ^= 1u;
    tc::fence_after_sync();
    // A hi is free: the next tile's rows can land during this tile's read-back and epilogue
    const long next = tile + gridDim.x;
    if (next < ntiles) {
      unsigned* fln = fl + (fb ^ 1) * kTcRows;
      flags_of(next * kTcRows, fln);
      __syncthreads();
      stage(next * kTcRows, fln);
    }
    // accumulator rows (warps 0-3), summed over the accumulators (FP32 adds rounded to nearest: a
    // few ulp over the handful of partial sums), plus the inflow columns, to the output tile (A lo
    // is free now)
    if (warp < 4) {
      const int m = 32 * warp + lane;
      const unsigned f = flc[m];
      for (int c0 = 0; c0 < N; c0 += 32) {
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.0f;
        for (int a = 0; a < nacc; ++a) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(a * N + c0), v);
          tc::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[j] += v[j];
        }
        for (int e = 0; e < nbc; ++e) {
          const int tt = src.bc_term[e], ax = src.axis[tt];
          const bool lower_face = src.w[tt] > 0;
          const bool at_face = lower_face ? !((f >> (2 * ax)) & 1u) : !((f >> (2 * ax + 1)) & 1u);
          const float val = (at_face && row0 + m < nrows) ? (float)src.bcval[e * src.G + (int)(f >> 8)] : 0.0f;
          if (val != 0.0f) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (c0 + j < N) acc[j] = fmaf(val, Wbc[e * N + c0 + j], acc[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < N) Os[(size_t)m * ldo + c0 + j] = acc[j];
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    update_epilogue<float, kTcRows>(epi, Os, ldo, kcap, vJs, vJ != nullptr, rowv, row0, nrows, e0t, e1t);
    fb ^= 1;
  }
  if (!ok) {
    // the MMAs of the tile may still be running: wait for them again (bounded) before the
    // accumulator is released, and report the timeout
    if (tid == 0) latch(epi.status, TT_ERR_TIMEOUT);
    (void)__syncthreads_and(tc::mbar_wait(&bar, phase));
  }
  if (partials) update_partials(red, e0t, e1t, partials);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, ncols);
  }
}

// Whether the tensor-core update takes a pass: FP32 storage, rank capacity 8, 16 or 32 (the
// kernel's instantiations; 16-byte aligned rows of whole MMA K steps), 1 to 3 axes, at most 256
// output columns, fewer than 2^31 rows, and its shared memory.
inline bool update_tc_fits(const SrcStencil<float>& src, const LivePattern& lp, long nrows, int kcap,
                           int smem_optin) {
  if ((src.rcap != 8 && src.rcap != 16 && src.rcap != 32) || src.ldz != src.rcap || ((size_t)src.Z % 16) != 0 ||
      src.rcap != lp.rcap || src.nax < 1 || src.nax > 3 || nrows >= (1L << 31))
    return false;
  if (kcap < 1 || update_tc_n(kcap) > 256) return false;
  const int K = (1 + 2 * src.nax) * src.rcap;
  const size_t need = update_tc_smem_bytes(K, update_tc_n(kcap), lp.nextra);
  return (need > 117 * 1024 ? need : 117 * 1024) <= (size_t)smem_optin;
}

template <class Epi, int NB, int RCAP>
tt_status launch_update_tc_k(cudaStream_t s, int num_sms, const SrcStencil<float>& src, LivePattern lp, long nrows,
                             const double* W, int kcap, const Epi& epi, double* partials, long* grid_out, int cat) {
  const int K = NB * RCAP, N = update_tc_n(kcap);
  // at least half an SM's shared memory, so that one CTA is resident per SM and its tensor-memory
  // accumulators never wait for another CTA's
  size_t smem = update_tc_smem_bytes(K, N, lp.nextra);
  if (smem < 117 * 1024) smem = 117 * 1024;
  auto kern = k_update_tc<Epi, NB, RCAP>;
  if (const tt_status a = smem_optin(kern, smem); a != TT_OK) return a;
  const long ntiles = (nrows + kTcRows - 1) / kTcRows;
  long grid = num_sms;  // one CTA per SM: its shared memory and accumulators stay resident
  if (grid > ntiles) grid = ntiles > 0 ? ntiles : 1;
  if (grid_out) *grid_out = grid;
  TimerScope scope(cat, s);
  kern<<<(unsigned)grid, kTcThreads, smem, s>>>(src, lp, nrows, W, kcap, epi, partials);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// Dispatch on (1 + 2 d_X, rcap); update_tc_fits has checked that an instantiation exists.
template <class Epi>
tt_status launch_update_tc(cudaStream_t s, int num_sms, const SrcStencil<float>& src, LivePattern lp, long nrows,
                           const double* W, int kcap, const Epi& epi, double* partials, long* grid_out,
                           int cat = kUpdate) {
#define TT_UPDATE_TC_CASE(NB_, RC_)                                                                          \
  if (1 + 2 * src.nax == NB_ && src.rcap == RC_)                                                            \
    return launch_update_tc_k<Epi, NB_, RC_>(s, num_sms, src, lp, nrows, W, kcap, epi, partials, grid_out, cat);
  TT_UPDATE_TC_CASE(3, 8) TT_UPDATE_TC_CASE(3, 16) TT_UPDATE_TC_CASE(3, 32)
  TT_UPDATE_TC_CASE(5, 8) TT_UPDATE_TC_CASE(5, 16) TT_UPDATE_TC_CASE(5, 32)
  TT_UPDATE_TC_CASE(7, 8) TT_UPDATE_TC_CASE(7, 16) TT_UPDATE_TC_CASE(7, 32)
#undef TT_UPDATE_TC_CASE
  return TT_ERR_UNSUPPORTED;
}

}  // namespace ttk
