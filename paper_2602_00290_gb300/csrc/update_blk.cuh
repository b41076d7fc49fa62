// Update pass over the stencil sum from staged row blocks (FP32 arithmetic).
//
// Column block t of the transport sum is, in the columns of Z, a combination of the differences
// of the centre rows C (row0 ..) with their neighbours along the operator's axis a: the lower
// difference D_L,a = C - L_a (L_a: rows row0 - s_a ..) and the upper difference
// D_H,a = H_a - C (H_a: rows row0 + s_a ..), a missing neighbour being zero (vacuum ghost cells):
//   upwind, w > 0       -lambda D_L,a
//   upwind, w < 0       -lambda D_H,a
//   Rusanov central     -lambda/2 (D_H,a + D_L,a)
//   Rusanov diffusion    lambda/2 (D_H,a - D_L,a)
// so Z_sum W = C W_0 + sum_a (D_L,a WL_a + D_H,a WH_a) + (inflow columns) W_bc, with the combined
// weights WL_a, WH_a formed once per CTA in FP64 from W and the operators' coefficients.  The
// neighbour differences are formed once per tile in shared memory, before any weight multiplies
// them: two close neighbours subtract exactly, as in the stencil columns themselves.  A tile is
// then a GEMM of the staged blocks (K = (1 + 2 d_X) rcap, the stencil sum's width) without a
// tile of the stencil sum in shared memory.  The inflow columns (at most 6) are added per row.
// The epilogue is the update pass's.
#pragma once
#include "bigpass.cuh"

namespace ttk {

// Padded row stride of a staged block: one 16-byte granule past the row, so that the rows that
// the threads of a warp read at once fall on different banks.
template <typename S>
__host__ __device__ inline int blk_ldp(int ldz) { return ldz + 16 / (int)sizeof(S); }

// Shared memory of k_update_blk: combined weights [(1 + 2 nax) rcap][kpad] and inflow weights
// [nbc][kpad] (FP32), staged blocks [(1 + 2 nax)][TM][ldp] (S), output tile [TM][kpad] (FP32),
// row scalars [3][TM] (FP64), vJ [kpad] (FP32), row flags [TM].
template <int TM, typename S>
__host__ __device__ inline size_t update_blk_smem_bytes(const SrcStencil<S>& src, int kpad, int nbc) {
  const int nb = 1 + 2 * src.nax;
  size_t b = sizeof(float) * ((size_t)nb * src.rcap * kpad + (size_t)nbc * kpad);
  b = (b + 15) & ~(size_t)15;
  size_t raw = sizeof(S) * (size_t)nb * TM * blk_ldp<S>(src.ldz);
  if (raw < sizeof(double) * 2 * 256) raw = sizeof(double) * 2 * 256;  // energy partials reuse it
  b += (raw + 15) & ~(size_t)15;
  b += sizeof(float) * (size_t)TM * kpad;
  b = (b + 15) & ~(size_t)15;
  return b + sizeof(double) * 3 * TM + sizeof(float) * (size_t)kpad + sizeof(unsigned) * TM;
}

// Coefficients of column block t (1 .. nterm) on the lower and upper differences of its axis.
template <typename S>
__device__ __forceinline__ void blk_coefs(const SrcStencil<S>& src, int t, double& cL, double& cH) {
  const int w = src.w[t - 1];
  const double lam = src.lam[t - 1];
  if (w == 2) {  // Rusanov central term
    cL = -0.5 * lam;
    cH = -0.5 * lam;
  } else if (w == -2) {  // Rusanov diffusion term
    cL = -0.5 * lam;
    cH = 0.5 * lam;
  } else if (w > 0) {
    cL = -lam;
    cH = 0.0;
  } else {
    cL = 0.0;
    cH = -lam;
  }
}

template <int TM, typename S, class Epi>
__global__ void __launch_bounds__(256) k_update_blk(SrcStencil<S> src, LivePattern lp, long nrows,
                                                    const double* __restrict__ W, int kcap, Epi epi,
                                                    double* __restrict__ partials) {
  static_assert(TM % 32 == 0, "rows per tile: a multiple of 32");
  constexpr int RPT = TM / 32;  // output rows per thread
  extern __shared__ __align__(16) unsigned char blk_smem[];
  const int rcap = src.rcap, nb = 1 + 2 * src.nax, nbc = lp.nextra;
  const int kpad = update_kpad<Epi>(kcap);
  const int ldp = blk_ldp<S>(src.ldz);
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  const int rq = r < rcap ? r : rcap;  // live columns of each Z block
  float* Wb = reinterpret_cast<float*>(blk_smem);      // [nb rcap][kpad]
  float* Wbc = Wb + (size_t)nb * rcap * kpad;          // [nbc][kpad]
  size_t off = sizeof(float) * ((size_t)nb * rcap * kpad + (size_t)nbc * kpad);
  off = (off + 15) & ~(size_t)15;
  S* raw = reinterpret_cast<S*>(blk_smem + off);       // [nb][TM][ldp]
  size_t rawb = sizeof(S) * (size_t)nb * TM * ldp;
  if (rawb < sizeof(double) * 2 * 256) rawb = sizeof(double) * 2 * 256;
  off += (rawb + 15) & ~(size_t)15;
  float* Os = reinterpret_cast<float*>(blk_smem + off);  // [TM][kpad]
  off += sizeof(float) * (size_t)TM * kpad;
  off = (off + 15) & ~(size_t)15;
  double* rowv = reinterpret_cast<double*>(blk_smem + off);  // [3][TM]
  float* vJs = reinterpret_cast<float*>(rowv + 3 * TM);      // [kpad]
  unsigned* fl = reinterpret_cast<unsigned*>(vJs + kpad);    // [TM]
  double* red = reinterpret_cast<double*>(raw);              // energy partials, after the last tile
  const int tid = threadIdx.x;
  const double* vJ = epi_vj(epi);

  // combined weights (FP64 sums, stored in FP32); dead columns of the stencil sum contribute nothing
  for (int i = tid; i < nb * rcap * kpad; i += blockDim.x) {
    const int row = i / kpad, j = i - (i / kpad) * kpad;
    const int b = row / rcap, q = row - (row / rcap) * rcap;
    double sum = 0.0;
    if (j < kcap && q < rq) {
      if (b == 0) {
        sum = W[(size_t)q * kcap + j];
      } else {
        for (int t = 1; t <= src.nterm; ++t) {
          const int ax = src.axis[t - 1];
          if (b != 1 + 2 * ax && b != 2 + 2 * ax) continue;
          double cL, cH;
          blk_coefs(src, t, cL, cH);
          const double cf = (b == 1 + 2 * ax) ? cL : cH;
          if (cf != 0.0) sum += cf * W[(size_t)(t * rcap + q) * kcap + j];
        }
      }
    }
    Wb[i] = (float)sum;
  }
  for (int i = tid; i < nbc * kpad; i += blockDim.x) {
    const int e = i / kpad, j = i - (i / kpad) * kpad;
    const int c = (src.nterm + 1) * rcap + e;
    Wbc[i] = (j < kcap && lp.live(c, r)) ? (float)W[(size_t)c * kcap + j] : 0.0f;
  }
  for (int j = tid; j < kpad; j += blockDim.x) vJs[j] = (vJ && j < kcap) ? (float)vJ[j] : 0.0f;

  constexpr int kPer = 16 / (int)sizeof(S);  // elements per cp.async granule
  const int gpr = src.ldz / kPer;            // granules per row
  const long ntiles = (nrows + TM - 1) / TM;
  double e0t = 0.0, e1t = 0.0;
  const int jg = tid & 7, mp = tid >> 3;  // 4 columns at 4*jg (+32 per column block), rows mp*RPT..
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long row0 = tile * TM;
    __syncthreads();  // the previous tile's buffers are free (and the weights are in place)
    for (int m = tid; m < TM; m += blockDim.x) fl[m] = (row0 + m < nrows) ? src.row_flags(row0 + m) : 0u;
    __syncthreads();
    // every granule of the tile's row blocks in flight at once; rows outside the core, and
    // neighbour rows that the row does not have, zero-filled
    const int per_block = TM * gpr;
    for (int i = tid; i < nb * per_block; i += blockDim.x) {
      const int b = i / per_block, rem = i - b * per_block;
      const int m = rem / gpr, g = rem - m * gpr;
      long k = row0 + m;
      bool ok = k < nrows;
      if (b > 0) {
        const int ax = (b - 1) >> 1;
        const bool upper = ((b - 1) & 1) != 0;
        ok = ok && ((fl[m] >> (2 * ax + (upper ? 1 : 0))) & 1u);
        k += upper ? src.stride[ax] : -src.stride[ax];
      }
      S* dst = raw + ((size_t)b * TM + m) * ldp + (size_t)g * kPer;
      const S* from = ok ? src.Z + k * src.ldz + (size_t)g * kPer : src.Z;
      cp_async16(dst, from, ok ? 16 : 0);
    }
    cp_async_wait_all();
    __syncthreads();
    // neighbour rows to differences with the centre rows: L_a -> C - L_a, H_a -> H_a - C
    {
      const int per = TM * rq;
      for (int i = tid; i < (nb - 1) * per; i += blockDim.x) {
        const int bb = i / per, rem = i - bb * per;
        const int m = rem / rq, q = rem - (rem / rq) * rq;
        const S c = raw[(size_t)m * ldp + q];
        S* v = raw + ((size_t)(1 + bb) * TM + m) * ldp + q;
        *v = (bb & 1) ? (*v - c) : (c - *v);
      }
    }
    __syncthreads();
    for (int jb = 0; jb < kpad; jb += 32) {
      const int j0 = jb + 4 * jg;
      if (j0 < kpad) {
        float acc[RPT][4];
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[q][u] = 0.0f;
        for (int b = 0; b < nb; ++b) {
          const S* ab = raw + ((size_t)b * TM + mp * RPT) * ldp;
          const float* wb = Wb + (size_t)b * rcap * kpad + j0;
#pragma unroll 4
          for (int q = 0; q < rq; ++q) {
            const float4 w = *reinterpret_cast<const float4*>(wb + (size_t)q * kpad);
#pragma unroll
            for (int rr = 0; rr < RPT; ++rr) {
              const float a = (float)ab[(size_t)rr * ldp + q];
              const float2 lo = __ffma2_rn(make_float2(a, a), make_float2(w.x, w.y), make_float2(acc[rr][0], acc[rr][1]));
              const float2 hi = __ffma2_rn(make_float2(a, a), make_float2(w.z, w.w), make_float2(acc[rr][2], acc[rr][3]));
              acc[rr][0] = lo.x; acc[rr][1] = lo.y; acc[rr][2] = hi.x; acc[rr][3] = hi.y;
            }
          }
        }
        // inflow columns: the face's inflow value on rows at that face, zero elsewhere
        for (int e = 0; e < nbc; ++e) {
          const int tt = src.bc_term[e], ax = src.axis[tt];
          const bool lower_face = src.w[tt] > 0;
          const float4 w = *reinterpret_cast<const float4*>(Wbc + (size_t)e * kpad + j0);
#pragma unroll
          for (int rr = 0; rr < RPT; ++rr) {
            const unsigned f = fl[mp * RPT + rr];
            const bool at_face = lower_face ? !((f >> (2 * ax)) & 1u) : !((f >> (2 * ax + 1)) & 1u);
            const float v = (at_face && row0 + mp * RPT + rr < nrows) ? (float)src.bcval[e * src.G + (int)(f >> 8)] : 0.0f;
            acc[rr][0] += v * w.x;
            acc[rr][1] += v * w.y;
            acc[rr][2] += v * w.z;
            acc[rr][3] += v * w.w;
          }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) Os[(size_t)(mp * RPT + q) * kpad + j0 + u] = acc[q][u];
      }
    }
    __syncthreads();
    update_epilogue<float, TM>(epi, Os, kpad, kcap, vJs, vJ != nullptr, rowv, row0, nrows, e0t, e1t);
  }
  if (partials) update_partials(red, e0t, e1t, partials);
}

}  // namespace ttk
