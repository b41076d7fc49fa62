// Blocked Householder TSQR leaf (FP32), with the block of rows held in tensor memory.
//
// The leaf of the column-owner kernels forms one reflector per column for every block of 32
// rows, so a row costs 160 dependent reflector steps over 32-row chains.  Here a CTA of 256
// threads takes blocks of 256 rows, one row per thread, and factors them against its running
// upper-triangular R (packed in shared memory) panel by panel, 32 columns at a time:
//   * panel: for each column k of the panel, the reflector of [R_kk; C(:, k)] (the same
//     structured Householder step as the other leaves: v = [1; u], u = C(:, k) / (alpha - beta),
//     tau = (beta - alpha) / beta), from a block-wide norm, and in one batched block reduction the
//     dots of u with every other panel column (w_c = R_kc + u . C(:, c), applied at once) and with
//     the previous reflectors of the panel (the column of the compact-WY factor T);
//   * trailing columns: the panel's block reflector I - V T V^T (V = [I; U]) applied as a whole,
//     W = R(panel rows, trailing) + U^T C(:, trailing), Y = T^T W, R(panel rows, trailing) -= Y,
//     C(:, trailing) -= U Y (FP32 FMAs, 32-column chunks).
// So a row costs 160 reflector steps over 256-row block reductions, and the trailing work is
// dense.  The block (256 rows x ncap columns, FP32) lives in tensor memory: thread t's row is
// TMEM lane 32 (warp mod 4) + lane, in the column half warp / 4 (cb columns each); tcgen05.ld and
// tcgen05.st move a row's 32-column chunk to and from registers.  One CTA per SM (the block takes
// 2 cb of the 512 TMEM columns).  Same contract as the other leaves: R of the CTA's row range,
// FP64 row-major ncap x ncap, into Rout.
#pragma once
#include "bigpass.cuh"
#include "tc.cuh"

namespace ttk {

constexpr int kBlkRows = 256;  // rows per block: one per thread
constexpr int kBlkUld = 36;    // row stride of the U and C-chunk tiles (16-byte rows, conflict-free)

// TMEM columns of one half of the block (ncap rounded up to 32) and of the allocation.
__host__ __device__ inline int blk_cb(int ncap) { return (ncap + 31) & ~31; }

// Shared memory: column descriptors, packed R, U and C-chunk tiles [256][36], W/Y [32][ncap],
// T [32][33], reduction scratch (norm partials [8], dot partials [8][32], per-warp sums [8][32]),
// row flags [256].  At least 117 KB, so that one CTA is resident per SM.
template <class Src>
__host__ __device__ inline size_t tsqr_blk_smem_bytes(int ncap) {
  size_t b = (sizeof(typename Src::Col) * (size_t)ncap + 15) & ~(size_t)15;
  b += sizeof(float) * tsqr_r_elems(ncap);
  b += sizeof(float) * 2 * (size_t)kBlkRows * kBlkUld;
  b += sizeof(float) * 32 * (size_t)ncap;
  b += sizeof(float) * 32 * 33;
  b += sizeof(float) * (8 + 8 * 32 + 8 * 32);
  b += sizeof(unsigned) * kBlkRows;
  b = (b + 15) & ~(size_t)15;
  return b < 117 * 1024 ? 117 * 1024 : b;
}

// Sum over the 32 lanes of a[c], for every c, leaving lane l with the sum of a[l]
// (a butterfly that halves the vector at every level: 31 shuffles).
__device__ __forceinline__ float warp_reduce_scatter32(float (&a)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = upper ? a[i] : a[i + off];
      const float keep = upper ? a[i + off] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return a[0];
}

template <class Src>
__global__ void __launch_bounds__(256, 1) k_tsqr_leaf_blk(Src src, LivePattern lp, long nrows, long rpc,
                                                          double* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char blk_smem[];
  using Col = typename Src::Col;
  const int ncap = lp.ncap();
  const int cb = blk_cb(ncap);
  Col* cols = reinterpret_cast<Col*>(blk_smem);
  size_t off = (sizeof(Col) * (size_t)ncap + 15) & ~(size_t)15;
  float* Rs = reinterpret_cast<float*>(blk_smem + off);
  off += sizeof(float) * tsqr_r_elems(ncap);
  float* Us = reinterpret_cast<float*>(blk_smem + off);  // [256][36]: the panel's reflectors by row
  off += sizeof(float) * kBlkRows * kBlkUld;
  float* Cc = reinterpret_cast<float*>(blk_smem + off);  // [256][36]: a 32-column chunk of the block
  off += sizeof(float) * kBlkRows * kBlkUld;
  float* Ws = reinterpret_cast<float*>(blk_smem + off);  // [32][ncap]: W, then Y, of the trailing columns
  off += sizeof(float) * 32 * (size_t)ncap;
  float* Ts = reinterpret_cast<float*>(blk_smem + off);  // [32][33]: T of the panel
  off += sizeof(float) * 32 * 33;
  float* redn = reinterpret_cast<float*>(blk_smem + off);  // [8]
  float* redq = redn + 8;                                   // [8][32]
  float* qw = redq + 8 * 32;                                // [8][32]
  unsigned* fl = reinterpret_cast<unsigned*>(qw + 8 * 32);  // [256]
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  for (int c = tid; c < ncap; c += blockDim.x) cols[c] = src.col(c);
  for (int i = tid; i < ncap * (ncap + 1) / 2; i += blockDim.x) Rs[i] = 0.0f;
  const uint32_t ncols = tc::tmem_cols(2 * cb);
  if (warp == 0) {
    tc::tmem_alloc(&tbase, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t trow = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * cb);
  const long beg = (long)blockIdx.x * rpc;
  const long end = (beg + rpc < nrows) ? beg + rpc : nrows;

  for (long row0 = beg; row0 < end; row0 += kBlkRows) {
    // ---- the block's rows into TMEM (dead columns and rows beyond the range are zero)
    const long k = row0 + tid;
    const bool rowok = k < end;
    fl[tid] = rowok ? src.row_flags(k) : 0u;
    const unsigned f = fl[tid];
    for (int c0 = 0; c0 < cb; c0 += 32) {
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        v[j] = (rowok && c < ncap && lp.live(c, r)) ? src.template loadT<float>(cols[c], k, f) : 0.0f;
      }
      tc::tmem_st32(trow + (uint32_t)c0, v);
    }
    tc::tmem_wait_st();

    // ---- panels of 32 columns; thread t's row of the panel is row t of Us (columns, then from
    // step k on the reflector entries u), so that every index into it may be a run-time one
    float* xr = Us + (size_t)tid * kBlkUld;
    for (int j0 = 0; j0 < ncap; j0 += 32) {
      const int pw = (ncap - j0 < 32) ? ncap - j0 : 32;
      {
        float v[32];
        tc::tmem_ld32(trow + (uint32_t)j0, v);
        tc::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; c += 4)
          *reinterpret_cast<float4*>(xr + c) = make_float4(c < pw ? v[c] : 0.0f, c + 1 < pw ? v[c + 1] : 0.0f,
                                                           c + 2 < pw ? v[c + 2] : 0.0f, c + 3 < pw ? v[c + 3] : 0.0f);
      }
      for (int i = tid; i < 32 * 33; i += blockDim.x) Ts[i] = 0.0f;
      float pend = 0.0f;  // warp 0, lane c: the new R(k, j0 + c) of the last step, written after
      int pend_at = -1;   // the next barrier (every thread reads the old one in that step)
      for (int kk = 0; kk < pw; ++kk) {
        const int kc = j0 + kk;
        if (!lp.live(kc, r)) continue;  // the same for every thread
        const float xk = xr[kk];
        // norm of the column below R(k, k)
        {
          const float s = warp_sum(xk * xk);
          if (lane == 0) redn[warp] = s;
        }
        __syncthreads();
        if (warp == 0 && pend_at >= 0) {
          Rs[pend_at] = pend;
          pend_at = -1;
        }
        float s2 = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) s2 += redn[w];
        const int rk = tri_off(kc, ncap);  // R(k, k) in the packed triangle; R(k, c) at rk + c - k
        const float alpha = Rs[rk];
        float tau = 0.0f, sc = 0.0f, beta = alpha;
        if (s2 > 0.0f) {
          const float nrm = sqrtf(alpha * alpha + s2);
          beta = (alpha >= 0.0f) ? -nrm : nrm;
          sc = chain_div<float>(1.0f, alpha - beta);
          tau = chain_div<float>(beta - alpha, beta);
        }
        const float u = xk * sc;
        xr[kk] = u;
        // dots of u with the other panel columns (c > kk) and the earlier reflectors (c < kk)
        float q[32];
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          const float4 xv = *reinterpret_cast<const float4*>(xr + c);
          q[c] = u * xv.x;
          q[c + 1] = u * xv.y;
          q[c + 2] = u * xv.z;
          q[c + 3] = u * xv.w;
        }
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (c == kk) q[c] = 0.0f;
        redq[warp * 32 + lane] = warp_reduce_scatter32(q, lane);
        __syncthreads();
        {
          float Q = 0.0f;
#pragma unroll
          for (int w = 0; w < 8; ++w) Q += redq[w * 32 + lane];
          qw[warp * 32 + lane] = Q;
        }
        __syncwarp();
        const float* Qw = qw + warp * 32;
        // w_c = R(k, c) + u . C(:, c) for the panel columns c > kk; C(:, c) -= tau w_c u
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          float4 xv = *reinterpret_cast<const float4*>(xr + c);
          float xe[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int cc = c + e;
            if (cc > kk && cc < pw) {
              const float wc = Rs[rk + cc - kk] + Qw[cc];
              xe[e] = fmaf(-tau * wc, u, xe[e]);
              if (warp == 0 && lane == cc) {
                pend = Rs[rk + cc - kk] - tau * wc;
                pend_at = rk + cc - kk;
              }
            }
          }
          *reinterpret_cast<float4*>(xr + c) = make_float4(xe[0], xe[1], xe[2], xe[3]);
        }
        if (warp == 0 && lane == kk) {
          pend = beta;
          pend_at = rk;
        }
        // column kk of T: T(l, kk) = -tau sum_{m = l}^{kk-1} T(l, m) (u_m . u_kk), T(kk, kk) = tau
        if (warp == 1) {
          if (lane < kk) {
            float t = 0.0f;
            for (int m = lane; m < kk; ++m) t = fmaf(Ts[lane * 33 + m], Qw[m], t);
            Ts[lane * 33 + kk] = -tau * t;
          } else if (lane == kk) {
            Ts[kk * 33 + kk] = tau;
          }
        }
      }
      __syncthreads();
      if (warp == 0 && pend_at >= 0) Rs[pend_at] = pend;
      __syncthreads();

      // ---- the panel's block reflector on the trailing columns
      const int t0 = j0 + 32;
      const int nc = ncap - t0;
      if (nc > 0) {
        // W = R(panel rows, trailing) + U^T C(:, trailing), 32 columns at a time
        const int kq = tid >> 3, cq = (tid & 7) * 4;
        for (int c0 = t0; c0 < ncap; c0 += 32) {
          float v[32];
          tc::tmem_ld32(trow + (uint32_t)c0, v);
          tc::tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 32; c += 4)
            *reinterpret_cast<float4*>(Cc + (size_t)tid * kBlkUld + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
          __syncthreads();
          float2 a01 = make_float2(0.0f, 0.0f), a23 = make_float2(0.0f, 0.0f);
#pragma unroll 8
          for (int i = 0; i < kBlkRows; ++i) {
            const float uk = Us[(size_t)i * kBlkUld + kq];
            const float4 c4 = *reinterpret_cast<const float4*>(Cc + (size_t)i * kBlkUld + cq);
            a01 = __ffma2_rn(make_float2(uk, uk), make_float2(c4.x, c4.y), a01);
            a23 = __ffma2_rn(make_float2(uk, uk), make_float2(c4.z, c4.w), a23);
          }
          const float acc[4] = {a01.x, a01.y, a23.x, a23.y};
          const int kr = j0 + kq;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int col = c0 + cq + q;
            if (col < ncap && kr < ncap) Ws[(size_t)kq * ncap + (col - t0)] = acc[q] + Rs[tri_off(kr, ncap) + col - kr];
          }
          __syncthreads();
        }
        // Y = T^T W (in place), and R(panel rows, trailing) -= Y: a thread per trailing column
        if (tid < nc) {
          float wv[32];
#pragma unroll
          for (int l = 0; l < 32; ++l) wv[l] = (j0 + l < ncap) ? Ws[(size_t)l * ncap + tid] : 0.0f;
#pragma unroll
          for (int kk = 0; kk < 32; ++kk) {
            float y = 0.0f;
#pragma unroll
            for (int l = 0; l <= kk; ++l) y = fmaf(Ts[l * 33 + kk], wv[l], y);
            if (j0 + kk < ncap) {
              Ws[(size_t)kk * ncap + tid] = y;
              Rs[tri_off(j0 + kk, ncap) + (t0 + tid) - (j0 + kk)] -= y;
            }
          }
        }
        __syncthreads();
        // C(:, trailing) -= U Y: every thread its own row, 32 columns at a time
        for (int c0 = t0; c0 < ncap; c0 += 32) {
          float v[32];
          tc::tmem_ld32(trow + (uint32_t)c0, v);
          tc::tmem_wait_ld();
          const int cw = (ncap - c0 < 32) ? ncap - c0 : 32;
          for (int kk = 0; kk < 32; ++kk) {
            const float nu = -xr[kk];
            const float* yk = Ws + (size_t)kk * ncap + (c0 - t0);
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              if (j < cw) {
                const float2 yy = make_float2(yk[j], (j + 1 < cw) ? yk[j + 1] : 0.0f);
                const float2 o = __ffma2_rn(make_float2(nu, nu), yy, make_float2(v[j], v[j + 1]));
                v[j] = o.x;
                v[j + 1] = o.y;
              }
            }
          }
          tc::tmem_st32(trow + (uint32_t)c0, v);
        }
        tc::tmem_wait_st();
      }
      __syncthreads();
    }
  }
  __syncthreads();
  write_R<float, 32>(Rs, ncap, Rout + (size_t)blockIdx.x * ncap * ncap);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, ncols);
  }
}

// Host driver: one leaf per SM at most (the block takes the tensor memory of an SM), rows split
// in whole 256-row blocks, then the merge tree; the same contract as run_tsqr.
template <class Src>
tt_status run_tsqr_blk(cudaStream_t s, int num_sms, const Src& src, LivePattern lp, long nrows, int max_leaves,
                       double* ws_a, double* ws_b, double** Rfinal, int leaf_cat = kTsqrLeaf) {
  const int ncap = lp.ncap();
  if (ncap > 224) return TT_ERR_UNSUPPORTED;
  const size_t smem = tsqr_blk_smem_bytes<Src>(ncap);
  if (smem > 227 * 1024) return TT_ERR_UNSUPPORTED;
  auto leaf = k_tsqr_leaf_blk<Src>;
  if (const tt_status a = smem_optin(leaf, smem); a != TT_OK) return a;
  const LeafSplit sp = tsqr_split(nrows, kBlkRows, num_sms, 1, max_leaves, 0);
  {
    TimerScope scope(leaf_cat, s);
    leaf<<<(unsigned)sp.leaves, kBlkRows, smem, s>>>(src, lp, nrows, sp.rpc, ws_a);
    count_launch();
  }
  return merge_tree<float>(s, lp, (int)sp.leaves, ws_a, ws_b, Rfinal);
}

}  // namespace ttk
