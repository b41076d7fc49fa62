// Gram-based factor of the merged core (the Gram method among the paper's rounding methods,
// Sec. 3.1): G = A^T A of the (possibly virtual) N_Z x R matrix A in FP64, then a square root
// R of G (R^T R = G, from a diagonally pivoted Cholesky), which stands in for the TSQR's R factor
// (the small-core sweep uses R only through R^T R).  Forming G squares the condition
// number: singular values below about sqrt(eps) |A| are not resolved.
#pragma once
#include "bigpass.cuh"
#include "small.cuh"

namespace ttk {

constexpr int kGramBlk = 64;    // G is computed in 64 x 64 blocks (bi <= bj)
constexpr int kGramTM = 64;     // rows per tile

__host__ __device__ inline int gram_nblk(int ncap) { return (ncap + kGramBlk - 1) / kGramBlk; }
__host__ __device__ inline int gram_npairs(int ncap) { const int b = gram_nblk(ncap); return b * (b + 1) / 2; }
template <class Src>
__host__ __device__ inline size_t gram_smem_bytes() {
  size_t b = sizeof(double) * 2 * (size_t)kGramTM * kGramBlk;
  b += sizeof(typename Src::Col) * 2 * kGramBlk;
  b = (b + 15) & ~(size_t)15;
  return b + sizeof(unsigned) * kGramTM + 2 * kGramBlk;
}

// CTA (split, pair): partial G block (bi, bj) over rows [split * rps, (split + 1) * rps).
// Thread (ty, tx) accumulates rows 4ty..4ty+3 x columns 4tx..4tx+3 of the block; in a diagonal
// block the micro-tiles wholly below the diagonal are skipped (the reduction reads the mirror).
template <class Src>
__global__ void __launch_bounds__(256) k_gram_tiles(Src src, LivePattern lp, long nrows, long rps,
                                                    double* __restrict__ part) {
  using Col = typename Src::Col;
  extern __shared__ __align__(16) unsigned char gram_smem[];
  const int ncap = lp.ncap();
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  double* Ai = reinterpret_cast<double*>(gram_smem);  // [TM][BLK]
  double* Aj = Ai + (size_t)kGramTM * kGramBlk;       // [TM][BLK]
  Col* cols = reinterpret_cast<Col*>(Aj + (size_t)kGramTM * kGramBlk);  // [2][BLK]
  size_t off = sizeof(double) * 2 * (size_t)kGramTM * kGramBlk + sizeof(Col) * 2 * kGramBlk;
  off = (off + 15) & ~(size_t)15;
  unsigned* fl = reinterpret_cast<unsigned*>(gram_smem + off);
  unsigned char* livec = reinterpret_cast<unsigned char*>(fl + kGramTM);  // [2][BLK]
  // pair index -> (bi, bj), bi <= bj, row-major over the upper triangle of blocks
  const int nb = gram_nblk(ncap);
  int p = blockIdx.y, bi = 0;
  while (p >= nb - bi) {
    p -= nb - bi;
    ++bi;
  }
  const int bj = bi + p;
  const bool diag = (bi == bj);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 2 * kGramBlk; i += blockDim.x) {
    const int c = (i < kGramBlk ? bi : bj) * kGramBlk + (i % kGramBlk);
    const bool ok = c < ncap;
    cols[i] = src.col(ok ? c : 0);
    livec[i] = (ok && lp.live(c, r)) ? 1 : 0;
  }
  const int ty = tid >> 4, tx = tid & 15;
  // micro-tiles wholly below the diagonal of a diagonal block, or wholly beyond the last
  // column (the last block of a width that is not a multiple of 64), have nothing to compute
  const bool active = !(diag && ty > tx) && (bi * kGramBlk + 4 * ty < ncap) && (bj * kGramBlk + 4 * tx < ncap);
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const long beg = (long)blockIdx.x * rps;
  const long end = (beg + rps < nrows) ? beg + rps : nrows;
  for (long row0 = beg; row0 < end; row0 += kGramTM) {
    __syncthreads();  // previous tile consumed (and the column set-up above done)
    for (int m = tid; m < kGramTM; m += blockDim.x) fl[m] = (row0 + m < end) ? src.row_flags(row0 + m) : 0u;
    __syncthreads();
    for (int m = warp; m < kGramTM; m += 8) {
      const long k = row0 + m;
      const unsigned f = fl[m];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        Ai[m * kGramBlk + c] = (k < end && livec[c]) ? src.template loadT<double>(cols[c], k, f) : 0.0;
        if (!diag)
          Aj[m * kGramBlk + c] =
              (k < end && livec[kGramBlk + c]) ? src.template loadT<double>(cols[kGramBlk + c], k, f) : 0.0;
      }
    }
    __syncthreads();
    if (active) {
      const double* Bj = diag ? Ai : Aj;
#pragma unroll 4
      for (int m = 0; m < kGramTM; ++m) {
        double a[4], b[4];
        ld4(Ai + m * kGramBlk + 4 * ty, a);
        ld4(Bj + m * kGramBlk + 4 * tx, b);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
      }
    }
  }
  double* out = part + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * kGramBlk * kGramBlk;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[(4 * ty + u) * kGramBlk + 4 * tx + v] = active ? acc[u][v] : 0.0;
}

// G[a][b] (full ncap x ncap) = sum over splits, in split order, of the canonical block entry.
static __global__ void k_gram_reduce(int ncap, int nsplit, int npairs, const double* __restrict__ part,
                              double* __restrict__ G) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)ncap * ncap) return;
  int a = (int)(idx / ncap), b = (int)(idx % ncap);
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  const int nb = gram_nblk(ncap);
  const int bi = a / kGramBlk, bj = b / kGramBlk;
  int p = 0;
  for (int q = 0; q < bi; ++q) p += nb - q;
  p += bj - bi;
  int ia = a % kGramBlk, ib = b % kGramBlk;
  if (bi == bj && (ia >> 2) > (ib >> 2)) {
    const int t = ia;
    ia = ib;
    ib = t;
  }
  double s = 0.0;
  for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * npairs + p) * kGramBlk * kGramBlk + ia * kGramBlk + ib];
  G[idx] = s;
}

// Diagonally pivoted Cholesky of the PSD Gram matrix G (n x n, overwritten): P^T G P = R^T R,
// stopped once the largest remaining pivot is at the round-off level of the largest diagonal
// entry (the rank of a rank-deficient sum).  Writes RZ = R P^T (n x n row-major, rows beyond the
// rank zero), so that RZ^T RZ = G.  One CTA; G stays in global memory (L2).
static __global__ void __launch_bounds__(1024) k_gram_pchol(int n, double* __restrict__ G, double* __restrict__ RZ,
                                                     int* __restrict__ perm) {
  __shared__ double rowj[512];
  __shared__ double redv[32];
  __shared__ int redi[32];
  __shared__ double d0;
  __shared__ int pj;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < n; i += blockDim.x) perm[i] = i;
  for (long i = tid; i < (long)n * n; i += blockDim.x) RZ[i] = 0.0;
  __syncthreads();
  const double thr_rel = 4.0 * n * 2.220446049250313e-16;
  for (int j = 0; j < n; ++j) {
    // largest remaining diagonal entry
    double best = -1.0;
    int bi = j;
    for (int q = j + tid; q < n; q += blockDim.x) {
      const int a = perm[q];
      const double v = G[(size_t)a * n + a];
      if (v > best) { best = v; bi = q; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = redv[0];
      int q = redi[0];
      for (int w = 1; w < nw; ++w)
        if (redv[w] > b || (redv[w] == b && redi[w] < q)) { b = redv[w]; q = redi[w]; }
      if (j == 0) d0 = b;
      const int t = perm[j];
      perm[j] = perm[q];
      perm[q] = t;
      pj = (b > thr_rel * d0 && b > 0.0) ? 1 : 0;
    }
    __syncthreads();
    if (!pj) break;  // the rest is round-off: rows j.. of RZ stay zero
    const int aj = perm[j];
    const double rjj = sqrt(G[(size_t)aj * n + aj]);
    const double inv = 1.0 / rjj;
    for (int q = j + tid; q < n; q += blockDim.x) {
      const int a = perm[q];
      const double r = (q == j) ? rjj : G[(size_t)aj * n + a] * inv;
      rowj[q] = r;
      RZ[(size_t)j * n + a] = r;
    }
    __syncthreads();
    const int m = n - j - 1;
    for (long idx = tid; idx < (long)m * m; idx += blockDim.x) {
      const int q1 = j + 1 + (int)(idx / m), q2 = j + 1 + (int)(idx % m);
      G[(size_t)perm[q1] * n + perm[q2]] -= rowj[q1] * rowj[q2];
    }
    __syncthreads();
  }
}

// Gram matrix G = A^T A (ncap x ncap, row-major, FP64) of the source's columns.  Takes its
// workspace from `ws` in dry runs too (same order) and launches nothing then.
template <class Src>
tt_status gram_matrix(cudaStream_t s, int num_sms, const Src& src, LivePattern lp, long nrows, Bump& ws,
                      double** G_out, int timer_cat = kTsqrLeaf) {
  const int ncap = lp.ncap();
  const int npairs = gram_npairs(ncap);
  const size_t smem = gram_smem_bytes<Src>();
  // about 8 waves of CTAs (3 per SM): the block pairs differ in work (diagonal and edge blocks
  // skip micro-tiles), and many short CTAs let the scheduler balance them
  const int occ = 3, waves = 8;
  long nsplit = ((long)num_sms * occ * waves + npairs - 1) / npairs;
  const long maxsplit = (nrows + kGramTM - 1) / kGramTM;
  if (nsplit > maxsplit) nsplit = maxsplit;
  if (nsplit < 1) nsplit = 1;
  long rps = (nrows + nsplit - 1) / nsplit;
  rps = ((rps + kGramTM - 1) / kGramTM) * kGramTM;
  nsplit = (nrows + rps - 1) / rps;
  if (nsplit < 1) nsplit = 1;
  double* part = ws.take<double>((size_t)nsplit * npairs * kGramBlk * kGramBlk);
  double* G = ws.take<double>((size_t)ncap * ncap);
  *G_out = G;
  if (ws.dry) return TT_OK;
  if (const tt_status a = smem_optin(k_gram_tiles<Src>, smem); a != TT_OK) return a;
  TimerScope scope(timer_cat, s);
  k_gram_tiles<Src><<<dim3((unsigned)nsplit, (unsigned)npairs), 256, smem, s>>>(src, lp, nrows, rps, part);
  count_launch();
  const long nn = (long)ncap * ncap;
  k_gram_reduce<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(ncap, (int)nsplit, npairs, part, G); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// Square-root factor RZ (ncap x ncap, row-major) of the Gram matrix of the source's columns.
// Takes its workspace from `ws` in dry runs too (same order), launches nothing then.
template <class Src>
tt_status gram_factor(cudaStream_t s, int num_sms, const Src& src, LivePattern lp, long nrows, Bump& ws,
                      DevCtrl* ctrl, int coop_grid_max, double** RZ_out, int timer_cat = kTsqrLeaf) {
  const int ncap = lp.ncap();
  if (ncap > 512) return TT_ERR_UNSUPPORTED;
  double* G = nullptr;
  tt_status st = gram_matrix(s, num_sms, src, lp, nrows, ws, &G, timer_cat);
  if (st != TT_OK) return st;
  int* perm = ws.take<int>(ncap);
  double* RZ = ws.take<double>((size_t)ncap * ncap);
  *RZ_out = RZ;
  if (ws.dry) return TT_OK;
  k_gram_pchol<<<1, 1024, 0, s>>>(ncap, G, RZ, perm); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

}  // namespace ttk
