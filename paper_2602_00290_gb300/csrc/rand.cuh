// Randomized factor of the merged core (the randomized method among the paper's rounding
// methods, Sec. 3.1): the first unfolding X_(1) = A B0 is sketched as Y = A (B0 omega) with a
// caller-drawn omega (n_2..n_d x l), Q = Y R_Y^{-1} from a Householder TSQR of Y's l columns, and
// C = Q^T A (l x R, FP64 accumulation) stands in for the TSQR's R factor of A (R^T R is then the
// Gram matrix of A restricted to the sketched range; the small-core sweep uses R only through
// R^T R).  No Gram matrix of A is formed, so the condition number is not squared.
#pragma once
#include "bigpass.cuh"
#include "small.cuh"

namespace ttk {

constexpr int kCrossTM = 64;  // rows per tile of the cross product

// Q[row][:l] <- Y[row][:l] R^{-1} in place (R upper triangular l x l, row-major); a pivot with
// |R_jj| <= 8 l eps max|R_ii| is round-off (the sketch has no more directions): its column is 0.
static __global__ void __launch_bounds__(128) k_rand_solve(long nrows, int l, const double* __restrict__ R, float* Yf,
                                                    double* Yd) {
  extern __shared__ double rsm[];
  double* Rs = rsm;  // [l][l]
  __shared__ double rmax;
  for (int i = threadIdx.x; i < l * l; i += blockDim.x) Rs[i] = R[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < l; ++i) m = fmax(m, fabs(Rs[i * l + i]));
    rmax = m;
  }
  __syncthreads();
  const double thr = 8.0 * l * 2.220446049250313e-16 * rmax;
  for (long row = blockIdx.x * (long)blockDim.x + threadIdx.x; row < nrows; row += (long)gridDim.x * blockDim.x) {
    double q[64];
    for (int j = 0; j < l; ++j) {
      double v = Yd ? Yd[row * l + j] : (double)Yf[row * l + j];
      for (int i = 0; i < j; ++i) v -= q[i] * Rs[i * l + j];
      const double rjj = Rs[j * l + j];
      q[j] = (fabs(rjj) > thr) ? v / rjj : 0.0;
    }
    for (int j = 0; j < l; ++j) {
      if (Yd) Yd[row * l + j] = q[j];
      else Yf[row * l + j] = (float)q[j];
    }
  }
}

// Partial cross products P[split] = sum over the split's rows of QL[row][a] * AR[row][b] for a
// 64 x 64 block (bi of the left columns, bj of the right columns); 4x4 FP64 register tiles.
template <class SrcL, class SrcR>
__global__ void __launch_bounds__(256) k_cross_tiles(SrcL srcL, int ncapL, SrcR srcR, LivePattern lpR, long nrows,
                                                     long rps, int nbj, double* __restrict__ part) {
  __shared__ __align__(16) double Ai[kCrossTM * 64];
  __shared__ __align__(16) double Aj[kCrossTM * 64];
  __shared__ typename SrcR::Col colsR[64];
  __shared__ unsigned char liveR[64];
  __shared__ unsigned fl[kCrossTM];
  const int ncapR = lpR.ncap();
  const int r = lpR.r_ptr ? *lpR.r_ptr : lpR.rcap;
  const int bi = blockIdx.y / nbj, bj = blockIdx.y % nbj;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 64; i += blockDim.x) {
    const int c = bj * 64 + i;
    colsR[i] = srcR.col(c < ncapR ? c : 0);
    liveR[i] = (c < ncapR && lpR.live(c, r)) ? 1 : 0;
  }
  const int ty = tid >> 4, tx = tid & 15;
  const bool active = (bi * 64 + 4 * ty < ncapL) && (bj * 64 + 4 * tx < ncapR);
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const long beg = (long)blockIdx.x * rps;
  const long end = (beg + rps < nrows) ? beg + rps : nrows;
  for (long row0 = beg; row0 < end; row0 += kCrossTM) {
    __syncthreads();
    for (int m = tid; m < kCrossTM; m += blockDim.x) fl[m] = (row0 + m < end) ? srcR.row_flags(row0 + m) : 0u;
    __syncthreads();
    for (int m = warp; m < kCrossTM; m += 8) {
      const long k = row0 + m;
      const unsigned f = fl[m];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        const int cl = bi * 64 + c;
        Ai[m * 64 + c] = (k < end && cl < ncapL) ? srcL.template loadT<double>(srcL.col(cl), k, 0u) : 0.0;
        Aj[m * 64 + c] = (k < end && liveR[c]) ? srcR.template loadT<double>(colsR[c], k, f) : 0.0;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll 4
      for (int m = 0; m < kCrossTM; ++m) {
        double a[4], b[4];
        ld4(Ai + m * 64 + 4 * ty, a);
        ld4(Aj + m * 64 + 4 * tx, b);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
      }
    }
  }
  double* out = part + ((size_t)blockIdx.x * gridDim.y + blockIdx.y) * 64 * 64;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[(4 * ty + u) * 64 + 4 * tx + v] = active ? acc[u][v] : 0.0;
}

// RZ (R x R, rows >= l zero) <- sum over splits of the cross blocks (C = Q^T A in its first l rows).
static __global__ void k_cross_reduce(int l, int R, int nsplit, int nbi, int nbj, const double* __restrict__ part,
                                      double* __restrict__ RZ) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)R * R) return;
  const int a = (int)(idx / R), b = (int)(idx % R);
  double s = 0.0;
  if (a < l) {
    const int p = (a / 64) * nbj + b / 64;
    const size_t off = (size_t)(a % 64) * 64 + (b % 64);
    for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * nbi * nbj + p) * 64 * 64 + off];
  }
  RZ[idx] = s;
}

// Mixed precision: Q = Y R_Y^{-1} with R_Y from an FP32 TSQR is orthonormal only to about
// kappa(Y) FP32 epsilon, and C = Q^T A then misses the projection onto span(Q).  With the FP64
// Gram G = Q^T Q = L L^T the projection is Q G^{-1} Q^T A, whose Gram in the A-columns equals
// that of L^{-1} C: the first l rows of RZ become L^{-1} C.  Columns of Q that the solve zeroed
// (no sketch direction) have a zero pivot here and keep zero rows.  One CTA (l <= 64).
static __global__ void __launch_bounds__(128) k_rand_correct(int l, int R, const double* __restrict__ G,
                                                             double* __restrict__ RZ) {
  __shared__ double Ls[64 * 64];
  __shared__ int ok[64];
  for (int i = threadIdx.x; i < l * l; i += blockDim.x) Ls[i] = G[i];
  __syncthreads();
  double gmax = 0.0;
  for (int j = 0; j < l; ++j) gmax = fmax(gmax, Ls[j * l + j]);
  for (int j = 0; j < l; ++j) {
    if (threadIdx.x == 0) {
      double d = Ls[j * l + j];
      for (int k = 0; k < j; ++k) d -= Ls[j * l + k] * Ls[j * l + k];
      ok[j] = d > 1e-12 * gmax;
      Ls[j * l + j] = ok[j] ? sqrt(d) : 0.0;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < l; i += blockDim.x) {
      double v = Ls[i * l + j];
      for (int k = 0; k < j; ++k) v -= Ls[i * l + k] * Ls[j * l + k];
      Ls[i * l + j] = ok[j] ? v / Ls[j * l + j] : 0.0;
    }
    __syncthreads();
  }
  for (int b = threadIdx.x; b < R; b += blockDim.x) {
    double y[64];
    for (int j = 0; j < l; ++j) {
      double v = RZ[(size_t)j * R + b];
      for (int k = 0; k < j; ++k) v -= Ls[j * l + k] * y[k];
      y[j] = ok[j] ? v / Ls[j * l + j] : 0.0;
    }
    for (int j = 0; j < l; ++j) RZ[(size_t)j * R + b] = y[j];
  }
}

}  // namespace ttk
