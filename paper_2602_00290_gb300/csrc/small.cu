// Small-core sweep of SVD-based TT rounding (Sec. 3.1 footnote, Oseledets 2011) for the
// merged topologies d = 2 (Z, mu) and d = 3 (Z, Theta, Phi).
//
// Given R_Z from the QR of the merged core of a (possibly virtual) TT sum and the dense
// right part B0 of that sum (B0[c][l][p] = sum_b Theta_sum[c][l][b] Phi_sum[b][p]), the TT is
// X = Q_Z * Y with Y = R_Z B0.  The left-to-right orthogonalisation of the small cores and
// the right-to-left truncated SVDs of the rounding act on Y only:
//   bond 2: SVD of Y viewed as (R n1) x n2 -> sigma_2, V_2; ||X|| = ||Y||_F,
//           delta = tol ||X|| / sqrt(d-1); k_2 by the tail rule; Phi_new = V_2(:, :k_2)^T.
//   bond 1: SVD of Y_2 = Y x_3 V_2k viewed as R x (n1 k_2) -> sigma_1, V_1; k_1;
//           Theta_new = V_1(:, :k_1)^T.
// The new merged core is the projection of X onto the new right frame,
//   Z_new = Z_sum W,   W = (B0 x_3 V_2k) V_1k,
// which equals Q_Z U_1 S_1 of the textbook sweep and needs no inverse of R_Z.
// Every SVD is a one-sided (Hestenes) Jacobi sweep run by a cooperative grid directly on the
// unfolding (bond 2: Y as (R n1) x n2 with accumulated rotations; bond 1: Y_2^T, whose
// normalised converged columns are the right singular vectors).
#include <cstddef>
#include <cstdio>

#include "bigpass.cuh"
#include "small.cuh"

namespace ttk {
namespace {

constexpr double kPi = 3.14159265358979323846;

template <typename TA, typename TB>
__global__ void k_small_gemm(int M, int N, int K, const TA* __restrict__ A, long sa0, long sa1,
                             const TB* __restrict__ B, long sb0, long sb1, double* __restrict__ C, long ldc,
                             const int* __restrict__ nlive, const double* __restrict__ inv_colscale,
                             const TA* __restrict__ A2, double* __restrict__ C2) {
  // a second product with the same B, shape and strides (A2 B into C2) in the CTAs of z = 1
  if (blockIdx.z == 1) {
    A = A2;
    C = C2;
  }
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.y * 16 + ty;
  const int j = blockIdx.x * 16 + tx;
  const int nl = nlive ? *nlive : N;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + tx, kb = k0 + ty;
    As[ty][tx] = (i < M && ka < K) ? (double)A[i * sa0 + ka * sa1] : 0.0;
    const int jb = blockIdx.x * 16 + tx;
    Bs[ty][tx] = (kb < K && jb < N && jb < nl) ? (double)B[kb * sb0 + jb * sb1] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc += As[ty][kk] * Bs[kk][tx];
    __syncthreads();
  }
  if (i < M && j < N) {
    double v = 0.0;
    if (j < nl) {
      v = acc;
      if (inv_colscale) {
        const double sg = inv_colscale[j];
        v = (sg > 0.0) ? v / sg : 0.0;
      }
    }
    C[i * ldc + j] = v;
  }
}

// C = A B with the K range split over gridDim.z slices of kslice (a multiple of 16): slice z writes
// its partial product, unmasked, to part[z] (M x N, row-major); k_small_gemm_sum adds the slices in
// order.  For products with few output tiles and a long K (W = B0p V1: 10 x 2 tiles, K = 512),
// where one CTA per tile leaves most SMs idle and each tile's FP64 chain runs on one SM.
__global__ void k_small_gemm_part(int M, int N, int K, int kslice, const double* __restrict__ A, long sa0, long sa1,
                                  const double* __restrict__ B, long sb0, long sb1, double* __restrict__ part) {
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.y * 16 + ty;
  const int j = blockIdx.x * 16 + tx;
  const int kbeg = blockIdx.z * kslice;
  const int kend = min(kbeg + kslice, K);
  double acc = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    const int ka = k0 + tx, kb = k0 + ty;
    As[ty][tx] = (i < M && ka < kend) ? A[i * sa0 + ka * sa1] : 0.0;
    const int jb = blockIdx.x * 16 + tx;
    Bs[ty][tx] = (kb < kend && jb < N) ? B[kb * sb0 + jb * sb1] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc += As[ty][kk] * Bs[kk][tx];
    __syncthreads();
  }
  if (i < M && j < N) part[((size_t)blockIdx.z * M + i) * N + j] = acc;
}

__global__ void k_small_gemm_sum(int M, int N, int nslice, const double* __restrict__ part, double* __restrict__ C,
                                 long ldc, const int* __restrict__ nlive) {
  const int nl = nlive ? *nlive : N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)M * N; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx - (long)i * N);
    double v = 0.0;
    if (j < nl)
      for (int z = 0; z < nslice; ++z) v += part[(size_t)z * M * N + idx];
    C[i * ldc + j] = v;
  }
}

// Rank decision for one bond.  first != 0: this is the first SVD of the right-to-left sweep,
// which also fixes ||X|| = sqrt(sum sigma^2) and delta = tol ||X|| / sqrt(d-1).  The kept rank
// is the smallest k >= 1 with sqrt(sum_{j>=k} sigma_j^2) <= delta (tol > 0), or the full rank
// of the unfolding (tol == 0), then capped by rmax and kcap.
__global__ void k_decide(const double* __restrict__ sigma, int n, int first, int dcores, double tol, int rmax,
                         int kcap, long full_rank_cap, const int* rptr, int nblk, int nextra, int rows_mul,
                         const int* r2ptr, int r2_nblk, int r2_nextra, const int* kprev, int cols_mul,
                         int cols_fixed, DevCtrl* ctrl, int slot, const double* extra_tail) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double tail_beyond = extra_tail ? *extra_tail : 0.0;  // energy beyond the n listed values
  if (first) {
    double s2 = tail_beyond;
    for (int j = n - 1; j >= 0; --j) s2 += sigma[j] * sigma[j];
    const double nrm = sqrt(s2);
    ctrl->norm = nrm;
    ctrl->delta = tol * nrm / sqrt((double)(dcores - 1 > 0 ? dcores - 1 : 1));
    if (!isfinite(nrm)) latch(&ctrl->status, TT_ERR_NONFINITE);
  }
  const double delta = ctrl->delta;
  // live dimensions of the unfolding
  const long rlive = (long)nblk * (rptr ? *rptr : 0) + nextra;
  long rows = rlive * rows_mul;
  if (r2ptr) {
    const long r2 = (long)r2_nblk * (*r2ptr) + r2_nextra;
    if (r2 < rows) rows = r2;
  }
  if (full_rank_cap > 0 && full_rank_cap < rows) rows = full_rank_cap;
  const long cols = kprev ? (long)(*kprev) * cols_mul : (long)cols_fixed;
  long full = rows < cols ? rows : cols;
  if (full > n) full = n;
  long k;
  if (tol == 0.0) {
    k = full;
  } else {
    k = n;
    double tail2 = tail_beyond;
    // tail(k) = sqrt(sum_{j>=k} sigma_j^2); smallest k >= 1 with tail(k) <= delta
    long best = n;
    for (long kk = n; kk >= 1; --kk) {
      if (kk < n) tail2 += sigma[kk] * sigma[kk];
      if (sqrt(tail2) <= delta) best = kk;
      else break;
    }
    k = best;
    if (k > full) k = full;
  }
  if (k > rmax) k = rmax;
  if (k > kcap) k = kcap;
  if (k < 1) k = 1;
  ctrl->k[slot] = (int)k;
}

// Classical Gram-Schmidt applied twice (FP64) to the first k columns of V (nv x ldv,
// row-major), in column order, normalising each.  The columns come sorted by decreasing
// singular value, so every column is cleaned of its components along the larger ones; a column
// with nothing left (relative remainder <= 1e-12) is replaced by the first canonical vector on a
// live row (row % rowmod < rowlive) that is independent of the earlier columns.
__global__ void __launch_bounds__(1024) k_orthonormalise(int nv, int ldv, double* __restrict__ V, const int* kptr,
                                                         int rowmod, const int* rowlive_ptr) {
  __shared__ double red[33];
  __shared__ double h[1024];
  const int k = *kptr;
  const int rowlive = rowlive_ptr ? *rowlive_ptr : rowmod;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    int cand = -1;
    for (int attempt = 0; attempt <= nv; ++attempt) {
      if (attempt > 0) {
        do {
          ++cand;
        } while (cand < nv && (cand % rowmod) >= rowlive);
        if (cand >= nv) break;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) V[(size_t)i * ldv + j] = (i == cand) ? 1.0 : 0.0;
        __syncthreads();
      }
      double n0 = 0.0;
      for (int i = threadIdx.x; i < nv; i += blockDim.x) n0 += V[(size_t)i * ldv + j] * V[(size_t)i * ldv + j];
      n0 = sqrt(block_sum(n0, red));
      for (int pass = 0; pass < 2; ++pass) {
        for (int i2 = warp; i2 < j; i2 += nwarps) {
          double sacc = 0.0;
          for (int i = lane; i < nv; i += 32) sacc += V[(size_t)i * ldv + i2] * V[(size_t)i * ldv + j];
          sacc = warp_sum(sacc);
          if (lane == 0) h[i2] = sacc;
        }
        __syncthreads();
        // warp per row: the sum over the earlier columns is split across lanes and reduced by
        // shuffles, instead of one dependent FP64 chain of length j per row
        for (int i = warp; i < nv; i += nwarps) {
          double part = 0.0;
          for (int i2 = lane; i2 < j; i2 += 32) part += h[i2] * V[(size_t)i * ldv + i2];
          part = warp_sum(part);
          if (lane == 0) V[(size_t)i * ldv + j] -= part;
        }
        __syncthreads();
      }
      double n1 = 0.0;
      for (int i = threadIdx.x; i < nv; i += blockDim.x) n1 += V[(size_t)i * ldv + j] * V[(size_t)i * ldv + j];
      n1 = sqrt(block_sum(n1, red));
      if (n1 > 1e-12 * n0 && n1 > 0.0) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) V[(size_t)i * ldv + j] /= n1;
        __syncthreads();
        break;
      }
    }
  }
}

// k_orthonormalise for nv <= 32 rows and k <= 32 columns in one warp, on V staged in shared
// memory (row i at V[i * 33 + c]): column dots with one lane per earlier column, the update with
// one lane per row, warp shuffles for norms; no block-wide barriers.  Same algorithm and outputs.
__device__ void cgs2_warp_staged(int nv, int k, int rowmod, int rowlive, double* V, double* h) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < k; ++j) {
    int cand = -1;
    for (int attempt = 0; attempt <= nv; ++attempt) {
      if (attempt > 0) {
        do {
          ++cand;
        } while (cand < nv && (cand % rowmod) >= rowlive);
        if (cand >= nv) break;
        if (lane < nv) V[lane * 33 + j] = (lane == cand) ? 1.0 : 0.0;
        __syncwarp();
      }
      double x = (lane < nv) ? V[lane * 33 + j] : 0.0;
      const double n0 = sqrt(warp_sum(x * x));
      for (int pass = 0; pass < 2; ++pass) {
        // both dependent FP64 chains in four partial sums
        double h0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0;
        if (lane < j) {
          int i = 0;
          for (; i + 3 < nv; i += 4) {
            h0 += V[i * 33 + lane] * V[i * 33 + j];
            h1 += V[(i + 1) * 33 + lane] * V[(i + 1) * 33 + j];
            h2 += V[(i + 2) * 33 + lane] * V[(i + 2) * 33 + j];
            h3 += V[(i + 3) * 33 + lane] * V[(i + 3) * 33 + j];
          }
          for (; i < nv; ++i) h0 += V[i * 33 + lane] * V[i * 33 + j];
        }
        h[lane] = (h0 + h1) + (h2 + h3);
        __syncwarp();
        if (lane < nv) {
          double v0 = V[lane * 33 + j], v1 = 0.0, v2 = 0.0, v3 = 0.0;
          int c = 0;
          for (; c + 3 < j; c += 4) {
            v0 -= h[c] * V[lane * 33 + c];
            v1 -= h[c + 1] * V[lane * 33 + c + 1];
            v2 -= h[c + 2] * V[lane * 33 + c + 2];
            v3 -= h[c + 3] * V[lane * 33 + c + 3];
          }
          for (; c < j; ++c) v0 -= h[c] * V[lane * 33 + c];
          V[lane * 33 + j] = (v0 + v1) + (v2 + v3);
        }
        __syncwarp();
      }
      x = (lane < nv) ? V[lane * 33 + j] : 0.0;
      const double n1 = sqrt(warp_sum(x * x));
      if (n1 > 1e-12 * n0 && n1 > 0.0) {
        if (lane < nv) V[lane * 33 + j] = x / n1;
        __syncwarp();
        break;
      }
    }
  }
  __syncwarp();
}

// The first k columns of V (nv <= 32 rows, k <= ldv <= 32) made orthonormal by Newton-Schulz steps
// towards the polar factor, V <- V (3 I - V^T V) / 2, when they are already close to
// orthonormal (the right singular vectors of a Jacobi sweep, normalised in FP64): with
// e = max |V^T V - I| <= 1e-4 each step takes e to about 1.5 e^2, so one step suffices for e <=
// 1e-8 (FP64 Jacobi) and two for FP32-accurate columns.  The span of the columns is unchanged and
// the columns move by O(e).  Other inputs (a vanishing or far from orthogonal column) take the
// column-by-column Gram-Schmidt of cgs2_warp_staged, which also replaces dependent columns.
// Four warps compute V^T V and the update as small matrix products in shared memory: no
// dependent chain longer than nv, against the column-by-column chains of Gram-Schmidt.
__global__ void __launch_bounds__(128) k_orthonormalise_polar(int nv, int ldv, double* __restrict__ Vg,
                                                              const int* kptr, int rowmod, const int* rowlive_ptr) {
  __shared__ double V[32 * 33];
  __shared__ double G[32 * 33];
  __shared__ double h[32];
  __shared__ double emax[4];
  __shared__ int nsteps;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = *kptr;
  const int rowlive = rowlive_ptr ? *rowlive_ptr : rowmod;
  for (int idx = tid; idx < nv * ldv; idx += blockDim.x) {
    const int i = idx / ldv, c = idx - (idx / ldv) * ldv;
    V[i * 33 + c] = Vg[idx];
  }
  __syncthreads();
  // G = V^T V over the first k columns; returns max |G - I| over this thread's entries
  auto gram = [&]() -> double {
    double e = 0.0;
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
      const int a = idx / k, b = idx - (idx / k) * k;
      double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
      int i = 0;
      for (; i + 3 < nv; i += 4) {
        g0 += V[i * 33 + a] * V[i * 33 + b];
        g1 += V[(i + 1) * 33 + a] * V[(i + 1) * 33 + b];
        g2 += V[(i + 2) * 33 + a] * V[(i + 2) * 33 + b];
        g3 += V[(i + 3) * 33 + a] * V[(i + 3) * 33 + b];
      }
      for (; i < nv; ++i) g0 += V[i * 33 + a] * V[i * 33 + b];
      const double g = (g0 + g1) + (g2 + g3);
      G[a * 33 + b] = g;
      const double d = fabs(g - (a == b ? 1.0 : 0.0));
      e = (d > e || d != d) ? d : e;  // a NaN counts as far from orthonormal
    }
    return e;
  };
  double e = gram();
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, e, o);
    e = (t > e || t != t) ? t : e;
  }
  if (lane == 0) emax[warp] = e;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = (emax[w] > m || emax[w] != emax[w]) ? emax[w] : m;
    // no step below the FP64 round-off of a k-term sum; one from e <= 1e-8; two from e <= 1e-4;
    // otherwise Gram-Schmidt (-1)
    const double floor64 = 8.0 * 2.220446049250313e-16 * (k > 1 ? k : 1);
    nsteps = (m <= floor64) ? 0 : (m <= 1e-8) ? 1 : (m <= 1e-4) ? 2 : -1;
  }
  __syncthreads();
  const int ns = nsteps;
  if (ns < 0) {
    if (warp == 0) cgs2_warp_staged(nv, k, rowmod, rowlive, V, h);
    __syncthreads();
  }
  for (int step = 0; step < ns; ++step) {
    if (step > 0) {
      (void)gram();
      __syncthreads();
    }
    // V[i][b] <- 1.5 V[i][b] - 0.5 sum_a V[i][a] G[a][b] (b < k): nv k <= 1024 entries, 8 a thread
    double w[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int idx = tid + r * (int)blockDim.x;
      w[r] = 0.0;
      if (idx < nv * k) {
        const int i = idx / k, b = idx - (idx / k) * k;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int a = 0;
        for (; a + 3 < k; a += 4) {
          s0 += V[i * 33 + a] * G[a * 33 + b];
          s1 += V[i * 33 + a + 1] * G[(a + 1) * 33 + b];
          s2 += V[i * 33 + a + 2] * G[(a + 2) * 33 + b];
          s3 += V[i * 33 + a + 3] * G[(a + 3) * 33 + b];
        }
        for (; a < k; ++a) s0 += V[i * 33 + a] * G[a * 33 + b];
        w[r] = 1.5 * V[i * 33 + b] - 0.5 * ((s0 + s1) + (s2 + s3));
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int idx = tid + r * (int)blockDim.x;
      if (idx < nv * k) {
        const int i = idx / k, b = idx - (idx / k) * k;
        V[i * 33 + b] = w[r];
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nv * ldv; idx += blockDim.x) {
    const int i = idx / ldv, c = idx - (idx / ldv) * ldv;
    Vg[idx] = V[i * 33 + c];
  }
}

// Mixed-path form of k_orthonormalise_polar, for columns that are FP32-accurate right singular
// vectors (~1e-2 from orthonormal where the FP32 sweep resolves a small singular value only to its
// round-off floor).  Newton-Schulz steps V <- V (3 I - V^T V) / 2 converge to the polar factor of
// V whenever the singular values of V lie in (0, sqrt 3), i.e. ||V^T V - I||_2 < 1; with
// E = V^T V - I each step takes E to about -(3/4) E^2 - (1/4) E^3.  The steps run in FP32 while
// ||E||_F is above the FP32 floor (||E||_F <= 1/2 bounds ||E||_2 <= 1/2 on entry), then in FP64
// from the FP32 result (one step from e = max |E_ij| <= 1.5e-7, two from e <= 1e-4), so the FP64
// pipe, which holds a sub-partition for ~64 cycles per warp instruction, runs one or two small
// products instead of the 2 nv k^2 dependent products of Gram-Schmidt.  The columns end
// orthonormal to FP64 round-off and span a space within the FP32 round-off of span(V), the
// accuracy V itself has.  Inputs outside the bounds (a vanishing, dependent or far from
// orthogonal column, a NaN) take the column-by-column Gram-Schmidt of cgs2_warp_staged on
// the original columns, which also replaces dependent columns.
__global__ void __launch_bounds__(128) k_orthonormalise_polar_mixed(int nv, int ldv, double* __restrict__ Vg,
                                                                    const int* kptr, int rowmod,
                                                                    const int* rowlive_ptr) {
  __shared__ double V[32 * 33];
  __shared__ double G[32 * 33];
  __shared__ float Vf[32 * 33];
  __shared__ float Gf[32 * 33];
  __shared__ double h[32];
  __shared__ double emax[4];
  __shared__ double red[33];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = *kptr;
  const int rowlive = rowlive_ptr ? *rowlive_ptr : rowmod;
  for (int idx = tid; idx < nv * ldv; idx += blockDim.x) {
    const int i = idx / ldv, c = idx - (idx / ldv) * ldv;
    V[i * 33 + c] = Vg[idx];
    Vf[i * 33 + c] = (float)Vg[idx];
  }
  __syncthreads();
  // block-wide maximum of one value per thread (a NaN wins)
  auto block_max = [&](double e) -> double {
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, e, o);
      e = (t > e || t != t) ? t : e;
    }
    if (lane == 0) emax[warp] = e;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = (emax[w] > m || emax[w] != emax[w]) ? emax[w] : m;
    __syncthreads();
    return m;
  };
  // ---- FP32 steps: Gf = Vf^T Vf over the first k columns, ||Gf - I||_F and max |Gf - I|
  const int n_entries = k * k;
  int mode32 = 0;  // 1: at the FP32 floor, -1: outside the bounds
  int steps32 = 0;  // FP32 updates made (none: V keeps its FP64 columns)
  double e_prev = 1e300;
  for (int step = 0; step < 6; ++step) {
    double f2 = 0.0, e = 0.0;
    for (int idx = tid; idx < n_entries; idx += blockDim.x) {
      const int a = idx / k, b = idx - (idx / k) * k;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
      int i = 0;
      for (; i + 3 < nv; i += 4) {
        g0 = fmaf(Vf[i * 33 + a], Vf[i * 33 + b], g0);
        g1 = fmaf(Vf[(i + 1) * 33 + a], Vf[(i + 1) * 33 + b], g1);
        g2 = fmaf(Vf[(i + 2) * 33 + a], Vf[(i + 2) * 33 + b], g2);
        g3 = fmaf(Vf[(i + 3) * 33 + a], Vf[(i + 3) * 33 + b], g3);
      }
      for (; i < nv; ++i) g0 = fmaf(Vf[i * 33 + a], Vf[i * 33 + b], g0);
      const float g = (g0 + g1) + (g2 + g3);
      Gf[a * 33 + b] = g;
      const double d = (double)g - (a == b ? 1.0 : 0.0);
      f2 += d * d;
      e = (fabs(d) > e || d != d) ? fabs(d) : e;
    }
    const double fro2 = block_sum(f2, red);
    const double e32 = block_max(e);
    // ||E||_2 <= ||E||_F <= 1/2 keeps every singular value of V inside the convergence region;
    // the comparison is false for a NaN
    if (!(fro2 <= 0.25)) {
      mode32 = -1;
      break;
    }
    // at the FP32 floor: small, or no longer falling quadratically
    if (e32 <= 1e-6 || e32 > 0.5 * e_prev) {
      mode32 = 1;
      break;
    }
    e_prev = e32;
    float w[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int idx = tid + r * (int)blockDim.x;
      w[r] = 0.f;
      if (idx < nv * k) {
        const int i = idx / k, b = idx - (idx / k) * k;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int a = 0;
        for (; a + 3 < k; a += 4) {
          s0 = fmaf(Vf[i * 33 + a], Gf[a * 33 + b], s0);
          s1 = fmaf(Vf[i * 33 + a + 1], Gf[(a + 1) * 33 + b], s1);
          s2 = fmaf(Vf[i * 33 + a + 2], Gf[(a + 2) * 33 + b], s2);
          s3 = fmaf(Vf[i * 33 + a + 3], Gf[(a + 3) * 33 + b], s3);
        }
        for (; a < k; ++a) s0 = fmaf(Vf[i * 33 + a], Gf[a * 33 + b], s0);
        w[r] = 1.5f * Vf[i * 33 + b] - 0.5f * ((s0 + s1) + (s2 + s3));
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int idx = tid + r * (int)blockDim.x;
      if (idx < nv * k) {
        const int i = idx / k, b = idx - (idx / k) * k;
        Vf[i * 33 + b] = w[r];
      }
    }
    __syncthreads();
    ++steps32;
  }
  // six steps without reaching the floor: the FP64 check below decides
  const int ok32 = (mode32 < 0) ? -1 : 1;
  int ns = -1;
  if (ok32 == 1) {
    // ---- FP64 steps from the FP32 result
    if (steps32 > 0) {
      for (int idx = tid; idx < nv * k; idx += blockDim.x) {
        const int i = idx / k, b = idx - (idx / k) * k;
        V[i * 33 + b] = (double)Vf[i * 33 + b];
      }
    }
    __syncthreads();
    for (int step = 0; step < 3; ++step) {
      if (step > 0 && step >= ns) break;
      double e = 0.0;
      for (int idx = tid; idx < n_entries; idx += blockDim.x) {
        const int a = idx / k, b = idx - (idx / k) * k;
        double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
        int i = 0;
        for (; i + 3 < nv; i += 4) {
          g0 += V[i * 33 + a] * V[i * 33 + b];
          g1 += V[(i + 1) * 33 + a] * V[(i + 1) * 33 + b];
          g2 += V[(i + 2) * 33 + a] * V[(i + 2) * 33 + b];
          g3 += V[(i + 3) * 33 + a] * V[(i + 3) * 33 + b];
        }
        for (; i < nv; ++i) g0 += V[i * 33 + a] * V[i * 33 + b];
        const double g = (g0 + g1) + (g2 + g3);
        G[a * 33 + b] = g;
        const double d = fabs(g - (a == b ? 1.0 : 0.0));
        e = (d > e || d != d) ? d : e;
      }
      const double m = block_max(e);
      // no step below the FP64 round-off of a k-term sum; one from e <= 1.5e-7 (1.5 e^2 is then
      // below that floor); two from e <= 1e-4; otherwise Gram-Schmidt
      const double floor64 = 8.0 * 2.220446049250313e-16 * (k > 1 ? k : 1);
      if (step == 0) ns = (m <= floor64) ? 0 : (m <= 1.5e-7) ? 1 : (m <= 1e-4) ? 2 : -1;
      if (ns < 0 || step >= ns) break;
      double w[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int idx = tid + r * (int)blockDim.x;
        w[r] = 0.0;
        if (idx < nv * k) {
          const int i = idx / k, b = idx - (idx / k) * k;
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int a = 0;
          for (; a + 3 < k; a += 4) {
            s0 += V[i * 33 + a] * G[a * 33 + b];
            s1 += V[i * 33 + a + 1] * G[(a + 1) * 33 + b];
            s2 += V[i * 33 + a + 2] * G[(a + 2) * 33 + b];
            s3 += V[i * 33 + a + 3] * G[(a + 3) * 33 + b];
          }
          for (; a < k; ++a) s0 += V[i * 33 + a] * G[a * 33 + b];
          w[r] = 1.5 * V[i * 33 + b] - 0.5 * ((s0 + s1) + (s2 + s3));
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int idx = tid + r * (int)blockDim.x;
        if (idx < nv * k) {
          const int i = idx / k, b = idx - (idx / k) * k;
          V[i * 33 + b] = w[r];
        }
      }
      __syncthreads();
    }
  }
  if (ns < 0) {
    // Gram-Schmidt on the original columns
    for (int idx = tid; idx < nv * ldv; idx += blockDim.x) {
      const int i = idx / ldv, c = idx - (idx / ldv) * ldv;
      V[i * 33 + c] = Vg[idx];
    }
    __syncthreads();
    if (warp == 0) cgs2_warp_staged(nv, k, rowmod, rowlive, V, h);
    __syncthreads();
  }
  for (int idx = tid; idx < nv * ldv; idx += blockDim.x) {
    const int i = idx / ldv, c = idx - (idx / ldv) * ldv;
    Vg[idx] = V[i * 33 + c];
  }
}

// Classical Gram-Schmidt applied twice (FP64) to the first K columns of V (nv x ldv), in
// column order: V[:, :K] becomes Q of V[:, :K] = Q T and sig[j] = |T_jj|.  With the columns in
// order of decreasing norm and P = A U for nearly orthogonal U, T is upper triangular with
// T_ij (i < j) at most eps_32 sigma_i, which moves the singular values only at second order, so
// |T_jj| are the singular values to about 1e-14 relative and Q are FP64-orthonormal left
// singular vectors.  A column with nothing left stays zero with sig = 0.
__global__ void __launch_bounds__(1024) k_cgs2_sigma(int nv, int ldv, double* __restrict__ V, int K,
                                                     double* __restrict__ sig) {
  __shared__ double red[33];
  __shared__ double h[1024];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int j = 0; j < K; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int i2 = warp; i2 < j; i2 += nwarps) {
        double sacc = 0.0;
        for (int i = lane; i < nv; i += 32) sacc += V[(size_t)i * ldv + i2] * V[(size_t)i * ldv + j];
        sacc = warp_sum(sacc);
        if (lane == 0) h[i2] = sacc;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double v = V[(size_t)i * ldv + j];
        for (int i2 = 0; i2 < j; ++i2) v -= h[i2] * V[(size_t)i * ldv + i2];
        V[(size_t)i * ldv + j] = v;
      }
      __syncthreads();
    }
    double n1 = 0.0;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) n1 += V[(size_t)i * ldv + j] * V[(size_t)i * ldv + j];
    n1 = sqrt(block_sum(n1, red));
    if (threadIdx.x == 0) sig[j] = n1;
    const double inv = (n1 > 0.0) ? 1.0 / n1 : 0.0;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) V[(size_t)i * ldv + j] *= inv;
    __syncthreads();
  }
}

// ---- CholeskyQR of the first K columns of V (FP64) -----------------------------------------
// The same factorisation V[:, :K] = Q T as Gram-Schmidt in column order, computed as: Gram
// matrix G = V^T V (row chunks spread over many CTAs), upper Cholesky factor G = T^T T (one
// CTA), V <- V T^{-1} (explicit triangular inverse in one CTA, then a row-parallel product over
// many CTAs).  Column j of T depends on columns 0..j of V only, so leading columns are
// unaffected by what follows them.  The columns here are P = A U for nearly orthogonal U, i.e.
// graded: V = W D with D the column norms and W of condition near 1 on the columns that matter;
// Cholesky and triangular solves are invariant under that scaling, so one pass gives Q
// orthonormal to about kappa(W)^2 eps_64 and |T_jj| to FP64 relative accuracy.  A column whose
// Cholesky pivot is at the round-off level of its own diagonal has nothing left beyond the
// earlier columns: its row of T and its column of Q are set to zero.

constexpr int kGramTileRows = 32;   // rows staged in shared memory per step
constexpr int kGramChunkRows = 64;  // rows per CTA (one partial Gram matrix each)
constexpr int kGramEntries = 2048;  // Gram entries per CTA (8 per thread)

__global__ void __launch_bounds__(256) k_gram_chunks(int nv, int ldv, const double* __restrict__ V, int K,
                                                     double* __restrict__ part) {
  __shared__ double gs[kGramTileRows * 129];
  const int KK = K * K;
  const int beg = blockIdx.x * kGramChunkRows;
  const int end = min(beg + kGramChunkRows, nv);
  const int e0 = blockIdx.y * kGramEntries;
  double acc[kGramEntries / 256];
#pragma unroll
  for (int i = 0; i < kGramEntries / 256; ++i) acc[i] = 0.0;
  for (int r0 = beg; r0 < end; r0 += kGramTileRows) {
    const int nr = min(kGramTileRows, end - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * K; idx += blockDim.x) {
      const int rr = idx / K, c = idx - rr * K;
      gs[rr * K + c] = V[(size_t)(r0 + rr) * ldv + c];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kGramEntries / 256; ++i) {
      const int e = e0 + threadIdx.x + 256 * i;
      if (e < KK) {
        const int a = e / K, b = e - (e / K) * K;
        double t = acc[i];
        for (int rr = 0; rr < nr; ++rr) t += gs[rr * K + a] * gs[rr * K + b];
        acc[i] = t;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kGramEntries / 256; ++i) {
    const int e = e0 + threadIdx.x + 256 * i;
    if (e < KK) part[(size_t)blockIdx.x * KK + e] = acc[i];
  }
}

// Entry e of the sum of the nchunks partial Gram matrices, in four independent chains (chunk c
// goes to chain c mod 4) so that the loads of several chunks are in flight at once instead of one
// memory round trip per chunk.
__device__ __forceinline__ double gram_partials_sum(int nchunks, int KK, const double* __restrict__ part, int e) {
  double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
  int c = 0;
#pragma unroll 2
  for (; c + 3 < nchunks; c += 4) {
    t0 += part[(size_t)c * KK + e];
    t1 += part[(size_t)(c + 1) * KK + e];
    t2 += part[(size_t)(c + 2) * KK + e];
    t3 += part[(size_t)(c + 3) * KK + e];
  }
  for (; c < nchunks; ++c) t0 += part[(size_t)c * KK + e];
  return (t0 + t1) + (t2 + t3);
}

__global__ void k_gram_sum(int nchunks, int KK, const double* __restrict__ part, double* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= KK) return;
  G[e] = gram_partials_sum(nchunks, KK, part, e);
}

// Upper Cholesky factor T (K x K, row-major, zero below the diagonal) of the symmetric G.
// Upper Cholesky factor of the K x K Gram matrix in A (shared memory, overwritten: T in the upper
// triangle, zero rows at dead pivots), d0 (shared, K) its original diagonal.  A pivot at the
// round-off level of its own diagonal is dead: its row of T is zero.  Block-wide.
__device__ void chol_upper_smem(int K, double* A, double* d0) {
  for (int j = threadIdx.x; j < K; j += blockDim.x) d0[j] = A[(size_t)j * K + j];
  __syncthreads();
  const double thr = 64.0 * K * 2.220446049250313e-16;
  for (int j = 0; j < K; ++j) {
    const double piv = A[j * K + j];
    const bool live = piv > thr * d0[j] && piv > 0.0;
    const double tjj = live ? sqrt(piv) : 0.0;
    const double inv = live ? 1.0 / tjj : 0.0;
    __syncthreads();
    for (int c = j + threadIdx.x; c < K; c += blockDim.x) A[j * K + c] = (c == j) ? tjj : A[j * K + c] * inv;
    __syncthreads();
    const int m = K - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int a = j + 1 + idx / m, b = j + 1 + (idx - (idx / m) * m);
      if (b >= a) A[a * K + b] -= A[j * K + a] * A[j * K + b];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_chol_upper(int K, const double* __restrict__ G, double* __restrict__ T) {
  extern __shared__ double chs[];
  double* A = chs;           // [K][K] working copy (upper triangle used)
  double* d0 = chs + K * K;  // original diagonal
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) A[idx] = G[idx];
  __syncthreads();
  chol_upper_smem(K, A, d0);
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int i = idx / K, c = idx - (idx / K) * K;
    T[idx] = (c >= i) ? A[idx] : 0.0;
  }
}

// M = T^{-1} for the upper-triangular T restricted to its live pivots (T_jj > 0), with zero rows
// and columns at dead pivots, so that v M equals the forward substitution v T^{-1} over the live
// pivots (dead columns give 0).  One thread per column of M, back substitution up the column.  One CTA.
// The reciprocals of the pivots are formed once, in parallel, and each step's dot product runs in
// four partial sums: on this part an FP64 division or a long dependent FP64 chain inside the
// sequential substitution costs hundreds of cycles per step.
// Ms <- T^{-1} over the live pivots of the upper-triangular Ts (both K x K in shared memory,
// rinv: K doubles of shared scratch), one thread per column.  Block-wide.
__device__ void tri_inv_smem(int K, const double* Ts, double* Ms, double* rinv) {
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) Ms[idx] = 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const double tii = Ts[i * K + i];
    rinv[i] = (tii > 0.0) ? 1.0 / tii : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    if (!(rinv[j] > 0.0)) continue;
    Ms[j * K + j] = rinv[j];
    for (int i = j - 1; i >= 0; --i) {
      const double ri = rinv[i];
      if (!(ri > 0.0)) continue;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int k = i + 1;
      for (; k + 3 <= j; k += 4) {
        a0 += Ts[i * K + k] * Ms[k * K + j];
        a1 += Ts[i * K + k + 1] * Ms[(k + 1) * K + j];
        a2 += Ts[i * K + k + 2] * Ms[(k + 2) * K + j];
        a3 += Ts[i * K + k + 3] * Ms[(k + 3) * K + j];
      }
      for (; k <= j; ++k) a0 += Ts[i * K + k] * Ms[k * K + j];
      Ms[i * K + j] = -((a0 + a1) + (a2 + a3)) * ri;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(128) k_tri_inv(int K, const double* __restrict__ T, double* __restrict__ M) {
  extern __shared__ double tis[];
  double* Ts = tis;                // [K][K]
  double* Ms = tis + K * K;        // [K][K]
  double* rinv = tis + 2 * K * K;  // [K] 1 / T_ii at live pivots, else 0
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) Ts[idx] = T[idx];
  __syncthreads();
  tri_inv_smem(K, Ts, Ms, rinv);
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) M[idx] = Ms[idx];
}

// The one-CTA part of a CholeskyQR pass in one launch, for K <= 64: the Gram partials summed
// (fixed order), the upper Cholesky factor T, its inverse over the live pivots into M, and
// sig[j] = T_jj.  Shared memory: 2 K^2 + 2 K doubles.
constexpr int kCholFusedMaxK = 64;
__global__ void __launch_bounds__(256) k_chol_inv_sig(int K, int nchunks, const double* __restrict__ part,
                                                      double* __restrict__ M, double* __restrict__ sig) {
  extern __shared__ double cis[];
  const int KK = K * K;
  double* A = cis;         // [K][K]: G, then T in the upper triangle
  double* Ms = A + KK;     // [K][K]
  double* d0 = Ms + KK;    // [K]
  double* rinv = d0 + K;   // [K]
  for (int e = threadIdx.x; e < KK; e += blockDim.x) A[e] = gram_partials_sum(nchunks, KK, part, e);
  __syncthreads();
  chol_upper_smem(K, A, d0);
  // below the diagonal A still holds Gram entries; the inverse reads the upper triangle only
  tri_inv_smem(K, A, Ms, rinv);
  for (int idx = threadIdx.x; idx < KK; idx += blockDim.x) M[idx] = Ms[idx];
  for (int j = threadIdx.x; j < K; j += blockDim.x) sig[j] = A[(size_t)j * K + j];
}

// V[row][:K] <- V[row][:K] M for upper-triangular M (K x K): rows staged kRowsTile per CTA in
// shared memory, one thread per output entry (no dependent chain), spread over many CTAs.
constexpr int kRowsTile = 16;
__global__ void __launch_bounds__(256) k_rows_times_upper(int nv, int ldv, double* __restrict__ V, int K,
                                                          const double* __restrict__ M) {
  extern __shared__ double rtu[];
  double* Ms = rtu;          // [K][K]
  double* Vs = rtu + K * K;  // [kRowsTile][K]
  const int row0 = blockIdx.x * kRowsTile;
  const int nr = min(kRowsTile, nv - row0);
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) Ms[idx] = M[idx];
  for (int idx = threadIdx.x; idx < nr * K; idx += blockDim.x) {
    const int rr = idx / K, c = idx - (idx / K) * K;
    Vs[rr * K + c] = V[(size_t)(row0 + rr) * ldv + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nr * K; idx += blockDim.x) {
    const int rr = idx / K, j = idx - (idx / K) * K;
    double acc = 0.0;
    for (int i = 0; i <= j; ++i) acc += Vs[rr * K + i] * Ms[i * K + j];
    V[(size_t)(row0 + rr) * ldv + j] = acc;
  }
}

__global__ void k_sig_from_chol(int K, const double* __restrict__ T1, const double* __restrict__ T2,
                                double* __restrict__ sig) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < K) sig[j] = T1[(size_t)j * K + j] * (T2 ? T2[(size_t)j * K + j] : 1.0);
}

// Sort the first K columns of V (nv x ldv) and sig[0..K) by decreasing sig (ties by index).
__global__ void __launch_bounds__(1024) k_sort_cols(int nv, int ldv, int K, double* __restrict__ sig,
                                                    double* __restrict__ V, double* __restrict__ tmp) {
  __shared__ int rank_of[1024];
  __shared__ double sg[1024];
  for (int c = threadIdx.x; c < K; c += blockDim.x) sg[c] = sig[c];
  __syncthreads();
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const double v = rank_key(sg[c]);
    int r = 0;
    for (int q = 0; q < K; ++q) {
      const double w = rank_key(sg[q]);
      r += (w > v) || (w == v && q < c);
    }
    rank_of[c] = r;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nv * K; idx += blockDim.x) {
    const int i = idx / K, c = idx - (idx / K) * K;
    tmp[(size_t)i * K + rank_of[c]] = V[(size_t)i * ldv + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nv * K; idx += blockDim.x) {
    const int i = idx / K, c = idx - (idx / K) * K;
    V[(size_t)i * ldv + c] = tmp[idx];
  }
  for (int c = threadIdx.x; c < K; c += blockDim.x) sig[rank_of[c]] = sg[c];
}

// *tail = max(0, ||A||_F^2 - sum_{j<K} sig_j^2): the energy of A outside its K leading singular
// pairs, with ||A||_F^2 over `count` entries of A, from partial sums: k_sumsq_parts writes
// gridDim.x partial sums of squares over a fixed grid-stride partition of A, k_tail_from_parts adds
// them in order (one SM's FP64 pipe took ~20 us for the 82k entries of the bench's bond-1 matrix
// in one CTA).  With concurrent problems (batches) one CTA does both, in one launch: parts = nullptr
// and a single CTA write fro2 and the tail directly.
__device__ __forceinline__ void tail_finish(double s, int K, const double* __restrict__ sig,
                                            double* __restrict__ fro2, double* __restrict__ tail) {
  *fro2 = s;
  double s2 = 0.0;
  for (int j = K - 1; j >= 0; --j) s2 += sig[j] * sig[j];
  const double t = s - s2;
  *tail = t > 0.0 ? t : 0.0;
}
__global__ void k_sumsq_parts(long count, const double* __restrict__ A, double* __restrict__ parts, int K,
                              const double* __restrict__ sig, double* __restrict__ fro2, double* __restrict__ tail) {
  __shared__ double red[33];
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    s += A[i] * A[i];
  s = block_sum(s, red);
  if (threadIdx.x != 0) return;
  if (parts)
    parts[blockIdx.x] = s;
  else
    tail_finish(s, K, sig, fro2, tail);
}
__global__ void k_tail_from_parts(int nparts, const double* __restrict__ parts, int K, const double* __restrict__ sig,
                                  double* __restrict__ fro2, double* __restrict__ tail) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int b = 0; b < nparts; ++b) s += parts[b];
  tail_finish(s, K, sig, fro2, tail);
}
constexpr int kTailParts = 32;

// k_sort_cols in two launches for tall V: the rank of each of the first K values of sig (decreasing,
// ties by index) into rank_of and sig sorted, in one CTA; then every row of V permuted in place
// through shared memory, kPermRows rows a CTA (one CTA moving the whole matrix took ~20 us).
__global__ void __launch_bounds__(1024) k_sort_keys(int K, double* __restrict__ sig, int* __restrict__ rank_of) {
  __shared__ double sg[1024];
  for (int c = threadIdx.x; c < K; c += blockDim.x) sg[c] = sig[c];
  __syncthreads();
  for (int c = threadIdx.x; c < K; c += blockDim.x) {
    const double v = rank_key(sg[c]);
    int r = 0;
    for (int q = 0; q < K; ++q) {
      const double w = rank_key(sg[q]);
      r += (w > v) || (w == v && q < c);
    }
    rank_of[c] = r;
    sig[r] = sg[c];
  }
}
constexpr int kPermRows = 4;
__global__ void __launch_bounds__(256) k_permute_cols(int nv, int ldv, int K, const int* __restrict__ rank_of,
                                                      double* __restrict__ V) {
  __shared__ double buf[kPermRows * 1024];
  const int row0 = blockIdx.x * kPermRows;
  const int nr = min(kPermRows, nv - row0);
  for (int idx = threadIdx.x; idx < nr * K; idx += blockDim.x) {
    const int r = idx / K, c = idx - (idx / K) * K;
    buf[idx] = V[(size_t)(row0 + r) * ldv + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nr * K; idx += blockDim.x) {
    const int r = idx / K, c = idx - (idx / K) * K;
    V[(size_t)(row0 + r) * ldv + rank_of[c]] = buf[idx];
  }
}

// Energy beyond the first K of n sorted singular values that are accurate to FP64 (the squared
// tail, like k_tail_from_parts, but without the cancellation of ||A||^2 - sum sigma^2).
__global__ void k_tail_from_sigma(int n, int K, const double* __restrict__ sig, double* __restrict__ tail) {
  if (threadIdx.x || blockIdx.x) return;
  double s2 = 0.0;
  for (int j = n - 1; j >= K; --j) s2 += sig[j] * sig[j];
  *tail = s2;
}

// Columns j < k of V (nv x ldv, row-major) whose singular value is exactly zero carry no
// direction (zero tensor, or a zero kept by tol = 0); each is replaced by the first canonical
// vector on a live row (row % rowmod < rowlive) that is independent of the earlier columns,
// orthonormalised against them twice (classical Gram-Schmidt).  Columns with sigma > 0 come
// out of the converged Jacobi sweep orthonormal and are left as they are.
__global__ void __launch_bounds__(1024) k_fix_zero_columns(int nv, int ldv, double* __restrict__ V,
                                                           const double* __restrict__ sigma, const int* kptr,
                                                           int rowmod, const int* rowlive_ptr,
                                                           const double* __restrict__ from, int ldfrom) {
  __shared__ double red[33];
  __shared__ double h[1024];
  // V[:, :ldv] <- from[:, :ldv] first (the leading columns of a wider matrix), when given
  if (from) {
    for (long idx = threadIdx.x; idx < (long)nv * ldv; idx += blockDim.x) {
      const int i = (int)(idx / ldv), j = (int)(idx - (long)i * ldv);
      V[(size_t)i * ldv + j] = from[(size_t)i * ldfrom + j];
    }
    __syncthreads();
  }
  const int k = *kptr;
  const int rowlive = rowlive_ptr ? *rowlive_ptr : rowmod;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    if (sigma[j] > 0.0) continue;
    int cand = -1;
    for (int attempt = 0; attempt < nv; ++attempt) {
      do {
        ++cand;
      } while (cand < nv && (cand % rowmod) >= rowlive);
      if (cand >= nv) break;
      for (int i = threadIdx.x; i < nv; i += blockDim.x) V[(size_t)i * ldv + j] = (i == cand) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int i2 = warp; i2 < k; i2 += nwarps) {
          double s = 0.0;
          if (i2 != j && (i2 < j || sigma[i2] > 0.0))
            for (int i = lane; i < nv; i += 32) s += V[(size_t)i * ldv + i2] * V[(size_t)i * ldv + j];
          s = warp_sum(s);
          if (lane == 0) h[i2] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nv; i += blockDim.x) {
          double v = V[(size_t)i * ldv + j];
          for (int i2 = 0; i2 < k; ++i2) v -= h[i2] * V[(size_t)i * ldv + i2];
          V[(size_t)i * ldv + j] = v;
        }
        __syncthreads();
      }
      double n1 = 0.0;
      for (int i = threadIdx.x; i < nv; i += blockDim.x) n1 += V[(size_t)i * ldv + j] * V[(size_t)i * ldv + j];
      n1 = sqrt(block_sum(n1, red));
      if (n1 > 0.5) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) V[(size_t)i * ldv + j] /= n1;
        __syncthreads();
        break;
      }
    }
  }
}

// out[c * rows + r] = in[r * cols + c] (row-major to column-major)
__global__ void k_transpose(int rows, int cols, const double* __restrict__ in, double* __restrict__ out) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)rows * cols;
       idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx - (long)r * cols);
    out[(size_t)c * rows + r] = in[idx];
  }
}

// Expand R x n right-singular-vector matrices into new cores and the new right part.
__global__ void k_write_cores3(int n1, int n2, int K1cap, int K2cap, const double* __restrict__ V1,
                               const double* __restrict__ V2, const DevCtrl* ctrl, double* __restrict__ core1,
                               double* __restrict__ core2) {
  const int k1 = ctrl->k[0], k2 = ctrl->k[1];
  const int tot1 = K1cap * n1 * K2cap;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot1 + K2cap * n2; idx += gridDim.x * blockDim.x) {
    if (idx < tot1) {
      const int j = idx / (n1 * K2cap);
      const int rem = idx - j * n1 * K2cap;
      const int l = rem / K2cap, b = rem - (rem / K2cap) * K2cap;
      core1[idx] = (j < k1 && b < k2) ? V1[(size_t)(l * K2cap + b) * K1cap + j] : 0.0;
    } else {
      const int i2 = idx - tot1;
      const int b = i2 / n2, p = i2 - (i2 / n2) * n2;
      core2[i2] = (b < k2) ? V2[(size_t)p * n2 + b] : 0.0;
    }
  }
}

__global__ void k_write_cores2(int n1, int K1cap, const double* __restrict__ V, const DevCtrl* ctrl,
                               double* __restrict__ core1) {
  const int k1 = ctrl->k[0];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < K1cap * n1; idx += gridDim.x * blockDim.x) {
    const int j = idx / n1, i = idx - (idx / n1) * n1;
    core1[idx] = (j < k1) ? V[(size_t)i * n1 + j] : 0.0;
  }
}

// vJ[j] = (1/4 pi) sum_i dOmega_i Bnew[j][i]
__global__ void k_vj(int K1cap, int nang, const double* __restrict__ Bnew, const double* __restrict__ domega,
                     double* __restrict__ vJ) {
  const int j = blockIdx.x;
  if (j >= K1cap) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nang; i += blockDim.x) s += domega[i] * Bnew[(size_t)j * nang + i];
  __shared__ double red[33];
  s = block_sum(s, red);
  if (threadIdx.x == 0) vJ[j] = s / (4.0 * kPi);
}

template <typename S>
__global__ void k_right_part2(int rcap1, int n1, const S* __restrict__ core1, double* __restrict__ Bbase) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rcap1 * n1; idx += gridDim.x * blockDim.x)
    Bbase[idx] = (double)core1[idx];
}

__global__ void k_reduce_partials(const double* __restrict__ partials, long nblocks, int stride,
                                  double* __restrict__ out, double scale) {
  __shared__ double red[33];
  for (int comp = 0; comp < stride; ++comp) {
    double s = 0.0;
    // fixed assignment of blocks to threads and fixed tree order: deterministic
    for (long b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[b * stride + comp];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[comp] = s * scale;
  }
}


// Grid-wide barrier for cooperative launches, with a bounded spin (ctrl->spin_limit, else 2^24
// spins of about 64 ns).  If the wait gives up, the barrier latches TT_ERR_TIMEOUT and raises
// the abort flag so every CTA leaves.  ctrl->barrier_extra > 0 (a test setting) makes it wait
// for arrivals that never come.
__device__ bool grid_barrier(DevCtrl* ctrl, unsigned nblocks) {
  __shared__ int sh_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* genp = &ctrl->bar_gen;
    volatile int* abortp = &ctrl->abort;
    const unsigned g = *genp;
    const unsigned target = nblocks + (unsigned)ctrl->barrier_extra;
    const long long limit = ctrl->spin_limit > 0 ? ctrl->spin_limit : (1LL << 24);
    __threadfence();
    const unsigned arrived = atomicAdd(&ctrl->bar_count, 1u) + 1u;
    if (arrived == target) {
      atomicExch(&ctrl->bar_count, 0u);
      __threadfence();
      atomicAdd(&ctrl->bar_gen, 1u);
    } else {
      long long spins = 0;
      while (*genp == g && *abortp == 0) {
        if (++spins > limit) {
          atomicExch(&ctrl->abort, 1);
          latch(&ctrl->status, TT_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    sh_ok = (*abortp == 0);
  }
  __syncthreads();
  return sh_ok != 0;
}

__global__ void k_fro2(long count, const double* __restrict__ A, double* out) {
  __shared__ double red[33];
  double s = 0.0;
  for (long i = threadIdx.x; i < count; i += blockDim.x) s += A[i] * A[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// Cooperative one-sided Jacobi: CTA b handles pairs b, b + gridDim.x, ... of each round.
// Each thread keeps E elements of both columns of its pair in registers; the three inner
// products are reduced through shared memory by one warp, and one lane forms the rotation,
// so every FP64 instruction that is not proportional to m is issued once per pair.  With
// V != null the rotations are also applied to the columns of V (n x n, column-major).
template <int E>
__global__ void __launch_bounds__(256) k_coop_jacobi(int m, int n, double* __restrict__ A, double* __restrict__ V,
                                                     DevCtrl* ctrl, int maxsweep) {
  __shared__ double part[3][256];
  __shared__ double rot[3];  // cs, sn, flag
  const unsigned nb = gridDim.x;
  const int np = n + (n & 1);
  const int npairs = np / 2;
  const int tid = threadIdx.x;
  const double floor_abs = 1e-32 * ctrl->fro2;
  const double rel_tol = 2.0 * m * 2.220446049250313e-16;  // round-off of a length-m inner product
  if (ctrl->jac_sweep_cap > 0 && ctrl->jac_sweep_cap < maxsweep) maxsweep = ctrl->jac_sweep_cap;
  int sweeps = 0;
  for (int sweep = 0; sweep < maxsweep; ++sweep) {
    sweeps = sweep + 1;
    for (int round = 0; round < np - 1; ++round) {
      for (int pr = blockIdx.x; pr < npairs; pr += nb) {
        int p, q;
        if (pr == 0) {
          p = round;
          q = np - 1;
        } else {
          p = (round + pr) % (np - 1);
          q = (round - pr + (np - 1)) % (np - 1);
        }
        if (p >= n || q >= n) continue;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double* ap = A + (size_t)p * m;
        double* aq = A + (size_t)q * m;
        double x[E], y[E];
        double a = 0.0, b = 0.0, g = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = tid + e * 256;
          x[e] = (i < m) ? ap[i] : 0.0;
          y[e] = (i < m) ? aq[i] : 0.0;
          a += x[e] * x[e];
          b += y[e] * y[e];
          g += x[e] * y[e];
        }
        part[0][tid] = a;
        part[1][tid] = b;
        part[2][tid] = g;
        __syncthreads();
        if (tid < 32) {
          double sa = 0.0, sb = 0.0, sg = 0.0;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            sa += part[0][tid + 32 * k];
            sb += part[1][tid + 32 * k];
            sg += part[2][tid + 32 * k];
          }
          sa = warp_sum(sa);
          sb = warp_sum(sb);
          sg = warp_sum(sg);
          if (tid == 0) {
            // One lane forms the rotation, and an FP64 instruction with one active lane holds
            // the FP64 pipe as long as a full warp: the test compares squares, and the angle is
            // tan(theta) = sg sign(d) / (|d| + sqrt(d^2 + sg^2)) with d = (sb - sa) / 2, i.e.
            // sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) with zeta = d / sg, without forming zeta.
            double cs = 1.0, sn = 0.0, flag = 0.0;
            if (fabs(sg) > floor_abs && sg * sg > rel_tol * rel_tol * sa * sb) {
              const double d = 0.5 * (sb - sa);
              const double t = (d >= 0.0 ? sg : -sg) / (fabs(d) + sqrt(fma(d, d, sg * sg)));
              cs = rsqrt(fma(t, t, 1.0));
              sn = cs * t;
              flag = 1.0;
              atomicAdd(&ctrl->jac_rot[sweep], 1);
            }
            rot[0] = cs;
            rot[1] = sn;
            rot[2] = flag;
          }
        }
        __syncthreads();
        if (rot[2] != 0.0) {
          const double cs = rot[0], sn = rot[1];
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int i = tid + e * 256;
            if (i < m) {
              ap[i] = cs * x[e] - sn * y[e];
              aq[i] = sn * x[e] + cs * y[e];
            }
          }
          if (V) {
            double* vp = V + (size_t)p * n;
            double* vq = V + (size_t)q * n;
            for (int i = tid; i < n; i += 256) {
              const double u = vp[i], w = vq[i];
              vp[i] = cs * u - sn * w;
              vq[i] = sn * u + cs * w;
            }
          }
        }
        __syncthreads();
      }
      if (!grid_barrier(ctrl, nb)) return;
    }
    const int nrot = *(volatile int*)&ctrl->jac_rot[sweep];
    if (nrot == 0) break;
    if (sweep == maxsweep - 1 && blockIdx.x == 0 && threadIdx.x == 0) latch(&ctrl->status, TT_ERR_TIMEOUT);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl->jac_sweeps = sweeps;
    atomicMax(&ctrl->jac_sweeps_max, sweeps);
    atomicAdd(&ctrl->jac_calls, 1);
    atomicAdd(&ctrl->jac_sweeps_sum, sweeps);
  }
}

__global__ void k_identity(int n, double* __restrict__ V) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x)
    V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

// Vout[i][j] = V[perm j][i] (columns of V as right singular vectors, sorted), row-major n x n.
__global__ void k_jacobi_write_v(int n, const double* __restrict__ V, const int* __restrict__ perm,
                                 double* __restrict__ Vout) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
    const int i = idx / n, j = idx - (idx / n) * n;
    Vout[idx] = V[(size_t)perm[j] * n + i];
  }
}

// One-CTA one-sided Jacobi on R^T (R: n x n upper-triangular factor of a tall matrix A,
// row-major FP64 in global memory) in arithmetic T, with the n columns of R^T (= rows of R)
// in shared memory.  Jacobi on the transposed triangular factor converges in a few sweeps
// (Drmac-Veselic preconditioning).  The normalised converged columns are the right singular
// vectors of R, hence of A; they are written unsorted to U (row-major n x n, column c).
// Teams of up to 32 lanes take the n/2 pairs of each round side by side; one barrier per round.
// Sweep counts go to the context's Jacobi statistics (ctrl, nullable).
// Lanes per column pair of the one-CTA Jacobi (1024 threads): the largest power of two <= 32 that
// lets the pairs of a round run side by side.
__host__ __device__ inline int jrt_ts(int n) {
  const int np = n + (n & 1);
  int ts = 32;
  while (ts > 1 && (np / 2) * ts > 1024) ts >>= 1;
  return ts;
}
// Column stride of the Jacobi copy of R^T: = ts (mod 32), so that the 32/ts teams of a warp, which
// work on consecutive columns, read disjoint bank windows.
__host__ __device__ inline int jrt_ld(int n) {
  const int ts = jrt_ts(n);
  return ((n + 31) / 32) * 32 + (ts < 32 ? ts : 0);
}

// Rotation arithmetic: FP32 takes the fast quotient and reciprocal square root (a few ulp; the
// FP64 refinement that follows the FP32 sweep absorbs them), FP64 the IEEE operations.
template <typename T>
__device__ __forceinline__ T jrt_div(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float jrt_div<float>(float a, float b) { return __fdividef(a, b); }
template <typename T>
__device__ __forceinline__ T jrt_rsqrt(T x) { return T(1) / sqrt(x); }
template <>
__device__ __forceinline__ float jrt_rsqrt<float>(float x) { return rsqrtf(x); }

template <typename T, bool SMEM>
__global__ void __launch_bounds__(1024) k_jacobi_rt(int n, const double* __restrict__ R, double* __restrict__ U,
                                                    double* __restrict__ raw, int maxsweep, T* gwork,
                                                    DevCtrl* ctrl) {
  extern __shared__ __align__(16) unsigned char jrt_smem[];
  // column c at At[c * ld]: in shared memory (SMEM, so that every access compiles to a
  // shared-memory load or store), or in global scratch when it does not fit; the stride
  // puts the columns of the pairs that share a warp on different banks
  const int ld = jrt_ld(n);
  T* At = SMEM ? reinterpret_cast<T*>(jrt_smem) : gwork;
  __shared__ int rot_flag;
  __shared__ float red[33];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int c = idx / n;
    At[(size_t)c * ld + (idx - c * n)] = (T)R[idx];
  }
  // scale-free thresholds: pairs below the matrix round-off level are left alone
  float fro = 0.f;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) fro += (float)(R[idx] * R[idx]);
  fro = warp_sum(fro);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = fro;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
    v = warp_sum(v);
    if (threadIdx.x == 0) red[32] = v;
  }
  __syncthreads();
  const T eps = sizeof(T) == 4 ? T(1.1920929e-7) : T(2.220446049250313e-16);
  const T rel_tol = T(4) * sqrt(T(n)) * eps;
  const T floor_abs = (sizeof(T) == 4 ? T(1e-14) : T(1e-32)) * (T)red[32];
  const int np = n + (n & 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // a team of ts lanes (power of two, <= 32) per column pair, so that the np/2 pairs of a
  // round run side by side; team sums are xor butterflies inside the team
  const int ts = jrt_ts(n);  // launched with 1024 threads
  const int team = threadIdx.x / ts, tl = threadIdx.x & (ts - 1), nteams = blockDim.x / ts;
  const unsigned tmask = (ts == 32) ? 0xffffffffu : (((1u << ts) - 1u) << (lane & ~(ts - 1)));
  int sweeps = 0;
  for (int sweep = 0; sweep < maxsweep; ++sweep) {
    if (threadIdx.x == 0) rot_flag = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int pr = team; pr < np / 2; pr += nteams) {
        int p, q;
        if (pr == 0) {
          p = round;
          q = np - 1;
        } else {
          p = round + pr;
          if (p >= np - 1) p -= np - 1;
          q = round - pr;
          if (q < 0) q += np - 1;
        }
        if (p >= n || q >= n) continue;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        T* ap = At + (size_t)p * ld;
        T* aq = At + (size_t)q * ld;
        T a = 0, b = 0, g = 0;
        // unrolled by 4: the loads of four elements issue back to back
#pragma unroll 4
        for (int i = tl; i < n; i += ts) {
          const T xi = ap[i], yi = aq[i];
          a += xi * xi;
          b += yi * yi;
          g += xi * yi;
        }
        for (int o = 1; o < ts; o <<= 1) {
          a += __shfl_xor_sync(tmask, a, o);
          b += __shfl_xor_sync(tmask, b, o);
          g += __shfl_xor_sync(tmask, g, o);
        }
        if (fabs(g) > floor_abs && fabs(g) > rel_tol * sqrt(a) * sqrt(b)) {
          const T zeta = (b - a) / (T(2) * g);
          T t;
          if (fabs(zeta) > (sizeof(T) == 4 ? T(1e18) : T(1e150)))
            t = T(0.5) / zeta;
          else  // the divisor lies in [1, 2e18]: the fast quotient is exact to 2 ulp
            t = jrt_div<T>(zeta >= T(0) ? T(1) : T(-1), fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T cs = jrt_rsqrt<T>(T(1) + t * t), sn = cs * t;
#pragma unroll 4
          for (int i = tl; i < n; i += ts) {
            const T xi = ap[i], yi = aq[i];
            ap[i] = cs * xi - sn * yi;
            aq[i] = sn * xi + cs * yi;
          }
          if (tl == 0) rot_flag = 1;
        }
      }
      __syncthreads();
    }
    const int f = rot_flag;
    __syncthreads();
    sweeps = sweep + 1;
    if (!f) break;
  }
  if (ctrl && threadIdx.x == 0) {
    atomicMax(&ctrl->jac_sweeps_max, sweeps);
    atomicAdd(&ctrl->jac_calls, 1);
    atomicAdd(&ctrl->jac_sweeps_sum, sweeps);
  }
  // normalised columns -> U[i][c]
  for (int c = warp; c < n; c += nwarps) {
    const T* ac = At + (size_t)c * ld;
    // FP64 norm of the stored column: U gets unit columns to FP64 accuracy, so that |A u_j|
    // differs from sigma_j only at second order in the FP32 rotation error
    double s2 = 0.0;
    for (int i = lane; i < n; i += 32) s2 += (double)ac[i] * (double)ac[i];
    s2 = warp_sum(s2);
    const double inv = (s2 > 0.0) ? 1.0 / sqrt(s2) : 0.0;
    for (int i = lane; i < n; i += 32) U[(size_t)i * n + c] = (double)ac[i] * inv;
    // the column norm before normalising is the singular value to FP32 accuracy; columns the
    // FP32 sweep cannot resolve have tiny norms here even though A u can be large
    if (lane == 0) raw[c] = sqrt(s2);
  }
}


// The same sweep with each pair's columns in registers, for n up to 160 columns: lane tl of a team
// of ts lanes holds the contiguous elements [tl vv, tl vv + vv) of both columns of its pair, vv a
// multiple of 4 with vv / 4 odd, so that the 16-byte loads and stores of the 8 lanes served
// together fall on distinct banks; columns are padded with zeros to ts vv = ld elements.  The
// dot products and the rotation run on the packed two-lane FP32 FMA.  The sweep is bound by the
// dependent chain of a round (loads, dots, team sums, rotation, stores, barrier), so:
//   * R is scaled by 1 / ||R||_F as it is loaded (every column norm <= 1), the test for a pair
//     becomes g^2 > tol^2 a b without square roots, and the raw values are scaled back at the end;
//   * the rotation takes the fast reciprocal and reciprocal square root (a few ulp: cs^2 + sn^2 = 1
//     to FP32 accuracy, and the FP64 refinement that follows the FP32 sweep absorbs the rest);
//   * rows of R below 2^-30 ||R||_F (the zero rows of capacity columns beyond the live ranks, and
//     round-off rows) stay out of the sweep, as in k_jacobi_rt's statement of the error: they
//     change R by less than sqrt(n) 2^-30 ||R||_F; their columns of U and raw values are zero.
// The team geometry (ts, vv, ld) is that of all n columns; the rounds run over the nk kept ones.
struct JrtRegGeom {
  int ts, vv, ld;
};
constexpr int kJrtThreadsReg = 640;  // 80 pairs x 8 lanes at 160 columns
constexpr int kJrtMaxV = 20;
constexpr float kJrtDropRel = 9.31322574615478515625e-10f;  // 2^-30
__host__ __device__ inline JrtRegGeom jrt_reg_geom(int n) {
  JrtRegGeom g;
  const int np = n + (n & 1);
  int ts = 32;
  while (ts > 1 && (np / 2) * ts > kJrtThreadsReg) ts >>= 1;
  int v = (n + ts - 1) / ts;
  v = (v + 3) & ~3;
  if (((v / 4) & 1) == 0) v += 4;
  g.ts = ts;
  g.vv = v;
  g.ld = ts * v;
  return g;
}
__host__ __device__ inline bool jrt_reg_fits(int n) {
  return n >= 2 && n <= kJrtThreadsReg / 4 && jrt_reg_geom(n).vv <= kJrtMaxV;
}
// the column copy, then the kept-row list
__host__ __device__ inline size_t jrt_reg_smem_bytes(int n) {
  return sizeof(float) * (size_t)n * jrt_reg_geom(n).ld + sizeof(int) * (size_t)n;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Rotation of the pair (a = |x|^2, b = |y|^2, g = x.y) of columns scaled to norms <= 1, or false
// when the pair is orthogonal to the working accuracy (or below the round-off level).
__device__ __forceinline__ bool jrt_rotation_scaled(float a, float b, float g, float tol2, float floor_abs,
                                                    float& cs, float& sn) {
  if (!(fabsf(g) > floor_abs && g * g > tol2 * a * b)) return false;
  const float zeta = __fdividef(b - a, 2.f * g);  // |2g| > 2e-14: inside the fast quotient's range
  const float az = fabsf(zeta);
  float t;
  if (az > 1e18f) {
    t = __fdividef(0.5f, zeta);
  } else {
    const float s = fmaf(zeta, zeta, 1.f);
    t = copysignf(__fdividef(1.f, az + s * rsqrtf(s)), zeta);
  }
  cs = rsqrtf(fmaf(t, t, 1.f));
  sn = cs * t;
  return true;
}

__global__ void __launch_bounds__(kJrtThreadsReg) k_jacobi_rt_reg(int n, const double* __restrict__ R,
                                                                  double* __restrict__ U, double* __restrict__ raw,
                                                                  int maxsweep, DevCtrl* ctrl, int* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char jrr_smem[];
  const JrtRegGeom geo = jrt_reg_geom(n);
  const int ts = geo.ts, vv = geo.vv, ld = geo.ld;
  float* At = reinterpret_cast<float*>(jrr_smem);
  int* kept = reinterpret_cast<int*>(At + (size_t)n * ld);
  __shared__ int rot_flag, nk_s;
  __shared__ double red[33];
  __shared__ float rnorm[kJrtThreadsReg / 8 * 2];  // row norms^2 (n <= 160), FP32
  __shared__ double rawk[kJrtThreadsReg / 4];      // rank keys of the raw values (n <= 160)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // FP64 Frobenius norm and FP32 row norms of R
  double fl = 0.0;
  for (int c = warp; c < n; c += nwarps) {
    double s2 = 0.0;
    for (int i = lane; i < n; i += 32) s2 += R[(size_t)c * n + i] * R[(size_t)c * n + i];
    s2 = warp_sum(s2);
    if (lane == 0) rnorm[c] = (float)s2;
    fl += s2;
  }
  if (lane == 0) red[warp] = fl;
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int w = 0; w < nwarps; ++w) f += red[w];
    red[32] = f;
    const float thr = (float)(f * (double)kJrtDropRel * (double)kJrtDropRel);
    int m = 0;
    for (int c = 0; c < n; ++c)
      if (rnorm[c] > thr) kept[m++] = c;
    nk_s = m;
  }
  __syncthreads();
  const int nk = nk_s;
  const double fro = sqrt(red[32]);
  const float scale = fro > 0.0 ? (float)(1.0 / fro) : 0.f;
  for (int idx = threadIdx.x; idx < nk * ld; idx += blockDim.x) {
    const int s = idx / ld, i = idx - (idx / ld) * ld;
    At[idx] = (i < n) ? (float)R[(size_t)kept[s] * n + i] * scale : 0.f;
  }
  __syncthreads();
  const float rel_tol = 4.f * sqrtf((float)n) * 1.1920929e-7f;
  const float tol2 = rel_tol * rel_tol;
  const float floor_abs = 1e-14f;  // of the scaled ||R||_F^2 = 1
  const int np = nk + (nk & 1);
  const int team = threadIdx.x / ts, tl = threadIdx.x & (ts - 1), nteams = blockDim.x / ts;
  const unsigned tmask = (ts == 32) ? 0xffffffffu : (((1u << ts) - 1u) << (lane & ~(ts - 1)));
  const int nv4 = vv / 4;
  int sweeps = 0;
  for (int sweep = 0; sweep < maxsweep && np > 1; ++sweep) {
    if (threadIdx.x == 0) rot_flag = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int pr = team; pr < np / 2; pr += nteams) {
        int p, q;
        if (pr == 0) {
          p = round;
          q = np - 1;
        } else {
          p = round + pr;
          if (p >= np - 1) p -= np - 1;
          q = round - pr;
          if (q < 0) q += np - 1;
        }
        if (p >= nk || q >= nk) continue;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        float4* ap = reinterpret_cast<float4*>(At + (size_t)p * ld + tl * vv);
        float4* aq = reinterpret_cast<float4*>(At + (size_t)q * ld + tl * vv);
        float4 x[kJrtMaxV / 4], y[kJrtMaxV / 4];
        float2 sa0 = f2(0.f, 0.f), sa1 = sa0, sb0 = sa0, sb1 = sa0, sg0 = sa0, sg1 = sa0;
#pragma unroll
        for (int k = 0; k < kJrtMaxV / 4; ++k) {
          if (k < nv4) {
            x[k] = ap[k];
            y[k] = aq[k];
          }
        }
#pragma unroll
        for (int k = 0; k < kJrtMaxV / 4; ++k) {
          if (k < nv4) {
            const float2 xl = f2(x[k].x, x[k].y), xh = f2(x[k].z, x[k].w);
            const float2 yl = f2(y[k].x, y[k].y), yh = f2(y[k].z, y[k].w);
            sa0 = __ffma2_rn(xl, xl, sa0);
            sa1 = __ffma2_rn(xh, xh, sa1);
            sb0 = __ffma2_rn(yl, yl, sb0);
            sb1 = __ffma2_rn(yh, yh, sb1);
            sg0 = __ffma2_rn(xl, yl, sg0);
            sg1 = __ffma2_rn(xh, yh, sg1);
          }
        }
        float a = (sa0.x + sa0.y) + (sa1.x + sa1.y);
        float b = (sb0.x + sb0.y) + (sb1.x + sb1.y);
        float g = (sg0.x + sg0.y) + (sg1.x + sg1.y);
        for (int o = 1; o < ts; o <<= 1) {
          a += __shfl_xor_sync(tmask, a, o);
          b += __shfl_xor_sync(tmask, b, o);
          g += __shfl_xor_sync(tmask, g, o);
        }
        float cs, sn;
        if (jrt_rotation_scaled(a, b, g, tol2, floor_abs, cs, sn)) {
          const float2 c2 = f2(cs, cs), s2 = f2(sn, sn), ns2 = f2(-sn, -sn);
#pragma unroll
          for (int k = 0; k < kJrtMaxV / 4; ++k) {
            if (k < nv4) {
              const float2 xl = f2(x[k].x, x[k].y), xh = f2(x[k].z, x[k].w);
              const float2 yl = f2(y[k].x, y[k].y), yh = f2(y[k].z, y[k].w);
              const float2 pl = __ffma2_rn(c2, xl, __fmul2_rn(ns2, yl));
              const float2 ph = __ffma2_rn(c2, xh, __fmul2_rn(ns2, yh));
              const float2 ql = __ffma2_rn(s2, xl, __fmul2_rn(c2, yl));
              const float2 qh = __ffma2_rn(s2, xh, __fmul2_rn(c2, yh));
              ap[k] = make_float4(pl.x, pl.y, ph.x, ph.y);
              aq[k] = make_float4(ql.x, ql.y, qh.x, qh.y);
            }
          }
          if (tl == 0) rot_flag = 1;
        }
      }
      __syncthreads();
    }
    const int f = rot_flag;
    __syncthreads();
    sweeps = sweep + 1;
    if (!f) break;
  }
  if (ctrl && threadIdx.x == 0) {
    atomicMax(&ctrl->jac_sweeps_max, sweeps);
    atomicAdd(&ctrl->jac_calls, 1);
    atomicAdd(&ctrl->jac_sweeps_sum, sweeps);
  }
  // normalised columns -> U[i][s] (s < nk), zero columns and raw values beyond; raw in R's scale
  for (int c = warp; c < n; c += nwarps) {
    if (c >= nk) {
      for (int i = lane; i < n; i += 32) U[(size_t)i * n + c] = 0.0;
      if (lane == 0) {
        raw[c] = 0.0;
        rawk[c] = 0.0;
      }
      continue;
    }
    const float* ac = At + (size_t)c * ld;
    double s2 = 0.0;
    for (int i = lane; i < n; i += 32) s2 += (double)ac[i] * (double)ac[i];
    s2 = warp_sum(s2);
    const double inv = (s2 > 0.0) ? 1.0 / sqrt(s2) : 0.0;
    for (int i = lane; i < n; i += 32) U[(size_t)i * n + c] = (double)ac[i] * inv;
    if (lane == 0) {
      const double rv = sqrt(s2) * fro;
      raw[c] = rv;
      rawk[c] = rank_key(rv);
    }
  }
  // perm[r] = the column of rank r by decreasing raw value (ties by index), as k_rank_perm
  if (perm) {
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const double v = rawk[c];
      int rk = 0;
      for (int q = 0; q < n; ++q) {
        const double w = rawk[q];
        rk += (w > v) || (w == v && q < c);
      }
      perm[rk] = c;
    }
  }
}

// The same FP32 one-sided Jacobi on R^T for n <= 32 in one warp: lane c holds column c of R^T
// (row c of R) in registers, a round exchanges columns between the two lanes of each pair by
// shuffles, and both lanes compute the rotation from the pair in the same order (x = the lower
// column), so they agree bit for bit.  No barriers.  As in k_jacobi_rt_reg, R is scaled to unit
// Frobenius norm (the pair test needs no square roots), the rotation takes the fast reciprocal
// and reciprocal square root, and the dot products run in four partial sums (the round is one
// dependent chain).  Same outputs as k_jacobi_rt.
__global__ void __launch_bounds__(32) k_jacobi_warp(int n, const double* __restrict__ R, double* __restrict__ U,
                                                    double* __restrict__ raw, int maxsweep, DevCtrl* ctrl,
                                                    int* __restrict__ perm) {
  const int lane = threadIdx.x;
  double f = 0.0;
  if (lane < n)
    for (int i = 0; i < n; ++i) f += R[(size_t)lane * n + i] * R[(size_t)lane * n + i];
  f = warp_sum(f);
  const double fro = sqrt(f);
  const float scale = fro > 0.0 ? (float)(1.0 / fro) : 0.f;
  float col[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) col[i] = (lane < n && i < n) ? (float)R[(size_t)lane * n + i] * scale : 0.f;
  const float rel_tol = 4.f * sqrtf((float)n) * 1.1920929e-7f;
  const float tol2 = rel_tol * rel_tol;
  const float floor_abs = 1e-14f;  // of the scaled ||R||_F^2 = 1
  const int np = n + (n & 1);
  int sweeps = 0;
  for (int sweep = 0; sweep < maxsweep; ++sweep) {
    int rotated = 0;
    for (int round = 0; round < np - 1; ++round) {
      // round-robin partner: (round, np - 1), else p + q = 2 round (mod np - 1)
      int partner;
      if (lane == np - 1) partner = round;
      else if (lane == round) partner = np - 1;
      else {
        partner = 2 * round - lane;
        if (partner < 0) partner += np - 1;
        if (partner >= np - 1) partner -= np - 1;
      }
      if (lane >= np) partner = lane;
      float other[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) other[i] = __shfl_sync(0xffffffffu, col[i], partner);
      const bool pair = lane < n && partner < n && partner != lane;
      const bool low = lane < partner;
      float pa[4] = {0.f, 0.f, 0.f, 0.f}, pb[4] = {0.f, 0.f, 0.f, 0.f}, pg[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float x = low ? col[i] : other[i], y = low ? other[i] : col[i];
        pa[i & 3] = fmaf(x, x, pa[i & 3]);
        pb[i & 3] = fmaf(y, y, pb[i & 3]);
        pg[i & 3] = fmaf(x, y, pg[i & 3]);
      }
      const float a = (pa[0] + pa[1]) + (pa[2] + pa[3]);
      const float b = (pb[0] + pb[1]) + (pb[2] + pb[3]);
      const float g = (pg[0] + pg[1]) + (pg[2] + pg[3]);
      float cs, sn;
      if (pair && jrt_rotation_scaled(a, b, g, tol2, floor_abs, cs, sn)) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float x = low ? col[i] : other[i], y = low ? other[i] : col[i];
          col[i] = low ? (cs * x - sn * y) : (sn * x + cs * y);
        }
        rotated = 1;
      }
    }
    sweeps = sweep + 1;
    if (!__any_sync(0xffffffffu, rotated)) break;
  }
  if (ctrl && lane == 0) {
    atomicMax(&ctrl->jac_sweeps_max, sweeps);
    atomicAdd(&ctrl->jac_calls, 1);
    atomicAdd(&ctrl->jac_sweeps_sum, sweeps);
  }
  double rawv = 0.0;
  if (lane < n) {
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < 32; ++i) s2 += (double)col[i] * (double)col[i];
    const double inv = (s2 > 0.0) ? 1.0 / sqrt(s2) : 0.0;
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < n) U[(size_t)i * n + lane] = (double)col[i] * inv;
    rawv = sqrt(s2) * fro;
    raw[lane] = rawv;
  }
  // perm[r] = the column of rank r by decreasing raw value (ties by index), as k_rank_perm
  if (perm) {
    const double v = rank_key(rawv);
    int rk = 0;
    for (int q = 0; q < n; ++q) {
      const double w = __shfl_sync(0xffffffffu, v, q);
      rk += (w > v) || (w == v && q < lane);
    }
    if (lane < n) perm[rk] = lane;
  }
}

// perm[r] = the column of rank r by decreasing vals (ties by index)
__global__ void __launch_bounds__(1024) k_rank_perm(int n, const double* __restrict__ vals, int* __restrict__ perm) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double v = rank_key(vals[c]);
    int r = 0;
    for (int q = 0; q < n; ++q) {
      const double w = rank_key(vals[q]);
      r += (w > v) || (w == v && q < c);
    }
    perm[r] = c;
  }
}

// Vout[i][j] = P[i][perm j] (divided by sigma_j when normalise != 0) for j < ncols.
__global__ void k_write_sorted(int m, int n, int ncols, const double* __restrict__ P, const double* __restrict__ sigma,
                               const int* __restrict__ perm, double* __restrict__ Vout, int ldv, int normalise) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)m * ncols;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / ncols), j = (int)(idx - (long)i * ncols);
    const double v = P[(size_t)i * n + perm[j]];
    Vout[(size_t)i * ldv + j] = normalise ? (sigma[j] > 0.0 ? v / sigma[j] : 0.0) : v;
  }
}

// Column norms of the converged matrix, rank-sorted descending (ties by index).
__global__ void __launch_bounds__(1024) k_jacobi_sort(int m, int n, const double* __restrict__ A,
                                                      double* __restrict__ sigma, int* __restrict__ perm,
                                                      double* __restrict__ tmp, int* status) {
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double a = 0.0;
    const double* ap = A + (size_t)p * m;
    for (int i = 0; i < m; ++i) a += ap[i] * ap[i];
    tmp[p] = sqrt(a);
    if (!isfinite(a)) latch(status, TT_ERR_NONFINITE);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const double sp = rank_key(tmp[p]);
    int rank = 0;
    for (int q = 0; q < n; ++q) {
      const double sq = rank_key(tmp[q]);
      rank += (sq > sp) || (sq == sp && q < p);
    }
    perm[rank] = p;
    sigma[rank] = tmp[p];
  }
}

// U[i][j] = A[i][perm j] / sigma_j for j < ncols (0 where sigma_j = 0).
__global__ void k_jacobi_write_u(int m, int ncols, const double* __restrict__ A, const double* __restrict__ sigma,
                                 const int* __restrict__ perm, double* __restrict__ U, int ldu) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)m * ncols;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / ncols), j = (int)(idx - (long)i * ncols);
    const double sg = sigma[j];
    U[(size_t)i * ldu + j] = (sg > 0.0) ? A[(size_t)perm[j] * m + i] / sg : 0.0;
  }
}

}  // namespace

template <typename TA, typename TB>
void small_gemm(cudaStream_t s, int M, int N, int K, const TA* A, long sa0, long sa1, const TB* B, long sb0,
                long sb1, double* C, long ldc, const int* nlive, const double* inv_colscale) {
  dim3 grid((N + 15) / 16, (M + 15) / 16);
  k_small_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, sa0, sa1, B, sb0, sb1, C, ldc, nlive, inv_colscale,
                                            nullptr, nullptr); count_launch();
}

// small_gemm (FP64, no column scaling) with K split over up to kMaxKSlices slices when the output
// has fewer tiles than half the SMs; part holds kMaxKSlices M N doubles (small_gemm_ksplit_elems).
constexpr int kMaxKSlices = 16;
static size_t small_gemm_ksplit_elems(int M, int N) { return (size_t)kMaxKSlices * M * N; }
static void small_gemm_ksplit(cudaStream_t s, int num_sms, int M, int N, int K, const double* A, long sa0, long sa1,
                              const double* B, long sb0, long sb1, double* C, long ldc, const int* nlive,
                              double* part) {
  const int tiles = ((N + 15) / 16) * ((M + 15) / 16);
  int ns = (num_sms / 2) / (tiles > 0 ? tiles : 1);
  if (ns > kMaxKSlices) ns = kMaxKSlices;
  const int kmin = 64;  // at least four 16-wide chunks a slice
  if (ns > (K + kmin - 1) / kmin) ns = (K + kmin - 1) / kmin;
  if (ns <= 1) {
    small_gemm<double, double>(s, M, N, K, A, sa0, sa1, B, sb0, sb1, C, ldc, nlive, nullptr);
    return;
  }
  int kslice = (K + ns - 1) / ns;
  kslice = (kslice + 15) / 16 * 16;
  ns = (K + kslice - 1) / kslice;
  dim3 grid((N + 15) / 16, (M + 15) / 16, ns);
  k_small_gemm_part<<<grid, 256, 0, s>>>(M, N, K, kslice, A, sa0, sa1, B, sb0, sb1, part); count_launch();
  const long tot = (long)M * N;
  k_small_gemm_sum<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, N, ns, part, C, ldc, nlive); count_launch();
}

// A B -> C and A2 B -> C2 in one launch (same shape, strides and B).
template <typename TA, typename TB>
void small_gemm_pair(cudaStream_t s, int M, int N, int K, const TA* A, const TA* A2, long sa0, long sa1, const TB* B,
                     long sb0, long sb1, double* C, double* C2, long ldc, const int* nlive) {
  dim3 grid((N + 15) / 16, (M + 15) / 16, 2);
  k_small_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, sa0, sa1, B, sb0, sb1, C, ldc, nlive, nullptr, A2, C2);
  count_launch();
}

template void small_gemm<double, double>(cudaStream_t, int, int, int, const double*, long, long, const double*,
                                         long, long, double*, long, const int*, const double*);
template void small_gemm<float, float>(cudaStream_t, int, int, int, const float*, long, long, const float*, long,
                                       long, double*, long, const int*, const double*);

template <typename S>
void right_part(cudaStream_t s, int d, int rcap1, int n1, int rcap2, int n2, const S* core1, const S* core2,
                double* Bbase) {
  if (d == 3) {
    small_gemm<S, S>(s, rcap1 * n1, n2, rcap2, core1, rcap2, 1, core2, n2, 1, Bbase, n2, nullptr, nullptr);
  } else {
    k_right_part2<S><<<(rcap1 * n1 + 255) / 256, 256, 0, s>>>(rcap1, n1, core1, Bbase); count_launch();
  }
}
template void right_part<double>(cudaStream_t, int, int, int, int, int, const double*, const double*, double*);
template void right_part<float>(cudaStream_t, int, int, int, int, int, const float*, const float*, double*);

void k_vj_host_launch(cudaStream_t s, int K1, int nang, const double* B, const double* domega, double* vJ) {
  k_vj<<<K1, 128, 0, s>>>(K1, nang, B, domega, vJ); count_launch();
}

void reduce_partials(cudaStream_t s, const double* partials, long nblocks, int stride, double* out, double scale) {
  k_reduce_partials<<<1, 1024, 0, s>>>(partials, nblocks, stride, out, scale); count_launch();
}

// grid: the CTAs wanted, capped here by the CTAs of this instantiation that are resident at once
// (a cooperative launch beyond that is refused).
template <int E>
static cudaError_t launch_coop(int grid, int num_sms, int m, int n, double* A, double* V, DevCtrl* ctrl,
                               int maxsweep, cudaStream_t s) {
  int occ = 0;
  const cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_coop_jacobi<E>, 256, 0);
  if (oe != cudaSuccess) return oe;
  const int resident = num_sms * (occ > 0 ? occ : 1);
  if (grid > resident) grid = resident;
  // a single CTA is always co-resident with itself: plain launch (capturable in any graph)
  if (grid == 1) {
    k_coop_jacobi<E><<<1, 256, 0, s>>>(m, n, A, V, ctrl, maxsweep);
    return cudaGetLastError();
  }
  void* args[] = {&m, &n, &A, &V, &ctrl, &maxsweep};
  return cudaLaunchCooperativeKernel((const void*)k_coop_jacobi<E>, dim3(grid), dim3(256), args, 0, s);
}

tt_status coop_jacobi(cudaStream_t s, int num_sms, int m, int n, double* A, double* V, double* sigma, double* U,
                      int ldu, int ncols_out, double* Vout, int* perm, double* tmp, DevCtrl* ctrl,
                      int grid_max) {
  if (m > 16 * 256) return TT_ERR_UNSUPPORTED;
  // barrier state, abort flag and sweep counters start at zero for every launch
  const size_t off = offsetof(DevCtrl, bar_count);
  cudaMemsetAsync(reinterpret_cast<char*>(ctrl) + off, 0, sizeof(DevCtrl) - off, s);
  k_fro2<<<1, 1024, 0, s>>>((long)m * n, A, &ctrl->fro2); count_launch();
  if (V) {
    k_identity<<<(n * n + 255) / 256, 256, 0, s>>>(n, V); count_launch();
  }
  const int npairs = (n + 1) / 2;
  int grid = npairs;
  if (grid_max > 0 && grid > grid_max) grid = grid_max;
  if (grid < 1) grid = 1;
  const int maxsweep = 40;
  cudaError_t e;
  if (m <= 256) e = launch_coop<1>(grid, num_sms, m, n, A, V, ctrl, maxsweep, s);
  else if (m <= 512) e = launch_coop<2>(grid, num_sms, m, n, A, V, ctrl, maxsweep, s);
  else if (m <= 1024) e = launch_coop<4>(grid, num_sms, m, n, A, V, ctrl, maxsweep, s);
  else if (m <= 2048) e = launch_coop<8>(grid, num_sms, m, n, A, V, ctrl, maxsweep, s);
  else e = launch_coop<16>(grid, num_sms, m, n, A, V, ctrl, maxsweep, s);
  if (e != cudaSuccess) return TT_ERR_CUDA;
  count_launch();
  k_jacobi_sort<<<1, 1024, 0, s>>>(m, n, A, sigma, perm, tmp, &ctrl->status); count_launch();
  if (U) {
    const long tot = (long)m * ncols_out;
    k_jacobi_write_u<<<(unsigned)((tot + 255) / 256 < 1024 ? (tot + 255) / 256 : 1024), 256, 0, s>>>(
        m, ncols_out, A, sigma, perm, U, ldu); count_launch();
  }
  if (V && Vout) {
    k_jacobi_write_v<<<(n * n + 255) / 256, 256, 0, s>>>(n, V, perm, Vout); count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// SVD of an m x n row-major matrix M (right singular vectors and singular values) by the
// cooperative Jacobi sweep on its transpose copy: sigma (n, sorted) and Vout (n x n,
// row-major, column j for sigma_j).
tt_status svd_right(cudaStream_t s, int num_sms, int m, int n, const double* M, Bump& ws, double* sigma,
                    double* Vout, DevCtrl* ctrl, int grid_max) {
  double* At = ws.take<double>((size_t)m * n);
  double* V = ws.take<double>((size_t)n * n);
  double* tmp = ws.take<double>(n);
  int* perm = ws.take<int>(n);
  if (ws.dry) return TT_OK;
  k_transpose<<<(unsigned)(((long)m * n + 255) / 256 < 1024 ? ((long)m * n + 255) / 256 : 1024), 256, 0, s>>>(
      m, n, M, At); count_launch();
  return coop_jacobi(s, num_sms, m, n, At, V, sigma, nullptr, 0, 0, Vout, perm, tmp, ctrl, grid_max);
}

// V[:, :K] (nv x ldv, row-major) <- Q and sig[j] = |T_jj| of V[:, :K] = Q T, by CholeskyQR in
// FP64 for K <= 112, by one-CTA Gram-Schmidt beyond.  One pass: the columns are P = A U for U
// from a converged Jacobi sweep, nearly orthogonal once each is normalised, and the error of a
// Cholesky factor is governed by the condition number of the column-equilibrated Gram matrix,
// not by that of P (whose column norms are the singular values), so Q is orthonormal to about
// kappa(P D^-1)^2 eps_64 in one pass; columns that are numerically dependent in that scaled
// sense meet a dead pivot (k_chol_upper) and give zero columns, as in the two-pass form.
static tt_status cholqr_sigma(cudaStream_t s, int nv, int ldv, double* V, int K, double* sig, Bump& ws) {
  const int KK = K * K;
  const int nchunks = (nv + kGramChunkRows - 1) / kGramChunkRows;
  double* part = ws.take<double>((size_t)nchunks * KK);
  double* G = ws.take<double>(KK);
  double* T1 = ws.take<double>(KK);
  double* Minv = ws.take<double>(KK);
  if (ws.dry) return TT_OK;
  if (K > 112 || nv < 1) {  // the inverse kernel holds 2 K^2 doubles in shared memory
    k_cgs2_sigma<<<1, 1024, 0, s>>>(nv, ldv, V, K, sig); count_launch();
    return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  const size_t chol_smem = sizeof(double) * ((size_t)KK + K);
  const size_t inv_smem = sizeof(double) * (2 * (size_t)KK + K);
  const size_t fused_smem = sizeof(double) * (2 * (size_t)KK + 2 * K);
  const size_t rtu_smem = sizeof(double) * ((size_t)KK + (size_t)kRowsTile * K);
  const bool fused = K <= kCholFusedMaxK;
  for (const auto& [f, b] : {std::make_pair((const void*)k_chol_upper, chol_smem),
                              std::make_pair((const void*)k_tri_inv, inv_smem),
                              std::make_pair((const void*)k_chol_inv_sig, fused ? fused_smem : (size_t)0),
                              std::make_pair((const void*)k_rows_times_upper, rtu_smem)})
    if (const tt_status a = smem_optin_impl(f, b); a != TT_OK) return a;
  k_gram_chunks<<<dim3((unsigned)nchunks, (unsigned)((KK + kGramEntries - 1) / kGramEntries)), 256, 0, s>>>(
      nv, ldv, V, K, part); count_launch();
  if (fused) {
    // partial sums, Cholesky, inverse and |T_jj| in one CTA
    k_chol_inv_sig<<<1, 256, fused_smem, s>>>(K, nchunks, part, Minv, sig); count_launch();
  } else {
    k_gram_sum<<<(KK + 255) / 256, 256, 0, s>>>(nchunks, KK, part, G); count_launch();
    k_chol_upper<<<1, 256, chol_smem, s>>>(K, G, T1); count_launch();
    // V <- V T^{-1} as a product with the explicit inverse: row-parallel without a dependent chain
    k_tri_inv<<<1, 128, inv_smem, s>>>(K, T1, Minv); count_launch();
    k_sig_from_chol<<<(K + 127) / 128, 128, 0, s>>>(K, T1, nullptr, sig); count_launch();
  }
  k_rows_times_upper<<<(nv + kRowsTile - 1) / kRowsTile, 256, rtu_smem, s>>>(nv, ldv, V, K, Minv);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// Mixed-precision SVD of an explicit tall matrix A (source `src`, rows x cols): FP32 TSQR
// factor R and one-CTA FP32 Jacobi on R^T giving the right singular vectors U (cols x cols)
// and their FP32 singular values `raw`, with perm the order of decreasing raw.
template <class Src>
static tt_status svd_right_mixed(cudaStream_t s, int num_sms, const Src& src, long rows, int cols, Bump& ws,
                                 double** U_out, double** P_out, double* raw, int* perm, DevCtrl* ctrl) {
  LivePattern lp{nullptr, cols, 1, 0};
  const long L = tsqr_max_leaves<float, 64>(num_sms, cols, rows, 8);
  double* a = ws.take<double>((size_t)L * cols * cols);
  double* b = ws.take<double>((size_t)((L + 1) / 2) * cols * cols);
  double* U = ws.take<double>((size_t)cols * cols);
  double* P = ws.take<double>((size_t)rows * cols);
  double* tmp = ws.take<double>(cols);
  const bool reg = cols > 32 && jrt_reg_fits(cols) && jrt_reg_smem_bytes(cols) <= 200 * 1024;
  const size_t at_bytes = sizeof(float) * (size_t)cols * jrt_ld(cols);
  const bool in_smem = at_bytes <= 200 * 1024;
  float* gwork = in_smem ? nullptr : ws.take<float>((size_t)cols * jrt_ld(cols));
  *U_out = U;
  *P_out = P;
  if (ws.dry) return TT_OK;
  double* R = nullptr;
  tt_status st = run_tsqr<float, 64>(s, num_sms, src, lp, rows, 8, a, b, &R);
  if (st != TT_OK) return st;
  if (cols <= 32) {
    k_jacobi_warp<<<1, 32, 0, s>>>(cols, R, U, raw, 40, ctrl, perm); count_launch();
  } else if (reg) {
    const size_t smem = jrt_reg_smem_bytes(cols);
    if (const tt_status a = smem_optin(k_jacobi_rt_reg, smem); a != TT_OK) return a;
    k_jacobi_rt_reg<<<1, kJrtThreadsReg, smem, s>>>(cols, R, U, raw, 40, ctrl, perm); count_launch();
  } else if (in_smem) {
    if (const tt_status a = smem_optin(k_jacobi_rt<float, true>, at_bytes); a != TT_OK) return a;
    k_jacobi_rt<float, true><<<1, 1024, at_bytes, s>>>(cols, R, U, raw, 40, nullptr, ctrl); count_launch();
    k_rank_perm<<<1, 1024, 0, s>>>(cols, raw, perm); count_launch();
  } else {
    k_jacobi_rt<float, false><<<1, 1024, 0, s>>>(cols, R, U, raw, 40, gwork, ctrl); count_launch();
    k_rank_perm<<<1, 1024, 0, s>>>(cols, raw, perm); count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

__global__ void k_iota(int n, int* __restrict__ p) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

// The same outputs as svd_right_mixed in FP64: FP64 Householder TSQR of the small matrix, then
// the cooperative FP64 one-sided Jacobi on R^T (row p of R is column p of R^T, contiguous),
// which converges in fewer sweeps than Jacobi on the matrix itself (Drmac-Veselic) and works on
// columns of length cols instead of rows.  U comes sorted by decreasing singular value, so perm is
// the identity; raw holds the FP64 singular values.
template <class Src>
static tt_status svd_right_f64pre(cudaStream_t s, int num_sms, const Src& src, long rows, int cols, Bump& ws,
                                  double** U_out, double** P_out, double* raw, int* perm, DevCtrl* ctrl,
                                  int grid_max) {
  LivePattern lp{nullptr, cols, 1, 0};
  const long L = tsqr_max_leaves<double, 32>(num_sms, cols, rows, 8);
  double* a = ws.take<double>((size_t)L * cols * cols);
  double* b = ws.take<double>((size_t)((L + 1) / 2) * cols * cols);
  double* U = ws.take<double>((size_t)cols * cols);
  double* P = ws.take<double>((size_t)rows * cols);
  double* tmp = ws.take<double>(cols);
  int* perm_j = ws.take<int>(cols);
  *U_out = U;
  *P_out = P;
  if (ws.dry) return TT_OK;
  double* R = nullptr;
  tt_status st = run_tsqr<double, 32>(s, num_sms, src, lp, rows, 8, a, b, &R);
  if (st != TT_OK) return st;
  st = coop_jacobi(s, num_sms, cols, cols, R, nullptr, raw, U, cols, cols, nullptr, perm_j, tmp, ctrl, grid_max);
  if (st != TT_OK) return st;
  k_iota<<<(cols + 255) / 256, 256, 0, s>>>(cols, perm); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

template <bool F64, class Src>
static tt_status svd_right_pre(cudaStream_t s, int num_sms, const Src& src, long rows, int cols, Bump& ws,
                               double** U_out, double** P_out, double* raw, int* perm, DevCtrl* ctrl, int grid_max) {
  if (F64) return svd_right_f64pre(s, num_sms, src, rows, cols, ws, U_out, P_out, raw, perm, ctrl, grid_max);
  return svd_right_mixed(s, num_sms, src, rows, cols, ws, U_out, P_out, raw, perm, ctrl);
}

// d = 3 small-core sweep.  For each bond a TSQR of the small matrix A and a one-sided Jacobi on
// R^T give right vectors U (mixed path: FP32 TSQR and one-CTA FP32 Jacobi, U nearly orthogonal;
// F64: FP64 TSQR and the cooperative FP64 Jacobi).  P = A U in FP64, sorted by column norm;
// CholeskyQR of the leading columns gives FP64 singular values |T_jj| and orthonormal left
// vectors; the energy beyond them comes from the FP64 Jacobi singular values (F64) or from
// Pythagoras (mixed).
template <bool F64>
static tt_status small_round_mixed3(cudaStream_t s, int num_sms, const SmallJob& j, Bump& ws, const double* Y) {
  const int R = j.lp.ncap();
  const int n1 = j.n1, n2 = j.n2, nang = n1 * n2;
  const int K1 = j.K1cap, K2 = j.K2cap;
  // ---- bond 2: A2 = Y viewed as (R n1) x n2; right vectors needed
  double* sigc2 = ws.take<double>(n2);
  int* perm2 = ws.take<int>(n2);
  double* sig2 = ws.take<double>(n2);
  double* V2 = ws.take<double>((size_t)n2 * n2);
  double* tmp2 = ws.take<double>((size_t)n2 * n2);
  double *U2 = nullptr, *P2 = nullptr;
  tt_status st = svd_right_pre<F64>(s, num_sms, SrcRows<double>{Y, n2}, (long)R * n1, n2, ws, &U2, &P2, sigc2,
                                   perm2, j.ctrl, j.coop_grid_max);
  if (st != TT_OK) return st;
  double* P2s = ws.take<double>((size_t)R * n1 * n2);
  const int nv = n1 * K2;
  double* Y2 = ws.take<double>((size_t)R * nv);
  double* B0p = ws.take<double>((size_t)R * nv);
  if (!ws.dry) {
    small_gemm<double, double>(s, R * n1, n2, n2, Y, n2, 1, U2, n2, 1, P2, n2, nullptr, nullptr);
    k_write_sorted<<<(unsigned)(((long)R * n1 * n2 + 255) / 256 < 1024 ? ((long)R * n1 * n2 + 255) / 256 : 1024), 256, 0,
                     s>>>(R * n1, n2, n2, P2, sigc2, perm2, P2s, n2, 0); count_launch();
    k_write_sorted<<<(n2 * n2 + 255) / 256, 256, 0, s>>>(n2, n2, n2, U2, sigc2, perm2, V2, n2, 0); count_launch();
  }
  st = cholqr_sigma(s, R * n1, n2, P2s, n2, sig2, ws);
  if (st != TT_OK) return st;
  if (!ws.dry) {
    k_sort_cols<<<1, 1024, 0, s>>>(n2, n2, n2, sig2, V2, tmp2); count_launch();
    k_decide<<<1, 32, 0, s>>>(sig2, n2, 1, 3, j.tol, j.rmax, K2, 0, j.lp.r_ptr, j.lp.nblk, j.lp.nextra, n1,
                              j.r2_ptr, j.r2_nblk, j.r2_nextra, nullptr, 0, n2, j.ctrl, 1, nullptr); count_launch();
    // FP64 path: the columns come from the FP64 Jacobi, orthonormal to round-off, and take at most
    // one polar step; the mixed path's FP32-accurate small columns are only ~1e-2 orthogonal
    // (the FP32 sweep stops at its round-off floor): their polar steps start in FP32
    if (n2 <= 32 && F64)
      k_orthonormalise_polar<<<1, 128, 0, s>>>(n2, n2, V2, &j.ctrl->k[1], n2, nullptr);
    else if (n2 <= 32)
      k_orthonormalise_polar_mixed<<<1, 128, 0, s>>>(n2, n2, V2, &j.ctrl->k[1], n2, nullptr);
    else
      k_orthonormalise<<<1, 1024, 0, s>>>(n2, n2, V2, &j.ctrl->k[1], n2, nullptr);
    count_launch();
    small_gemm_pair<double, double>(s, R * n1, K2, n2, Y, j.B0, n2, 1, V2, n2, 1, Y2, B0p, K2, &j.ctrl->k[1]);
  }
  // ---- bond 1: A1 = Y2^T (nv x R); its left vectors are V1
  double* sigc1 = ws.take<double>(R);
  int* perm1 = ws.take<int>(R);
  const int Kr = (K1 + 8 < R) ? K1 + 8 : R;  // leading columns refined in FP64
  double* sig1 = ws.take<double>(Kr);
  double* P1s = ws.take<double>((size_t)nv * R);
  double* fro1 = ws.take<double>(1);
  double* fparts = ws.take<double>(kTailParts);
  int* rank1 = ws.take<int>(R);
  double* tmpK = ws.take<double>((size_t)nv * Kr);
  // concurrent problems (batch views, one-CTA cooperative launches): the GPU is already full, so
  // the bond-1 tail, column sort and W product take the forms with the fewest launches and CTAs
  const bool few_launches = (j.coop_grid_max == 1);
  double* tailK = ws.take<double>(1);
  double* V1 = ws.take<double>((size_t)nv * K1);
  double* wpart = ws.take<double>(small_gemm_ksplit_elems(R, K1));
  double *U1 = nullptr, *P1 = nullptr;
  st = svd_right_pre<F64>(s, num_sms, SrcCols<double>{Y2, nv}, nv, R, ws, &U1, &P1, sigc1, perm1, j.ctrl,
                          j.coop_grid_max);
  if (st != TT_OK) return st;
  if (!ws.dry) {
    small_gemm<double, double>(s, nv, R, R, Y2, 1, nv, U1, R, 1, P1, R, nullptr, nullptr);  // P1 = A1 U1
    k_write_sorted<<<(unsigned)(((long)nv * R + 255) / 256 < 1024 ? ((long)nv * R + 255) / 256 : 1024), 256, 0,
                     s>>>(nv, R, R, P1, sigc1, perm1, P1s, R, 0); count_launch();
  }
  st = cholqr_sigma(s, nv, R, P1s, Kr, sig1, ws);
  if (st != TT_OK || ws.dry) return st;
  // energy beyond the Kr refined values: from the FP64 Jacobi singular values (FP64 path), or
  // ||A1||_F^2 - sum sigma_j^2 (mixed path; accurate to about sqrt(eps_64) ||A1||)
  if (F64) {  // the FP64 Jacobi singular values resolve the whole tail
    k_tail_from_sigma<<<1, 32, 0, s>>>(R, Kr, sigc1, tailK); count_launch();
  } else {
    if (few_launches) {
      k_sumsq_parts<<<1, 1024, 0, s>>>((long)R * nv, Y2, nullptr, Kr, sig1, fro1, tailK); count_launch();
    } else {
      k_sumsq_parts<<<kTailParts, 256, 0, s>>>((long)R * nv, Y2, fparts, 0, nullptr, nullptr, nullptr);
      count_launch();
      k_tail_from_parts<<<1, 32, 0, s>>>(kTailParts, fparts, Kr, sig1, fro1, tailK); count_launch();
    }
  }
  if (few_launches) {
    k_sort_cols<<<1, 1024, 0, s>>>(nv, R, Kr, sig1, P1s, tmpK); count_launch();
  } else {
    k_sort_keys<<<1, 1024, 0, s>>>(Kr, sig1, rank1); count_launch();
    k_permute_cols<<<(nv + kPermRows - 1) / kPermRows, 256, 0, s>>>(nv, R, Kr, rank1, P1s); count_launch();
  }
  k_decide<<<1, 32, 0, s>>>(sig1, Kr, 0, 3, j.tol, j.rmax, K1, j.nrowsZ, j.lp.r_ptr, j.lp.nblk, j.lp.nextra, 1,
                            nullptr, 0, 0, &j.ctrl->k[1], n1, 0, j.ctrl, 0, tailK); count_launch();
  // V1 <- the leading K1 columns of P1s, with the zero ones replaced by independent unit vectors
  k_fix_zero_columns<<<1, 1024, 0, s>>>(nv, K1, V1, sig1, &j.ctrl->k[0], K2, &j.ctrl->k[1], P1s, R); count_launch();
  k_write_cores3<<<64, 256, 0, s>>>(n1, n2, K1, K2, V1, V2, j.ctrl, j.core1, j.core2); count_launch();
  small_gemm_ksplit(s, few_launches ? 0 : num_sms, R, K1, nv, B0p, nv, 1, V1, K1, 1, j.W, K1, &j.ctrl->k[0], wpart);
  small_gemm<double, double>(s, K1 * n1, n2, K2, j.core1, K2, 1, j.core2, n2, 1, j.Bnew, n2, nullptr, nullptr);
  k_vj<<<K1, 128, 0, s>>>(K1, nang, j.Bnew, j.domega, j.vJ); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

tt_status small_round(cudaStream_t s, int num_sms, const SmallJob& j, Bump& ws) {
  TimerScope scope(kSmall, s);
  const int R = j.lp.ncap();
  const int n1 = j.n1, n2 = j.n2, nang = n1 * n2;
  tt_status st;
  double* Y = ws.take<double>((size_t)R * nang);
  if (!ws.dry) small_gemm<double, double>(s, R, nang, R, j.RZ, R, 1, j.B0, nang, 1, Y, nang, nullptr, nullptr);
  if (j.d == 2) {
    // the only bond: SVD of Y (R x n1)
    double* sig = ws.take<double>(n1);
    double* V = ws.take<double>((size_t)n1 * n1);
    st = svd_right(s, num_sms, R, n1, Y, ws, sig, V, j.ctrl, j.coop_grid_max);
    if (st != TT_OK || ws.dry) return st;
    k_decide<<<1, 32, 0, s>>>(sig, n1, 1, 2, j.tol, j.rmax, j.K1cap, j.nrowsZ, j.lp.r_ptr, j.lp.nblk,
                              j.lp.nextra, 1, nullptr, 0, 0, nullptr, 0, n1, j.ctrl, 0, nullptr); count_launch();
    small_gemm<double, double>(s, R, j.K1cap, n1, j.B0, n1, 1, V, n1, 1, j.W, j.K1cap, &j.ctrl->k[0], nullptr);
    k_write_cores2<<<(j.K1cap * n1 + 255) / 256, 256, 0, s>>>(n1, j.K1cap, V, j.ctrl, j.core1); count_launch();
    cudaMemcpyAsync(j.Bnew, j.core1, sizeof(double) * (size_t)j.K1cap * n1, cudaMemcpyDeviceToDevice, s);
    k_vj<<<j.K1cap, 128, 0, s>>>(j.K1cap, nang, j.Bnew, j.domega, j.vJ); count_launch();
    return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  // ---- d = 3 ----
  const int K1 = j.K1cap, K2 = j.K2cap;
  return j.mixed ? small_round_mixed3<false>(s, num_sms, j, ws, Y) : small_round_mixed3<true>(s, num_sms, j, ws, Y);
}

}  // namespace ttk
