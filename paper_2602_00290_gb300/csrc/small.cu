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
// Every SVD is a QR (TSQR) followed by a one-sided Jacobi SVD of the triangular factor.
#include <cstdio>

#include "bigpass.cuh"
#include "small.cuh"

namespace ttk {
namespace {

constexpr double kPi = 3.14159265358979323846;

template <typename TA, typename TB>
__global__ void k_small_gemm(int M, int N, int K, const TA* __restrict__ A, long sa0, long sa1,
                             const TB* __restrict__ B, long sb0, long sb1, double* __restrict__ C, long ldc,
                             const int* __restrict__ nlive, const double* __restrict__ inv_colscale) {
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

// One-sided (Hestenes) Jacobi SVD of an n x n matrix R (row-major) in one CTA: columns are
// orthogonalised by plane rotations in round-robin order (n/2 independent pairs per round,
// one warp per pair), accumulating V.  Output: sigma sorted descending and V_out row-major
// with column j the right singular vector of sigma_j.  At most `maxsweep` sweeps.
__global__ void __launch_bounds__(1024) k_jacobi(int n, const double* __restrict__ R, double* __restrict__ Aw,
                                                 double* __restrict__ Vw, double* __restrict__ sigma_out,
                                                 double* __restrict__ V_out, int* __restrict__ perm, int maxsweep,
                                                 int* status) {
  __shared__ int rot_flag;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int row = idx / n, col = idx - row * n;
    Aw[(size_t)col * n + row] = R[idx];
    Vw[(size_t)col * n + row] = (row == col) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int np = n + (n & 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int sweep = 0; sweep < maxsweep; ++sweep) {
    if (threadIdx.x == 0) rot_flag = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int pr = warp; pr < np / 2; pr += nwarps) {
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
        double* ap = Aw + (size_t)p * n;
        double* aq = Aw + (size_t)q * n;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = lane; i < n; i += 32) {
          const double x = ap[i], y = aq[i];
          a += x * x;
          b += y * y;
          g += x * y;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (g != 0.0 && fabs(g) > 1e-15 * sqrt(a) * sqrt(b)) {
          const double zeta = (b - a) / (2.0 * g);
          double t;
          if (fabs(zeta) > 1e150)
            t = 0.5 / zeta;
          else
            t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          for (int i = lane; i < n; i += 32) {
            const double x = ap[i], y = aq[i];
            ap[i] = cs * x - sn * y;
            aq[i] = sn * x + cs * y;
          }
          double* vp = Vw + (size_t)p * n;
          double* vq = Vw + (size_t)q * n;
          for (int i = lane; i < n; i += 32) {
            const double x = vp[i], y = vq[i];
            vp[i] = cs * x - sn * y;
            vq[i] = sn * x + cs * y;
          }
          if (lane == 0) rot_flag = 1;
        }
      }
      __syncthreads();
    }
    const int f = rot_flag;
    __syncthreads();
    if (!f) break;
    if (sweep == maxsweep - 1 && threadIdx.x == 0) latch(status, TT_ERR_TIMEOUT);
  }
  // singular values = column norms; rank-sort descending (ties by index)
  double* sig = sigma_out;  // temporary: unsorted norms in V_out's last use? use perm-sorted write below
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double a = 0.0;
    const double* ap = Aw + (size_t)p * n;
    for (int i = 0; i < n; ++i) a += ap[i] * ap[i];
    Aw[(size_t)p * n] = sqrt(a);  // column p is no longer needed beyond its norm
    if (!isfinite(a)) latch(status, TT_ERR_NONFINITE);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const double sp = Aw[(size_t)p * n];
    int rank = 0;
    for (int q = 0; q < n; ++q) {
      const double sq = Aw[(size_t)q * n];
      rank += (sq > sp) || (sq == sp && q < p);
    }
    perm[rank] = p;
    sig[rank] = sp;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    V_out[idx] = Vw[(size_t)perm[j] * n + i];
  }
}

// Rank decision for one bond.  first != 0: this is the first SVD of the right-to-left sweep,
// which also fixes ||X|| = sqrt(sum sigma^2) and delta = tol ||X|| / sqrt(d-1).  The kept rank
// is the smallest k >= 1 with sqrt(sum_{j>=k} sigma_j^2) <= delta (tol > 0), or the full rank
// of the unfolding (tol == 0), then capped by rmax and kcap.
__global__ void k_decide(const double* __restrict__ sigma, int n, int first, int dcores, double tol, int rmax,
                         int kcap, long full_rank_cap, const int* rptr, int nblk, int nextra, int rows_mul,
                         const int* r2ptr, int r2_nblk, int r2_nextra, const int* kprev, int cols_mul,
                         int cols_fixed, DevCtrl* ctrl, int slot) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (first) {
    double s2 = 0.0;
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
    double tail2 = 0.0;
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

// Re-orthonormalise the first k columns of V (nv x ldv, row-major) by classical Gram-Schmidt
// applied twice.  Rows with row % rowmod >= rowlive are structurally zero and stay zero; a
// column that vanishes (zero singular value) is replaced by the first canonical vector that
// is independent of the earlier columns.
__global__ void __launch_bounds__(1024) k_reorth(int nv, int ldv, double* __restrict__ V, const int* kptr,
                                                 int rowmod, const int* rowlive_ptr) {
  __shared__ double red[33];
  __shared__ double h[1024];
  const int k = *kptr;
  const int rowlive = rowlive_ptr ? *rowlive_ptr : rowmod;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    int cand = -1;  // canonical replacement index in use (-1: original column)
    for (int attempt = 0; attempt <= nv; ++attempt) {
      if (attempt > 0) {
        // next canonical vector on a live row
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
          double s = 0.0;
          for (int i = lane; i < nv; i += 32) s += V[(size_t)i * ldv + i2] * V[(size_t)i * ldv + j];
          s = warp_sum(s);
          if (lane == 0) h[i2] = s;
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
      if (n1 > 0.5 * n0 && n1 > 0.0) {
        for (int i = threadIdx.x; i < nv; i += blockDim.x) V[(size_t)i * ldv + j] /= n1;
        __syncthreads();
        break;
      }
    }
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

}  // namespace

template <typename TA, typename TB>
void small_gemm(cudaStream_t s, int M, int N, int K, const TA* A, long sa0, long sa1, const TB* B, long sb0,
                long sb1, double* C, long ldc, const int* nlive, const double* inv_colscale) {
  dim3 grid((N + 15) / 16, (M + 15) / 16);
  k_small_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, sa0, sa1, B, sb0, sb1, C, ldc, nlive, inv_colscale); count_launch();
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

static tt_status jacobi(cudaStream_t s, int n, const double* R, Bump& ws, double* sigma, double* V,
                        DevCtrl* ctrl) {
  double* Aw = ws.take<double>((size_t)n * n);
  double* Vw = ws.take<double>((size_t)n * n);
  int* perm = ws.take<int>(n);
  if (ws.dry) return TT_OK;
  if (n > 1024) return TT_ERR_UNSUPPORTED;
  k_jacobi<<<1, 1024, 0, s>>>(n, R, Aw, Vw, sigma, V, perm, 60, &ctrl->status); count_launch();
  return TT_OK;
}

// QR of an explicit small matrix (rows x cols) through the TSQR kernels; returns R (cols x cols).
template <class Src>
static tt_status small_qr(cudaStream_t s, int num_sms, const Src& src, long rows, int cols, Bump& ws,
                          double** Rout) {
  LivePattern lp{nullptr, cols, 1, 0};
  const long L = tsqr_max_leaves<double, 16>(num_sms, cols, rows, 64);
  double* a = ws.take<double>((size_t)L * cols * cols);
  double* b = ws.take<double>((size_t)((L + 1) / 2) * cols * cols);
  if (ws.dry) {
    *Rout = nullptr;
    return TT_OK;
  }
  return run_tsqr<double, 16>(s, num_sms, src, lp, rows, 64, a, b, Rout);
}

tt_status small_round(cudaStream_t s, int num_sms, const SmallJob& j, Bump& ws) {
  TimerScope scope(kSmall, s);
  const int R = j.lp.ncap();
  const int n1 = j.n1, n2 = j.n2, nang = n1 * n2;
  tt_status st;
  double* Y = ws.take<double>((size_t)R * nang);
  if (!ws.dry) small_gemm<double, double>(s, R, nang, R, j.RZ, R, 1, j.B0, nang, 1, Y, nang, nullptr, nullptr);
  if (j.d == 2) {
    double* Rq = nullptr;
    st = small_qr(s, num_sms, SrcRows<double>{Y, n1}, R, n1, ws, &Rq);
    if (st != TT_OK) return st;
    double* sig = ws.take<double>(n1);
    double* V = ws.take<double>((size_t)n1 * n1);
    st = jacobi(s, n1, Rq, ws, sig, V, j.ctrl);
    if (st != TT_OK) return st;
    if (ws.dry) return TT_OK;
    k_decide<<<1, 32, 0, s>>>(sig, n1, 1, 2, j.tol, j.rmax, j.K1cap, j.nrowsZ, j.lp.r_ptr, j.lp.nblk,
                              j.lp.nextra, 1, nullptr, 0, 0, nullptr, 0, n1, j.ctrl, 0); count_launch();
    small_gemm<double, double>(s, R, j.K1cap, n1, j.B0, n1, 1, V, n1, 1, j.W, j.K1cap, &j.ctrl->k[0], nullptr);
    k_write_cores2<<<(j.K1cap * n1 + 255) / 256, 256, 0, s>>>(n1, j.K1cap, V, j.ctrl, j.core1); count_launch();
    cudaMemcpyAsync(j.Bnew, j.core1, sizeof(double) * (size_t)j.K1cap * n1, cudaMemcpyDeviceToDevice, s);
    k_vj<<<j.K1cap, 128, 0, s>>>(j.K1cap, nang, j.Bnew, j.domega, j.vJ); count_launch();
    return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  // ---- d = 3 ----
  const int K1 = j.K1cap, K2 = j.K2cap;
  // bond 2: SVD of Y as (R n1) x n2
  double* R2 = nullptr;
  st = small_qr(s, num_sms, SrcRows<double>{Y, n2}, (long)R * n1, n2, ws, &R2);
  if (st != TT_OK) return st;
  double* sig2 = ws.take<double>(n2);
  double* V2 = ws.take<double>((size_t)n2 * n2);
  st = jacobi(s, n2, R2, ws, sig2, V2, j.ctrl);
  if (st != TT_OK) return st;
  const int nv = n1 * K2;
  double* Y2 = ws.take<double>((size_t)R * nv);
  double* B0p = ws.take<double>((size_t)R * nv);
  if (!ws.dry) {
    k_decide<<<1, 32, 0, s>>>(sig2, n2, 1, 3, j.tol, j.rmax, K2, 0, j.lp.r_ptr, j.lp.nblk, j.lp.nextra, n1,
                              j.r2_ptr, j.r2_nblk, j.r2_nextra, nullptr, 0, n2, j.ctrl, 1); count_launch();
    small_gemm<double, double>(s, R * n1, K2, n2, Y, n2, 1, V2, n2, 1, Y2, K2, &j.ctrl->k[1], nullptr);
    small_gemm<double, double>(s, R * n1, K2, n2, j.B0, n2, 1, V2, n2, 1, B0p, K2, &j.ctrl->k[1], nullptr);
  }
  // bond 1: SVD of Y2 as R x (n1 K2) through the QR of its transpose
  double* R1 = nullptr;
  st = small_qr(s, num_sms, SrcCols<double>{Y2, nv}, nv, R, ws, &R1);
  if (st != TT_OK) return st;
  double* sig1 = ws.take<double>(R);
  double* U1 = ws.take<double>((size_t)R * R);
  st = jacobi(s, R, R1, ws, sig1, U1, j.ctrl);
  if (st != TT_OK) return st;
  double* V1 = ws.take<double>((size_t)nv * K1);
  if (ws.dry) return TT_OK;
  k_decide<<<1, 32, 0, s>>>(sig1, R, 0, 3, j.tol, j.rmax, K1, j.nrowsZ, j.lp.r_ptr, j.lp.nblk, j.lp.nextra, 1,
                            nullptr, 0, 0, &j.ctrl->k[1], n1, 0, j.ctrl, 0); count_launch();
  // V1 = Y2^T U1(:, :k1) diag(1/sigma1)
  small_gemm<double, double>(s, nv, K1, R, Y2, 1, nv, U1, R, 1, V1, K1, &j.ctrl->k[0], sig1);
  k_reorth<<<1, 1024, 0, s>>>(nv, K1, V1, &j.ctrl->k[0], K2, &j.ctrl->k[1]); count_launch();
  k_write_cores3<<<64, 256, 0, s>>>(n1, n2, K1, K2, V1, V2, j.ctrl, j.core1, j.core2); count_launch();
  // W = B0p (R x nv) V1 (nv x K1)
  small_gemm<double, double>(s, R, K1, nv, B0p, nv, 1, V1, K1, 1, j.W, K1, &j.ctrl->k[0], nullptr);
  // Bnew = core1 (K1 n1 x K2) core2 (K2 x n2); vJ
  small_gemm<double, double>(s, K1 * n1, n2, K2, j.core1, K2, 1, j.core2, n2, 1, j.Bnew, n2, nullptr, nullptr);
  k_vj<<<K1, 128, 0, s>>>(K1, nang, j.Bnew, j.domega, j.vJ); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

}  // namespace ttk
