// Small-core part of SVD-based TT rounding (Sec. 3.1 footnote): everything after the QR of
// the merged core, on matrices whose sizes are set by ranks and angular mode sizes only.
#pragma once
#include "common.cuh"

namespace ttk {

// Bump allocator over the context workspace (dry run = size query).
struct Bump {
  char* base;
  size_t off;
  size_t cap;
  bool dry;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = ((sizeof(T) * (count ? count : 1)) + 255) & ~(size_t)255;
    char* p = dry ? nullptr : base + off;
    off += bytes;
    return reinterpret_cast<T*>(p);
  }
  bool ok() const { return dry || off <= cap; }
};

// Inputs/outputs of one small-core sweep (all FP64, capacity layout).
struct SmallJob {
  int coop_grid_max;  // > 0: cap on the CTAs of the cooperative Jacobi
  int d;          // 2 or 3
  int n1, n2;     // angular mode sizes (n2 = 1 for d = 2)
  long nrowsZ;    // N_Z (bounds the rank of the merged-core unfolding)
  LivePattern lp; // columns of the sum (Rcap = lp.ncap())
  const int* r2_ptr;  // live bond-2 rank of the sum's blocks (d = 3), else null
  int r2_nblk, r2_nextra;  // bond-2 width of the sum = r2_nblk * r2 + r2_nextra
  double tol;
  int rmax;
  int K1cap, K2cap;   // output rank capacities
  const double* B0;   // [Rcap][n1*n2] right part of the sum
  const double* RZ;   // [Rcap][Rcap] upper triangular
  const double* domega;  // [n1*n2]
  // outputs
  double* W;          // [Rcap][K1cap]
  double* core1;      // d=3: [K1cap][n1][K2cap]; d=2: [K1cap][n1]
  double* core2;      // d=3: [K2cap][n2]
  double* Bnew;       // [K1cap][n1*n2]
  double* vJ;         // [K1cap]
  DevCtrl* ctrl;      // ranks -> ctrl->k[0] (bond 1), ctrl->k[1] (bond 2)
  bool mixed;         // FP32 rotations (Jacobi on R^T of an FP32 TSQR), FP64 singular values/vectors
};

tt_status small_round(cudaStream_t s, int num_sms, const SmallJob& job, Bump& ws);

// C[i][j] = sum_k A(i,k) B(k,j) * colscale(j) for j < Nlive (device count) else 0.
// A(i,k) = A[i*sa0 + k*sa1], B(k,j) = B[k*sb0 + j*sb1], C row-major with ldc.
template <typename TA, typename TB>
void small_gemm(cudaStream_t s, int M, int N, int K, const TA* A, long sa0, long sa1, const TB* B, long sb0,
                long sb1, double* C, long ldc, const int* nlive, const double* inv_colscale);

// B_base[q][l][p] = sum_b core1[q][l][b] core2[b][p] (d = 3) or core1[q][l] (d = 2), cast to FP64.
template <typename S>
void right_part(cudaStream_t s, int d, int rcap1, int n1, int rcap2, int n2, const S* core1, const S* core2,
                double* Bbase);

// vJ[j] = (1/4 pi) sum_i dOmega_i B[j][i] for j < K1 (angle integral weights of a right part).
void k_vj_host_launch(cudaStream_t s, int K1, int nang, const double* B, const double* domega, double* vJ);

// Energy-type reductions: out[i] = sum over CTA partials (fixed order).
void reduce_partials(cudaStream_t s, const double* partials, long nblocks, int stride, double* out,
                     double scale);

}  // namespace ttk

namespace ttk {
// One-sided Jacobi SVD of an m x n column-major matrix A (in place) by a cooperative grid:
// one CTA per column pair per round (round-robin order), bounded-spin grid barrier between
// rounds.  On return the columns of A are orthogonal; sigma[j] (sorted descending) and, if
// U != null, U[i][j] = A[i][perm j] / sigma_j (row-major m x ldu, j < ncols_out, zero
// columns for sigma = 0) are written.  Rotations stop when no pair in a sweep exceeds the
// thresholds (at most 40 sweeps, else TT_ERR_TIMEOUT is latched).
// With V != null the rotations are accumulated in V (n x n) and Vout (row-major n x n,
// column j the right singular vector of sigma_j) is written.
// SVD of an m x n row-major matrix M by the cooperative one-sided Jacobi on its transpose: sigma (n,
// decreasing) and Vout (n x n row-major, column j the right singular vector of sigma_j).
tt_status svd_right(cudaStream_t s, int num_sms, int m, int n, const double* M, Bump& ws, double* sigma,
                    double* Vout, DevCtrl* ctrl, int grid_max);
tt_status coop_jacobi(cudaStream_t s, int num_sms, int m, int n, double* A, double* V, double* sigma, double* U,
                      int ldu, int ncols_out, double* Vout, int* perm, double* tmp, DevCtrl* ctrl,
                      int grid_max = 0);
}  // namespace ttk
