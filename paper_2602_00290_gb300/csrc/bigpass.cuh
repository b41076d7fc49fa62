// Passes over the merged spatio-spectral core Z (N_Z rows): tall-skinny QR (TSQR) of a
// possibly virtual N_Z x R matrix, and the rank-reducing update Z_new = A W with the
// source-step epilogue.  These are the kernels that touch every row of the TT state.
#pragma once
#include "common.cuh"
#include "instr.cuh"

namespace ttk {

// ---------------------------------------------------------------------------------------
// Column sources.  A source maps (row k, column c) of a tall matrix to a value; `col(c)`
// precomputes what a thread that owns column c needs.

// Explicit row-major matrix A[k * ld + c].
template <typename S>
struct SrcRows {
  const S* A;
  long ld;
  struct Col { int c; };
  __device__ __forceinline__ Col col(int c) const { return Col{c}; }
  __device__ __forceinline__ double load(const Col& cc, long k) const {
    return (double)A[k * ld + cc.c];
  }
};

// Explicit matrix read transposed: element (row i, column c) = A[c * ld + i].
template <typename S>
struct SrcCols {
  const S* A;
  long ld;
  struct Col { int c; };
  __device__ __forceinline__ Col col(int c) const { return Col{c}; }
  __device__ __forceinline__ double load(const Col& cc, long k) const {
    return (double)A[(long)cc.c * ld + k];
  }
};

// The forward-Euler upwind transport sum of Appendix A as a virtual matrix over the rows of
// Z, in capacity layout: column block 0 is Z itself, block t = 1..nterm is
// -lambda_a D_{a,w} Z with D_{a,+} Z_i = Z_i - Z_{i-1} and D_{a,-} Z_i = Z_{i+1} - Z_i (zero
// ghost rows outside the grid), and each of the nbc trailing columns is the rank-1 Dirichlet
// inflow column of one operator (+-lambda_a * inflow spectrum on the face-adjacent rows).
template <typename S>
struct SrcStencil {
  const S* Z;
  int ldz;   // rank capacity of Z (row stride)
  int rcap;  // column block width
  int nterm;
  int G;
  int ext[3];
  long stride[3];
  double lam[kMaxTerms];   // lambda_a of each operator
  int axis[kMaxTerms];
  int w[kMaxTerms];
  int bc_term[kMaxTerms];  // operator of each inflow column
  const double* bcval;     // [nbc][G] signed lambda * inflow
  struct Col {
    int kind;  // 0: Z, 1: operator image, 2: inflow column, 3: none
    int q, ax, w, b;
    double lam;
  };
  __device__ __forceinline__ Col col(int c) const {
    Col cc{3, 0, 0, 0, 0, 0.0};
    const int t = c / rcap;
    if (t == 0) {
      cc.kind = 0;
      cc.q = c;
    } else if (t <= nterm) {
      cc.kind = 1;
      cc.q = c - t * rcap;
      cc.ax = axis[t - 1];
      cc.w = w[t - 1];
      cc.lam = lam[t - 1];
    } else {
      cc.kind = 2;
      cc.b = c - (nterm + 1) * rcap;
      const int tt = bc_term[cc.b];
      cc.ax = axis[tt];
      cc.w = w[tt];
    }
    return cc;
  }
  __device__ __forceinline__ double load(const Col& cc, long k) const {
    if (cc.kind == 0) return (double)Z[k * ldz + cc.q];
    if (cc.kind == 3) return 0.0;
    const long s = stride[cc.ax];
    const int idx = (int)((k / s) % ext[cc.ax]);
    if (cc.kind == 1) {
      const double zk = (double)Z[k * ldz + cc.q];
      double diff;
      if (cc.w > 0) {
        const double up = (idx > 0) ? (double)Z[(k - s) * ldz + cc.q] : 0.0;
        diff = zk - up;
      } else {
        const double dn = (idx < ext[cc.ax] - 1) ? (double)Z[(k + s) * ldz + cc.q] : 0.0;
        diff = dn - zk;
      }
      return -cc.lam * diff;
    }
    const bool at_face = (cc.w > 0) ? (idx == 0) : (idx == ext[cc.ax] - 1);
    return at_face ? bcval[cc.b * G + (int)(k % G)] : 0.0;
  }
};

// ---------------------------------------------------------------------------------------
// Householder TSQR.  A CTA owns a contiguous range of rows and keeps the upper-triangular
// factor R of everything it has read in shared memory (row-major packed: row j holds
// columns j..ncap-1).  Thread c owns column c: it holds column c of the current block of
// BR rows in registers and is the only thread that ever touches R[.][c].  For each live
// column j the reflector that annihilates column j of the block against R[j][j] is formed
// by thread j and applied by every thread c > j; one barrier per reflector (the reflector
// vector is double-buffered).

__device__ __forceinline__ int tri_off(int j, int n) { return j * n - (j * (j - 1)) / 2; }

template <typename T, int BR>
__device__ __forceinline__ void hh_absorb(T* Rs, int ncap, T (&B)[BR], T* vbuf, T* taub, int& buf,
                                          int jbeg, const LivePattern& lp, int r, bool mycol) {
  const int c = threadIdx.x;
  for (int j = jbeg; j < ncap; ++j) {
    if (!lp.live(j, r)) continue;
    T* vb = vbuf + buf * BR;
    if (c == j) {
      T xp[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int i = 0; i < BR; ++i) xp[i & 3] += B[i] * B[i];
      const T x2 = (xp[0] + xp[1]) + (xp[2] + xp[3]);
      T tau = T(0);
      if (x2 > T(0)) {
        T* rjj = Rs + tri_off(j, ncap);
        const T alpha = *rjj;
        const T nrm = sqrt(alpha * alpha + x2);
        const T beta = (alpha >= T(0)) ? -nrm : nrm;
        const T sc = T(1) / (alpha - beta);
#pragma unroll
        for (int i = 0; i < BR; ++i) vb[i] = B[i] * sc;
        tau = (beta - alpha) / beta;
        *rjj = beta;
#pragma unroll
        for (int i = 0; i < BR; ++i) B[i] = T(0);
      }
      taub[buf] = tau;
    }
    __syncthreads();
    const T tau = taub[buf];
    if (tau != T(0) && c > j && mycol) {
      T* rjc = Rs + tri_off(j, ncap) + (c - j);
      T wp[4] = {*rjc, T(0), T(0), T(0)};
#pragma unroll
      for (int i = 0; i < BR; ++i) wp[i & 3] += vb[i] * B[i];
      T wv = (wp[0] + wp[1]) + (wp[2] + wp[3]);
      wv *= tau;
      *rjc -= wv;
#pragma unroll
      for (int i = 0; i < BR; ++i) B[i] -= wv * vb[i];
    }
    buf ^= 1;
  }
}

template <typename T, int BR>
__device__ __forceinline__ void write_R(const T* Rs, int ncap, double* Ro) {
  for (int idx = threadIdx.x; idx < ncap * ncap; idx += blockDim.x) {
    const int i = idx / ncap, j = idx - (idx / ncap) * ncap;
    Ro[idx] = (j >= i) ? (double)Rs[tri_off(i, ncap) + (j - i)] : 0.0;
  }
}

// packed R, then the double-buffered reflector (16-byte aligned) and its two scalars
__host__ __device__ inline size_t tsqr_r_elems(int ncap) { return (((size_t)ncap * (ncap + 1) / 2) + 3) & ~(size_t)3; }
template <typename T, int BR>
__host__ __device__ inline size_t tsqr_smem_bytes(int ncap) {
  return sizeof(T) * (tsqr_r_elems(ncap) + 2 * BR + 4);
}

template <typename T, int BR, class Src>
__global__ void __launch_bounds__(256) k_tsqr_leaf(Src src, LivePattern lp, long nrows, long rpc,
                                                   double* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char tsqr_smem[];
  const int ncap = lp.ncap();
  T* Rs = reinterpret_cast<T*>(tsqr_smem);
  T* vbuf = Rs + tsqr_r_elems(ncap);
  T* taub = vbuf + 2 * BR;
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  for (int i = threadIdx.x; i < ncap * (ncap + 1) / 2; i += blockDim.x) Rs[i] = T(0);
  const int c = threadIdx.x;
  const bool mycol = (c < ncap) && lp.live(c, r);
  const auto cc = src.col(c < ncap ? c : 0);
  __syncthreads();
  const long beg = (long)blockIdx.x * rpc;
  const long end = (beg + rpc < nrows) ? beg + rpc : nrows;
  int buf = 0;
  for (long r0 = beg; r0 < end; r0 += BR) {
    T B[BR];
#pragma unroll
    for (int i = 0; i < BR; ++i) B[i] = (mycol && r0 + i < end) ? (T)src.load(cc, r0 + i) : T(0);
    hh_absorb<T, BR>(Rs, ncap, B, vbuf, taub, buf, 0, lp, r, mycol);
  }
  __syncthreads();
  write_R<T, BR>(Rs, ncap, Rout + (size_t)blockIdx.x * ncap * ncap);
}

// One level of the binary merge tree: output m = QR([R_{2m}; R_{2m+1}]).R
template <typename T, int BR>
__global__ void __launch_bounds__(256) k_tsqr_merge(LivePattern lp, int nin, const double* __restrict__ Rin,
                                                    double* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char tsqr_smem[];
  const int ncap = lp.ncap();
  const size_t nn = (size_t)ncap * ncap;
  const int a = 2 * blockIdx.x, b = a + 1;
  const double* Ra = Rin + (size_t)a * nn;
  double* Ro = Rout + (size_t)blockIdx.x * nn;
  if (b >= nin) {
    for (size_t i = threadIdx.x; i < nn; i += blockDim.x) Ro[i] = Ra[i];
    return;
  }
  const double* Rb = Rin + (size_t)b * nn;
  T* Rs = reinterpret_cast<T*>(tsqr_smem);
  T* vbuf = Rs + tsqr_r_elems(ncap);
  T* taub = vbuf + 2 * BR;
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  for (int idx = threadIdx.x; idx < ncap * ncap; idx += blockDim.x) {
    const int i = idx / ncap, j = idx - (idx / ncap) * ncap;
    if (j >= i) Rs[tri_off(i, ncap) + (j - i)] = (T)Ra[idx];
  }
  const int c = threadIdx.x;
  const bool mycol = (c < ncap) && lp.live(c, r);
  __syncthreads();
  int buf = 0;
  for (int i0 = 0; i0 < ncap; i0 += BR) {
    T B[BR];
#pragma unroll
    for (int i = 0; i < BR; ++i) B[i] = (mycol && i0 + i < ncap) ? (T)Rb[(size_t)(i0 + i) * ncap + c] : T(0);
    // rows i0.. of an upper-triangular factor vanish in columns < i0
    hh_absorb<T, BR>(Rs, ncap, B, vbuf, taub, buf, i0, lp, r, mycol);
  }
  __syncthreads();
  write_R<T, BR>(Rs, ncap, Ro);
}

// Host driver: leaves then merge levels; returns the device pointer of the final R
// (ncap x ncap, row-major, upper triangular) inside ws_a or ws_b.
template <typename T, int BR, class Src>
tt_status run_tsqr(cudaStream_t s, int num_sms, const Src& src, LivePattern lp, long nrows, int max_leaves,
                   double* ws_a, double* ws_b, double** Rfinal) {
  const int ncap = lp.ncap();
  const size_t smem = tsqr_smem_bytes<T, BR>(ncap);
  if (smem > 227 * 1024) return TT_ERR_UNSUPPORTED;
  const int threads = ((ncap + 31) / 32) * 32;
  if (threads > 1024) return TT_ERR_UNSUPPORTED;
  static_assert(BR > 0, "block rows");
  const int per_sm = (int)((228 * 1024) / (smem + 1024));
  long L = (nrows + BR - 1) / BR;
  long cap = (long)num_sms * (per_sm > 0 ? per_sm : 1);
  if (max_leaves > 0 && cap > max_leaves) cap = max_leaves;
  if (L > cap) L = cap;
  if (L < 1) L = 1;
  long rpc = (nrows + L - 1) / L;
  rpc = ((rpc + BR - 1) / BR) * BR;
  L = (nrows + rpc - 1) / rpc;
  if (L < 1) L = 1;
  cudaFuncSetAttribute(k_tsqr_leaf<T, BR, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_tsqr_merge<T, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  {
    TimerScope scope(kTsqrLeaf, s);
    k_tsqr_leaf<T, BR, Src><<<(unsigned)L, threads, smem, s>>>(src, lp, nrows, rpc, ws_a); count_launch();
  }
  TimerScope scope(kTsqrMerge, s);
  double* in = ws_a;
  double* out = ws_b;
  int n = (int)L;
  while (n > 1) {
    const int m = (n + 1) / 2;
    k_tsqr_merge<T, BR><<<m, threads, smem, s>>>(lp, n, in, out); count_launch();
    double* t = in;
    in = out;
    out = t;
    n = m;
  }
  *Rfinal = in;
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// Leaves needed for a TSQR of nrows rows (bounds workspace sizing).
template <typename T, int BR>
inline long tsqr_max_leaves(int num_sms, int ncap, long nrows, int max_leaves) {
  const size_t smem = tsqr_smem_bytes<T, BR>(ncap);
  const int per_sm = (int)((228 * 1024) / (smem + 1024));
  long L = (nrows + BR - 1) / BR;
  long cap = (long)num_sms * (per_sm > 0 ? per_sm : 1);
  if (max_leaves > 0 && cap > max_leaves) cap = max_leaves;
  if (L > cap) L = cap;
  return L < 1 ? 1 : L;
}

// ---------------------------------------------------------------------------------------
// Update pass: out[k][j] = scale_k * sum_c A[k][c] W[c][j] over the live columns c of A,
// j < kcap, plus an optional extra column out[k][kcap].  A tile of TM rows of A (formed from
// the source, e.g. the stencil sum) and W sit in shared memory; each thread accumulates a
// strip of outputs.  Per-row epilogue values (scale, extra column, two energy partials) are
// computed by thread m < TM from the full output row; partial sums per CTA go to
// partials[2*cta + {0,1}] in a fixed order.

template <typename SO>
struct EpiPlain {
  SO* out;
  long ld;
  static constexpr bool kExtra = false;
  __device__ __forceinline__ void prep(long, const double*, int, double& scale, double& extra, double& e0,
                                       double& e1) const {
    scale = 1.0;
    extra = 0.0;
    e0 = 0.0;
    e1 = 0.0;
  }
};

// Backward-Euler source update of Eq. (discRTsource) at fixed T on a freshly rounded row:
// J* = Z_new[k,:] . vJ, J^{m+1} = (J* + a eps)/(1 + a), row scale 1/(1 + a + s) and the
// isotropic column g = (a eps + s J^{m+1})/(1 + a + s).
template <typename SO>
struct EpiSource {
  SO* out;
  long ld;
  const double* vJ;
  const double* acoef;
  const double* scoef;
  const double* eps;
  static constexpr bool kExtra = true;
  __device__ __forceinline__ void prep(long k, const double* o, int kcap, double& scale, double& extra,
                                       double& e0, double& e1) const {
    double js = 0.0;
    for (int j = 0; j < kcap; ++j) js += o[j] * vJ[j];
    const double a = acoef[k], s = scoef[k], e = eps[k];
    const double jn = (js + a * e) / (1.0 + a);
    const double dinv = 1.0 / (1.0 + a + s);
    scale = dinv;
    extra = (a * e + s * jn) * dinv;
    e0 = js;
    e1 = a * (e - jn);
  }
};

// Final write of a rounded row plus its mean intensity for the energy report.
template <typename SO>
struct EpiFinal {
  SO* out;
  long ld;
  const double* vJ;
  static constexpr bool kExtra = false;
  __device__ __forceinline__ void prep(long, const double* o, int kcap, double& scale, double& extra,
                                       double& e0, double& e1) const {
    double js = 0.0;
    for (int j = 0; j < kcap; ++j) js += o[j] * vJ[j];
    scale = 1.0;
    extra = 0.0;
    e0 = js;
    e1 = 0.0;
  }
};

template <typename T, int TM>
__host__ __device__ inline size_t update_smem_bytes(int ncap, int kcap) {
  return ((sizeof(T) * ((size_t)TM * (ncap + 1) + (size_t)ncap * kcap) + 15) & ~(size_t)15) +
         sizeof(double) * ((size_t)TM * (kcap + 1) + 4 * TM);
}

template <typename T, int TM, class Src, class Epi>
__global__ void __launch_bounds__(256) k_update(Src src, LivePattern lp, long nrows, const double* __restrict__ W,
                                                int kcap, Epi epi, double* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char upd_smem[];
  const int ncap = lp.ncap();
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  T* As = reinterpret_cast<T*>(upd_smem);                            // [TM][ncap+1]
  T* Ws = As + (size_t)TM * (ncap + 1);                              // [ncap][kcap]
  const size_t os_off = ((sizeof(T) * ((size_t)TM * (ncap + 1) + (size_t)ncap * kcap) + 15) & ~(size_t)15);
  double* Os = reinterpret_cast<double*>(upd_smem + os_off);         // [TM][kcap+1]
  double* rowv = Os + (size_t)TM * (kcap + 1);                       // [4][TM]
  const long row0 = (long)blockIdx.x * TM;
  for (int i = threadIdx.x; i < ncap * kcap; i += blockDim.x) Ws[i] = (T)W[i];
  for (int c = threadIdx.x; c < ncap; c += blockDim.x) {
    const bool live = lp.live(c, r);
    const auto cc = src.col(c);
    for (int m = 0; m < TM; ++m) {
      const long k = row0 + m;
      As[(size_t)m * (ncap + 1) + c] = (live && k < nrows) ? (T)src.load(cc, k) : T(0);
    }
  }
  __syncthreads();
  const int m = threadIdx.x % TM;
  const int strip = threadIdx.x / TM;
  const int nstrip = blockDim.x / TM;
  for (int j0 = strip; j0 < kcap; j0 += nstrip * 4) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int c = 0; c < ncap; ++c) {
      const T a = As[(size_t)m * (ncap + 1) + c];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u * nstrip;
        if (j < kcap) acc[u] += a * Ws[(size_t)c * kcap + j];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u * nstrip;
      if (j < kcap) Os[(size_t)m * (kcap + 1) + j] = (double)acc[u];
    }
  }
  __syncthreads();
  if (threadIdx.x < TM) {
    const long k = row0 + threadIdx.x;
    double sc = 0.0, ex = 0.0, e0 = 0.0, e1 = 0.0;
    if (k < nrows) epi.prep(k, Os + (size_t)threadIdx.x * (kcap + 1), kcap, sc, ex, e0, e1);
    rowv[threadIdx.x] = sc;
    rowv[TM + threadIdx.x] = ex;
    rowv[2 * TM + threadIdx.x] = e0;
    rowv[3 * TM + threadIdx.x] = e1;
  }
  __syncthreads();
  const int width = kcap + (Epi::kExtra ? 1 : 0);
  for (int idx = threadIdx.x; idx < TM * width; idx += blockDim.x) {
    const int mm = idx / width, j = idx - mm * width;
    const long k = row0 + mm;
    if (k >= nrows) continue;
    const double v = (j < kcap) ? rowv[mm] * Os[(size_t)mm * (kcap + 1) + j] : rowv[TM + mm];
    epi.out[k * epi.ld + j] = (decltype(+epi.out[0]))v;
  }
  if (partials && threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int mm = 0; mm < TM; ++mm) {
      s0 += rowv[2 * TM + mm];
      s1 += rowv[3 * TM + mm];
    }
    partials[2 * (size_t)blockIdx.x] = s0;
    partials[2 * (size_t)blockIdx.x + 1] = s1;
  }
}

}  // namespace ttk
