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
  __device__ __forceinline__ unsigned row_flags(long) const { return 0u; }
  template <typename T>
  __device__ __forceinline__ T loadT(const Col& cc, long k, unsigned) const {
    return (T)A[k * ld + cc.c];
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
  __device__ __forceinline__ unsigned row_flags(long) const { return 0u; }
  template <typename T>
  __device__ __forceinline__ T loadT(const Col& cc, long k, unsigned) const {
    return (T)A[(long)cc.c * ld + k];
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
    int kind;  // 0: Z, 1: upwind image, 2: inflow column, 3: none, 4/5: Rusanov central/diffusion
    int q, ax, w, b;
    double lam;
    float lamf;
    long s;    // row stride of the operator's axis
  };
  __device__ __forceinline__ Col col(int c) const {
    Col cc{3, 0, 0, 0, 0, 0.0, 0.0f, 0};
    const int t = c / rcap;
    if (t == 0) {
      cc.kind = 0;
      cc.q = c;
    } else if (t <= nterm) {
      const int wc = w[t - 1];
      cc.kind = (wc == 2) ? 4 : (wc == -2) ? 5 : 1;
      cc.q = c - t * rcap;
      cc.ax = axis[t - 1];
      cc.w = w[t - 1];
      cc.lam = lam[t - 1];
      cc.lamf = (float)cc.lam;
      cc.s = stride[cc.ax];
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
    if (cc.kind >= 4) {  // Rusanov (vacuum ghost cells)
      const double lo = (idx > 0) ? (double)Z[(k - s) * ldz + cc.q] : 0.0;
      const double hi = (idx < ext[cc.ax] - 1) ? (double)Z[(k + s) * ldz + cc.q] : 0.0;
      if (cc.kind == 4) return -0.5 * cc.lam * (hi - lo);
      return 0.5 * cc.lam * (hi - 2.0 * (double)Z[k * ldz + cc.q] + lo);
    }
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
  // Per-row neighbour flags, computed once per row and shared by all columns: bit 2a is set
  // when row k has a lower neighbour along axis a, bit 2a+1 an upper one; the group index
  // k mod G sits in bits 8 and up.
  __device__ __forceinline__ unsigned row_flags(long k) const {
    unsigned f = 0u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long idx = (k / stride[a]) % ext[a];
      f |= (idx > 0 ? 1u : 0u) << (2 * a);
      f |= (idx < ext[a] - 1 ? 1u : 0u) << (2 * a + 1);
    }
    return f | ((unsigned)(k % G) << 8);
  }
  // The value of load() in arithmetic T, from the row's flags.
  template <typename T>
  __device__ __forceinline__ T loadT(const Col& cc, long k, unsigned fl) const {
    if (cc.kind == 0) return (T)Z[k * ldz + cc.q];
    if (cc.kind == 3) return T(0);
    if (cc.kind >= 4) {  // Rusanov (vacuum ghost cells)
      const T lamT = (sizeof(T) == 8) ? (T)cc.lam : (T)cc.lamf;
      const T lo = ((fl >> (2 * cc.ax)) & 1u) ? (T)Z[(k - cc.s) * ldz + cc.q] : T(0);
      const T hi = ((fl >> (2 * cc.ax + 1)) & 1u) ? (T)Z[(k + cc.s) * ldz + cc.q] : T(0);
      if (cc.kind == 4) return T(-0.5) * lamT * (hi - lo);
      return T(0.5) * lamT * (hi - T(2) * (T)Z[k * ldz + cc.q] + lo);
    }
    if (cc.kind == 1) {
      const T lamT = (sizeof(T) == 8) ? (T)cc.lam : (T)cc.lamf;
      const T zk = (T)Z[k * ldz + cc.q];
      T diff;
      if (cc.w > 0) {
        const T up = ((fl >> (2 * cc.ax)) & 1u) ? (T)Z[(k - cc.s) * ldz + cc.q] : T(0);
        diff = zk - up;
      } else {
        const T dn = ((fl >> (2 * cc.ax + 1)) & 1u) ? (T)Z[(k + cc.s) * ldz + cc.q] : T(0);
        diff = dn - zk;
      }
      return -lamT * diff;
    }
    const bool at_face = (cc.w > 0) ? !((fl >> (2 * cc.ax)) & 1u) : !((fl >> (2 * cc.ax + 1)) & 1u);
    return at_face ? (T)bcval[cc.b * G + (int)(fl >> 8)] : T(0);
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

__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Quotient on the reflector chain: FP32 takes the fast reciprocal-based divide (2 ulp; both
// divisors are at least sqrt(x2) >= 3.7e-23 and below the FP32 overflow range), FP64 the
// IEEE one.
template <typename T>
__device__ __forceinline__ T chain_div(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float chain_div<float>(float a, float b) { return __fdividef(a, b); }

// Live test of reflector j without a division per step: (block, offset) of j advanced with j.
struct LiveWalk {
  int t, o;
  __device__ __forceinline__ LiveWalk(const LivePattern& lp, int j) : t(j / lp.rcap), o(j - (j / lp.rcap) * lp.rcap) {}
  __device__ __forceinline__ bool next(const LivePattern& lp, int r) {
    const bool live = (t < lp.nblk) ? (o < r) : true;
    if (++o == lp.rcap) {
      o = 0;
      ++t;
    }
    return live;
  }
};

template <typename T, int BR>
__device__ __forceinline__ void hh_absorb(T* Rs, int ncap, T (&B)[BR], T* vbuf, T* taub, int& buf,
                                          int jbeg, const LivePattern& lp, int r, bool mycol) {
  const int c = threadIdx.x;
  LiveWalk walk(lp, jbeg);
  for (int j = jbeg; j < ncap; ++j) {
    if (!walk.next(lp, r)) continue;
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
        const T sc = chain_div<T>(T(1), alpha - beta);
#pragma unroll
        for (int i = 0; i < BR; ++i) vb[i] = B[i] * sc;
        tau = chain_div<T>(beta - alpha, beta);
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

// packed R, then the double-buffered reflector (16-byte aligned), its two scalars and the row
// flags of the current block
__host__ __device__ inline size_t tsqr_r_elems(int ncap) { return (((size_t)ncap * (ncap + 1) / 2) + 3) & ~(size_t)3; }
template <typename T, int BR>
__host__ __device__ inline size_t tsqr_smem_bytes(int ncap) {
  return sizeof(T) * (tsqr_r_elems(ncap) + 2 * BR + 4) + sizeof(unsigned) * BR;
}

template <typename T, int BR, class Src, int MAXT = 256, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) k_tsqr_leaf(Src src, LivePattern lp, long nrows, long rpc,
                                                          double* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char tsqr_smem[];
  const int ncap = lp.ncap();
  T* Rs = reinterpret_cast<T*>(tsqr_smem);
  T* vbuf = Rs + tsqr_r_elems(ncap);
  T* taub = vbuf + 2 * BR;
  unsigned* flags = reinterpret_cast<unsigned*>(taub + 4);
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  for (int i = threadIdx.x; i < ncap * (ncap + 1) / 2; i += blockDim.x) Rs[i] = T(0);
  const int c = threadIdx.x;
  const bool mycol = (c < ncap) && lp.live(c, r);
  const auto cc = src.col(c < ncap ? c : 0);
  const long beg = (long)blockIdx.x * rpc;
  const long end = (beg + rpc < nrows) ? beg + rpc : nrows;
  int buf = 0;
  for (long r0 = beg; r0 < end; r0 += BR) {
    // neighbour flags once per row of the block, shared by all columns; values in arithmetic T
    __syncthreads();  // the previous block's loads of `flags` are done
    for (int i = threadIdx.x; i < BR; i += blockDim.x) flags[i] = (r0 + i < end) ? src.row_flags(r0 + i) : 0u;
    __syncthreads();
    T B[BR];
#pragma unroll
    for (int i = 0; i < BR; ++i) B[i] = (mycol && r0 + i < end) ? src.template loadT<T>(cc, r0 + i, flags[i]) : T(0);
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

// Merge tree over the leaves' R factors (defined with the row-split kernels in tsqr_rs.cuh).
template <typename T>
tt_status merge_tree(cudaStream_t s, LivePattern lp, int nleaves, double* ws_a, double* ws_b, double** Rfinal);

// Host driver: leaves then merge levels; returns the device pointer of the final R
// (ncap x ncap, row-major, upper triangular) inside ws_a or ws_b.
// Leaf kernels are instantiated with launch bounds (MAXT threads, MINB resident CTAs; FP32 by
// default at most 128 registers, so that three 160-thread CTAs share an SM); the leaf count is
// capped by the CTAs that are resident at once.
template <typename T, int BR, int MAXT = 256, int MINB = (sizeof(T) == 4 ? 2 : 1), class Src>
tt_status run_tsqr(cudaStream_t s, int num_sms, const Src& src, LivePattern lp, long nrows, int max_leaves,
                   double* ws_a, double* ws_b, double** Rfinal, int leaf_cat = kTsqrLeaf) {
  const int ncap = lp.ncap();
  const size_t smem = tsqr_smem_bytes<T, BR>(ncap);
  if (smem > 227 * 1024) return TT_ERR_UNSUPPORTED;
  const int threads = ((ncap + 31) / 32) * 32;
  if (threads > MAXT || threads > 256) return TT_ERR_UNSUPPORTED;
  static_assert(BR > 0, "block rows");
  auto leaf = k_tsqr_leaf<T, BR, Src, MAXT, MINB>;
  cudaFuncSetAttribute(leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, leaf, threads, smem) != cudaSuccess) return TT_ERR_CUDA;
  long L = (nrows + BR - 1) / BR;
  long cap = (long)num_sms * (per_sm > 0 ? per_sm : 1);
  if (max_leaves > 0 && cap > max_leaves) cap = max_leaves;
  if (L > cap) L = cap;
  if (L < 1) L = 1;
  long rpc = (nrows + L - 1) / L;
  rpc = ((rpc + BR - 1) / BR) * BR;
  L = (nrows + rpc - 1) / rpc;
  if (L < 1) L = 1;
  {
    TimerScope scope(leaf_cat, s);
    leaf<<<(unsigned)L, threads, smem, s>>>(src, lp, nrows, rpc, ws_a); count_launch();
  }
  return merge_tree<T>(s, lp, (int)L, ws_a, ws_b, Rfinal);
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
// j < kcap, plus an optional extra column out[k][kcap].  Persistent CTAs: W is staged in
// shared memory once per CTA, which then walks row tiles of TM rows.  A tile of A is formed
// from the source (e.g. the stencil sum, with per-row neighbour flags) into shared memory;
// each thread accumulates a TM/32-row x 4-column block of the output over all columns of A.
// The per-row epilogue (the dot with vJ, scale, extra column, two energy partials) runs one
// warp per row; per-CTA energy partials go to partials[2*cta + {0,1}] in a fixed order.

template <typename SO>
struct EpiPlain {
  SO* out;
  long ld;
  static constexpr bool kExtra = false;
  static constexpr bool kDot = false;
  const double* vj() const { return nullptr; }
  __device__ __forceinline__ void prep(long, double, double& scale, double& extra, double& e0, double& e1) const {
    scale = 1.0;
    extra = 0.0;
    e0 = 0.0;
    e1 = 0.0;
  }
};

// Backward-Euler source update of Eq. (discRTsource) at fixed T on a freshly rounded row with
// J* = Z_new[k,:] . vJ: J^{m+1} = (J* + a eps)/(1 + a), row scale 1/(1 + a + s) and the
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
  static constexpr bool kDot = true;
  __device__ __forceinline__ void prep(long k, double js, double& scale, double& extra, double& e0,
                                       double& e1) const {
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
  double* jout;  // optional: J of every final row (the coupled temperature update reads it)
  static constexpr bool kExtra = false;
  static constexpr bool kDot = true;
  __device__ __forceinline__ void prep(long k, double js, double& scale, double& extra, double& e0,
                                       double& e1) const {
    if (jout) jout[k] = js;
    scale = 1.0;
    extra = 0.0;
    e0 = js;
    e1 = 0.0;
  }
};

template <class Epi>
__device__ __forceinline__ const double* epi_vj(const Epi& e) {
  if constexpr (Epi::kDot) return e.vJ;
  else return nullptr;
}

// Output columns of the update GEMM: kcap rounded up to a multiple of 4.
template <class Epi>
__host__ __device__ inline int update_kpad(int kcap) { return (kcap + 3) & ~3; }
template <typename T, int TM, class Src, class Epi>
__host__ __device__ inline size_t update_smem_bytes(int ncap, int kcap) {
  const int kpad = update_kpad<Epi>(kcap);
  size_t b = sizeof(T) * ((size_t)ncap * kpad + (size_t)TM * (ncap + 1) + (size_t)TM * kpad);
  b = (b + 15) & ~(size_t)15;
  b += sizeof(typename Src::Col) * (size_t)ncap;
  b = (b + 15) & ~(size_t)15;
  return b + sizeof(double) * (3 * TM + 2 * 256) + sizeof(T) * (size_t)kpad + sizeof(unsigned) * TM + (size_t)ncap;
}

template <typename T, int TM, class Src, class Epi>
__global__ void __launch_bounds__(256) k_update(Src src, LivePattern lp, long nrows, const double* __restrict__ W,
                                                int kcap, Epi epi, double* __restrict__ partials) {
  static_assert(TM % 32 == 0, "rows per tile: a multiple of 32");
  constexpr int RPT = TM / 32;  // output rows per thread
  using Col = typename Src::Col;
  extern __shared__ __align__(16) unsigned char upd_smem[];
  const int ncap = lp.ncap();
  const int kpad = update_kpad<Epi>(kcap);
  const int lda = ncap + 1;
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  T* Ws = reinterpret_cast<T*>(upd_smem);    // [ncap][kpad]: W, then W vJ
  T* As = Ws + (size_t)ncap * kpad;          // [TM][ncap + 1]
  T* Os = As + (size_t)TM * lda;             // [TM][kpad]
  size_t off = sizeof(T) * ((size_t)ncap * kpad + (size_t)TM * lda + (size_t)TM * kpad);
  off = (off + 15) & ~(size_t)15;
  Col* cols = reinterpret_cast<Col*>(upd_smem + off);
  off += sizeof(Col) * (size_t)ncap;
  off = (off + 15) & ~(size_t)15;
  double* rowv = reinterpret_cast<double*>(upd_smem + off);  // [3][TM]: J*, scale, extra
  double* red = rowv + 3 * TM;                                // [blockDim][2] energy partials
  T* vJs = reinterpret_cast<T*>(red + 2 * 256);               // [kpad] vJ in arithmetic T
  unsigned* fl = reinterpret_cast<unsigned*>(vJs + kpad);
  unsigned char* livec = reinterpret_cast<unsigned char*>(fl + TM);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = (int)(blockDim.x >> 5);
  const double* vJ = epi_vj(epi);
  for (int c = tid; c < ncap; c += blockDim.x) {
    cols[c] = src.col(c);
    livec[c] = lp.live(c, r) ? 1 : 0;
  }
  for (int i = tid; i < ncap * kpad; i += blockDim.x) {
    const int c = i / kpad, j = i - (i / kpad) * kpad;
    Ws[i] = (j < kcap) ? (T)W[(size_t)c * kcap + j] : T(0);
  }
  for (int j = tid; j < kpad; j += blockDim.x) vJs[j] = (vJ && j < kcap) ? (T)vJ[j] : T(0);
  const long ntiles = (nrows + TM - 1) / TM;
  double e0t = 0.0, e1t = 0.0;  // this thread's energy partials (rows it prepared)
  const int jg = tid & 7, mp = tid >> 3;  // 4 columns at 4*jg (+32 per column block), rows mp*RPT..
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long row0 = tile * TM;
    __syncthreads();  // previous tile's buffers are free (and the staging above is done)
    for (int m = tid; m < TM; m += blockDim.x) fl[m] = (row0 + m < nrows) ? src.row_flags(row0 + m) : 0u;
    __syncthreads();
    // tile of A: one warp per row, lanes over columns (coalesced row reads)
#pragma unroll
    for (int q = 0; q < TM / 8; ++q) {
      const int m = warp + 8 * q;
      if (m < TM) {
        const long k = row0 + m;
        const unsigned f = fl[m];
        for (int c = lane; c < ncap; c += 32)
          As[(size_t)m * lda + c] = (k < nrows && livec[c]) ? src.template loadT<T>(cols[c], k, f) : T(0);
      }
    }
    __syncthreads();
    for (int jb = 0; jb < kpad; jb += 32) {
      const int j0 = jb + 4 * jg;
      if (j0 < kpad) {
        T acc[RPT][4];
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[q][u] = T(0);
        const T* arow = As + (size_t)(mp * RPT) * lda;
#pragma unroll 4
        for (int c = 0; c < ncap; ++c) {
          T w[4];
          ld4(Ws + (size_t)c * kpad + j0, w);
#pragma unroll
          for (int q = 0; q < RPT; ++q) {
            const T a = arow[(size_t)q * lda + c];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[q][u] += a * w[u];
          }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) Os[(size_t)(mp * RPT + q) * kpad + j0 + u] = acc[q][u];
      }
    }
    __syncthreads();
    // epilogue: (a) one warp per row for J* = o . vJ in arithmetic T, (b) one thread per row
    // for the row scalars (FP64), (c) coalesced writes of the output rows
    if (vJ) {
      for (int mm = warp; mm < TM; mm += nwarps) {
        const T* o = Os + (size_t)mm * kpad;
        T js = T(0);
        for (int j = lane; j < kcap; j += 32) js += o[j] * vJs[j];
        js = warp_sum(js);
        if (lane == 0) rowv[2 * TM + mm] = (double)js;
      }
      __syncthreads();
    }
    for (int m = tid; m < TM; m += blockDim.x) {
      const long k = row0 + m;
      double sc = 0.0, ex = 0.0, e0 = 0.0, e1 = 0.0;
      if (k < nrows) epi.prep(k, vJ ? rowv[2 * TM + m] : 0.0, sc, ex, e0, e1);
      rowv[m] = sc;
      rowv[TM + m] = ex;
      e0t += e0;
      e1t += e1;
    }
    __syncthreads();
    const int width = kcap + (Epi::kExtra ? 1 : 0);
    for (int mm = warp; mm < TM; mm += nwarps) {
      const long k = row0 + mm;
      if (k >= nrows) break;
      const T* o = Os + (size_t)mm * kpad;
      const T sc = (T)rowv[mm];
      const double ex = rowv[TM + mm];
      for (int j = lane; j < width; j += 32) {
        if (j < kcap) epi.out[k * epi.ld + j] = (decltype(+epi.out[0]))(sc * o[j]);
        else epi.out[k * epi.ld + j] = (decltype(+epi.out[0]))ex;
      }
    }
  }
  if (partials) {
    // fixed-order reduction of the per-thread partials
    __syncthreads();
    red[2 * tid] = e0t;
    red[2 * tid + 1] = e1t;
    __syncthreads();
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int t = 0; t < (int)blockDim.x; ++t) {
        s0 += red[2 * t];
        s1 += red[2 * t + 1];
      }
      partials[2 * (size_t)blockIdx.x] = s0;
      partials[2 * (size_t)blockIdx.x + 1] = s1;
    }
  }
}

// Persistent grid of the update pass (also the number of energy partials it writes).
template <typename T, int TM, class Src, class Epi>
inline long update_grid(int num_sms, int ncap, int kcap, long nrows) {
  const size_t smem = update_smem_bytes<T, TM, Src, Epi>(ncap, kcap);
  cudaFuncSetAttribute(k_update<T, TM, Src, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_update<T, TM, Src, Epi>, 256, smem) != cudaSuccess ||
      occ < 1)
    occ = 1;
  const long ntiles = (nrows + TM - 1) / TM;
  long g = (long)num_sms * occ;
  return g < ntiles ? g : (ntiles > 0 ? ntiles : 1);
}

}  // namespace ttk

// the row-split kernels and the merge tree
#include "tsqr_rs.cuh"
