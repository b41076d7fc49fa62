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
  int nax;                 // spatial axes d_X (every operator's axis is below it)
  int staged;              // update pass: stage the tile's row blocks in shared memory (host choice)
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
  // Staged form for a tile of TM rows starting at row0: block 0 holds Z rows row0.., block
  // 1 + 2a rows row0 - s_a.., block 2 + 2a rows row0 + s_a.. (TM x ldz each, rows outside
  // [0, nrows) zero).  Bytes of the staging buffer:
  __host__ __device__ size_t stage_bytes(int TM) const { return sizeof(S) * (size_t)TM * ldz * (1 + 2 * nax); }
  // The value of loadT(cc, row0 + m, fl) read from the staged blocks (same arithmetic).
  template <typename T>
  __device__ __forceinline__ T stagedT(const S* raw, int TM, const Col& cc, int m, unsigned fl) const {
    const S* C = raw + (size_t)m * ldz + cc.q;
    if (cc.kind == 0) return (T)*C;
    if (cc.kind == 3) return T(0);
    if (cc.kind == 2) {
      const bool at_face = (cc.w > 0) ? !((fl >> (2 * cc.ax)) & 1u) : !((fl >> (2 * cc.ax + 1)) & 1u);
      return at_face ? (T)bcval[cc.b * G + (int)(fl >> 8)] : T(0);
    }
    const S* L = C + (size_t)(1 + 2 * cc.ax) * TM * ldz;
    const S* H = L + (size_t)TM * ldz;
    const T lamT = (sizeof(T) == 8) ? (T)cc.lam : (T)cc.lamf;
    if (cc.kind >= 4) {
      const T lo = ((fl >> (2 * cc.ax)) & 1u) ? (T)*L : T(0);
      const T hi = ((fl >> (2 * cc.ax + 1)) & 1u) ? (T)*H : T(0);
      if (cc.kind == 4) return T(-0.5) * lamT * (hi - lo);
      return T(0.5) * lamT * (hi - T(2) * (T)*C + lo);
    }
    const T zk = (T)*C;
    T diff;
    if (cc.w > 0) {
      const T up = ((fl >> (2 * cc.ax)) & 1u) ? (T)*L : T(0);
      diff = zk - up;
    } else {
      const T dn = ((fl >> (2 * cc.ax + 1)) & 1u) ? (T)*H : T(0);
      diff = dn - zk;
    }
    return -lamT * diff;
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

// FP32 form of the reflector loop on the packed two-lane FMA of sm_100+ (__ffma2_rn: each lane
// rounds as one fmaf): the column owner's norm, the dot of the reflector with a column and the
// column update each run BR/2 packed FMAs in four partial sums, and the reflector is read from
// shared memory in 16-byte vectors.  The pivot thread's work is the critical path of every
// reflector step (the other columns wait for it at the barrier), so, as in the FP64 form, it
// stores the reflector unscaled, u = [alpha - beta; B], and the other columns apply
// sc = 1/(alpha - beta) (H x = x - tau v (v^T x), v = sc u); its own rows are not cleared (no
// later step of this block reads them: the pivot column takes no further update).  Same
// arithmetic as the generic loop below up to the order of the partial sums and the place of sc.
template <int BR>
__device__ __forceinline__ void hh_absorb_x2(float* Rs, int ncap, float (&B)[BR], float* vbuf, float* taub,
                                             int& buf, int jbeg, const LivePattern& lp, int r, bool mycol) {
  static_assert(BR % 8 == 0, "block rows in pairs of float4 groups");
  const int c = threadIdx.x;
  LiveWalk walk(lp, jbeg);
  for (int j = jbeg; j < ncap; ++j) {
    if (!walk.next(lp, r)) continue;
    float* vb = vbuf + buf * BR;
    if (c == j) {
      float2 xp0 = make_float2(0.f, 0.f), xp1 = xp0, xp2 = xp0, xp3 = xp0;
#pragma unroll
      for (int i = 0; i < BR; i += 8) {
        xp0 = __ffma2_rn(make_float2(B[i], B[i + 1]), make_float2(B[i], B[i + 1]), xp0);
        xp1 = __ffma2_rn(make_float2(B[i + 2], B[i + 3]), make_float2(B[i + 2], B[i + 3]), xp1);
        xp2 = __ffma2_rn(make_float2(B[i + 4], B[i + 5]), make_float2(B[i + 4], B[i + 5]), xp2);
        xp3 = __ffma2_rn(make_float2(B[i + 6], B[i + 7]), make_float2(B[i + 6], B[i + 7]), xp3);
      }
      const float x2 = ((xp0.x + xp0.y) + (xp1.x + xp1.y)) + ((xp2.x + xp2.y) + (xp3.x + xp3.y));
      float tau = 0.f, sc = 0.f;
      if (x2 > 0.f) {
#pragma unroll
        for (int i = 0; i < BR; i += 4)
          *reinterpret_cast<float4*>(vb + i) = make_float4(B[i], B[i + 1], B[i + 2], B[i + 3]);
        float* rjj = Rs + tri_off(j, ncap);
        const float alpha = *rjj;
        const float nrm = sqrtf(alpha * alpha + x2);
        const float beta = (alpha >= 0.f) ? -nrm : nrm;
        sc = chain_div<float>(1.f, alpha - beta);
        tau = chain_div<float>(beta - alpha, beta);
        *rjj = beta;
      }
      taub[buf] = tau;
      taub[2 + buf] = sc;
    }
    __syncthreads();
    const float tau = taub[buf];
    if (tau != 0.f && c > j && mycol) {
      const float sc = taub[2 + buf];
      float* rjc = Rs + tri_off(j, ncap) + (c - j);
      // up to 32 block rows the reflector stays in registers between the dot and the update;
      // wider blocks read it again (their B already fills the register budget)
      constexpr bool kKeep = BR <= 32;
      float2 w0 = make_float2(0.f, 0.f), w1 = w0, w2 = w0, w3 = w0;
      float v[kKeep ? BR : 1];
#pragma unroll
      for (int i = 0; i < BR; i += 8) {
        const float4 t = *reinterpret_cast<const float4*>(vb + i);
        const float4 t2 = *reinterpret_cast<const float4*>(vb + i + 4);
        if constexpr (kKeep) {
          v[i] = t.x; v[i + 1] = t.y; v[i + 2] = t.z; v[i + 3] = t.w;
          v[i + 4] = t2.x; v[i + 5] = t2.y; v[i + 6] = t2.z; v[i + 7] = t2.w;
        }
        w0 = __ffma2_rn(make_float2(t.x, t.y), make_float2(B[i], B[i + 1]), w0);
        w1 = __ffma2_rn(make_float2(t.z, t.w), make_float2(B[i + 2], B[i + 3]), w1);
        w2 = __ffma2_rn(make_float2(t2.x, t2.y), make_float2(B[i + 4], B[i + 5]), w2);
        w3 = __ffma2_rn(make_float2(t2.z, t2.w), make_float2(B[i + 6], B[i + 7]), w3);
      }
      const float d = ((w0.x + w0.y) + (w1.x + w1.y)) + ((w2.x + w2.y) + (w3.x + w3.y));
      const float wv = fmaf(sc, d, *rjc) * tau;
      *rjc -= wv;
      const float ws = wv * sc;
      const float2 nw = make_float2(-ws, -ws);
#pragma unroll
      for (int i = 0; i < BR; i += 4) {
        float4 t;
        if constexpr (kKeep) {
          t = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
          t = *reinterpret_cast<const float4*>(vb + i);
        }
        const float2 u0 = __ffma2_rn(nw, make_float2(t.x, t.y), make_float2(B[i], B[i + 1]));
        const float2 u1 = __ffma2_rn(nw, make_float2(t.z, t.w), make_float2(B[i + 2], B[i + 3]));
        B[i] = u0.x; B[i + 1] = u0.y; B[i + 2] = u1.x; B[i + 3] = u1.y;
      }
    }
    buf ^= 1;
  }
}

// FP64 form.  An FP64 warp instruction occupies the SM sub-partition's FP64 pipe for the same
// time whether one lane or 32 are active, so the pivot thread's serial work (norm, scaling) is
// moved off single-lane instructions: the pivot's warp takes the column's rows by shuffles (lane
// l holds rows l, l + 32, ...) and sums their squares by a butterfly, and the reflector is
// stored unscaled, u = [alpha - beta; B], with sc = 1/(alpha - beta) applied by the other
// columns (H x = x - tau v (v^T x) with v = sc u).  Needs every lane of the pivot's warp present.
template <int BR>
__device__ __forceinline__ void hh_absorb_f64(double* Rs, int ncap, double (&B)[BR], double* vbuf, double* taub,
                                              int& buf, int jbeg, const LivePattern& lp, int r, bool mycol) {
  static_assert(BR % 32 == 0, "rows in whole warps");
  const int c = threadIdx.x, lane = c & 31;
  LiveWalk walk(lp, jbeg);
  for (int j = jbeg; j < ncap; ++j) {
    if (!walk.next(lp, r)) continue;
    double* vb = vbuf + buf * BR;
    if ((c >> 5) == (j >> 5)) {
      const int jl = j & 31;
      double part = 0.0;
#pragma unroll
      for (int h = 0; h < BR / 32; ++h) {
        double mine = 0.0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const double t = __shfl_sync(0xffffffffu, B[32 * h + i], jl);
          if (lane == i) mine = t;
        }
        part = fma(mine, mine, part);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == jl) {
        const double x2 = part;
        double tau = 0.0, sc = 0.0;
        if (x2 > 0.0) {
          double* rjj = Rs + tri_off(j, ncap);
          const double alpha = *rjj;
          const double nrm = sqrt(alpha * alpha + x2);
          const double beta = (alpha >= 0.0) ? -nrm : nrm;
          sc = 1.0 / (alpha - beta);
#pragma unroll
          for (int i = 0; i < BR; i += 2) *reinterpret_cast<double2*>(vb + i) = make_double2(B[i], B[i + 1]);
          tau = (beta - alpha) / beta;
          *rjj = beta;
#pragma unroll
          for (int i = 0; i < BR; ++i) B[i] = 0.0;
        }
        taub[buf] = tau;
        taub[2 + buf] = sc;
      }
    }
    __syncthreads();
    const double tau = taub[buf];
    if (tau != 0.0 && c > j && mycol) {
      const double sc = taub[2 + buf];
      double* rjc = Rs + tri_off(j, ncap) + (c - j);
      double wp[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int i = 0; i < BR; ++i) wp[i & 3] += vb[i] * B[i];
      const double w = tau * fma(sc, (wp[0] + wp[1]) + (wp[2] + wp[3]), *rjc);
      *rjc -= w;
      const double ws = w * sc;
#pragma unroll
      for (int i = 0; i < BR; ++i) B[i] -= ws * vb[i];
    }
    buf ^= 1;
  }
}

template <typename T, int BR>
__device__ __forceinline__ void hh_absorb(T* Rs, int ncap, T (&B)[BR], T* vbuf, T* taub, int& buf,
                                          int jbeg, const LivePattern& lp, int r, bool mycol) {
  if constexpr (sizeof(T) == 8 && BR % 32 == 0) {
    hh_absorb_f64<BR>(Rs, ncap, B, vbuf, taub, buf, jbeg, lp, r, mycol);
    return;
  }
  // the packed form measured faster for 64-row blocks (5.57 against 5.76 ms for the bench's
  // transport-sum leaf) and slower for 32-row blocks (5.51 against 5.39 ms)
  if constexpr (sizeof(T) == 4 && BR % 4 == 0 && BR > 32) {
    hh_absorb_x2<BR>(Rs, ncap, B, vbuf, taub, buf, jbeg, lp, r, mycol);
    return;
  }
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
      // the reflector goes out unscaled, u = [alpha - beta; B], with sc = 1/(alpha - beta) for
      // the other columns, and the pivot's rows are not cleared (as in hh_absorb_x2)
      T tau = T(0), sc = T(0);
      if (x2 > T(0)) {
#pragma unroll
        for (int i = 0; i < BR; ++i) vb[i] = B[i];
        T* rjj = Rs + tri_off(j, ncap);
        const T alpha = *rjj;
        const T nrm = sqrt(alpha * alpha + x2);
        const T beta = (alpha >= T(0)) ? -nrm : nrm;
        sc = chain_div<T>(T(1), alpha - beta);
        tau = chain_div<T>(beta - alpha, beta);
        *rjj = beta;
      }
      taub[buf] = tau;
      taub[2 + buf] = sc;
    }
    __syncthreads();
    const T tau = taub[buf];
    if (tau != T(0) && c > j && mycol) {
      const T sc = taub[2 + buf];
      T* rjc = Rs + tri_off(j, ncap) + (c - j);
      T wp[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int i = 0; i < BR; ++i) wp[i & 3] += vb[i] * B[i];
      const T wv = (*rjc + sc * ((wp[0] + wp[1]) + (wp[2] + wp[3]))) * tau;
      *rjc -= wv;
      const T ws = wv * sc;
#pragma unroll
      for (int i = 0; i < BR; ++i) B[i] -= ws * vb[i];
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

// Leaves of a TSQR leaf launch over nrows rows in blocks of BR rows: at most one wave of
// resident CTAs (num_sms x per_sm), the caller's cap max_leaves (> 0) and cap2 (> 0); every leaf
// takes rpc rows, a whole number of blocks, and the last one the ragged rest.  The workspace of
// the R factors is sized by tsqr_max_leaves<T, 32>, which bounds every launch this returns.
struct LeafSplit {
  long leaves, rpc;
};
inline LeafSplit tsqr_split(long nrows, int BR, int num_sms, int per_sm, int max_leaves, long cap2) {
  long L = (nrows + BR - 1) / BR;
  long cap = (long)num_sms * (per_sm > 0 ? per_sm : 1);
  if (max_leaves > 0 && cap > max_leaves) cap = max_leaves;
  if (cap2 > 0 && cap > cap2) cap = cap2;
  if (L > cap) L = cap;
  if (L < 1) L = 1;
  long rpc = (nrows + L - 1) / L;
  rpc = ((rpc + BR - 1) / BR) * BR;
  if (rpc < BR) rpc = BR;
  L = (nrows + rpc - 1) / rpc;
  if (L < 1) L = 1;
  return {L, rpc};
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
  if (const tt_status a = smem_optin(leaf, smem); a != TT_OK) return a;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, leaf, threads, smem) != cudaSuccess) return TT_ERR_CUDA;
  const LeafSplit sp = tsqr_split(nrows, BR, num_sms, per_sm, max_leaves, 0);
  const long L = sp.leaves, rpc = sp.rpc;
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

// Bytes the update pass stages per tile: the stencil source's row blocks when the host chose
// staging and its rows are 16-byte multiples at a 16-byte aligned base (cp.async granules),
// else nothing.
template <class Src>
__host__ __device__ inline size_t update_stage_bytes(const Src&, int) { return 0; }
template <typename S>
__host__ __device__ inline size_t update_stage_bytes(const SrcStencil<S>& src, int TM) {
  const bool ok = src.staged && ((size_t)src.ldz * sizeof(S)) % 16 == 0 && ((size_t)src.Z % 16) == 0 &&
                  src.nax >= 1;
  return ok ? src.stage_bytes(TM) : 0;
}

template <class Src>
inline void set_staged(Src&, int) {}
template <typename S>
inline void set_staged(SrcStencil<S>& src, int on) { src.staged = on; }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Every epilogue latches TT_ERR_NONFINITE in *status (nullable) when a value it writes is not
// finite: a NaN or Inf anywhere in the inputs of a rounding reaches every row it mixes into, even
// where the factorisation passes over it (a non-finite column norm gives no reflector).
template <typename SO>
struct EpiPlain {
  SO* out;
  long ld;
  int* status;
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
  int* status;
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
  int* status;
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
// Output tile bytes; the staged source rows share that region (they are consumed before the
// GEMM writes it).
template <typename T, int TM>
__host__ __device__ inline size_t update_out_bytes(int kpad, size_t stage) {
  const size_t o = sizeof(T) * (size_t)TM * kpad;
  return ((o > stage ? o : stage) + 15) & ~(size_t)15;
}
// A tile bytes; after the last tile the region holds the 256 threads' energy partial pairs.
template <typename T, int TM>
__host__ __device__ inline size_t update_a_bytes(int ncap) {
  const size_t a = sizeof(T) * (size_t)TM * (ncap + 1), red = sizeof(double) * 2 * 256;
  return a > red ? a : red;
}
template <typename T, int TM, class Src, class Epi>
__host__ __device__ inline size_t update_smem_bytes(int ncap, int kcap, size_t stage = 0) {
  const int kpad = update_kpad<Epi>(kcap);
  size_t b = sizeof(T) * (size_t)ncap * kpad + update_a_bytes<T, TM>(ncap);
  b = (b + 15) & ~(size_t)15;
  b += update_out_bytes<T, TM>(kpad, stage);
  b += sizeof(typename Src::Col) * (size_t)ncap;
  b = (b + 15) & ~(size_t)15;
  return b + sizeof(double) * (3 * TM) + sizeof(T) * (size_t)kpad + sizeof(unsigned) * TM + (size_t)ncap;
}

// Epilogue of one output tile (Os: TM x kpad in arithmetic T): (a) one warp per row for
// J* = o . vJ, (b) one thread per row for the row scalars (FP64), (c) coalesced writes of the
// output rows.  e0t/e1t accumulate this thread's energy partials.
template <typename T, int TM, class Epi>
__device__ __forceinline__ void update_epilogue(const Epi& epi, const T* Os, int kpad, int kcap, const T* vJs,
                                                bool dot, double* rowv, long row0, long nrows, double& e0t,
                                                double& e1t) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = (int)(blockDim.x >> 5);
  if (dot) {
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
    if (k < nrows) epi.prep(k, dot ? rowv[2 * TM + m] : 0.0, sc, ex, e0, e1);
    rowv[m] = sc;
    rowv[TM + m] = ex;
    e0t += e0;
    e1t += e1;
  }
  __syncthreads();
  const int width = kcap + (Epi::kExtra ? 1 : 0);
  bool finite = true;
  for (int mm = warp; mm < TM; mm += nwarps) {
    const long k = row0 + mm;
    if (k >= nrows) break;
    const T* o = Os + (size_t)mm * kpad;
    const T sc = (T)rowv[mm];
    const double ex = rowv[TM + mm];
    for (int j = lane; j < width; j += 32) {
      const auto v = (j < kcap) ? (decltype(+epi.out[0]))(sc * o[j]) : (decltype(+epi.out[0]))ex;
      finite = finite && isfinite(v);
      epi.out[k * epi.ld + j] = v;
    }
  }
  if (!finite) latch(epi.status, TT_ERR_NONFINITE);
}

// Fixed-order reduction of the threads' energy partials into partials[2 cta + {0, 1}] (red:
// 2 blockDim doubles of shared memory that are free by now).
__device__ __forceinline__ void update_partials(double* red, double e0t, double e1t, double* partials) {
  const int tid = threadIdx.x;
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

// Issue the cp.async copies of a tile's stencil row blocks (a no-op for other sources).
template <int TM, class Src, typename T>
__device__ __forceinline__ void stage_rows(const Src&, long, long, T*, int) {}
template <int TM, typename S, typename T>
__device__ __forceinline__ void stage_rows(const SrcStencil<S>& src, long row0, long nrows, T* buf, int tid) {
  S* raw = reinterpret_cast<S*>(buf);
  constexpr int kPer = 16 / (int)sizeof(S);  // elements per granule
  const int gpr = src.ldz / kPer;            // granules per row
  const int per_block = TM * gpr;
  const int total = (1 + 2 * src.nax) * per_block;
  for (int i = tid; i < total; i += (int)blockDim.x) {
    const int b = i / per_block, rem = i - b * per_block;
    const int m = rem / gpr, g = rem - m * gpr;
    long k = row0 + m;
    if (b > 0) {
      const long sa = src.stride[(b - 1) >> 1];
      k += ((b - 1) & 1) ? sa : -sa;
    }
    const bool ok = (k >= 0 && k < nrows);
    S* dst = raw + ((size_t)b * TM + m) * src.ldz + (size_t)g * kPer;
    const S* from = ok ? src.Z + k * src.ldz + (size_t)g * kPer : src.Z;
    cp_async16(dst, from, ok ? 16 : 0);
  }
}
template <typename T, int TM, class Src, typename B>
__device__ __forceinline__ T staged_value(const Src& src, const B* buf, const typename Src::Col& cc, int m, unsigned f) {
  return T(0);
}
template <typename T, int TM, typename S, typename B>
__device__ __forceinline__ T staged_value(const SrcStencil<S>& src, const B* buf, const typename SrcStencil<S>::Col& cc,
                                          int m, unsigned f) {
  return src.template stagedT<T>(reinterpret_cast<const S*>(buf), TM, cc, m, f);
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
  const size_t stage = update_stage_bytes(src, TM);
  T* Ws = reinterpret_cast<T*>(upd_smem);    // [ncap][kpad]: W, then W vJ
  T* As = Ws + (size_t)ncap * kpad;          // [TM][ncap + 1]
  size_t off = sizeof(T) * (size_t)ncap * kpad + update_a_bytes<T, TM>(ncap);
  off = (off + 15) & ~(size_t)15;
  T* Os = reinterpret_cast<T*>(upd_smem + off);  // [TM][kpad], or the staged source rows
  off += update_out_bytes<T, TM>(kpad, stage);
  Col* cols = reinterpret_cast<Col*>(upd_smem + off);
  off += sizeof(Col) * (size_t)ncap;
  off = (off + 15) & ~(size_t)15;
  double* rowv = reinterpret_cast<double*>(upd_smem + off);  // [3][TM]: J*, scale, extra
  // [blockDim][2] energy partials, after the last tile: in the A tile's region
  double* red = reinterpret_cast<double*>(As);
  T* vJs = reinterpret_cast<T*>(rowv + 3 * TM);               // [kpad] vJ in arithmetic T
  unsigned* fl = reinterpret_cast<unsigned*>(vJs + kpad);
  unsigned char* livec = reinterpret_cast<unsigned char*>(fl + TM);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
    if (stage > 0) {
      // every 16-byte granule of the tile's source row blocks in flight at once (cp.async),
      // rows outside [0, nrows) zero-filled; then the stencil columns from shared memory
      stage_rows<TM>(src, row0, nrows, Os, tid);
      cp_async_wait_all();
      __syncthreads();
#pragma unroll
      for (int q = 0; q < TM / 8; ++q) {
        const int m = warp + 8 * q;
        if (m < TM) {
          const long k = row0 + m;
          const unsigned f = fl[m];
          for (int c = lane; c < ncap; c += 32)
            As[(size_t)m * lda + c] = (k < nrows && livec[c]) ? staged_value<T, TM>(src, Os, cols[c], m, f) : T(0);
        }
      }
    } else {
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
        if constexpr (sizeof(T) == 4) {
          // packed two-lane FMAs: each lane rounds as one fmaf, same sums as the generic loop
#pragma unroll 4
          for (int c = 0; c < ncap; ++c) {
            const float4 w = *reinterpret_cast<const float4*>(Ws + (size_t)c * kpad + j0);
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
              const float a = arow[(size_t)q * lda + c];
              const float2 lo = __ffma2_rn(make_float2(a, a), make_float2(w.x, w.y), make_float2(acc[q][0], acc[q][1]));
              const float2 hi = __ffma2_rn(make_float2(a, a), make_float2(w.z, w.w), make_float2(acc[q][2], acc[q][3]));
              acc[q][0] = lo.x; acc[q][1] = lo.y; acc[q][2] = hi.x; acc[q][3] = hi.y;
            }
          }
        } else {
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
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) Os[(size_t)(mp * RPT + q) * kpad + j0 + u] = acc[q][u];
      }
    }
    __syncthreads();
    update_epilogue<T, TM>(epi, Os, kpad, kcap, vJs, vJ != nullptr, rowv, row0, nrows, e0t, e1t);
  }
  if (partials) update_partials(red, e0t, e1t, partials);
}

// Persistent grid of the update pass (also the number of energy partials it writes); 0 when the
// runtime refuses the kernel's shared memory.
template <typename T, int TM, class Src, class Epi>
inline long update_grid(int num_sms, int ncap, int kcap, long nrows, size_t stage = 0) {
  const size_t smem = update_smem_bytes<T, TM, Src, Epi>(ncap, kcap, stage);
  if (smem_optin(k_update<T, TM, Src, Epi>, smem) != TT_OK) return 0;
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
// the update pass over staged row blocks of the stencil sum
#include "update_blk.cuh"
