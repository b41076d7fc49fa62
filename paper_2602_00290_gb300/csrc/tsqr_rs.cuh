// Row-split Householder TSQR: the same reflector sequence as the column-owner leaf and merge
// of bigpass.cuh (one reflector per live column, R kept packed in shared memory), with QS
// consecutive lanes sharing a column.  Lane q of a column group holds rows q*RPT .. q*RPT+RPT-1
// of the current block of BR rows in registers; norms and reflector dots are partial sums over
// those rows, combined by an xor butterfly inside the group (every lane ends with the same
// bits).  Against one thread per column this cuts the dependent chain of each reflector by QS
// and keeps QS times as many warps busy to the right of the pivot.
#pragma once
#include "bigpass.cuh"

namespace ttk {

template <typename T, int BR, int QS>
struct RsGeom {
  static_assert(BR % (4 * QS) == 0, "rows per lane must be a multiple of 4");
  static_assert(QS == 2 || QS == 4 || QS == 8, "group size");
  static constexpr int RPT = BR / QS;  // rows a lane holds
  static constexpr int SS = RPT + 4;   // reflector segment stride: the QS segments start on distinct banks
};

// packed R, the double-buffered reflector (QS segments each), two scalars, BR row flags
template <typename T, int BR, int QS>
__host__ __device__ inline size_t tsqr_rs_smem_bytes(int ncap) {
  return sizeof(T) * (tsqr_r_elems(ncap) + 2 * QS * RsGeom<T, BR, QS>::SS + 4) + sizeof(unsigned) * BR;
}
template <int QS>
__host__ __device__ inline int tsqr_rs_threads(int ncap) {
  return ((ncap * QS + 31) / 32) * 32;
}

template <typename T>
__device__ __forceinline__ void st4(T* p, T a, T b, T c, T d);
template <>
__device__ __forceinline__ void st4<float>(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void st4<double>(double* p, double a, double b, double c, double d) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
  *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
}

template <typename T, int QS>
__device__ __forceinline__ T group_sum(T v, unsigned gm) {
#pragma unroll
  for (int o = 1; o < QS; o <<= 1) v += __shfl_xor_sync(gm, v, o);
  return v;
}

// sum_i a[i] b[i] + init with four partial sums; FP32 on the packed two-lane FMA (__ffma2_rn)
template <typename T, int N>
__device__ __forceinline__ T dot4(const T* a, const T* b, T init) {
  static_assert(N % 4 == 0, "multiple of 4");
  if constexpr (sizeof(T) == 4) {
    float2 p0 = make_float2(init, 0.f), p1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < N; i += 4) {
      p0 = __ffma2_rn(make_float2(a[i], a[i + 1]), make_float2(b[i], b[i + 1]), p0);
      p1 = __ffma2_rn(make_float2(a[i + 2], a[i + 3]), make_float2(b[i + 2], b[i + 3]), p1);
    }
    return (p0.x + p0.y) + (p1.x + p1.y);
  } else {
    T p[4] = {init, T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < N; ++i) p[i & 3] += a[i] * b[i];
    return (p[0] + p[1]) + (p[2] + p[3]);
  }
}

// B[i] -= w v[i]; FP32 on the packed two-lane FMA
template <typename T, int N>
__device__ __forceinline__ void axpy_neg(T w, const T* v, T* B) {
  if constexpr (sizeof(T) == 4) {
    const float2 nw = make_float2(-w, -w);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const float2 u = __ffma2_rn(nw, make_float2(v[i], v[i + 1]), make_float2(B[i], B[i + 1]));
      B[i] = u.x;
      B[i + 1] = u.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) B[i] -= w * v[i];
  }
}

// Absorb a block held as B (rows of this lane's segment, column c) into the packed R.
// Reflectors jbeg..ncap-1; column j's reflector is formed by its group, lane 0 of the group
// owning R[.][c]; one barrier per reflector.
// VREG: the lane's reflector segment is held in registers between the dot and the update
// (else it is read from shared memory twice, which keeps long segments within 64 registers).
// FP64 form (see hh_absorb_f64 in bigpass.cuh): the pivot's warp gathers the pivot column's
// rows by shuffles (BR/32 per lane) and sums their squares with a butterfly, and the reflector is
// stored unscaled, u = [alpha - beta; B], with sc = 1/(alpha - beta) applied by the other columns.
template <int BR, int QS, bool VREG>
__device__ __forceinline__ void hh_absorb_rs_f64(double* Rs, int ncap, double (&B)[BR / QS], double* vbuf,
                                                 double* taub, int& buf, int jbeg, const LivePattern& lp, int r,
                                                 bool mycol, int c, int q, unsigned gm) {
  constexpr int RPT = RsGeom<double, BR, QS>::RPT, SS = RsGeom<double, BR, QS>::SS;
  constexpr int GPW = 32 / QS;  // column groups per warp
  static_assert(BR % 32 == 0, "rows in whole warps");
  const int lane = threadIdx.x & 31;
  LiveWalk walk(lp, jbeg);
  for (int j = jbeg; j < ncap; ++j) {
    if (!walk.next(lp, r)) continue;
    double* vb = vbuf + buf * (QS * SS);
    if ((int)(threadIdx.x >> 5) == (j * QS) >> 5) {
      const int src0 = (j * QS) & 31;
      double mine[BR / 32];
#pragma unroll
      for (int k = 0; k < BR / 32; ++k) mine[k] = 0.0;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const double t = __shfl_sync(0xffffffffu, B[i], src0 + (lane % QS));
        if (lane / QS == i % GPW) mine[i / GPW] = t;
      }
      double part = 0.0;
#pragma unroll
      for (int k = 0; k < BR / 32; ++k) part = fma(mine[k], mine[k], part);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (c == j) {
        const double x2 = part;
        if (x2 > 0.0) {
          double* seg = vb + q * SS;
#pragma unroll
          for (int i = 0; i < RPT; i += 4) st4<double>(seg + i, B[i], B[i + 1], B[i + 2], B[i + 3]);
#pragma unroll
          for (int i = 0; i < RPT; ++i) B[i] = 0.0;
        }
        if (q == 0) {
          double tau = 0.0, sc = 0.0;
          if (x2 > 0.0) {
            double* rjj = Rs + tri_off(j, ncap);
            const double alpha = *rjj;
            const double nrm = sqrt(alpha * alpha + x2);
            const double beta = (alpha >= 0.0) ? -nrm : nrm;
            sc = 1.0 / (alpha - beta);
            tau = (beta - alpha) / beta;
            *rjj = beta;
          }
          taub[buf] = tau;
          taub[2 + buf] = sc;
        }
      }
    }
    __syncthreads();
    const double tau = taub[buf];
    if (tau != 0.0 && c > j && mycol) {
      const double sc = taub[2 + buf];
      const double* seg = vb + q * SS;
      double* rjc = Rs + tri_off(j, ncap) + (c - j);
      double v[VREG ? RPT : 4];
      double d;
      if constexpr (VREG) {
#pragma unroll
        for (int i = 0; i < RPT; i += 4) ld4(seg + i, *reinterpret_cast<double(*)[4]>(v + i));
        d = dot4<double, RPT>(v, B, 0.0);
      } else {
        double wp[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < RPT; i += 4) {
          ld4(seg + i, *reinterpret_cast<double(*)[4]>(v));
          wp[0] += v[0] * B[i];
          wp[1] += v[1] * B[i + 1];
          wp[2] += v[2] * B[i + 2];
          wp[3] += v[3] * B[i + 3];
        }
        d = (wp[0] + wp[1]) + (wp[2] + wp[3]);
      }
      d = group_sum<double, QS>(d, gm);
      const double w = tau * fma(sc, d, *rjc);
      if (q == 0) *rjc -= w;
      const double ws = w * sc;
      if constexpr (VREG) {
        axpy_neg<double, RPT>(ws, v, B);
      } else {
#pragma unroll
        for (int i = 0; i < RPT; i += 4) {
          ld4(seg + i, *reinterpret_cast<double(*)[4]>(v));
          B[i] -= ws * v[0];
          B[i + 1] -= ws * v[1];
          B[i + 2] -= ws * v[2];
          B[i + 3] -= ws * v[3];
        }
      }
    }
    buf ^= 1;
  }
}

// TRI (merges): the block holds rows jbeg.. of an upper-triangular factor, so column c has no
// entries below block row c - jbeg, every reflector j keeps that shape, and its vector vanishes
// below block row j - jbeg; lanes whose whole segment lies below it skip the dot and the update
// (they still take part in the group's butterfly).
template <typename T, int BR, int QS, bool VREG = true, bool TRI = false>
__device__ __forceinline__ void hh_absorb_rs(T* Rs, int ncap, T (&B)[BR / QS], T* vbuf, T* taub, int& buf,
                                             int jbeg, const LivePattern& lp, int r, bool mycol, int c, int q,
                                             unsigned gm) {
  if constexpr (sizeof(T) == 8 && BR % 32 == 0) {
    hh_absorb_rs_f64<BR, QS, VREG>(Rs, ncap, B, vbuf, taub, buf, jbeg, lp, r, mycol, c, q, gm);
    return;
  }
  constexpr int RPT = RsGeom<T, BR, QS>::RPT, SS = RsGeom<T, BR, QS>::SS;
  LiveWalk walk(lp, jbeg);
  for (int j = jbeg; j < ncap; ++j) {
    if (!walk.next(lp, r)) continue;
    T* vb = vbuf + buf * (QS * SS);
    if (c == j) {
      // the reflector goes out unscaled, u = [alpha - beta; B], with sc = 1/(alpha - beta) for
      // the other columns, and the pivot's rows are not cleared (no later step of this block
      // reads them): the pivot group's part of the step is the critical path
      const T x2 = group_sum<T, QS>(dot4<T, RPT>(B, B, T(0)), gm);
      if (x2 > T(0)) {
        T* seg = vb + q * SS;
#pragma unroll
        for (int i = 0; i < RPT; i += 4) st4<T>(seg + i, B[i], B[i + 1], B[i + 2], B[i + 3]);
      }
      if (q == 0) {
        T tau = T(0), sc = T(0);
        if (x2 > T(0)) {
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
    }
    __syncthreads();
    const T tau = taub[buf];
    // this lane's rows meet the reflector (always, unless TRI)
    const bool meets = !TRI || q * RPT <= j - jbeg;
    if (tau != T(0) && c > j && mycol && VREG) {
      T v[RPT];
      const T* seg = vb + q * SS;
      T* rjc = Rs + tri_off(j, ncap) + (c - j);
      const T sc = taub[2 + buf];
      T part = T(0);
      if (meets) {
#pragma unroll
        for (int i = 0; i < RPT; i += 4) {
          T t4[4];
          ld4(seg + i, t4);
          v[i] = t4[0];
          v[i + 1] = t4[1];
          v[i + 2] = t4[2];
          v[i + 3] = t4[3];
        }
        part = dot4<T, RPT>(v, B, part);
      }
      const T wv = (*rjc + sc * group_sum<T, QS>(part, gm)) * tau;
      if (q == 0) *rjc -= wv;
      if (meets) axpy_neg<T, RPT>(wv * sc, v, B);
    } else if (tau != T(0) && c > j && mycol) {
      const T* seg = vb + q * SS;
      T* rjc = Rs + tri_off(j, ncap) + (c - j);
      const T sc = taub[2 + buf];
      T wp[4] = {T(0), T(0), T(0), T(0)};
      if (meets) {
#pragma unroll
        for (int i = 0; i < RPT; i += 4) {
          T t4[4];
          ld4(seg + i, t4);
          wp[0] += t4[0] * B[i];
          wp[1] += t4[1] * B[i + 1];
          wp[2] += t4[2] * B[i + 2];
          wp[3] += t4[3] * B[i + 3];
        }
      }
      const T wv = (*rjc + sc * group_sum<T, QS>((wp[0] + wp[1]) + (wp[2] + wp[3]), gm)) * tau;
      if (q == 0) *rjc -= wv;
      const T ws = wv * sc;
      if (meets) {
#pragma unroll
        for (int i = 0; i < RPT; i += 4) {
          T t4[4];
          ld4(seg + i, t4);
          B[i] -= ws * t4[0];
          B[i + 1] -= ws * t4[1];
          B[i + 2] -= ws * t4[2];
          B[i + 3] -= ws * t4[3];
        }
      }
    }
    buf ^= 1;
  }
}

template <typename T, int BR, int QS, class Src>
__global__ void __launch_bounds__(1024) k_tsqr_leaf_rs(Src src, LivePattern lp, long nrows, long rpc,
                                                       double* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char tsqr_smem[];
  constexpr int RPT = RsGeom<T, BR, QS>::RPT, SS = RsGeom<T, BR, QS>::SS;
  const int ncap = lp.ncap();
  T* Rs = reinterpret_cast<T*>(tsqr_smem);
  T* vbuf = Rs + tsqr_r_elems(ncap);
  T* taub = vbuf + 2 * QS * SS;
  unsigned* flags = reinterpret_cast<unsigned*>(taub + 4);
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  for (int i = threadIdx.x; i < ncap * (ncap + 1) / 2; i += blockDim.x) Rs[i] = T(0);
  const int c = threadIdx.x / QS, q = threadIdx.x % QS;
  const unsigned gm = ((1u << QS) - 1u) << ((threadIdx.x & 31) & ~(QS - 1));
  const bool mycol = (c < ncap) && lp.live(c, r);
  const auto cc = src.col(c < ncap ? c : 0);
  const long beg = (long)blockIdx.x * rpc;
  const long end = (beg + rpc < nrows) ? beg + rpc : nrows;
  int buf = 0;
  for (long r0 = beg; r0 < end; r0 += BR) {
    __syncthreads();  // the previous block's loads of `flags` are done
    for (int i = threadIdx.x; i < BR; i += blockDim.x) flags[i] = (r0 + i < end) ? src.row_flags(r0 + i) : 0u;
    __syncthreads();
    T B[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int ii = q * RPT + i;
      B[i] = (mycol && r0 + ii < end) ? src.template loadT<T>(cc, r0 + ii, flags[ii]) : T(0);
    }
    hh_absorb_rs<T, BR, QS>(Rs, ncap, B, vbuf, taub, buf, 0, lp, r, mycol, c, q, gm);
  }
  __syncthreads();
  write_R<T, BR>(Rs, ncap, Rout + (size_t)blockIdx.x * ncap * ncap);
}

// One level of the binary merge tree, row-split: output m = QR([R_{2m}; R_{2m+1}]).R
template <typename T, int BR, int QS, bool VREG = true>
__global__ void __launch_bounds__(BR == 160 ? 640 : 1024) k_tsqr_merge_rs(LivePattern lp, int nin,
                                                                         const double* __restrict__ Rin,
                                                        double* __restrict__ Rout) {
  extern __shared__ __align__(16) unsigned char tsqr_smem[];
  constexpr int RPT = RsGeom<T, BR, QS>::RPT, SS = RsGeom<T, BR, QS>::SS;
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
  T* taub = vbuf + 2 * QS * SS;
  const int r = lp.r_ptr ? *lp.r_ptr : lp.rcap;
  const int c = threadIdx.x / QS, q = threadIdx.x % QS;
  // the first factor's column c, rows q, q + QS, ... up to the diagonal, into packed R with eight
  // loads in flight per lane (a loop of one load per element waits out the memory latency each time)
  if (c < ncap) {
    for (int i0 = q; i0 <= c; i0 += 8 * QS) {
      T t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int row = i0 + u * QS;
        t[u] = (row <= c) ? (T)Ra[(size_t)row * ncap + c] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int row = i0 + u * QS;
        if (row <= c) Rs[tri_off(row, ncap) + (c - row)] = t[u];
      }
    }
  }
  const unsigned gm = ((1u << QS) - 1u) << ((threadIdx.x & 31) & ~(QS - 1));
  const bool mycol = (c < ncap) && lp.live(c, r);
  __syncthreads();
  int buf = 0;
  for (int i0 = 0; i0 < ncap; i0 += BR) {
    T B[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = i0 + q * RPT + i;
      B[i] = (mycol && row < ncap) ? (T)Rb[(size_t)row * ncap + c] : T(0);
    }
    // rows i0.. of an upper-triangular factor vanish in columns < i0
    hh_absorb_rs<T, BR, QS, VREG, true>(Rs, ncap, B, vbuf, taub, buf, i0, lp, r, mycol, c, q, gm);
  }
  __syncthreads();
  // column c of the result, rows q, q + QS, ... (zeros below the diagonal)
  if (c < ncap) {
#pragma unroll 4
    for (int row = q; row < ncap; row += QS)
      Ro[(size_t)row * ncap + c] = (row <= c) ? (double)Rs[tri_off(row, ncap) + (c - row)] : 0.0;
  }
}

// Host driver of the row-split TSQR; same contract as run_tsqr (final R, ncap x ncap row-major
// upper triangular, in ws_a or ws_b).  The leaf count is at most one wave of resident CTAs,
// max_leaves, and the column-owner driver's own bound (so workspace sized by tsqr_max_leaves
// always suffices).
template <typename T, int BR, int QS, class Src>
tt_status run_tsqr_rs(cudaStream_t s, int num_sms, const Src& src, LivePattern lp, long nrows, int max_leaves,
                      double* ws_a, double* ws_b, double** Rfinal, int leaf_cat = kTsqrLeaf) {
  const int ncap = lp.ncap();
  const size_t smem = tsqr_rs_smem_bytes<T, BR, QS>(ncap);
  if (smem > 227 * 1024) return TT_ERR_UNSUPPORTED;
  const int threads = tsqr_rs_threads<QS>(ncap);
  if (threads > 1024) return TT_ERR_UNSUPPORTED;
  auto leaf = k_tsqr_leaf_rs<T, BR, QS, Src>;
  if (const tt_status a = smem_optin(leaf, smem); a != TT_OK) return a;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, leaf, threads, smem) != cudaSuccess) return TT_ERR_CUDA;
  if (per_sm < 1) return TT_ERR_UNSUPPORTED;
  const long colcap = tsqr_max_leaves<T, BR>(num_sms, ncap, nrows, max_leaves);
  const LeafSplit sp = tsqr_split(nrows, BR, num_sms, per_sm, max_leaves, colcap);
  const long L = sp.leaves, rpc = sp.rpc;
  {
    TimerScope scope(leaf_cat, s);
    leaf<<<(unsigned)L, threads, smem, s>>>(src, lp, nrows, rpc, ws_a); count_launch();
  }
  return merge_tree<T>(s, lp, (int)L, ws_a, ws_b, Rfinal);
}

// Rows of the second factor the row-split merge absorbs at a time.  FP64: 64 (a 160-column
// level: 288 reflector steps instead of 480), its lanes reading the reflector from shared memory
// so that the longer row segments stay within 64 registers (measured 15.4 -> 14.4 ms of merges
// per step).  FP32: 64 rows with the reflector in registers up to 64 columns; wider factors are
// up to 160 columns are absorbed 160 rows at a time (one block: 160 reflector steps instead of
// 288 at 160 columns), the reflector read from shared memory, lanes below the reflector idle;
// that kernel is launched with at most 640 threads, which leaves it 96 registers a thread.
template <typename T>
__host__ __device__ inline int merge_rs_rows(int ncap) {
  return (sizeof(T) == 4 && ncap > 64 && ncap <= 160) ? 160 : 64;
}
template <typename T>
__host__ __device__ inline size_t merge_rs_smem_bytes(int ncap) {
  return merge_rs_rows<T>(ncap) == 160 ? tsqr_rs_smem_bytes<T, 160, 4>(ncap) : tsqr_rs_smem_bytes<T, 64, 4>(ncap);
}

// Merge tree of the TSQR: levels of pairwise QRs of stacked R factors, the last one in ws_a or
// ws_b.  Every leaf kernel merges with the row-split merge (measured faster than the
// column-owner merge for every pass shape tried) where 4 ncap <= 1024 lanes, else with the
// column-owner merge.
template <typename T>
tt_status merge_tree(cudaStream_t s, LivePattern lp, int nleaves, double* ws_a, double* ws_b, double** Rfinal) {
  constexpr int MBR = sizeof(T) == 4 ? 64 : 32;  // rows of the column-owner merge's blocks
  constexpr bool RVREG = sizeof(T) == 4;
  const int ncap = lp.ncap();
  const int rs_threads = tsqr_rs_threads<4>(ncap);
  const bool rs = rs_threads <= 1024 && merge_rs_smem_bytes<T>(ncap) <= 227 * 1024;
  const bool wide = merge_rs_rows<T>(ncap) == 160;
  auto merge64 = k_tsqr_merge_rs<T, 64, 4, RVREG>;
  // FP32 only (the FP64 merge never takes 160-row blocks)
  auto merge160 = k_tsqr_merge_rs<float, 160, 4, false>;
  size_t smem;
  int threads;
  if (rs) {
    smem = merge_rs_smem_bytes<T>(ncap);
    threads = rs_threads;
    const tt_status a = wide ? smem_optin(merge160, smem) : smem_optin(merge64, smem);
    if (a != TT_OK) return a;
  } else {
    smem = tsqr_smem_bytes<T, MBR>(ncap);
    threads = ((ncap + 31) / 32) * 32;
    if (smem > 227 * 1024 || threads > 256) return TT_ERR_UNSUPPORTED;
    if (const tt_status a = smem_optin(k_tsqr_merge<T, MBR>, smem); a != TT_OK) return a;
  }
  TimerScope scope(kTsqrMerge, s);
  double* in = ws_a;
  double* out = ws_b;
  int n = nleaves;
  while (n > 1) {
    const int m = (n + 1) / 2;
    if (rs && wide)
      merge160<<<m, threads, smem, s>>>(lp, n, in, out);
    else if (rs)
      merge64<<<m, threads, smem, s>>>(lp, n, in, out);
    else
      k_tsqr_merge<T, MBR><<<m, threads, smem, s>>>(lp, n, in, out);
    count_launch();
    double* t = in;
    in = out;
    out = t;
    n = m;
  }
  *Rfinal = in;
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

}  // namespace ttk
