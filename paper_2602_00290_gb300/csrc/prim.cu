// TT primitives: materialised transport sum, axpy by rank concatenation, inner product.
#include "bigpass.cuh"
#include "small.cuh"
#include "step.cuh"

namespace ttk {
namespace {

// Merged core of the materialised transport sum in compact layout: columns t*r + q
// (t = 0 state, t = 1..nterm operator images) and the nbc inflow columns after them.
template <typename S>
__global__ void k_transport_Z(long N, SrcStencil<S> src, const int* __restrict__ rank_in, S* __restrict__ Zo,
                              int ldo, int nbc, const int* __restrict__ rank_in2, int rcapo2, int* status) {
  const int r = rank_in[1];
  const int R = (src.nterm + 1) * r + nbc;
  bool over = R > ldo;
  if (rank_in2) over = over || ((src.nterm + 1) * (*rank_in2) + nbc > rcapo2);
  if (over) {
    if (blockIdx.x == 0 && threadIdx.x == 0) latch(status, TT_ERR_CAPACITY);
    return;
  }
  src.rcap = r > 0 ? r : 1;
  const long tot = N * (long)ldo;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const long k = idx / ldo;
    const int c = (int)(idx - k * ldo);
    double v = 0.0;
    if (c < R && r > 0) {
      const auto cc = src.col(c);
      v = src.load(cc, k);
    } else if (c < R) {  // r == 0 cannot happen for a valid tensor; inflow columns only
      v = 0.0;
    }
    Zo[idx] = (S)v;
  }
}

// Small cores of the materialised transport sum: block diagonal middle core, stacked last
// core (d = 3), or stacked mu core (d = 2); operator blocks scaled by the angular factors.
template <typename S>
__global__ void k_transport_small(int d, int nterm, int nbc, int n1, int n2, const S* __restrict__ c1,
                                  const S* __restrict__ c2, int rcapi1, int rcapi2, const int* __restrict__ rank_in,
                                  S* __restrict__ o1, S* __restrict__ o2, int rcapo1, int rcapo2,
                                  const double* __restrict__ fac1, const double* __restrict__ fac2,
                                  const int* __restrict__ bc_term) {
  const int r1 = rank_in[1];
  const int r2 = (d == 3) ? rank_in[2] : 1;
  const int R1 = (nterm + 1) * r1 + nbc;
  const int R2 = (nterm + 1) * r2 + nbc;
  if (R1 > rcapo1 || (d == 3 && R2 > rcapo2)) return;
  if (d == 2) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rcapo1 * n1; idx += gridDim.x * blockDim.x) {
      const int a = idx / n1, j = idx - (idx / n1) * n1;
      double v = 0.0;
      if (a < (nterm + 1) * r1) {
        const int t = a / r1, q = a - t * r1;
        v = (double)c1[q * n1 + j] * (t == 0 ? 1.0 : fac1[(t - 1) * n1 + j]);
      } else if (a < R1) {
        v = fac1[bc_term[a - (nterm + 1) * r1] * n1 + j];
      }
      o1[idx] = (S)v;
    }
    return;
  }
  const long tot1 = (long)rcapo1 * n1 * rcapo2;
  const long tot2 = (long)rcapo2 * n2;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot1 + tot2; idx += (long)gridDim.x * blockDim.x) {
    if (idx < tot1) {
      const int a = (int)(idx / ((long)n1 * rcapo2));
      const int rem = (int)(idx - (long)a * n1 * rcapo2);
      const int l = rem / rcapo2, b = rem - (rem / rcapo2) * rcapo2;
      double v = 0.0;
      if (a < (nterm + 1) * r1 && b < (nterm + 1) * r2) {
        const int ta = a / r1, tb = b / r2;
        if (ta == tb) {
          const int qa = a - ta * r1, qb = b - tb * r2;
          v = (double)c1[((size_t)qa * n1 + l) * rcapi2 + qb] * (ta == 0 ? 1.0 : fac1[(ta - 1) * n1 + l]);
        }
      } else if (a >= (nterm + 1) * r1 && a < R1 && b >= (nterm + 1) * r2 && b < R2) {
        const int ba = a - (nterm + 1) * r1, bb = b - (nterm + 1) * r2;
        if (ba == bb) v = fac1[bc_term[ba] * n1 + l];
      }
      o1[idx] = (S)v;
    } else {
      const long i2 = idx - tot1;
      const int b = (int)(i2 / n2), p = (int)(i2 - (long)b * n2);
      double v = 0.0;
      if (b < (nterm + 1) * r2) {
        const int tb = b / r2, qb = b - tb * r2;
        v = (double)c2[(size_t)qb * n2 + p] * (tb == 0 ? 1.0 : fac2[(tb - 1) * n2 + p]);
      } else if (b < R2) {
        v = fac2[bc_term[b - (nterm + 1) * r2] * n2 + p];
      }
      o2[i2] = (S)v;
    }
  }
  (void)rcapi1;
}

__global__ void k_transport_ranks(int d, int nterm, int nbc, const int* __restrict__ rank_in, int* __restrict__ rank_out,
                                  int rcapo1, int rcapo2) {
  if (threadIdx.x || blockIdx.x) return;
  const int R1 = (nterm + 1) * rank_in[1] + nbc;
  const int R2 = (d == 3) ? (nterm + 1) * rank_in[2] + nbc : 1;
  if (R1 > rcapo1 || (d == 3 && R2 > rcapo2)) return;
  rank_out[0] = 1;
  rank_out[1] = R1;
  if (d == 3) {
    rank_out[2] = R2;
    rank_out[3] = 1;
  } else {
    rank_out[2] = 1;
  }
}

// y <- alpha x + y: x's blocks appended after y's live ranks (TT addition, Sec. 3.1).
template <typename S>
__global__ void k_axpy_Z(long N, double alpha, const S* __restrict__ Zx, int ldx, const int* __restrict__ rx,
                         S* __restrict__ Zy, int ldy, const int* __restrict__ ry, int d, int rcapy2, int* status) {
  const int rx1 = rx[1], ry1 = ry[1];
  const bool over = (rx1 + ry1 > ldy) || (d == 3 && rx[2] + ry[2] > rcapy2);
  if (over) {
    if (blockIdx.x == 0 && threadIdx.x == 0) latch(status, TT_ERR_CAPACITY);
    return;
  }
  const long tot = N * (long)rx1;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const long k = idx / rx1;
    const int q = (int)(idx - k * rx1);
    Zy[k * ldy + ry1 + q] = (S)(alpha * (double)Zx[k * ldx + q]);
  }
}

template <typename S>
__global__ void k_axpy_small(int d, int n1, int n2, const S* __restrict__ x1, const S* __restrict__ x2, int rcapx1,
                             int rcapx2, const int* __restrict__ rx, S* __restrict__ y1, S* __restrict__ y2, int rcapy1,
                             int rcapy2, const int* __restrict__ ry) {
  const int rx1 = rx[1], ry1 = ry[1];
  const int rx2 = (d == 3) ? rx[2] : 0, ry2 = (d == 3) ? ry[2] : 0;
  if (rx1 + ry1 > rcapy1 || (d == 3 && rx2 + ry2 > rcapy2)) return;
  if (d == 2) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rx1 * n1; idx += gridDim.x * blockDim.x) {
      const int a = idx / n1, j = idx - (idx / n1) * n1;
      y1[(size_t)(ry1 + a) * n1 + j] = x1[(size_t)a * n1 + j];
    }
    return;
  }
  const int tot1 = rx1 * n1 * rx2, tot2 = rx2 * n2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot1 + tot2; idx += gridDim.x * blockDim.x) {
    if (idx < tot1) {
      const int a = idx / (n1 * rx2);
      const int rem = idx - a * n1 * rx2;
      const int l = rem / rx2, b = rem - (rem / rx2) * rx2;
      y1[((size_t)(ry1 + a) * n1 + l) * rcapy2 + ry2 + b] = x1[((size_t)a * n1 + l) * rcapx2 + b];
    } else {
      const int i2 = idx - tot1;
      const int b = i2 / n2, p = i2 - (i2 / n2) * n2;
      y2[(size_t)(ry2 + b) * n2 + p] = x2[(size_t)b * n2 + p];
    }
  }
  (void)rcapx1;
}

__global__ void k_axpy_ranks(int d, const int* __restrict__ rx, int* __restrict__ ry, int rcapy1, int rcapy2) {
  if (threadIdx.x || blockIdx.x) return;
  const int n1 = rx[1] + ry[1];
  const int n2 = (d == 3) ? rx[2] + ry[2] : 1;
  if (n1 > rcapy1 || (d == 3 && n2 > rcapy2)) return;
  ry[1] = n1;
  if (d == 3) ry[2] = n2;
}

// Per-chunk partial Gram entries W1[a][b] = sum_k X[k][a] Y[k][b].
template <typename S>
__global__ void k_gram_partials(long N, long rows_per, const S* __restrict__ X, int ldx, int rx,
                                const S* __restrict__ Y, int ldy, int ry, double* __restrict__ partials) {
  const int e = blockIdx.y * blockDim.x + threadIdx.x;
  if (e >= rx * ry) return;
  const int a = e / ry, b = e - (e / ry) * ry;
  const long beg = blockIdx.x * rows_per;
  const long end = (beg + rows_per < N) ? beg + rows_per : N;
  double acc = 0.0;
  for (long k = beg; k < end; ++k) acc += (double)X[k * ldx + a] * (double)Y[k * ldy + b];
  partials[(size_t)blockIdx.x * rx * ry + e] = acc;
}

__global__ void k_sum_chunks(const double* __restrict__ partials, long nchunks, int ne, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = 0.0;
  for (long c = 0; c < nchunks; ++c) s += partials[(size_t)c * ne + e];
  out[e] = s;
}

__global__ void k_dot_final(int ne, const double* __restrict__ W1, const double* __restrict__ G, double* __restrict__ out) {
  __shared__ double red[33];
  double s = 0.0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) s += W1[e] * G[e];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace

template <typename S>
tt_status apply_transport_impl(tt_context* ctx, const tt_plan* p, const tt_tensor* in, tt_tensor* out) {
  cudaStream_t s = ctx->stream;
  const int d = in->d;
  SrcStencil<S> src{};
  src.Z = (const S*)in->core[0];
  src.ldz = in->rcap[1];
  src.rcap = in->rcap[1];
  src.nterm = p->nterm;
  src.G = p->G;
  for (int a = 0; a < 3; ++a) {
    src.ext[a] = p->ext[a];
    src.stride[a] = p->stride[a];
  }
  for (int t = 0; t < kMaxTerms; ++t) {
    src.lam[t] = (t < p->nterm) ? p->lam[p->term_axis[t]] : 0.0;
    src.axis[t] = (t < p->nterm) ? p->term_axis[t] : 0;
    src.w[t] = (t < p->nterm) ? p->term_w[t] : 1;
    src.bc_term[t] = (t < p->nbc) ? p->bc_term[t] : 0;
  }
  src.bcval = p->bcval;
  src.nax = p->ndim;
  const long N = in->n[0];
  const int rcapo2 = (d == 3) ? out->rcap[2] : 1;
  k_transport_Z<S><<<1024, 256, 0, s>>>(N, src, in->rank, (S*)out->core[0], out->rcap[1], p->nbc,
                                        d == 3 ? in->rank + 2 : nullptr, rcapo2, &ctx->ctrl->status); count_launch();
  k_transport_small<S><<<64, 256, 0, s>>>(d, p->nterm, p->nbc, p->n1, p->n2, (const S*)in->core[1],
                                          d == 3 ? (const S*)in->core[2] : nullptr, in->rcap[1],
                                          d == 3 ? in->rcap[2] : 1, in->rank, (S*)out->core[1],
                                          d == 3 ? (S*)out->core[2] : nullptr, out->rcap[1], rcapo2, p->fac1, p->fac2,
                                          p->bc_term_dev); count_launch();
  k_transport_ranks<<<1, 32, 0, s>>>(d, p->nterm, p->nbc, in->rank, out->rank, out->rcap[1], rcapo2); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

template <typename S>
tt_status axpy_impl(tt_context* ctx, double alpha, const tt_tensor* x, tt_tensor* y) {
  cudaStream_t s = ctx->stream;
  const int d = x->d;
  const long N = x->n[0];
  const int rcapy2 = (d == 3) ? y->rcap[2] : 1;
  k_axpy_Z<S><<<1024, 256, 0, s>>>(N, alpha, (const S*)x->core[0], x->rcap[1], x->rank, (S*)y->core[0], y->rcap[1],
                                   y->rank, d, rcapy2, &ctx->ctrl->status); count_launch();
  k_axpy_small<S><<<64, 256, 0, s>>>(d, x->n[1], d == 3 ? x->n[2] : 1, (const S*)x->core[1],
                                     d == 3 ? (const S*)x->core[2] : nullptr, x->rcap[1], d == 3 ? x->rcap[2] : 1,
                                     x->rank, (S*)y->core[1], d == 3 ? (S*)y->core[2] : nullptr, y->rcap[1], rcapy2,
                                     y->rank); count_launch();
  k_axpy_ranks<<<1, 32, 0, s>>>(d, x->rank, y->rank, y->rcap[1], rcapy2); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

template <typename S>
tt_status dot_impl(tt_context* ctx, const tt_tensor* x, const tt_tensor* y, double* out, Bump& ws) {
  cudaStream_t s = ctx->stream;
  const int d = x->d;
  const long N = x->n[0];
  const int n1 = x->n[1], n2 = (d == 3) ? x->n[2] : 1, nang = n1 * n2;
  const int rx = x->rcap[1], ry = y->rcap[1];
  const int ne = rx * ry;
  long nchunks = (N + 1023) / 1024;
  if (nchunks > 2048) nchunks = 2048;
  const long rows_per = (N + nchunks - 1) / nchunks;
  nchunks = (N + rows_per - 1) / rows_per;
  double* part = ws.take<double>((size_t)nchunks * ne);
  double* W1 = ws.take<double>(ne);
  double* Bx = ws.take<double>((size_t)rx * nang);
  double* By = ws.take<double>((size_t)ry * nang);
  double* G = ws.take<double>(ne);
  if (ws.dry) return TT_OK;
  dim3 grid((unsigned)nchunks, (unsigned)((ne + 255) / 256));
  k_gram_partials<S><<<grid, 256, 0, s>>>(N, rows_per, (const S*)x->core[0], rx, rx, (const S*)y->core[0], ry, ry,
                                          part); count_launch();
  k_sum_chunks<<<(ne + 255) / 256, 256, 0, s>>>(part, nchunks, ne, W1); count_launch();
  right_part<S>(s, d, rx, n1, d == 3 ? x->rcap[2] : 1, n2, (const S*)x->core[1], d == 3 ? (const S*)x->core[2] : nullptr,
                Bx);
  right_part<S>(s, d, ry, n1, d == 3 ? y->rcap[2] : 1, n2, (const S*)y->core[1], d == 3 ? (const S*)y->core[2] : nullptr,
                By);
  small_gemm<double, double>(s, rx, ry, nang, Bx, nang, 1, By, 1, nang, G, ry, nullptr, nullptr);
  k_dot_final<<<1, 1024, 0, s>>>(ne, W1, G, out); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

// Inner product with caller-provided scratch (no workspace, no allocation): the same kernels
// as dot_impl with the number of row chunks reduced until everything fits in `cap` doubles.
template <typename S>
tt_status dot_into(cudaStream_t s, const tt_tensor* x, const tt_tensor* y, double* out, double* scratch,
                   size_t cap) {
  const int d = x->d;
  const long N = x->n[0];
  const int n1 = x->n[1], n2 = (d == 3) ? x->n[2] : 1, nang = n1 * n2;
  const int rx = x->rcap[1], ry = y->rcap[1];
  const size_t ne = (size_t)rx * ry;
  const size_t fixed = ne /*W1*/ + ne /*G*/ + (size_t)(rx + ry) * nang;
  if (fixed + ne > cap) return TT_ERR_WORKSPACE;
  long nchunks = (N + 1023) / 1024;
  if (nchunks > 2048) nchunks = 2048;
  const long fit = (long)((cap - fixed) / ne);
  if (nchunks > fit) nchunks = fit;
  if (nchunks < 1) nchunks = 1;
  const long rows_per = (N + nchunks - 1) / nchunks;
  nchunks = (N + rows_per - 1) / rows_per;
  double* part = scratch;
  double* W1 = part + (size_t)nchunks * ne;
  double* Bx = W1 + ne;
  double* By = Bx + (size_t)rx * nang;
  double* G = By + (size_t)ry * nang;
  dim3 grid((unsigned)nchunks, (unsigned)((ne + 255) / 256));
  k_gram_partials<S><<<grid, 256, 0, s>>>(N, rows_per, (const S*)x->core[0], rx, rx, (const S*)y->core[0], ry, ry,
                                          part); count_launch();
  k_sum_chunks<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(part, nchunks, (int)ne, W1); count_launch();
  right_part<S>(s, d, rx, n1, d == 3 ? x->rcap[2] : 1, n2, (const S*)x->core[1], d == 3 ? (const S*)x->core[2] : nullptr,
                Bx);
  right_part<S>(s, d, ry, n1, d == 3 ? y->rcap[2] : 1, n2, (const S*)y->core[1], d == 3 ? (const S*)y->core[2] : nullptr,
                By);
  small_gemm<double, double>(s, rx, ry, nang, Bx, nang, 1, By, 1, nang, G, ry, nullptr, nullptr);
  k_dot_final<<<1, 1024, 0, s>>>((int)ne, W1, G, out); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}
template tt_status dot_into<double>(cudaStream_t, const tt_tensor*, const tt_tensor*, double*, double*, size_t);
template tt_status dot_into<float>(cudaStream_t, const tt_tensor*, const tt_tensor*, double*, double*, size_t);

template tt_status apply_transport_impl<double>(tt_context*, const tt_plan*, const tt_tensor*, tt_tensor*);
template tt_status apply_transport_impl<float>(tt_context*, const tt_plan*, const tt_tensor*, tt_tensor*);
template tt_status axpy_impl<double>(tt_context*, double, const tt_tensor*, tt_tensor*);
template tt_status axpy_impl<float>(tt_context*, double, const tt_tensor*, tt_tensor*);
template tt_status dot_impl<double>(tt_context*, const tt_tensor*, const tt_tensor*, double*, Bump&);
template tt_status dot_impl<float>(tt_context*, const tt_tensor*, const tt_tensor*, double*, Bump&);

}  // namespace ttk
