// Internal structure of the merged core (Sec. 5.2): singular values of
// reshape(Z, [N_nu, N_X r]) (frequency-leading) and reshape(Z, [N_X, N_nu r]) (space-leading),
// each from the FP64 Gram matrix of its narrow side and the cooperative Jacobi eigen-solver,
// and the delta-ranks r1, r1x of Sec. 5.4's delta-SVD.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "gram.cuh"
#include "step.cuh"

namespace ttk {
namespace {

// Transposed frequency-leading unfolding: row rho = cell * ldz + q, column g:
// Z[(g + G cell) * ldz + q] (every column is one group's values over cells and ranks).
template <typename S>
struct SrcNu {
  const S* Z;
  int ldz;
  int G;
  struct Col { int g; };
  __device__ __forceinline__ Col col(int c) const { return Col{c}; }
  __device__ __forceinline__ unsigned row_flags(long) const { return 0u; }
  template <typename T>
  __device__ __forceinline__ T loadT(const Col& cc, long rho, unsigned) const {
    const long cell = rho / ldz, q = rho - (rho / ldz) * ldz;
    return (T)Z[((long)cc.g + (long)G * cell) * ldz + q];
  }
  __device__ __forceinline__ double load(const Col& cc, long rho) const { return loadT<double>(cc, rho, 0u); }
};

// Smallest k with sqrt(sum_{j>=k} s_j^2) <= delta * |s| (s sorted decreasing).
int delta_rank(const std::vector<double>& s, double delta) {
  double tot = 0.0;
  for (double v : s) tot += v * v;
  if (tot == 0.0) return 1;
  const double thr = delta * std::sqrt(tot);
  double tail = 0.0;
  int k = (int)s.size();
  for (int j = (int)s.size() - 1; j >= 0; --j) {
    if (std::sqrt(tail) <= thr) k = j + 1;
    else break;
    tail += s[j] * s[j];
  }
  // k is the smallest index whose tail (sum over j >= k) stays within the threshold
  return std::max(1, k);
}

}  // namespace

template <typename S>
tt_status internal_ranks_impl(tt_context* ctx, const tt_plan* p, const tt_tensor* x, double delta, int* ranks,
                              double* sig_nu, long nsig_nu, double* sig_x, long nsig_x, Bump& ws) {
  cudaStream_t s = ctx->stream;
  const int G = p->G;
  const int ldz = x->rcap[1];
  const long nX = x->n[0] / G;
  const int ncx = G * ldz;
  if (ncx > 4096 || G > 4096) return TT_ERR_UNSUPPORTED;
  double *Gnu = nullptr, *Gx = nullptr;
  SrcNu<S> snu{(const S*)x->core[0], ldz, G};
  tt_status st = gram_matrix(s, ctx->num_sms, snu, LivePattern{nullptr, G, 1, 0}, nX * ldz, ws, &Gnu, kOther);
  if (st != TT_OK) return st;
  st = gram_matrix(s, ctx->num_sms, SrcRows<S>{(const S*)x->core[0], (long)ncx}, LivePattern{nullptr, ncx, 1, 0}, nX,
                   ws, &Gx, kOther);
  if (st != TT_OK) return st;
  double* lnu = ws.take<double>(G);
  double* Vnu = ws.take<double>((size_t)G * G);
  double* lx = ws.take<double>(ncx);
  double* Vx = ws.take<double>((size_t)ncx * ncx);
  st = svd_right(s, ctx->num_sms, G, G, Gnu, ws, lnu, Vnu, ctx->ctrl, ctx->coop_grid_max);
  if (st != TT_OK) return st;
  st = svd_right(s, ctx->num_sms, ncx, ncx, Gx, ws, lx, Vx, ctx->ctrl, ctx->coop_grid_max);
  if (st != TT_OK || ws.dry) return st;
  std::vector<double> hnu(G), hx(ncx);
  if (cudaMemcpyAsync(hnu.data(), lnu, sizeof(double) * G, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hx.data(), lx, sizeof(double) * ncx, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TT_ERR_CUDA;
  // Gram eigenvalues lambda = sigma^2 (Jacobi returns them sorted, decreasing)
  for (double& v : hnu) v = v > 0.0 ? std::sqrt(v) : 0.0;
  for (double& v : hx) v = v > 0.0 ? std::sqrt(v) : 0.0;
  // the space-leading unfolding has at most min(N_X, G ldz) nonzero singular values
  if ((long)hx.size() > nX) hx.resize(nX);
  ranks[0] = delta_rank(hnu, delta);
  ranks[1] = delta_rank(hx, delta);
  for (long i = 0; sig_nu && i < nsig_nu; ++i) sig_nu[i] = i < (long)hnu.size() ? hnu[i] : 0.0;
  for (long i = 0; sig_x && i < nsig_x; ++i) sig_x[i] = i < (long)hx.size() ? hx[i] : 0.0;
  return TT_OK;
}

template tt_status internal_ranks_impl<double>(tt_context*, const tt_plan*, const tt_tensor*, double, int*, double*,
                                               long, double*, long, Bump&);
template tt_status internal_ranks_impl<float>(tt_context*, const tt_plan*, const tt_tensor*, double, int*, double*,
                                              long, double*, long, Bump&);

}  // namespace ttk
