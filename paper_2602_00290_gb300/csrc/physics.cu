// Per-problem setup on the device: angular quadrature, group emission by Planck integrals,
// backward-Euler source coefficients, and the angular factors of the rank-1 transport
// operators.  Runs once per plan, not per time step.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "instr.cuh"

namespace ttk {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kBern = 32;

// Quadrature (Sec. 4 preamble): lat/long midpoint rule in mu = cos(theta) and phi, or
// Gauss-Legendre nodes in mu for the planar slab (nodes by Newton's method on P_n).
__global__ void k_quadrature(int quad, int ntheta, int nphi, double* mu, double* phi,
                             double* domega) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (quad == TT_QUAD_GAUSS_LEGENDRE_MU) {
    const int n = ntheta;
    for (int i = 0; i < n; ++i) {
      double x = cos(kPi * (i + 0.75) / (n + 0.5));
      double dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p0 = 1.0; p1 = x; }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
      }
      // final derivative at the converged node for the weight
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = x; }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double w = 2.0 / ((1.0 - x * x) * dp * dp);
      mu[n - 1 - i] = x;
      domega[n - 1 - i] = 2.0 * kPi * w;
    }
    phi[0] = 0.0;
  } else {
    for (int l = 0; l < ntheta; ++l) mu[l] = -1.0 + (2.0 * l + 1.0) / ntheta;
    for (int p = 0; p < nphi; ++p) phi[p] = (2.0 * p + 1.0) * kPi / nphi;
    const double dom = (2.0 / ntheta) * (2.0 * kPi / nphi);
    for (int i = 0; i < ntheta * nphi; ++i) domega[i] = dom;
  }
}

// Angular factors of the rank-1 transport operators (Appendix A, 'Value of n'), split over the
// angular cores: upwind n_a * 1[n_a >= 0] (w = +1) or n_a * 1[n_a < 0] (w = -1); Rusanov and
// central n_a (w = +2) and, Rusanov only, 1 (w = -2).
__global__ void k_angular_factors(int d, int nterm, const int* axis, const int* w, int n1,
                                  int n2, const double* mu, const double* phi, double* fac1,
                                  double* fac2) {
  const int t = blockIdx.x;
  if (t >= nterm) return;
  const int ax = axis[t], ww = w[t];
  if (ww == 2 || ww == -2) {
    // Rusanov: the central term carries the full n_a, the diffusion term no angular factor
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
      const double m = mu[i];
      fac1[t * n1 + i] = (ww < 0) ? 1.0 : ((d == 2 || ax == 2) ? m : sqrt(1.0 - m * m));
    }
    for (int p = threadIdx.x; p < n2; p += blockDim.x) {
      double f = 1.0;
      if (ww > 0 && d == 3 && ax < 2) f = (ax == 0) ? cos(phi[p]) : sin(phi[p]);
      fac2[t * n2 + p] = f;
    }
    return;
  }
  for (int i = threadIdx.x; i < n1; i += blockDim.x) {
    double m = mu[i], f;
    if (d == 2) {
      f = (ww > 0) ? (m >= 0.0 ? m : 0.0) : (m < 0.0 ? m : 0.0);
    } else if (ax == 2) {
      f = (ww > 0) ? (m >= 0.0 ? m : 0.0) : (m < 0.0 ? m : 0.0);
    } else {
      f = sqrt(1.0 - m * m);
    }
    fac1[t * n1 + i] = f;
  }
  for (int p = threadIdx.x; p < n2; p += blockDim.x) {
    double f = 1.0;
    if (d == 3 && ax < 2) {
      double cp = (ax == 0) ? cos(phi[p]) : sin(phi[p]);
      f = (ww > 0) ? (cp >= 0.0 ? cp : 0.0) : (cp < 0.0 ? cp : 0.0);
    }
    fac2[t * n2 + p] = f;
  }
}

// Taylor coefficients b_m = B_m / m! of t/(e^t - 1), from t = (e^t - 1) sum b_j t^j.
__device__ void bernoulli_over_factorial(double* b) {
  b[0] = 1.0;
  for (int m = 1; m < kBern; ++m) {
    double s = 0.0, fact = 1.0;  // fact = (m+1-j)!
    for (int k = 2; k <= m + 1; ++k) fact *= k;
    for (int j = 0; j < m; ++j) {
      s += b[j] / fact;
      fact /= (m + 1 - j);
    }
    b[m] = -s;
  }
}

// Q(x) = int_0^x t^3/(e^t - 1) dt = sum_m b_m x^{m+3}/(m+3), for 0 <= x <= 1.
__device__ double planck_head(double x, const double* b) {
  if (x <= 0.0) return 0.0;
  double xp = x * x * x, s = 0.0;
  for (int m = 0; m < kBern; ++m) {
    s += b[m] * xp / (m + 3);
    xp *= x;
  }
  return s;
}

// P(x) = int_x^inf t^3/(e^t - 1) dt = sum_n e^{-n x}(x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4),
// i.e. x^3 Li_1(e^-x) + 3x^2 Li_2(e^-x) + 6x Li_3(e^-x) + 6 Li_4(e^-x), for x >= 1.
__device__ double planck_tail(double x) {
  if (!(x < 745.0)) return 0.0;
  const int nmax = (int)(42.0 / x) + 2;
  const double x2 = x * x, x3 = x2 * x;
  double s = 0.0;
  for (int n = nmax; n >= 1; --n) {  // small terms first
    const double dn = n;
    s += exp(-dn * x) * (x3 / dn + 3.0 * x2 / (dn * dn) + 6.0 * x / (dn * dn * dn) +
                         6.0 / (dn * dn * dn * dn));
  }
  return s;
}

// int_{x1}^{x2} t^3/(e^t-1) dt, split at x = 1 so neither series cancels badly.
__device__ double planck_segment(double x1, double x2, const double* b) {
  if (!(x2 > x1) || x1 >= 745.0) return 0.0;
  if (x2 <= 1.0) return planck_head(x2, b) - planck_head(x1, b);
  const double tail2 = isinf(x2) ? 0.0 : planck_tail(x2);
  if (x1 >= 1.0) return planck_tail(x1) - tail2;
  return (planck_head(1.0, b) - planck_head(x1, b)) + (planck_tail(1.0) - tail2);
}

// epsilon_f(T) = (c a T^4 / 4 pi)(15/pi^4) int_{nu_{f-1}/T}^{nu_f/T} t^3/(e^t-1) dt
// (Eqs. Ttoeps1-2), flushed to 0 below 1e-300.
__device__ double emission(double T, double lo, double hi, double c, double a, const double* b) {
  if (!(T > 0.0)) return 0.0;
  const double pref = c * a * T * T * T * T / (4.0 * kPi) * 15.0 / (kPi * kPi * kPi * kPi);
  const double x1 = lo / T;
  const double x2 = isinf(hi) ? hi : hi / T;
  double v = pref * planck_segment(x1, x2, b);
  return (v >= 1e-300) ? v : 0.0;
}

__global__ void k_emission_rows(long nrow, int G, const double* __restrict__ T,
                                const double* __restrict__ edges, double c, double a,
                                double* __restrict__ eps) {
  __shared__ double b[kBern];
  if (threadIdx.x == 0) bernoulli_over_factorial(b);
  __syncthreads();
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < nrow;
       k += (long)gridDim.x * blockDim.x) {
    const int g = (int)(k % G);
    eps[k] = emission(T[k / G], edges[g], edges[g + 1], c, a, b);
  }
}

__global__ void k_inflow(int G, const double* __restrict__ Tb6, const double* __restrict__ edges,
                         double c, double a, double* __restrict__ inflow) {
  __shared__ double b[kBern];
  if (threadIdx.x == 0) bernoulli_over_factorial(b);
  __syncthreads();
  for (int i = threadIdx.x; i < 6 * G; i += blockDim.x) {
    const int f = i / G, g = i % G;
    const double Tb = Tb6[f];
    inflow[i] = (Tb >= 0.0) ? emission(Tb, edges[g], edges[g + 1], c, a, b) : 0.0;
  }
}

__global__ void k_row_coef(long nrow, double cdt, const double* __restrict__ ka,
                           const double* __restrict__ ks, double* __restrict__ acoef,
                           double* __restrict__ scoef) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < nrow;
       k += (long)gridDim.x * blockDim.x) {
    acoef[k] = cdt * ka[k];
    scoef[k] = cdt * ks[k];
  }
}

__global__ void k_bcval(int nbc, int G, const int* __restrict__ face, const double* __restrict__ sgnlam,
                        const double* __restrict__ inflow, double* __restrict__ bcval) {
  for (int i = threadIdx.x; i < nbc * G; i += blockDim.x) {
    const int b = i / G, g = i % G;
    bcval[i] = sgnlam[b] * inflow[face[b] * G + g];
  }
}

// d epsilon_f / dT = 4 epsilon_f / T - (c a T^3 / 4 pi)(15/pi^4) [x^4/(e^x - 1)]_{x_lo}^{x_hi},
// x = nu / T (the derivative of the Planck group integral, Eqs. Ttoeps1-2).
__device__ double demission_dT(double T, double eps, double lo, double hi, double c, double a) {
  if (!(T > 0.0)) return 0.0;
  const double pref = c * a * T * T * T / (4.0 * kPi) * 15.0 / (kPi * kPi * kPi * kPi);
  auto edge = [](double x) { return (x > 0.0 && x < 700.0) ? x * x * x * x / expm1(x) : 0.0; };
  const double xl = lo / T, xh = isinf(hi) ? 0.0 : hi / T;
  return 4.0 * eps / T - pref * ((isinf(hi) ? 0.0 : edge(xh)) - edge(xl));
}

// One warp per cell: T^dagger = root of f(T) = T^m + C sum_f w_f (J*_f - eps_f(T)) - T with
// C = 4 pi / (c rho c_v), w_f = a_f / (1 + a_f) (the paper's f(T^dagger), Sec. 2.1), by Newton
// steps kept inside a shrinking bracket [lo, hi] (f(lo) > 0 > f(hi)); then eps rows <- eps(T^dagger).
__global__ void k_t_dagger(long ncell, int G, double c, double a, const double* __restrict__ edges,
                           const double* __restrict__ Tm, const double* __restrict__ rho_cv,
                           const double* __restrict__ acoef, const double* __restrict__ jstar,
                           double* __restrict__ tdag, double* __restrict__ eps) {
  __shared__ double b[kBern];
  if (threadIdx.x == 0) bernoulli_over_factorial(b);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long cell = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); cell < ncell; cell += warps) {
    const double T0 = Tm[cell];
    const double C = 4.0 * kPi / (c * rho_cv[cell]);
    // f(T) and f'(T), lanes over groups
    auto eval = [&](double T, double& f, double& df) {
      double s = 0.0, ds = 0.0;
      for (int g = lane; g < G; g += 32) {
        const long k = (long)cell * G + g;
        const double w = acoef[k] / (1.0 + acoef[k]);
        const double e = emission(T, edges[g], edges[g + 1], c, a, b);
        s += w * (jstar[k] - e);
        ds += w * demission_dT(T, e, edges[g], edges[g + 1], c, a);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        ds += __shfl_xor_sync(0xffffffffu, ds, o);
      }
      f = T0 + C * s - T;
      df = -C * ds - 1.0;
    };
    double f, df;
    eval(0.0, f, df);
    double T = 0.0;
    if (f > 0.0) {
      double lo = 0.0, hi = T0 > 1e-3 ? T0 : 1e-3;
      double fh, dh;
      eval(hi, fh, dh);
      for (int it = 0; it < 200 && fh > 0.0; ++it) {
        lo = hi;
        hi *= 2.0;
        eval(hi, fh, dh);
      }
      T = 0.5 * (lo + hi);
      for (int it = 0; it < 200; ++it) {
        eval(T, f, df);
        if (f > 0.0) lo = T; else hi = T;
        double Tn = T - f / df;
        if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
        const double step = fabs(Tn - T);
        T = Tn;
        if (step <= 1e-15 * T || hi - lo <= 1e-15 * hi) break;
      }
    }
    if (lane == 0) tdag[cell] = T;
    for (int g = lane; g < G; g += 32) eps[(long)cell * G + g] = emission(T, edges[g], edges[g + 1], c, a, b);
  }
}

// rho c_v (T^{m+1} - T^m) = (4 pi / c) sum_f (J*_f - J^{m+1}_f), one warp per cell.
__global__ void k_t_update(long ncell, int G, double c, const double* __restrict__ rho_cv,
                           const double* __restrict__ jstar, const double* __restrict__ jnew,
                           double* __restrict__ T) {
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long cell = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); cell < ncell; cell += warps) {
    double s = 0.0;
    for (int g = lane; g < G; g += 32) s += jstar[(long)cell * G + g] - jnew[(long)cell * G + g];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) T[cell] += 4.0 * kPi / (c * rho_cv[cell]) * s;
  }
}

}  // namespace

tt_status physics_setup(tt_context* ctx, const tt_problem* p, tt_plan* plan) {
  cudaStream_t s = ctx->stream;
  const int G = p->ngroup;
  plan->ndim = p->ndim_x;
  plan->nx = p->nx; plan->ny = p->ny; plan->nz = p->nz;
  plan->G = G;
  plan->quad = p->quadrature;
  plan->ntheta = p->ntheta; plan->nphi = p->nphi;
  plan->d = (p->ndim_x == 1) ? 2 : 3;
  plan->n1 = p->ntheta;
  plan->n2 = (plan->d == 3) ? p->nphi : 1;
  plan->nrow = (long)p->nx * p->ny * p->nz * G;
  plan->c = p->c; plan->dt = p->dt;
  const double dxs[3] = {p->dx, p->dy, p->dz};
  double dV = 1.0;
  for (int a = 0; a < 3; ++a) plan->lam[a] = 0.0;
  for (int a = 0; a < p->ndim_x; ++a) {
    plan->lam[a] = p->c * p->dt / dxs[a];
    dV *= dxs[a];
  }
  plan->dV = dV;
  plan->ext[0] = p->nx; plan->ext[1] = p->ny; plan->ext[2] = p->nz;
  plan->stride[0] = G;
  plan->stride[1] = (long)G * p->nx;
  plan->stride[2] = (long)G * p->nx * p->ny;
  // upwind and Rusanov: two terms per axis; central (Rusanov with wavespeed 0): one per axis
  const bool central = (p->flux == TT_FLUX_CENTRAL);
  const bool upwind = (p->flux == TT_FLUX_UPWIND);
  plan->nterm = (central ? 1 : 2) * p->ndim_x;
  int faces[kMaxTerms];
  double sgnlam[kMaxTerms];
  plan->nbc = 0;
  for (int t = 0; t < plan->nterm; ++t) {
    // upwind: +1 / -1 (one-sided differences); Rusanov: +2 (central) / -2 (diffusion);
    // central: +2 only
    plan->term_axis[t] = central ? t : t / 2;
    plan->term_w[t] = central ? 2 : ((t % 2 == 0) ? +1 : -1) * (upwind ? 1 : 2);
    const int face = 2 * (t / 2) + (t % 2);  // w=+ reads the minus-face ghost
    if (upwind && p->inflow_temperature[face] >= 0.0) {
      plan->bc_term[plan->nbc] = t;
      faces[plan->nbc] = face;
      sgnlam[plan->nbc] = (t % 2 == 0 ? 1.0 : -1.0) * plan->lam[t / 2];
      plan->nbc++;
    }
  }
  const int n1 = plan->n1, n2 = plan->n2;
  const size_t nang = (size_t)p->ntheta * (plan->d == 3 ? p->nphi : 1);
#define TT_ALLOC(ptr, count) \
  if (cudaMalloc((void**)&(ptr), sizeof(double) * (size_t)((count) > 0 ? (count) : 1)) != cudaSuccess) return TT_ERR_CUDA
  TT_ALLOC(plan->eps, plan->nrow);
  TT_ALLOC(plan->acoef, plan->nrow);
  TT_ALLOC(plan->scoef, plan->nrow);
  TT_ALLOC(plan->domega, nang);
  TT_ALLOC(plan->mu, p->ntheta);
  TT_ALLOC(plan->phi, p->nphi);
  TT_ALLOC(plan->fac1, plan->nterm * n1);
  TT_ALLOC(plan->fac2, plan->nterm * n2);
  TT_ALLOC(plan->inflow, 6 * G);
  TT_ALLOC(plan->bcval, plan->nbc * G);
  TT_ALLOC(plan->edges, G + 1);
  const long ncell = (long)p->nx * p->ny * p->nz;
  TT_ALLOC(plan->temp, ncell);
  plan->a_rad = p->a_rad;
  plan->coupled = (p->rho_cv != nullptr) ? 1 : 0;
  if (plan->coupled) {
    TT_ALLOC(plan->rho_cv, ncell);
    TT_ALLOC(plan->tdag, ncell);
  }
  if (cudaMalloc((void**)&plan->bc_term_dev, sizeof(int) * kMaxTerms) != cudaSuccess) return TT_ERR_CUDA;
#undef TT_ALLOC
  // small host->device parameter blocks
  int* d_axis = nullptr;
  double* d_tb = nullptr;
  if (cudaMalloc((void**)&d_axis, sizeof(int) * 4 * kMaxTerms) != cudaSuccess) return TT_ERR_CUDA;
  if (cudaMalloc((void**)&d_tb, sizeof(double) * (6 + kMaxTerms)) != cudaSuccess) return TT_ERR_CUDA;
  int hint[4 * kMaxTerms];
  for (int t = 0; t < kMaxTerms; ++t) {
    hint[t] = plan->term_axis[t];
    hint[kMaxTerms + t] = plan->term_w[t];
    hint[2 * kMaxTerms + t] = (t < plan->nbc) ? faces[t] : 0;
    hint[3 * kMaxTerms + t] = 0;
  }
  double hdb[6 + kMaxTerms];
  for (int f = 0; f < 6; ++f) hdb[f] = (f / 2 < p->ndim_x) ? p->inflow_temperature[f] : -1.0;
  for (int t = 0; t < kMaxTerms; ++t) hdb[6 + t] = (t < plan->nbc) ? sgnlam[t] : 0.0;
  cudaMemcpyAsync(d_axis, hint, sizeof(hint), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_tb, hdb, sizeof(hdb), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(plan->bc_term_dev, plan->bc_term, sizeof(int) * kMaxTerms, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(plan->edges, p->group_edges, sizeof(double) * (G + 1), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(plan->temp, p->temperature, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, s);
  if (plan->coupled) {
    cudaMemcpyAsync(plan->rho_cv, p->rho_cv, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(plan->tdag, 0, sizeof(double) * ncell, s);
  }
  k_quadrature<<<1, 32, 0, s>>>(p->quadrature, p->ntheta, plan->d == 3 ? p->nphi : 1, plan->mu,
                                plan->phi, plan->domega);
  k_angular_factors<<<plan->nterm, 128, 0, s>>>(plan->d, plan->nterm, d_axis, d_axis + kMaxTerms,
                                                n1, n2, plan->mu, plan->phi, plan->fac1, plan->fac2);
  const int blocks = (int)((plan->nrow + 255) / 256 < 4096 ? (plan->nrow + 255) / 256 : 4096);
  k_emission_rows<<<blocks, 256, 0, s>>>(plan->nrow, G, p->temperature, plan->edges, p->c, p->a_rad,
                                         plan->eps);
  k_row_coef<<<blocks, 256, 0, s>>>(plan->nrow, p->c * p->dt, p->rho_kappa_a, p->rho_kappa_s,
                                    plan->acoef, plan->scoef);
  k_inflow<<<1, 256, 0, s>>>(G, d_tb, plan->edges, p->c, p->a_rad, plan->inflow);
  if (plan->nbc > 0)
    k_bcval<<<1, 256, 0, s>>>(plan->nbc, G, d_axis + 2 * kMaxTerms, d_tb + 6, plan->inflow,
                              plan->bcval);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d_axis);
  cudaFree(d_tb);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
  return TT_OK;
}

tt_status coupled_t_dagger(cudaStream_t s, tt_plan* p, const double* jstar) {
  const long ncell = (long)p->nx * p->ny * p->nz;
  const long blocks = (ncell + 7) / 8 < 2048 ? (ncell + 7) / 8 : 2048;
  k_t_dagger<<<(unsigned)blocks, 256, 0, s>>>(ncell, p->G, p->c, p->a_rad, p->edges, p->temp, p->rho_cv, p->acoef,
                                              jstar, p->tdag, p->eps); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

tt_status coupled_t_update(cudaStream_t s, tt_plan* p, const double* jstar, const double* jnew) {
  const long ncell = (long)p->nx * p->ny * p->nz;
  const long blocks = (ncell + 7) / 8 < 2048 ? (ncell + 7) / 8 : 2048;
  k_t_update<<<(unsigned)blocks, 256, 0, s>>>(ncell, p->G, p->c, p->rho_cv, jstar, jnew, p->temp); count_launch();
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

}  // namespace ttk
