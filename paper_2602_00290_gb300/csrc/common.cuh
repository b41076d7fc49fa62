// Shared device/host definitions of the sm_103a tensor-train transport library.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tt.h"

namespace ttk {

constexpr int kMaxTerms = 6;  // 2 d_X transport operators for d_X <= 3 (Appendix A)

// Device control block of a context: latched status plus the per-rounding decisions that
// later kernels read (no host round trip inside a step).
struct DevCtrl {
  int status;          // first tt_status latched on the device (0 = TT_OK)
  int k[4];            // ranks decided by the last small-core sweep (bond 1, bond 2)
  int pad;
  double norm;         // ||X||_F of the last rounded tensor
  double delta;        // truncation threshold of the last rounding
  double energy[8];    // scratch for energy reports
  int jac_sweeps;      // sweeps of the last cooperative Jacobi SVD
  int jac_sweeps_max;  // max sweeps over Jacobi SVDs since the last counter reset
  int jac_calls;       // Jacobi SVDs since the last counter reset
  int jac_sweeps_sum;  // their total sweeps
  int jac_sweep_cap;   // > 0: cap on the sweeps of one FP64 Jacobi SVD (tt_context_set_limits)
  int barrier_extra;   // arrivals a grid barrier waits for beyond the grid (> 0: never met)
  long long spin_limit;  // > 0: spins of one grid-barrier wait before it gives up (else 2^24)
  unsigned bar_count;  // grid barrier of cooperative kernels: arrivals in this generation
  unsigned bar_gen;    // grid barrier generation
  int abort;           // set when a bounded wait gives up; every CTA then leaves
  int pad2;
  double fro2;         // ||A||_F^2 of the matrix in a cooperative Jacobi sweep
  int jac_rot[64];     // rotations per sweep of the cooperative Jacobi
};

__device__ __forceinline__ void latch(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Column-liveness pattern of a (possibly virtual) tall matrix in capacity layout:
// columns [t*rcap, t*rcap + rcap) for t < nblk are live iff their offset is < r (r read
// from device memory); the `nextra` columns after nblk*rcap are always live.
struct LivePattern {
  const int* r_ptr;
  int rcap;
  int nblk;
  int nextra;
  __host__ __device__ int ncap() const { return nblk * rcap + nextra; }
  __device__ __forceinline__ bool live(int c, int r) const {
    int t = c / rcap;
    if (t < nblk) return (c - t * rcap) < r;
    return c < nblk * rcap + nextra;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double per thread (blockDim multiple of 32, <= 1024).  All threads
// receive the result.  `red` is shared scratch of >= 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = (lane < nw) ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  double out = red[32];
  __syncthreads();
  return out;
}

template <typename S>
__device__ __forceinline__ double to_d(S x) { return (double)x; }

// Sort key of a singular value or column norm: NaN ranks below every number, so that ranks by
// decreasing key with ties broken by index always form a permutation (a non-finite input then
// still gives in-range indices; its status is latched where the value is formed).
__device__ __forceinline__ double rank_key(double v) { return (v == v) ? v : -INFINITY; }

// Argument checks of a tensor descriptor (d, dtype, capacities, non-null cores) and of two
// descriptors with equal mode sizes and dtype, shared by every entry point.
tt_status check_tensor(const tt_tensor* x);
tt_status same_modes(const tt_tensor* a, const tt_tensor* b);

// Unique id of the CUDA context current on the calling thread (0 when none is current).
unsigned long long current_context_id();
// Allow `bytes` of dynamic shared memory per CTA for kernel `func` (the opt-in above 48 KB),
// never lowering an earlier setting.  TT_ERR_CUDA if the runtime refuses, TT_ERR_UNSUPPORTED
// above the device's opt-in maximum.  Every launch site above 48 KB calls it and returns its
// status, so a refused attribute never reaches a launch (or a captured graph node).
tt_status smem_optin_impl(const void* func, size_t bytes);
template <class F>
inline tt_status smem_optin(F* func, size_t bytes) {
  return smem_optin_impl(reinterpret_cast<const void*>(func), bytes);
}

}  // namespace ttk

// Host-side context and plan (defined here so every translation unit sees one layout).
struct tt_context {
  int device;
  cudaStream_t stream;
  void* ws;
  size_t ws_bytes;
  ttk::DevCtrl* ctrl;  // device
  int num_sms;
  int smem_optin;
  void* instr;  // ttk::Instr, opt-in counters and kernel timers
  int coop_grid_max;  // > 0: cap on the CTAs of a cooperative launch (concurrent streams)
  int tsqr_leaf_cap;  // > 0: cap on the TSQR leaves over the merged core (batched problems)
  int rounding;       // tt_rounding of tt_round / tt_step
  const double* sketch;  // randomized rounding: omega (sketch_nang x sketch_ell, device, caller-owned)
  int sketch_nang, sketch_ell;
  void* tune;  // ttk::TsqrTune, TSQR kernel choice per shape (owned; batch views share it)
  int graphs;        // tt_step replays a captured CUDA graph of the step (tt_context_set_graphs)
  void* step_graph;  // the captured step and what it depends on (owned; not shared by batch views)
  long graph_replays, graph_captures, graph_failures;  // since the last diagnostics reset
  int tensor_cores;  // the call in progress runs TT_PREC_MIXED_3XTF32 (tensor-core contractions)
};

struct tt_plan {
  tt_context* ctx;
  unsigned long long serial;  // unique per created plan (a plan at a reused address differs)
  int ndim, nx, ny, nz, G, quad, ntheta, nphi;
  int d;          // TT cores: 2 (slab) or 3
  int n1, n2;     // angular mode sizes (n2 = 1 when d = 2)
  long nrow;      // N_Z
  double lam[3], c, dt, dV;
  int nterm;                    // 2 d_X (upwind, Rusanov) or d_X (central)
  int term_axis[ttk::kMaxTerms], term_w[ttk::kMaxTerms];
  int nbc;                      // operators whose upwind face has inflow
  int bc_term[ttk::kMaxTerms];  // operator index of each inflow column
  long stride[3];
  int ext[3];
  // device arrays owned by the plan
  double* eps;     // [N_Z]
  double* acoef;   // [N_Z] c dt rho kappa_a
  double* scoef;   // [N_Z] c dt rho kappa_s
  double* domega;  // [n1*n2]
  double* mu;      // [ntheta]
  double* phi;     // [nphi]
  double* fac1;    // [nterm][n1] angular factor on core 1
  double* fac2;    // [nterm][n2] angular factor on core 2 (ones when d = 2)
  double* inflow;  // [6][G] inflow spectra (0 for vacuum)
  double* bcval;   // [nbc][G] signed lambda * inflow spectrum of each inflow column
  double* edges;   // [G+1]
  int* bc_term_dev;  // [kMaxTerms] operator index of each inflow column
  double a_rad;
  int coupled;       // material temperature advanced by tt_step (Sec. 2.1, Eq. Tupdate)
  double* temp;      // [N_X] material temperature (coupled: state, else the fixed input)
  double* rho_cv;    // [N_X] volumetric heat capacity (coupled only)
  double* tdag;      // [N_X] T^dagger of the last step (coupled only)
};

// Internal entry points shared between translation units.
namespace ttk {
tt_status physics_setup(tt_context* ctx, const tt_problem* prob, tt_plan* plan);
// Coupled temperature (physics.cu): T^dagger per cell from J* per row, writing plan->tdag and
// epsilon(T^dagger) into plan->eps; then T^{m+1} from J* and the rounded state's J^{m+1}.
tt_status coupled_t_dagger(cudaStream_t s, tt_plan* p, const double* jstar);
tt_status coupled_t_update(cudaStream_t s, tt_plan* p, const double* jstar, const double* jnew);
}
