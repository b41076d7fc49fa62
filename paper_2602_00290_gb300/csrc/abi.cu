// C ABI of the library (declared in include/tt.h): argument checks, context and plan
// lifetime, workspace sizing, dtype dispatch.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include <atomic>

#include "common.cuh"
#include "instr.cuh"
#include "small.cuh"
#include "step.cuh"
#include "tune.cuh"

namespace ttk {
thread_local Instr* g_instr = nullptr;

tt_status check_tensor(const tt_tensor* x) {
  if (!x || !x->rank) return TT_ERR_ARG;
  if (x->d != 2 && x->d != 3) return TT_ERR_UNSUPPORTED;
  if (x->dtype != TT_F64 && x->dtype != TT_F32) return TT_ERR_ARG;
  if (x->rcap[0] != 1 || x->rcap[x->d] != 1) return TT_ERR_SHAPE;
  for (int j = 0; j < x->d; ++j) {
    if (x->n[j] <= 0 || x->rcap[j + 1] <= 0 || !x->core[j]) return TT_ERR_SHAPE;
  }
  return TT_OK;
}

tt_status same_modes(const tt_tensor* a, const tt_tensor* b) {
  if (a->d != b->d || a->dtype != b->dtype) return TT_ERR_SHAPE;
  for (int j = 0; j < a->d; ++j)
    if (a->n[j] != b->n[j]) return TT_ERR_SHAPE;
  return TT_OK;
}
}  // namespace ttk

namespace {

using ttk::check_tensor;
using ttk::same_modes;

struct InstrGuard {
  ttk::Instr* prev;
  explicit InstrGuard(tt_context* ctx) : prev(ttk::g_instr) { ttk::g_instr = static_cast<ttk::Instr*>(ctx->instr); }
  ~InstrGuard() { ttk::g_instr = prev; }
};

tt_status check_plan_tensor(const tt_plan* p, const tt_tensor* x) {
  if (!p) return TT_ERR_ARG;
  if (x->d != p->d || x->n[0] != p->nrow || x->n[1] != p->n1) return TT_ERR_SHAPE;
  if (x->d == 3 && x->n[2] != p->n2) return TT_ERR_SHAPE;
  return TT_OK;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
  return cs != cudaStreamCaptureStatusNone;
}

tt_status ensure_ws(tt_context* ctx, size_t need) {
  if (need <= ctx->ws_bytes) return TT_OK;
  if (capturing(ctx->stream)) return TT_ERR_WORKSPACE;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  if (cudaMalloc(&ctx->ws, need) != cudaSuccess) return TT_ERR_CUDA;
  ctx->ws_bytes = need;
  return TT_OK;
}

// Run `fn(Bump&)` once as a dry run to size the workspace, then for real.
template <class F>
tt_status with_ws(tt_context* ctx, F&& fn) {
  InstrGuard guard(ctx);
  ttk::Bump dry{nullptr, 0, 0, true};
  tt_status st = fn(dry);
  if (st != TT_OK) return st;
  st = ensure_ws(ctx, dry.off);
  if (st != TT_OK) return st;
  ttk::Bump real{static_cast<char*>(ctx->ws), 0, ctx->ws_bytes, false};
  return fn(real);
}

int set_device(tt_context* ctx) { return cudaSetDevice(ctx->device) == cudaSuccess; }

std::atomic<unsigned long long> g_plan_serial{0};

// A captured tt_step and everything its launch sequence depends on: the plan, the state's
// pointers and capacities, the step arguments, the workspace and the context settings that
// choose kernels.  Device data (ranks, cores, plan arrays, material temperature) may change
// between replays; none of it is read by the host.
struct StepGraph {
  const tt_plan* plan = nullptr;
  unsigned long long plan_serial = 0;  // the plan's device arrays belong to this serial
  int d = 0;
  tt_dtype dtype = TT_F64;
  void* core[TT_MAX_CORES] = {};
  int32_t* rank = nullptr;
  int32_t rcap[TT_MAX_CORES + 1] = {};
  double tol = 0.0;
  int32_t rmax = 0;
  tt_precision prec = TT_PREC_FP64;
  double* energy = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int rounding = 0, sketch_nang = 0, sketch_ell = 0, coop_grid_max = 0, tsqr_leaf_cap = 0;
  const double* sketch = nullptr;
  unsigned long tune_epoch = 0;
  // result of the capture
  cudaGraphExec_t exec = nullptr;
  bool warmed = false;  // one eager step ran with this key (captured on the next call)
  bool failed = false;  // the step could not be captured: run it eagerly
  long launches[ttk::kNumCat] = {};

  static StepGraph of(const tt_context* ctx, const tt_plan* plan, const tt_tensor* I, double tol, int32_t rmax,
                      tt_precision prec, double* energy) {
    StepGraph g;
    g.plan = plan;
    g.plan_serial = plan->serial;
    g.d = I->d;
    g.dtype = I->dtype;
    for (int j = 0; j < TT_MAX_CORES; ++j) g.core[j] = (j < I->d) ? I->core[j] : nullptr;
    g.rank = I->rank;
    for (int j = 0; j <= TT_MAX_CORES; ++j) g.rcap[j] = (j <= I->d) ? I->rcap[j] : 0;
    g.tol = tol;
    g.rmax = rmax;
    g.prec = prec;
    g.energy = energy;
    g.ws = ctx->ws;
    g.ws_bytes = ctx->ws_bytes;
    g.rounding = ctx->rounding;
    g.sketch = ctx->sketch;
    g.sketch_nang = ctx->sketch_nang;
    g.sketch_ell = ctx->sketch_ell;
    g.coop_grid_max = ctx->coop_grid_max;
    g.tsqr_leaf_cap = ctx->tsqr_leaf_cap;
    g.tune_epoch = ttk::tune_of(ctx)->epoch;
    return g;
  }
  bool same(const StepGraph& o) const {
    if (plan != o.plan || plan_serial != o.plan_serial || d != o.d || dtype != o.dtype || rank != o.rank || tol != o.tol || rmax != o.rmax ||
        prec != o.prec || energy != o.energy || ws != o.ws || ws_bytes != o.ws_bytes || rounding != o.rounding ||
        sketch != o.sketch || sketch_nang != o.sketch_nang || sketch_ell != o.sketch_ell ||
        coop_grid_max != o.coop_grid_max || tsqr_leaf_cap != o.tsqr_leaf_cap || tune_epoch != o.tune_epoch)
      return false;
    for (int j = 0; j < TT_MAX_CORES; ++j)
      if (core[j] != o.core[j]) return false;
    for (int j = 0; j <= TT_MAX_CORES; ++j)
      if (rcap[j] != o.rcap[j]) return false;
    return true;
  }
};

void drop_step_graph(tt_context* ctx) {
  StepGraph* g = static_cast<StepGraph*>(ctx->step_graph);
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  ctx->step_graph = nullptr;
}

}  // namespace

extern "C" {

const char* tt_status_string(tt_status s) {
  switch (s) {
    case TT_OK: return "ok";
    case TT_ERR_ARG: return "invalid argument";
    case TT_ERR_SHAPE: return "incompatible shapes";
    case TT_ERR_CAPACITY: return "rank capacity exceeded";
    case TT_ERR_CUDA: return "CUDA runtime error";
    case TT_ERR_NONFINITE: return "non-finite value";
    case TT_ERR_TIMEOUT: return "bounded device wait gave up";
    case TT_ERR_UNSUPPORTED: return "unsupported request";
    case TT_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

tt_status tt_context_create(tt_context** out, int device, void* stream, size_t workspace_bytes) {
  if (!out) return TT_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return TT_ERR_CUDA;
  tt_context* ctx = new tt_context();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  ctx->instr = new ttk::Instr();
  ctx->coop_grid_max = 0;
  ctx->tsqr_leaf_cap = 0;
  ctx->rounding = TT_ROUND_TSQR;
  ctx->sketch = nullptr;
  ctx->sketch_nang = 0;
  ctx->sketch_ell = 0;
  ctx->tune = new ttk::TsqrTune();
  ctx->graphs = 0;
  ctx->step_graph = nullptr;
  ctx->graph_replays = ctx->graph_captures = ctx->graph_failures = 0;
  ctx->tensor_cores = 0;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (cudaMalloc((void**)&ctx->ctrl, sizeof(ttk::DevCtrl)) != cudaSuccess) {
    delete ttk::tune_of(ctx);
    delete static_cast<ttk::Instr*>(ctx->instr);
    delete ctx;
    return TT_ERR_CUDA;
  }
  cudaMemsetAsync(ctx->ctrl, 0, sizeof(ttk::DevCtrl), ctx->stream);
  if (workspace_bytes > 0 && ensure_ws(ctx, workspace_bytes) != TT_OK) {
    cudaFree(ctx->ctrl);
    delete ttk::tune_of(ctx);
    delete static_cast<ttk::Instr*>(ctx->instr);
    delete ctx;
    return TT_ERR_CUDA;
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaFree(ctx->ctrl);
    delete ttk::tune_of(ctx);
    delete static_cast<ttk::Instr*>(ctx->instr);
    delete ctx;
    return TT_ERR_CUDA;
  }
  *out = ctx;
  return TT_OK;
}

tt_status tt_context_destroy(tt_context* ctx) {
  if (!ctx) return TT_ERR_ARG;
  set_device(ctx);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->ws) cudaFree(ctx->ws);
  cudaFree(ctx->ctrl);
  ttk::Instr* in = static_cast<ttk::Instr*>(ctx->instr);
  for (cudaEvent_t e : in->pool) cudaEventDestroy(e);
  delete in;
  delete ttk::tune_of(ctx);
  drop_step_graph(ctx);
  delete ctx;
  return TT_OK;
}

tt_status tt_context_set_graphs(tt_context* ctx, int enable) {
  if (!ctx) return TT_ERR_ARG;
  set_device(ctx);
  ctx->graphs = (enable != 0);
  if (!ctx->graphs) {
    cudaStreamSynchronize(ctx->stream);
    drop_step_graph(ctx);
  }
  return TT_OK;
}

tt_status tt_context_set_sketch(tt_context* ctx, const double* omega_dev, int32_t nang, int32_t ell) {
  if (!ctx || !omega_dev || nang < 1 || ell < 1 || ell > 64) return TT_ERR_ARG;
  ctx->sketch = omega_dev;
  ctx->sketch_nang = nang;
  ctx->sketch_ell = ell;
  return TT_OK;
}

tt_status tt_context_set_rounding(tt_context* ctx, tt_rounding method) {
  if (!ctx || (method != TT_ROUND_TSQR && method != TT_ROUND_GRAM && method != TT_ROUND_RANDOMIZED))
    return TT_ERR_ARG;
  ctx->rounding = method;
  return TT_OK;
}

tt_status tt_context_set_timing(tt_context* ctx, int enable) {
  if (!ctx) return TT_ERR_ARG;
  static_cast<ttk::Instr*>(ctx->instr)->timing = (enable != 0);
  return TT_OK;
}

tt_status tt_context_counters(tt_context* ctx, double* ms, int64_t* launches, int reset) {
  if (!ctx) return TT_ERR_ARG;
  ttk::Instr* in = static_cast<ttk::Instr*>(ctx->instr);
  set_device(ctx);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  double acc[ttk::kNumCat] = {};
  for (const auto& r : in->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return TT_ERR_CUDA;
    acc[r.cat] += t;
  }
  for (int c = 0; c < ttk::kNumCat; ++c) {
    if (ms) ms[c] = acc[c];
    if (launches) launches[c] = in->launches[c];
  }
  if (reset) {
    in->recs.clear();
    in->pool_used = 0;
    for (int c = 0; c < ttk::kNumCat; ++c) in->launches[c] = 0;
  }
  return TT_OK;
}

tt_status tt_context_diagnostics(tt_context* ctx, int64_t* out, int n, int reset) {
  if (!ctx || (n > 0 && !out) || n < 0 || n > 6) return TT_ERR_ARG;
  set_device(ctx);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  int v[3] = {0, 0, 0};
  if (cudaMemcpy(v, &ctx->ctrl->jac_sweeps_max, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return TT_ERR_CUDA;
  const int64_t w[6] = {v[0], v[1], v[2], ctx->graph_replays, ctx->graph_captures, ctx->graph_failures};
  for (int i = 0; i < n; ++i) out[i] = w[i];
  if (reset) {
    if (cudaMemset(&ctx->ctrl->jac_sweeps_max, 0, sizeof(v)) != cudaSuccess) return TT_ERR_CUDA;
    ctx->graph_replays = ctx->graph_captures = ctx->graph_failures = 0;
  }
  return TT_OK;
}

tt_status tt_context_set_limits(tt_context* ctx, int32_t jacobi_sweeps, int64_t barrier_spins,
                                int32_t barrier_extra) {
  if (!ctx || jacobi_sweeps < 0 || barrier_spins < 0 || barrier_extra < 0) return TT_ERR_ARG;
  set_device(ctx);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  struct {
    int sweeps, extra;
    long long spins;
  } v{jacobi_sweeps, barrier_extra, (long long)barrier_spins};
  static_assert(offsetof(ttk::DevCtrl, barrier_extra) == offsetof(ttk::DevCtrl, jac_sweep_cap) + sizeof(int),
                "limit fields are contiguous");
  static_assert(offsetof(ttk::DevCtrl, spin_limit) == offsetof(ttk::DevCtrl, jac_sweep_cap) + 2 * sizeof(int),
                "limit fields are contiguous");
  if (cudaMemcpy(&ctx->ctrl->jac_sweep_cap, &v, sizeof(v), cudaMemcpyHostToDevice) != cudaSuccess) return TT_ERR_CUDA;
  return TT_OK;
}

tt_status tt_sync(tt_context* ctx) {
  if (!ctx) return TT_ERR_ARG;
  set_device(ctx);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, &ctx->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TT_ERR_CUDA;
  if (st != 0) cudaMemset(&ctx->ctrl->status, 0, sizeof(int));
  if (cudaGetLastError() != cudaSuccess) return TT_ERR_CUDA;
  return static_cast<tt_status>(st);
}

tt_status tt_plan_create(tt_context* ctx, const tt_problem* prob, tt_plan** out) {
  if (!ctx || !prob || !out) return TT_ERR_ARG;
  *out = nullptr;
  if (prob->ndim_x < 1 || prob->ndim_x > 3) return TT_ERR_ARG;
  if (prob->ngroup < 1 || prob->nx < 1 || prob->ny < 1 || prob->nz < 1 || prob->ntheta < 1 || prob->nphi < 1)
    return TT_ERR_ARG;
  if (prob->ndim_x == 1 && (prob->quadrature != TT_QUAD_GAUSS_LEGENDRE_MU || prob->ny != 1 || prob->nz != 1))
    return TT_ERR_UNSUPPORTED;
  if (prob->ndim_x >= 2 && prob->quadrature != TT_QUAD_LATLONG_MIDPOINT) return TT_ERR_UNSUPPORTED;
  if (prob->ndim_x == 2 && prob->nz != 1) return TT_ERR_ARG;
  if (!prob->group_edges || !prob->temperature || !prob->rho_kappa_a || !prob->rho_kappa_s) return TT_ERR_ARG;
  if (!(prob->c > 0) || !(prob->dt > 0) || !(prob->dx > 0)) return TT_ERR_ARG;
  if (prob->ndim_x >= 2 && !(prob->dy > 0)) return TT_ERR_ARG;
  if (prob->ndim_x >= 3 && !(prob->dz > 0)) return TT_ERR_ARG;
  if (prob->flux != TT_FLUX_UPWIND && prob->flux != TT_FLUX_RUSANOV && prob->flux != TT_FLUX_CENTRAL)
    return TT_ERR_ARG;
  if (prob->topology != TT_TOPO_MERGED && prob->topology != TT_TOPO_MERGED_NUX_Y && prob->topology != TT_TOPO_SPLIT_X)
    return TT_ERR_ARG;
  if (prob->topology != TT_TOPO_MERGED) return TT_ERR_UNSUPPORTED;  // the d = 4 layouts are not built
  if (prob->flux != TT_FLUX_UPWIND)
    for (int f = 0; f < 2 * prob->ndim_x; ++f)
      if (prob->inflow_temperature[f] >= 0.0) return TT_ERR_UNSUPPORTED;
  set_device(ctx);
  tt_plan* p = new tt_plan();
  std::memset(p, 0, sizeof(tt_plan));
  p->ctx = ctx;
  p->serial = g_plan_serial.fetch_add(1) + 1;
  tt_status st = ttk::physics_setup(ctx, prob, p);
  if (st != TT_OK) {
    tt_plan_destroy(p);
    return st;
  }
  *out = p;
  return TT_OK;
}

tt_status tt_plan_destroy(tt_plan* p) {
  if (!p) return TT_ERR_ARG;
  double* arrs[] = {p->eps,    p->acoef,  p->scoef, p->domega, p->mu,     p->phi,  p->fac1,
                    p->fac2,   p->inflow, p->bcval, p->edges,  p->temp,   p->rho_cv, p->tdag};
  for (double* a : arrs)
    if (a) cudaFree(a);
  if (p->bc_term_dev) cudaFree(p->bc_term_dev);
  delete p;
  return TT_OK;
}

tt_status tt_plan_array(const tt_plan* p, int which, const double** ptr, int64_t* len) {
  if (!p || !ptr || !len) return TT_ERR_ARG;
  switch (which) {
    case 0: *ptr = p->eps; *len = p->nrow; break;
    case 1: *ptr = p->domega; *len = (int64_t)p->n1 * p->n2; break;
    case 2: *ptr = p->mu; *len = p->ntheta; break;
    case 3: *ptr = p->phi; *len = p->nphi; break;
    case 4: *ptr = p->acoef; *len = p->nrow; break;
    case 5: *ptr = p->scoef; *len = p->nrow; break;
    case 6: *ptr = p->inflow; *len = 6 * (int64_t)p->G; break;
    case 7: *ptr = p->temp; *len = (int64_t)p->nx * p->ny * p->nz; break;
    case 8:
      if (!p->coupled) return TT_ERR_ARG;
      *ptr = p->tdag; *len = (int64_t)p->nx * p->ny * p->nz; break;
    default: return TT_ERR_ARG;
  }
  return TT_OK;
}

tt_status tt_axpy(tt_context* ctx, double alpha, const tt_tensor* x, tt_tensor* y) {
  if (!ctx) return TT_ERR_ARG;
  tt_status st = check_tensor(x);
  if (st == TT_OK) st = check_tensor(y);
  if (st == TT_OK) st = same_modes(x, y);
  if (st != TT_OK) return st;
  if (!std::isfinite(alpha)) return TT_ERR_ARG;
  set_device(ctx);
  InstrGuard guard(ctx);
  return (x->dtype == TT_F64) ? ttk::axpy_impl<double>(ctx, alpha, x, y) : ttk::axpy_impl<float>(ctx, alpha, x, y);
}

tt_status tt_dot(tt_context* ctx, const tt_tensor* x, const tt_tensor* y, double* out_dev) {
  if (!ctx || !out_dev) return TT_ERR_ARG;
  tt_status st = check_tensor(x);
  if (st == TT_OK) st = check_tensor(y);
  if (st == TT_OK) st = same_modes(x, y);
  if (st != TT_OK) return st;
  set_device(ctx);
  return with_ws(ctx, [&](ttk::Bump& ws) {
    return (x->dtype == TT_F64) ? ttk::dot_impl<double>(ctx, x, y, out_dev, ws)
                                : ttk::dot_impl<float>(ctx, x, y, out_dev, ws);
  });
}

static tt_status check_round_args(const tt_tensor* x, double tol, int32_t rmax, tt_precision prec) {
  if (!(tol >= 0.0) || !std::isfinite(tol)) return TT_ERR_ARG;
  if (rmax < 1) return TT_ERR_ARG;
  if (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED && prec != TT_PREC_MIXED_3XTF32) return TT_ERR_ARG;
  for (int j = 1; j < x->d; ++j)
    if (rmax > x->rcap[j]) return TT_ERR_CAPACITY;
  return TT_OK;
}

tt_status tt_round(tt_context* ctx, tt_tensor* x, double tol, int32_t rmax, tt_precision prec) {
  if (!ctx) return TT_ERR_ARG;
  tt_status st = check_tensor(x);
  if (st == TT_OK) st = check_round_args(x, tol, rmax, prec);
  if (st != TT_OK) return st;
  set_device(ctx);
  ctx->tensor_cores = (prec == TT_PREC_MIXED_3XTF32);
  return with_ws(ctx, [&](ttk::Bump& ws) {
    const bool f64 = (x->dtype == TT_F64), mixed = (prec != TT_PREC_FP64);
    if (f64) return mixed ? ttk::round_impl<double, float>(ctx, x, tol, rmax, ws)
                          : ttk::round_impl<double, double>(ctx, x, tol, rmax, ws);
    return mixed ? ttk::round_impl<float, float>(ctx, x, tol, rmax, ws)
                 : ttk::round_impl<float, double>(ctx, x, tol, rmax, ws);
  });
}

tt_status tt_apply_transport(tt_context* ctx, const tt_plan* plan, const tt_tensor* in, tt_tensor* out) {
  if (!ctx || !plan) return TT_ERR_ARG;
  tt_status st = check_tensor(in);
  if (st == TT_OK) st = check_tensor(out);
  if (st == TT_OK) st = same_modes(in, out);
  if (st == TT_OK) st = check_plan_tensor(plan, in);
  if (st != TT_OK) return st;
  if (in->core[0] == out->core[0]) return TT_ERR_ARG;
  set_device(ctx);
  InstrGuard guard(ctx);
  return (in->dtype == TT_F64) ? ttk::apply_transport_impl<double>(ctx, plan, in, out)
                               : ttk::apply_transport_impl<float>(ctx, plan, in, out);
}

tt_status tt_step(tt_context* ctx, const tt_plan* plan, tt_tensor* I, double tol, int32_t rmax, tt_precision prec,
                  double* energy_dev) {
  if (!ctx || !plan) return TT_ERR_ARG;
  tt_status st = check_tensor(I);
  if (st == TT_OK) st = check_plan_tensor(plan, I);
  if (st == TT_OK) st = check_round_args(I, tol, rmax, prec);
  if (st != TT_OK) return st;
  set_device(ctx);
  ctx->tensor_cores = (prec == TT_PREC_MIXED_3XTF32);
  auto body = [&](ttk::Bump& ws) {
    const bool f64 = (I->dtype == TT_F64), mixed = (prec != TT_PREC_FP64);
    if (f64) return mixed ? ttk::step_impl<double, float>(ctx, plan, I, tol, rmax, energy_dev, ws)
                          : ttk::step_impl<double, double>(ctx, plan, I, tol, rmax, energy_dev, ws);
    return mixed ? ttk::step_impl<float, float>(ctx, plan, I, tol, rmax, energy_dev, ws)
                 : ttk::step_impl<float, double>(ctx, plan, I, tol, rmax, energy_dev, ws);
  };
  ttk::Instr* in = static_cast<ttk::Instr*>(ctx->instr);
  if (!ctx->graphs || (in && in->timing) || capturing(ctx->stream)) return with_ws(ctx, body);
  // Graph replay: size the workspace outside any capture, then replay the step captured for
  // the same key, or capture it now (the capture runs no kernel; launching the graph does).
  {
    InstrGuard guard(ctx);
    ttk::Bump dry{nullptr, 0, 0, true};
    st = body(dry);
    if (st != TT_OK) return st;
    st = ensure_ws(ctx, dry.off);
    if (st != TT_OK) return st;
  }
  const StepGraph key = StepGraph::of(ctx, plan, I, tol, rmax, prec, energy_dev);
  StepGraph* g = static_cast<StepGraph*>(ctx->step_graph);
  if (!g || !g->same(key)) {
    // A new key steps eagerly once: every kernel of the step is then loaded and has its
    // shared-memory limit set outside any capture, and the capture (next call) records only
    // launches whose configuration already launched successfully.
    drop_step_graph(ctx);
    g = new StepGraph(key);
    ctx->step_graph = g;
    return with_ws(ctx, body);
  }
  if (!g->warmed) {
    g->warmed = true;
    long before[ttk::kNumCat] = {};
    if (in)
      for (int c = 0; c < ttk::kNumCat; ++c) before[c] = in->launches[c];
    // capture on a private stream (the context's may be the legacy default stream, which
    // cannot be captured); the graph is launched on the context's stream
    cudaGraph_t graph = nullptr;
    tt_status cst = TT_ERR_CUDA;
    cudaStream_t own = ctx->stream, cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess) {
      ctx->stream = cap;
      if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        {
          InstrGuard guard(ctx);
          ttk::Bump real{static_cast<char*>(ctx->ws), 0, ctx->ws_bytes, false};
          cst = body(real);
        }
        if (cudaStreamEndCapture(cap, &graph) != cudaSuccess) cst = TT_ERR_CUDA;
      }
      ctx->stream = own;
      cudaStreamDestroy(cap);
    }
    if (cst == TT_OK && graph && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
      g->exec = nullptr;
      cst = TT_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    if (in)
      for (int c = 0; c < ttk::kNumCat; ++c) {
        g->launches[c] = in->launches[c] - before[c];
        in->launches[c] = before[c];  // counted again below, per launch of the step
      }
    ++ctx->graph_captures;
    if (cst != TT_OK || !g->exec) {
      (void)cudaGetLastError();  // the refused capture leaves nothing behind; run the step eagerly
      g->failed = true;
      ++ctx->graph_failures;
    }
  }
  if (g->failed) return with_ws(ctx, body);
  if (cudaGraphLaunch(g->exec, ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  ++ctx->graph_replays;
  if (in)
    for (int c = 0; c < ttk::kNumCat; ++c) in->launches[c] += g->launches[c];
  return TT_OK;
}

tt_status tt_internal_ranks(tt_context* ctx, const tt_plan* plan, const tt_tensor* x, double delta_rel,
                            int32_t* ranks, double* sigma_nu, int64_t nsigma_nu, double* sigma_x, int64_t nsigma_x) {
  if (!ctx || !plan || !ranks || !(delta_rel >= 0.0) || nsigma_nu < 0 || nsigma_x < 0) return TT_ERR_ARG;
  tt_status st = check_tensor(x);
  if (st == TT_OK) st = check_plan_tensor(plan, x);
  if (st != TT_OK) return st;
  set_device(ctx);
  int r[2] = {0, 0};
  st = with_ws(ctx, [&](ttk::Bump& ws) {
    return (x->dtype == TT_F64) ? ttk::internal_ranks_impl<double>(ctx, plan, x, delta_rel, r, sigma_nu, nsigma_nu,
                                                                   sigma_x, nsigma_x, ws)
                                : ttk::internal_ranks_impl<float>(ctx, plan, x, delta_rel, r, sigma_nu, nsigma_nu,
                                                                  sigma_x, nsigma_x, ws);
  });
  ranks[0] = r[0];
  ranks[1] = r[1];
  if (st != TT_OK) return st;
  // synchronous: report (and clear) what the analysis latched on the device, e.g. a Jacobi sweep
  // cap reached on a Gram matrix with many eigenvalues at round-off level (ranks still written)
  int dst = 0;
  if (cudaMemcpy(&dst, &ctx->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TT_ERR_CUDA;
  if (dst != 0 && cudaMemset(&ctx->ctrl->status, 0, sizeof(int)) != cudaSuccess) return TT_ERR_CUDA;
  return static_cast<tt_status>(dst);
}

tt_status tt_energy_density(tt_context* ctx, const tt_plan* plan, const tt_tensor* x, double* out_dev) {
  if (!ctx || !plan || !out_dev) return TT_ERR_ARG;
  tt_status st = check_tensor(x);
  if (st == TT_OK) st = check_plan_tensor(plan, x);
  if (st != TT_OK) return st;
  set_device(ctx);
  return with_ws(ctx, [&](ttk::Bump& ws) {
    return (x->dtype == TT_F64) ? ttk::energy_density_impl<double>(ctx, plan, x, out_dev, ws)
                                : ttk::energy_density_impl<float>(ctx, plan, x, out_dev, ws);
  });
}

tt_status tt_workspace_query(tt_context* ctx, const tt_plan* plan, const tt_tensor* x, tt_precision prec,
                             size_t* bytes) {
  if (!ctx || !x || !bytes) return TT_ERR_ARG;
  tt_status st = check_tensor(x);
  if (st != TT_OK) return st;
  ttk::Bump dry{nullptr, 0, 0, true};
  tt_tensor tmp = *x;
  if (plan) {
    st = check_plan_tensor(plan, x);
    if (st != TT_OK) return st;
    if (prec != TT_PREC_FP64)
      st = (x->dtype == TT_F64) ? ttk::step_impl<double, float>(ctx, plan, &tmp, 1e-6, 1, nullptr, dry)
                                : ttk::step_impl<float, float>(ctx, plan, &tmp, 1e-6, 1, nullptr, dry);
    else
      st = (x->dtype == TT_F64) ? ttk::step_impl<double, double>(ctx, plan, &tmp, 1e-6, 1, nullptr, dry)
                                : ttk::step_impl<float, double>(ctx, plan, &tmp, 1e-6, 1, nullptr, dry);
  } else {
    if (prec != TT_PREC_FP64)
      st = (x->dtype == TT_F64) ? ttk::round_impl<double, float>(ctx, &tmp, 1e-6, 1, dry)
                                : ttk::round_impl<float, float>(ctx, &tmp, 1e-6, 1, dry);
    else
      st = (x->dtype == TT_F64) ? ttk::round_impl<double, double>(ctx, &tmp, 1e-6, 1, dry)
                                : ttk::round_impl<float, double>(ctx, &tmp, 1e-6, 1, dry);
  }
  *bytes = dry.off;
  return st;
}

}  // extern "C"
