// Batched time stepping of independent problems (many TT states with their own plans, ranks,
// tolerances and shapes).  Each problem runs the same launch sequence as tt_step on its own
// control block and workspace region; problems are spread over a pool of streams (largest
// first onto the least-loaded stream) so that their latency-bound small-core phases overlap,
// and the whole batched step is captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "instr.cuh"
#include "step.cuh"

struct tt_batch {
  tt_context* ctx;
  int nprob;
  tt_precision prec;
  std::vector<const tt_plan*> plans;
  std::vector<tt_tensor> states;  // copies of the callers' descriptors (device memory stays theirs)
  std::vector<double> tol;
  std::vector<int> rmax;
  std::vector<size_t> ws_off, ws_len;
  std::vector<int> stream_of;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork;
  cudaStream_t origin;  // capture origin (the context stream may be the legacy default stream)
  std::vector<tt_context> sub;  // per-problem views of the context
  ttk::DevCtrl* ctrls;
  void* ws;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool warmed;  // the first batched step ran eagerly (the graph is captured at the next one)
  cudaEvent_t pre, post;  // order the eager step after / before the context stream's work
  ttk::Instr counts;  // launch counts of the captured step (timing off)
};

namespace {

tt_status step_dispatch(tt_context* c, const tt_plan* p, tt_tensor* I, double tol, int rmax, tt_precision prec,
                        ttk::Bump& ws) {
  const bool f64 = (I->dtype == TT_F64), mixed = (prec != TT_PREC_FP64);
  c->tensor_cores = (prec == TT_PREC_MIXED_3XTF32);
  if (f64) return mixed ? ttk::step_impl<double, float>(c, p, I, tol, rmax, nullptr, ws)
                        : ttk::step_impl<double, double>(c, p, I, tol, rmax, nullptr, ws);
  return mixed ? ttk::step_impl<float, float>(c, p, I, tol, rmax, nullptr, ws)
               : ttk::step_impl<float, double>(c, p, I, tol, rmax, nullptr, ws);
}

void release(tt_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->pre) cudaEventDestroy(b->pre);
  if (b->post) cudaEventDestroy(b->post);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->ws) cudaFree(b->ws);
  if (b->ctrls) cudaFree(b->ctrls);
  for (cudaEvent_t e : b->counts.pool) cudaEventDestroy(e);
  delete b;
}

// Issue one batched step on the origin stream (fork into the pool, join back).
tt_status issue_step(tt_batch* b) {
  if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) return TT_ERR_CUDA;
  for (cudaStream_t s : b->streams)
    if (cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) return TT_ERR_CUDA;
  ttk::Instr* prev = ttk::g_instr;
  ttk::g_instr = &b->counts;
  tt_status st = TT_OK;
  for (int i = 0; i < b->nprob && st == TT_OK; ++i) {
    ttk::Bump ws{static_cast<char*>(b->ws) + b->ws_off[i], 0, b->ws_len[i], false};
    st = step_dispatch(&b->sub[i], b->plans[i], &b->states[i], b->tol[i], b->rmax[i], b->prec, ws);
  }
  ttk::g_instr = prev;
  for (size_t k = 0; k < b->streams.size(); ++k) {
    if (cudaEventRecord(b->joins[k], b->streams[k]) != cudaSuccess) return TT_ERR_CUDA;
    if (cudaStreamWaitEvent(b->origin, b->joins[k], 0) != cudaSuccess) return TT_ERR_CUDA;
  }
  return st;
}

}  // namespace

extern "C" {

tt_status tt_batch_create(tt_context* ctx, int32_t nprob, const tt_plan* const* plans, const tt_tensor* states,
                          const double* tol, const int32_t* rmax, tt_precision prec, int32_t nstreams,
                          tt_batch** out) {
  if (!ctx || !out || nprob < 1 || !plans || !states || !tol || !rmax) return TT_ERR_ARG;
  if (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED && prec != TT_PREC_MIXED_3XTF32) return TT_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return TT_ERR_CUDA;
  for (int i = 0; i < nprob; ++i) {
    const tt_tensor* x = &states[i];
    const tt_plan* p = plans[i];
    if (!p || !x->rank) return TT_ERR_ARG;
    if (x->d != p->d || x->n[0] != p->nrow || x->n[1] != p->n1 || (x->d == 3 && x->n[2] != p->n2))
      return TT_ERR_SHAPE;
    if (x->dtype != TT_F64 && x->dtype != TT_F32) return TT_ERR_ARG;
    if (!(tol[i] >= 0.0) || rmax[i] < 1) return TT_ERR_ARG;
    for (int j = 1; j < x->d; ++j)
      if (rmax[i] > x->rcap[j]) return TT_ERR_CAPACITY;
  }
  tt_batch* b = new tt_batch();
  b->ctx = ctx;
  b->nprob = nprob;
  b->prec = prec;
  b->plans.assign(plans, plans + nprob);
  b->states.assign(states, states + nprob);
  b->tol.assign(tol, tol + nprob);
  b->rmax.assign(rmax, rmax + nprob);
  b->fork = nullptr;
  b->origin = nullptr;
  b->ctrls = nullptr;
  b->ws = nullptr;
  b->graph = nullptr;
  b->exec = nullptr;
  b->warmed = false;
  b->pre = nullptr;
  b->post = nullptr;
  if (cudaEventCreateWithFlags(&b->pre, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->post, cudaEventDisableTiming) != cudaSuccess) {
    release(b);
    return TT_ERR_CUDA;
  }
  // streams: at most one per problem
  // default pool: 128 streams.  A problem's step is a latency-bound chain (its small-core kernels
  // hold one SM each), so the batch step is about (problems per stream) x (one problem's chain):
  // measured on the 256-problem batch, 16 -> 128 streams took a step from 42.7 to 12.7 ms (cells
  // and groups / 4) and from 3.86 to 1.84 s (full size); 256 streams were no faster.
  int ns = nstreams > 0 ? nstreams : 128;
  if (ns > nprob) ns = nprob;
  for (int k = 0; k < ns; ++k) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { release(b); return TT_ERR_CUDA; }
    b->streams.push_back(s);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { release(b); return TT_ERR_CUDA; }
    b->joins.push_back(e);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) { release(b); return TT_ERR_CUDA; }
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess) { release(b); return TT_ERR_CUDA; }
  if (cudaMalloc((void**)&b->ctrls, sizeof(ttk::DevCtrl) * (size_t)nprob) != cudaSuccess) { release(b); return TT_ERR_CUDA; }
  if (cudaMemsetAsync(b->ctrls, 0, sizeof(ttk::DevCtrl) * (size_t)nprob, ctx->stream) != cudaSuccess) {
    release(b);
    return TT_ERR_CUDA;
  }
  // problems, largest first, onto the least-loaded stream; cost ~ rows x (5 rcap)^2
  std::vector<int> order(nprob);
  std::vector<double> cost(nprob);
  for (int i = 0; i < nprob; ++i) {
    order[i] = i;
    const double R1 = 5.0 * b->states[i].rcap[1];
    cost[i] = (double)b->states[i].n[0] * R1 * R1;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<double> load(ns, 0.0);
  b->stream_of.assign(nprob, 0);
  for (int i : order) {
    int best = 0;
    for (int k = 1; k < ns; ++k)
      if (load[k] < load[best]) best = k;
    b->stream_of[i] = best;
    load[best] += cost[i];
  }
  // per-problem views of the context: own stream, control block and workspace region; the
  // cooperative Jacobi runs as one CTA so that concurrent problems never wait on each other
  b->sub.assign(nprob, *ctx);
  b->ws_off.assign(nprob, 0);
  b->ws_len.assign(nprob, 0);
  size_t total = 0;
  double rows_all = 0.0;
  for (int i = 0; i < nprob; ++i) rows_all += (double)b->states[i].n[0];
  ttk::Instr* prev = ttk::g_instr;
  ttk::g_instr = &b->counts;
  for (int i = 0; i < nprob; ++i) {
    tt_context& c = b->sub[i];
    c.stream = b->streams[b->stream_of[i]];
    c.ctrl = b->ctrls + i;
    c.ws = nullptr;
    c.ws_bytes = 0;
    c.instr = &b->counts;
    c.coop_grid_max = 1;
    // TSQR leaves in proportion to the problem's share of the batch's rows (all problems run at
    // once): at least 8, at most the single-problem wave
    const double share = (double)b->states[i].n[0] / rows_all;
    int cap = (int)(share * 3.0 * ctx->num_sms + 0.5);
    c.tsqr_leaf_cap = cap < 8 ? 8 : cap;
    ttk::Bump dry{nullptr, 0, 0, true};
    tt_status st = step_dispatch(&c, b->plans[i], &b->states[i], b->tol[i], b->rmax[i], prec, dry);
    if (st != TT_OK) {
      ttk::g_instr = prev;
      release(b);
      return st;
    }
    b->ws_off[i] = total;
    b->ws_len[i] = dry.off;
    total += (dry.off + 255) & ~(size_t)255;
  }
  ttk::g_instr = prev;
  if (cudaMalloc(&b->ws, total > 0 ? total : 256) != cudaSuccess) { release(b); return TT_ERR_CUDA; }
  for (int i = 0; i < nprob; ++i) {
    b->sub[i].ws = static_cast<char*>(b->ws) + b->ws_off[i];
    b->sub[i].ws_bytes = b->ws_len[i];
  }
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { release(b); return TT_ERR_CUDA; }
  *out = b;
  return TT_OK;
}

tt_status tt_batch_step(tt_batch* b, int32_t nsteps) {
  if (!b || nsteps < 0) return TT_ERR_ARG;
  tt_context* ctx = b->ctx;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return TT_ERR_CUDA;
  if (!b->exec && !b->warmed && nsteps > 0) {
    // The first batched step runs eagerly: every kernel is loaded and has its shared-memory
    // limit set outside any capture; the graph is captured at the next step.
    b->warmed = true;
    if (cudaEventRecord(b->pre, ctx->stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->origin, b->pre, 0) != cudaSuccess)
      return TT_ERR_CUDA;
    long keep[ttk::kNumCat];
    for (int c = 0; c < ttk::kNumCat; ++c) keep[c] = b->counts.launches[c];
    const tt_status st = issue_step(b);
    for (int c = 0; c < ttk::kNumCat; ++c) b->counts.launches[c] = keep[c];  // not the captured step's
    if (cudaEventRecord(b->post, b->origin) != cudaSuccess || cudaStreamWaitEvent(ctx->stream, b->post, 0) != cudaSuccess)
      return TT_ERR_CUDA;
    if (st != TT_OK) return st;
    if (--nsteps == 0) return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  if (!b->exec && nsteps > 0) {
    b->counts.launches[ttk::kOther] = 0;
    for (int c = 0; c < ttk::kNumCat; ++c) b->counts.launches[c] = 0;
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TT_ERR_CUDA;
    tt_status st = issue_step(b);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->origin, &g);
    if (st != TT_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ce != cudaSuccess || !g) return TT_ERR_CUDA;
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      b->exec = nullptr;
      return TT_ERR_CUDA;
    }
  }
  for (int k = 0; k < nsteps; ++k)
    if (cudaGraphLaunch(b->exec, ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

tt_status tt_batch_sync(tt_batch* b, int32_t* status_out) {
  if (!b) return TT_ERR_ARG;
  tt_context* ctx = b->ctx;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return TT_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return TT_ERR_CUDA;
  std::vector<ttk::DevCtrl> h(b->nprob);
  if (cudaMemcpy(h.data(), b->ctrls, sizeof(ttk::DevCtrl) * (size_t)b->nprob, cudaMemcpyDeviceToHost) != cudaSuccess)
    return TT_ERR_CUDA;
  tt_status first = TT_OK;
  for (int i = 0; i < b->nprob; ++i) {
    if (status_out) status_out[i] = h[i].status;
    if (first == TT_OK && h[i].status != 0) first = static_cast<tt_status>(h[i].status);
  }
  return first;
}

tt_status tt_batch_info(const tt_batch* b, int64_t* launches_per_step, size_t* workspace_bytes, int32_t* nstreams) {
  if (!b) return TT_ERR_ARG;
  if (launches_per_step) {
    long n = 0;
    for (int c = 0; c < ttk::kNumCat; ++c) n += b->counts.launches[c];
    *launches_per_step = b->exec ? n : -1;
  }
  if (workspace_bytes) {
    size_t t = 0;
    for (int i = 0; i < b->nprob; ++i) t += (b->ws_len[i] + 255) & ~(size_t)255;
    *workspace_bytes = t;
  }
  if (nstreams) *nstreams = (int32_t)b->streams.size();
  return TT_OK;
}

tt_status tt_batch_destroy(tt_batch* b) {
  if (!b) return TT_ERR_ARG;
  cudaSetDevice(b->ctx->device);
  cudaStreamSynchronize(b->ctx->stream);
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  cudaStreamSynchronize(b->origin);
  release(b);
  return TT_OK;
}

}  // extern "C"
