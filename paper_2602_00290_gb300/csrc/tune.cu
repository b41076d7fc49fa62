// TSQR kernel choice per shape: explicit setting and autotuning by timing whole steps.
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tune.cuh"

namespace {

int esize_of(tt_precision prec) { return prec == TT_PREC_FP64 ? 8 : 4; }

// Default leaf wave of the passes over the merged core (the cap tsqr_cfg clamps to).
int default_wave(const tt_context* ctx, int esize) { return (esize == 8 ? 2 : 3) * ctx->num_sms; }

size_t core_bytes(const tt_tensor* x, int j) {
  return (size_t)x->rcap[j] * x->n[j] * x->rcap[j + 1] * (x->dtype == TT_F64 ? 8 : 4);
}

// Device copy of a tensor's cores and ranks (the autotuner steps it instead of the caller's).
struct Scratch {
  tt_tensor x{};
  std::vector<void*> bufs;
  ~Scratch() {
    for (void* p : bufs) cudaFree(p);
  }
  tt_status init(const tt_tensor* src) {
    x = *src;
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(int32_t) * (src->d + 1)) != cudaSuccess) return TT_ERR_CUDA;
    bufs.push_back(p);
    x.rank = static_cast<int32_t*>(p);
    for (int j = 0; j < src->d; ++j) {
      if (cudaMalloc(&p, core_bytes(src, j)) != cudaSuccess) return TT_ERR_CUDA;
      bufs.push_back(p);
      x.core[j] = p;
    }
    return TT_OK;
  }
  void load(const tt_tensor* src, cudaStream_t s) {
    cudaMemcpyAsync(x.rank, src->rank, sizeof(int32_t) * (src->d + 1), cudaMemcpyDeviceToDevice, s);
    for (int j = 0; j < src->d; ++j) cudaMemcpyAsync(x.core[j], src->core[j], core_bytes(src, j), cudaMemcpyDeviceToDevice, s);
  }
};

}  // namespace

extern "C" {

tt_status tt_context_set_tsqr(tt_context* ctx, tt_precision prec, int32_t ncap, int32_t variant, int32_t leaves) {
  if (!ctx || (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED && prec != TT_PREC_MIXED_3XTF32)) return TT_ERR_ARG;
  ttk::TsqrTune* tab = ttk::tune_of(ctx);
  if (ncap <= 0) {
    tab->m.clear();
    ++tab->epoch;
    return TT_OK;
  }
  if (variant < 0 || variant >= ttk::kTsqrVariants) return TT_ERR_ARG;
  tab->m[ttk::TsqrTune::key(esize_of(prec), ncap)] = ttk::TsqrCfg{variant, leaves > 0 ? leaves : 0};
  ++tab->epoch;
  return TT_OK;
}

tt_status tt_context_get_tsqr(const tt_context* ctx, tt_precision prec, int32_t ncap, int32_t* variant,
                              int32_t* leaves) {
  if (!ctx || ncap <= 0 || (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED && prec != TT_PREC_MIXED_3XTF32)) return TT_ERR_ARG;
  const int es = esize_of(prec);
  const ttk::TsqrCfg cfg = ttk::resolve_tsqr(ctx, es, ncap, default_wave(ctx, es));
  if (variant) *variant = cfg.variant;
  if (leaves) *leaves = cfg.leaves;
  return TT_OK;
}

tt_status tt_autotune(tt_context* ctx, const tt_plan* plan, const tt_tensor* I, double tol, int32_t rmax,
                      tt_precision prec, int32_t steps, int32_t* chosen, float* ms) {
  if (!ctx || !plan || !I || !I->rank || steps < 1 || steps > 64) return TT_ERR_ARG;
  if (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED && prec != TT_PREC_MIXED_3XTF32) return TT_ERR_ARG;
  if (ctx->rounding != TT_ROUND_TSQR) return TT_ERR_UNSUPPORTED;
  if (I->d != plan->d || I->n[0] != plan->nrow || I->rcap[1] <= 0) return TT_ERR_SHAPE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return TT_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return TT_ERR_ARG;
  cudaStream_t s = ctx->stream;
  const int es = esize_of(prec);
  const int K1 = I->rcap[1];
  const int ncaps[2] = {(plan->nterm + 1) * K1 + plan->nbc, K1 + 1};  // transport sum, source sum
  ttk::TsqrTune* tab = ttk::tune_of(ctx);
  const ttk::TsqrTune saved = *tab;

  Scratch sc;
  tt_status st = sc.init(I);
  if (st != TT_OK) return st;
  const long ncell = (long)plan->nx * plan->ny * plan->nz;
  double* temp0 = nullptr;
  if (plan->coupled) {
    if (cudaMalloc(&temp0, sizeof(double) * ncell) != cudaSuccess) return TT_ERR_CUDA;
    cudaMemcpyAsync(temp0, plan->temp, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, s);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);

  // One trial: the caller's state (and material temperature), one untimed step, `steps` timed.
  auto trial = [&](float* out) -> tt_status {
    sc.load(I, s);
    if (temp0) cudaMemcpyAsync(plan->temp, temp0, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, s);
    // two untimed steps: with step graphs on, the first steps eagerly and the second captures
    tt_status t = tt_step(ctx, plan, &sc.x, tol, rmax, prec, nullptr);
    if (t == TT_OK) t = tt_step(ctx, plan, &sc.x, tol, rmax, prec, nullptr);
    if (t != TT_OK) return t;
    cudaEventRecord(e0, s);
    for (int i = 0; i < steps && t == TT_OK; ++i) t = tt_step(ctx, plan, &sc.x, tol, rmax, prec, nullptr);
    cudaEventRecord(e1, s);
    if (t != TT_OK) return t;
    if (cudaEventSynchronize(e1) != cudaSuccess) return TT_ERR_CUDA;
    t = tt_sync(ctx);
    if (t != TT_OK) return t;
    float el = 0.0f;
    cudaEventElapsedTime(&el, e0, e1);
    *out = el / (float)steps;
    return TT_OK;
  };

  const int wave = default_wave(ctx, es);
  const int most = ttk::kTsqrMaxLeavesPerSm * ctx->num_sms;
  // leaf caps tried per variant (multiples of half the SM count): up to one default wave for
  // the column kernels, up to kTsqrMaxLeavesPerSm CTAs per SM for the row-split and dense column
  // kernels (measured: the 33-column row-split source leaf, six CTAs per SM, takes 0.39 ms at 912
  // leaves against 0.63 ms at 456)
  auto leaf_opts = [&](int v) {
    std::vector<int> o;
    for (int m : {1, 2, 3, 4, 6, 8, 12}) {
      const int l = m * ctx->num_sms / 2;
      const bool wide = (v == ttk::kTsqrColumnDense || v == ttk::kTsqrRowSplit);
      const int hi = wide ? most : (v == ttk::kTsqrBlocked) ? ctx->num_sms : wave;
      const int lo = (v == ttk::kTsqrColumnDense) ? ctx->num_sms : 8;
      if (l >= lo && l <= hi) o.push_back(l);
    }
    return o;
  };
  float base = 0.0f, best = 0.0f;
  int pick[2][2] = {{ttk::kTsqrColumn, wave}, {ttk::kTsqrColumn, wave}};
  for (int role = 0; role < 2; ++role) tab->m.erase(ttk::TsqrTune::key(es, ncaps[role]));
  ++tab->epoch;
  st = trial(&base);
  best = base;
  for (int role = 0; st == TT_OK && role < 2; ++role) {
    const long key = ttk::TsqrTune::key(es, ncaps[role]);
    for (int v = 0; st == TT_OK && v < ttk::kTsqrVariants; ++v) {
      tab->m[key] = ttk::TsqrCfg{v, wave};
      ++tab->epoch;
      if (ttk::resolve_tsqr(ctx, es, ncaps[role], wave).variant != v) continue;  // shape not taken by v
      for (int l : leaf_opts(v)) {
        if (v == ttk::kTsqrColumn && l == wave) continue;  // the default, timed as `base`
        tab->m[key] = ttk::TsqrCfg{v, l};
        ++tab->epoch;
        float t = 0.0f;
        st = trial(&t);
        if (st != TT_OK) break;
        if (t < best) {
          best = t;
          pick[role][0] = v;
          pick[role][1] = l;
        }
      }
    }
    tab->m[key] = ttk::TsqrCfg{pick[role][0], pick[role][1]};
    ++tab->epoch;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (temp0) {
    cudaMemcpyAsync(plan->temp, temp0, sizeof(double) * ncell, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    cudaFree(temp0);
  }
  cudaStreamSynchronize(s);
  if (st != TT_OK) {
    *tab = saved;
    return st;
  }
  if (chosen) {
    chosen[0] = pick[0][0];
    chosen[1] = pick[0][1];
    chosen[2] = pick[1][0];
    chosen[3] = pick[1][1];
  }
  if (ms) {
    ms[0] = base;
    ms[1] = best;
  }
  return TT_OK;
}

}  // extern "C"
