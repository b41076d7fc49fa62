// Opt-in instrumentation of a context: launch counts per category and CUDA-event timing of
// the hot kernels on the context stream.  Set per ABI call through a thread-local pointer.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace ttk {

enum TimerCat { kTsqrLeaf = 0, kTsqrMerge = 1, kSmall = 2, kUpdate = 3, kOther = 4, kTsqrLeafSrc = 5, kUpdateSrc = 6,
                kNumCat = 7 };

struct Instr {
  bool timing = false;
  long launches[kNumCat] = {};
  int active = -1;  // category of the open scope (scopes do not nest)
  struct Rec {
    int cat;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  cudaEvent_t take_event() {
    if (pool_used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[pool_used++];
  }
};

extern thread_local Instr* g_instr;

inline void count_launch(int n = 1) {
  if (g_instr) g_instr->launches[g_instr->active >= 0 ? g_instr->active : kOther] += n;
}

struct TimerScope {
  Instr* in;
  cudaStream_t s;
  bool own;
  Instr::Rec rec;
  TimerScope(int cat, cudaStream_t stream) : in(g_instr), s(stream), own(false) {
    if (!in || in->active >= 0) return;
    in->active = cat;
    own = true;
    rec.cat = cat;
    if (in->timing) {
      rec.a = in->take_event();
      rec.b = in->take_event();
      cudaEventRecord(rec.a, s);
    }
  }
  ~TimerScope() {
    if (!own) return;
    if (in->timing) {
      cudaEventRecord(rec.b, s);
      in->recs.push_back(rec);
    }
    in->active = -1;
  }
};

}  // namespace ttk
