// Per-context choice of the TSQR over the merged core: which leaf/merge kernels (one thread
// per column, or QS lanes per column) and how many leaves, per (arithmetic, column count).
// Filled by tt_context_set_tsqr or tt_autotune; absent entries take the defaults.
#pragma once
#include <map>

#include "common.cuh"

namespace ttk {

// kTsqrColumn: one thread per column over 64-row (FP32) / 32-row (FP64) blocks, default
// residency; kTsqrRowSplit: four lanes per column; kTsqrColumnDense: FP32 only, one thread per
// column over 32-row blocks with registers held to four resident CTAs per SM (passes of at most
// 160 columns; otherwise the column kernels run); kTsqrBlocked: FP32 only, 256-row blocks held in
// tensor memory, 32-column panels and compact-WY trailing updates, one CTA per SM (passes of at
// most 224 columns).
enum TsqrVariant : int { kTsqrColumn = 0, kTsqrRowSplit = 1, kTsqrColumnDense = 2, kTsqrBlocked = 3,
                         kTsqrVariants = 4 };

// Most leaves a tuned entry may ask for, per SM (workspace is sized for the entry in effect; the
// leaf launch itself stays within the CTAs its kernel keeps resident).  Narrow passes fit six:
// the row-split leaf of the 33-column source sum keeps six CTAs per SM.
constexpr int kTsqrMaxLeavesPerSm = 6;

struct TsqrCfg {
  int variant;
  int leaves;  // cap on the leaves; 0: one wave of resident CTAs
};

struct TsqrTune {
  std::map<long, TsqrCfg> m;
  unsigned long epoch = 0;  // advanced on every change of m (a captured step depends on m)
  static long key(int esize, int ncap) { return (long)esize * 1000000L + ncap; }
  bool find(int esize, int ncap, TsqrCfg* out) const {
    auto it = m.find(key(esize, ncap));
    if (it == m.end()) return false;
    *out = it->second;
    return true;
  }
};

inline TsqrTune* tune_of(const tt_context* ctx) { return static_cast<TsqrTune*>(ctx->tune); }

// What a pass of ncap columns in arithmetic of esize bytes runs: the tuned entry (or the column
// kernels), leaves = the entry's cap within kTsqrMaxLeavesPerSm per SM, else `wave` (a batch
// view's proportional cap, when set, always wins); variants that cannot take the shape fall
// back to the column kernels: the dense column kernels need FP32 and <= 160 threads, the
// row-split ones 4 ncap <= 1024 lanes.
inline TsqrCfg resolve_tsqr(const tt_context* ctx, int esize, int ncap, int wave) {
  TsqrCfg cfg{kTsqrColumn, 0};
  const TsqrTune* tab = tune_of(ctx);
  if (tab) tab->find(esize, ncap, &cfg);
  const int most = kTsqrMaxLeavesPerSm * ctx->num_sms;
  if (ctx->tsqr_leaf_cap > 0 || cfg.leaves <= 0) cfg.leaves = wave;
  else if (cfg.leaves > most) cfg.leaves = most;
  const int col_threads = ((ncap + 31) / 32) * 32;
  const int rs_threads = ((4 * ncap + 31) / 32) * 32;
  if (cfg.variant == kTsqrColumnDense && (esize != 4 || col_threads > 160)) cfg.variant = kTsqrColumn;
  if (cfg.variant == kTsqrBlocked && (esize != 4 || ncap > 224)) cfg.variant = kTsqrColumn;
  if (cfg.variant == kTsqrRowSplit && rs_threads > 1024) cfg.variant = kTsqrColumn;
  return cfg;
}

}  // namespace ttk
