// Launch geometry of the tall-skinny QR over the merged core, computed on the host by the same
// functions the launchers use (tsqr_split, tsqr_max_leaves, the shared-memory layouts), so that
// it can be checked without a GPU against the buffers a step sizes.
#include "bigpass.cuh"
#include "tsqr_blk.cuh"
#include "tsqr_rs.cuh"
#include "tune.cuh"

namespace {

template <typename T>
tt_status geometry(int variant, int ncap, long nrows, int num_sms, int per_sm, int max_leaves, int64_t* g) {
  constexpr int kBR = sizeof(T) == 8 ? 32 : 64;  // rows per block of the column and row-split leaves
  const int col_threads = ((ncap + 31) / 32) * 32;
  const int rs_threads = ttk::tsqr_rs_threads<4>(ncap);
  if (variant == ttk::kTsqrColumnDense && (sizeof(T) != 4 || col_threads > 160)) variant = ttk::kTsqrColumn;
  if (variant == ttk::kTsqrRowSplit && rs_threads > 1024) variant = ttk::kTsqrColumn;
  if (variant == ttk::kTsqrBlocked && (sizeof(T) != 4 || ncap > 224)) variant = ttk::kTsqrColumn;
  int br, threads;
  size_t smem;
  long cap2 = 0;
  if (variant == ttk::kTsqrBlocked) {
    // one CTA per SM (the block takes an SM's tensor memory), shared memory of the stencil source
    br = ttk::kBlkRows;
    threads = ttk::kBlkRows;
    smem = ttk::tsqr_blk_smem_bytes<ttk::SrcStencil<float>>(ncap);
    per_sm = 1;
  } else if (variant == ttk::kTsqrRowSplit) {
    br = kBR;
    threads = rs_threads;
    smem = ttk::tsqr_rs_smem_bytes<T, kBR, 4>(ncap);
    cap2 = ttk::tsqr_max_leaves<T, kBR>(num_sms, ncap, nrows, max_leaves);
    if (per_sm < 1) return TT_ERR_UNSUPPORTED;
  } else if (variant == ttk::kTsqrColumnDense) {
    br = 32;
    threads = col_threads;
    smem = ttk::tsqr_smem_bytes<float, 32>(ncap);
  } else {
    br = kBR;
    threads = col_threads;
    smem = ttk::tsqr_smem_bytes<T, kBR>(ncap);
    if (threads > 256) return TT_ERR_UNSUPPORTED;
  }
  if (smem > 227 * 1024) return TT_ERR_UNSUPPORTED;
  const ttk::LeafSplit sp = ttk::tsqr_split(nrows, br, num_sms, per_sm, max_leaves, cap2);
  // merge tree: the row-split merge where 4 ncap lanes fit a CTA, else the column-owner merge
  size_t msmem;
  int mthreads;
  int mrows;
  if (rs_threads <= 1024 && ttk::merge_rs_smem_bytes<T>(ncap) <= 227 * 1024) {
    msmem = ttk::merge_rs_smem_bytes<T>(ncap);
    mthreads = rs_threads;
    mrows = ttk::merge_rs_rows<T>(ncap);
  } else {
    mrows = sizeof(T) == 4 ? 64 : 32;
    msmem = ttk::tsqr_smem_bytes<T, sizeof(T) == 4 ? 64 : 32>(ncap);
    mthreads = col_threads;
    if (msmem > 227 * 1024 || mthreads > 256) return TT_ERR_UNSUPPORTED;
  }
  int levels = 0;
  for (long n = sp.leaves; n > 1; n = (n + 1) / 2) ++levels;
  const long bound = ttk::tsqr_max_leaves<T, 32>(num_sms, ncap, nrows, max_leaves);
  const int64_t nn = (int64_t)ncap * ncap;
  g[0] = sp.leaves;
  g[1] = sp.rpc;
  g[2] = br;
  g[3] = threads;
  g[4] = (int64_t)smem;
  g[5] = mthreads;
  g[6] = (int64_t)msmem;
  g[7] = levels;
  g[8] = bound * nn;
  g[9] = ((bound + 1) / 2) * nn;
  g[10] = variant;
  g[11] = mrows;
  return TT_OK;
}

}  // namespace

extern "C" tt_status tt_tsqr_geometry(tt_precision prec, int32_t variant, int32_t ncap, int64_t nrows,
                                      int32_t num_sms, int32_t per_sm, int32_t max_leaves, int64_t* out,
                                      int32_t nout) {
  if (!out || nout < 1 || nout > 12 || ncap < 1 || nrows < 1 || num_sms < 1 || variant < 0 ||
      variant >= ttk::kTsqrVariants || (prec != TT_PREC_FP64 && prec != TT_PREC_MIXED && prec != TT_PREC_MIXED_3XTF32))
    return TT_ERR_ARG;
  int64_t g[12] = {};
  const tt_status st = (prec == TT_PREC_FP64)
                           ? geometry<double>(variant, ncap, nrows, num_sms, per_sm, max_leaves, g)
                           : geometry<float>(variant, ncap, nrows, num_sms, per_sm, max_leaves, g);
  if (st != TT_OK) return st;
  for (int i = 0; i < nout; ++i) out[i] = g[i];
  return TT_OK;
}
