// Host runtime helpers shared by every translation unit: the identity of the current CUDA
// context and the checked opt-in to more than 48 KB of dynamic shared memory per CTA.
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace ttk {

namespace {
typedef int (*PfnCtxGetCurrent)(void**);
typedef int (*PfnCtxGetId)(void*, unsigned long long*);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
std::once_flag g_ctx_once;

void resolve_ctx_entry_points() {
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
  void* f1 = nullptr;
  void* f2 = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
      q1 == cudaDriverEntryPointSuccess)
    g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
      q2 == cudaDriverEntryPointSuccess)
    g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f2);
  (void)cudaGetLastError();
}
}  // namespace

unsigned long long current_context_id() {
  std::call_once(g_ctx_once, resolve_ctx_entry_points);
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  void* ctx = nullptr;
  if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
  unsigned long long id = 0;
  if (g_ctx_get_id(ctx, &id) != 0) return 0;
  return id;
}

// Largest dynamic shared memory already allowed, per (kernel, context).  A context that is
// destroyed and re-created (cudaDeviceReset) gets a new id, so its kernels are set again.
tt_status smem_optin_impl(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return TT_OK;
  static std::mutex mu;
  static std::map<std::pair<const void*, unsigned long long>, size_t> done;
  const unsigned long long cid = current_context_id();
  const auto key = std::make_pair(func, cid);
  if (cid != 0) {
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return TT_OK;
  }
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return TT_ERR_CUDA;
  }
  if (bytes > (size_t)optin) return TT_ERR_UNSUPPORTED;
  // never lower a limit that an earlier launch (or a captured graph node) relies on
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
    (void)cudaGetLastError();
    return TT_ERR_CUDA;
  }
  if ((size_t)fa.maxDynamicSharedSizeBytes < bytes &&
      cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return TT_ERR_CUDA;
  }
  if (cid != 0) {
    std::lock_guard<std::mutex> lock(mu);
    size_t& v = done[key];
    if (bytes > v) v = bytes;
  }
  return TT_OK;
}

}  // namespace ttk
