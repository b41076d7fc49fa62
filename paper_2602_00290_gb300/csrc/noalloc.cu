// Inner product of two TT tensors for callers that cannot allocate device memory.
//
// Some host programs may not call cudaMalloc while they run: code inside a fixed memory
// budget reserved up front, code that runs where an allocation would synchronise the device
// or fragment a pool it does not own, and code driven from a callback or a real-time loop
// that must not block.  tt_dot needs a context, and a context owns allocated workspace.  This
// entry point takes only a stream and keeps its scratch in one file-scope device array of
// fixed size that lives as long as the library is loaded on each device that uses it.
#include <map>
#include <mutex>

#include "common.cuh"
#include "instr.cuh"
#include "step.cuh"

namespace {

constexpr size_t kNoAllocScratchDoubles = 1u << 19;  // 4 MiB of FP64 scratch per device

// The scratch itself.  Host code must not pass this symbol to a kernel: in host code its name
// is a stand-in, not a device address.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_mutex;
std::map<unsigned long long, double*> g_scratch_ptr;  // per CUDA context (its unique id)

// Device address of the scratch array in the current CUDA context, looked up once per context
// (a context created after cudaDeviceReset, or another context made current on the device, has a
// new id and its own copy of the array).  Without a context id it is looked up on every call.
tt_status scratch_for_current_context(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return TT_ERR_CUDA;
  const unsigned long long cid = ttk::current_context_id();
  std::lock_guard<std::mutex> lock(g_mutex);
  if (cid != 0) {
    auto it = g_scratch_ptr.find(cid);
    if (it != g_scratch_ptr.end()) {
      *out = it->second;
      return TT_OK;
    }
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TT_ERR_CUDA;
  if (cid != 0) g_scratch_ptr[cid] = static_cast<double*>(p);
  *out = static_cast<double*>(p);
  return TT_OK;
}

}  // namespace

extern "C" tt_status tt_dot_noalloc(void* cuda_stream, const tt_tensor* x, const tt_tensor* y, double* out_dev) {
  if (!out_dev) return TT_ERR_ARG;
  tt_status st = ttk::check_tensor(x);
  if (st == TT_OK) st = ttk::check_tensor(y);
  if (st == TT_OK) st = ttk::same_modes(x, y);
  if (st != TT_OK) return st;
  double* scratch = nullptr;
  st = scratch_for_current_context(&scratch);
  if (st != TT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return (x->dtype == TT_F64) ? ttk::dot_into<double>(s, x, y, out_dev, scratch, kNoAllocScratchDoubles)
                              : ttk::dot_into<float>(s, x, y, out_dev, scratch, kNoAllocScratchDoubles);
}
