// Inner product of two TT tensors for callers that cannot allocate device memory.
//
// Some host programs may not call cudaMalloc while they run: code inside a fixed memory
// budget reserved up front, code that runs where an allocation would synchronise the device
// or fragment a pool it does not own, and code driven from a callback or a real-time loop
// that must not block.  tt_dot needs a context, and a context owns allocated workspace.  This
// entry point takes only a stream and keeps its scratch in one file-scope device array of
// fixed size that lives as long as the library is loaded on each device that uses it.
#include <mutex>

#include "common.cuh"
#include "instr.cuh"
#include "step.cuh"

namespace {

constexpr size_t kNoAllocScratchDoubles = 1u << 19;  // 4 MiB of FP64 scratch per device

// The scratch itself.  Host code must not pass this symbol to a kernel: in host code its name
// is a stand-in, not a device address.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
tt_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TT_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TT_OK;
}

tt_status check(const tt_tensor* x) {
  if (!x || !x->rank) return TT_ERR_ARG;
  if (x->d != 2 && x->d != 3) return TT_ERR_UNSUPPORTED;
  if (x->dtype != TT_F64 && x->dtype != TT_F32) return TT_ERR_ARG;
  if (x->rcap[0] != 1 || x->rcap[x->d] != 1) return TT_ERR_SHAPE;
  for (int j = 0; j < x->d; ++j)
    if (x->n[j] <= 0 || x->rcap[j + 1] <= 0 || !x->core[j]) return TT_ERR_SHAPE;
  return TT_OK;
}

}  // namespace

extern "C" tt_status tt_dot_noalloc(void* cuda_stream, const tt_tensor* x, const tt_tensor* y, double* out_dev) {
  if (!out_dev) return TT_ERR_ARG;
  tt_status st = check(x);
  if (st == TT_OK) st = check(y);
  if (st != TT_OK) return st;
  if (x->d != y->d || x->dtype != y->dtype) return TT_ERR_SHAPE;
  for (int j = 0; j < x->d; ++j)
    if (x->n[j] != y->n[j]) return TT_ERR_SHAPE;
  double* scratch = nullptr;
  st = scratch_for_current_device(&scratch);
  if (st != TT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return (x->dtype == TT_F64) ? ttk::dot_into<double>(s, x, y, out_dev, scratch, kNoAllocScratchDoubles)
                              : ttk::dot_into<float>(s, x, y, out_dev, scratch, kNoAllocScratchDoubles);
}
