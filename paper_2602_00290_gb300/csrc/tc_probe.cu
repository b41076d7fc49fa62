// A dense FP32 GEMM on the tcgen05 tensor cores in TF32 or split TF32 (3xTF32) arithmetic, and
// peak probes of the FP64 and FP32 FMA pipes and of the kind::tf32 tensor pipe.  The GEMM runs the
// same descriptors, operand layout and accumulator reads as the mixed path's tensor-core kernels,
// so that they can be checked in isolation against an FP64 product; the probes give the roofline
// denominators of the benchmark, measured on the GPU it runs on.
#include "common.cuh"
#include "tc.cuh"

namespace ttk {
namespace {

constexpr int kGemmKT = 32;  // K values staged per chunk

// D[m][n] = sum_k A[m][k] B[n][k]; A (M x K), B (N x K), D (M x N) row-major FP32.  One CTA of
// 128 threads per 128-row tile of D with all N columns (N a multiple of 16, at most 256); K in
// chunks of kGemmKT staged in shared memory as TF32 hi and lo parts; one thread issues the MMAs
// (passes = 3: hi hi + hi lo + lo hi, else hi hi) into the TMEM accumulator; each warp then reads
// its 32 rows.  A wait that runs out latches TT_ERR_TIMEOUT in *status and ends the tile.
__global__ void __launch_bounds__(128) k_tc_gemm(long M, int N, int K, const float* __restrict__ A,
                                                 const float* __restrict__ B, float* __restrict__ D, int passes,
                                                 int* status) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  constexpr int KT = kGemmKT;
  float* Ahi = reinterpret_cast<float*>(tc_smem);
  float* Alo = Ahi + 128 * KT;
  float* Bhi = Alo + 128 * KT;
  float* Blo = Bhi + (size_t)N * KT;
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long m0 = (long)blockIdx.x * 128;
  const uint32_t ncols = tc::tmem_cols(N);
  if (warp == 0) {
    tc::tmem_alloc(&tbase, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint32_t idesc = tc::idesc_tf32(128, N);
  const uint32_t lbo = 128, sbo = KT / 4 * 128;
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K && ok; k0 += KT) {
    for (int i = tid; i < 128 * KT; i += 128) {
      const int r = i / KT, k = i - (i / KT) * KT;
      const float a = (m0 + r < M && k0 + k < K) ? A[(m0 + r) * K + k0 + k] : 0.0f;
      const float h = tc::tf32_hi(a);
      const uint32_t o = tc::kmajor_off(r, k, KT) >> 2;
      Ahi[o] = h;
      Alo[o] = tc::tf32_hi(a - h);
    }
    for (int i = tid; i < N * KT; i += 128) {
      const int r = i / KT, k = i - (i / KT) * KT;
      const float b = (k0 + k < K) ? B[(long)r * K + k0 + k] : 0.0f;
      const float h = tc::tf32_hi(b);
      const uint32_t o = tc::kmajor_off(r, k, KT) >> 2;
      Bhi[o] = h;
      Blo[o] = tc::tf32_hi(b - h);
    }
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll
      for (int s = 0; s < KT / 8; ++s) {
        const uint32_t so = 256u * s;
        const uint32_t acc = (k0 > 0 || s > 0) ? 1u : 0u;
        tc::mma_tf32(tmem, tc::smem_desc(ah + so, lbo, sbo), tc::smem_desc(bh + so, lbo, sbo), idesc, acc);
        if (passes == 3) {
          tc::mma_tf32(tmem, tc::smem_desc(ah + so, lbo, sbo), tc::smem_desc(bl + so, lbo, sbo), idesc, 1u);
          tc::mma_tf32(tmem, tc::smem_desc(al + so, lbo, sbo), tc::smem_desc(bh + so, lbo, sbo), idesc, 1u);
        }
      }
      tc::mma_commit(&bar);
    }
    // every thread waits: the operands are rewritten only after the MMAs that read them are done;
    // the CTA decides together (a wait that runs out ends the tile in every thread)
    ok = __syncthreads_and(tc::mbar_wait(&bar, phase)) != 0;
    phase ^= 1u;
  }
  if (!ok) {
    if (tid == 0) latch(status, TT_ERR_TIMEOUT);
  } else {
    tc::fence_after_sync();
    const long row = m0 + 32 * warp + lane;
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      tc::tmem_wait_ld();
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < N) D[row * N + c0 + j] = v[j];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, ncols);
  }
}

// Tensor-pipe probe: one CTA per SM issues `iters` kind::tf32 MMAs of 128 x N x 8 on operands
// resident in shared memory into one TMEM accumulator, then waits for them.
__global__ void __launch_bounds__(128, 1) k_tc_peak(int N, long iters, float* __restrict__ sink, int* status) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  float* As = reinterpret_cast<float*>(tc_smem);  // 128 x 8
  float* Bs = As + 128 * 8;                      // N x 8
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (128 + N) * 8; i += 128) As[i] = 1.0f / 64.0f;
  if (warp == 0) {
    tc::tmem_alloc(&tbase, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  bool ok = true;
  if (tid == 0) {
    const uint64_t a = tc::smem_desc(tc::smem_u32(As), 128, 256);
    const uint64_t b = tc::smem_desc(tc::smem_u32(Bs), 128, 256);
    const uint32_t idesc = tc::idesc_tf32(128, N);
    for (long i = 0; i < iters; ++i) tc::mma_tf32(tmem, a, b, idesc, i > 0 ? 1u : 0u);
    tc::mma_commit(&bar);
  }
  ok = __syncthreads_and(tc::mbar_wait(&bar, 0, 1L << 26)) != 0;
  if (!ok) {
    if (tid == 0) latch(status, TT_ERR_TIMEOUT);
  } else {
    tc::fence_after_sync();
    float v[32];
    tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
    tc::tmem_wait_ld();
    if (tid == 0 && sink) sink[blockIdx.x] = v[0];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 256);
  }
}

// FMA-pipe probe: 8 independent chains of fused multiply-adds per thread (FP64 or FP32); the sum
// goes to sink only when flag is set (never in a probe), so the chains cannot be removed.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(long iters, T a, T b, T* __restrict__ sink, int flag) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c);
  for (long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (flag) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace ttk

extern "C" {

tt_status tt_tc_gemm(void* cuda_stream, int64_t M, int32_t N, int32_t K, const float* A, const float* B, float* D,
                     int32_t passes, int32_t* status_dev) {
  if (!A || !B || !D || M < 1 || K < 1 || N < 16 || N > 256 || (N & 15) || (passes != 1 && passes != 3))
    return TT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t smem = sizeof(float) * (size_t)ttk::kGemmKT * (2 * 128 + 2 * (size_t)N);
  if (const tt_status a = ttk::smem_optin(ttk::k_tc_gemm, smem); a != TT_OK) return a;
  const long tiles = (M + 127) / 128;
  ttk::k_tc_gemm<<<(unsigned)tiles, 128, smem, s>>>(M, N, K, A, B, D, passes, status_dev);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

tt_status tt_peak_probe(void* cuda_stream, int32_t kind, int64_t iters, double* flops, float* ms) {
  if (!flops || !ms || iters < 1 || kind < 0 || kind > 2) return TT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TT_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TT_ERR_CUDA;
  }
  tt_status st = TT_OK;
  if (kind == 2) {
    constexpr int N = 256;
    const size_t smem = sizeof(float) * (128 + N) * 8;
    int* status = nullptr;
    cudaEventRecord(e0, s);
    ttk::k_tc_peak<<<(unsigned)nsm, 128, smem, s>>>(N, (long)iters, nullptr, status);
    cudaEventRecord(e1, s);
    *flops = (double)nsm * (double)iters * 2.0 * 128.0 * N * 8.0;
  } else {
    int occ = 0;
    const unsigned threads = 256;
    if (kind == 0)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ttk::k_fma_peak<double>, threads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ttk::k_fma_peak<float>, threads, 0);
    const unsigned grid = (unsigned)nsm * (unsigned)(occ > 0 ? occ : 1);
    cudaEventRecord(e0, s);
    if (kind == 0)
      ttk::k_fma_peak<double><<<grid, threads, 0, s>>>((long)iters, 0.999999, 1e-7, nullptr, 0);
    else
      ttk::k_fma_peak<float><<<grid, threads, 0, s>>>((long)iters, 0.999f, 1e-3f, nullptr, 0);
    cudaEventRecord(e1, s);
    *flops = 2.0 * 8.0 * (double)iters * grid * threads;
  }
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
    st = TT_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // extern "C"
