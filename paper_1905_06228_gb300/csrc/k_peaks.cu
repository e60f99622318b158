// k_peaks.cu -- measured throughput peaks of the units that bound the
// kernels without a tensor-core or HBM roofline: the FP32 FMA pipe (the
// sub-pixel refinement) and shared-memory float atomic adds (the scatter of
// the ZNSSD adjoint).  No counterpart in the paper; the benchmark divides
// the kernels' algorithmic rates by these.
#include "dic_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

// Eight independent FMA chains per thread: enough in flight to keep the
// FP32 pipe busy at full occupancy.  The result is kept alive by a store
// that only happens if it is exactly zero.
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(float* sink, int iters) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (float)(threadIdx.x + c);
  const float b = 0.999999f, d = 1e-6f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], b, d);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 0.f) sink[blockIdx.x] = s;
}

// Shared-memory float atomic adds, one per thread per step, lanes of a warp
// on 32 consecutive words (distinct banks) as in the adjoint's scatter of
// neighbouring subset points; successive steps move to another row of the
// table so that each word sees few adds in a row.
__global__ void __launch_bounds__(kThreads) atomic_probe_kernel(float* sink, int iters) {
  __shared__ float tab[64 * 32];
  for (int i = threadIdx.x; i < 64 * 32; i += kThreads) tab[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < iters; ++i) atomicAdd(&tab[((wid * 8 + i) & 63) * 32 + lane], 1.f);
  __syncthreads();
  if (tab[threadIdx.x] < 0.f) sink[blockIdx.x] = tab[threadIdx.x];
}

}  // namespace

extern "C" dic_status dic_measure_peak(int kind, void* cuda_stream, double* rate) {
  if (!rate || (kind != DIC_PEAK_FP32_FMA && kind != DIC_PEAK_SMEM_ATOMIC_F32))
    return DIC_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DIC_ERR_CUDA;
  // blocks: 8 resident per SM at 256 threads (2048 threads per SM)
  const int blocks = sms * 8;
  const int iters = kind == DIC_PEAK_FP32_FMA ? 1 << 16 : 1 << 14;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dic_status out = DIC_OK;
  if (cudaMalloc(&sink, sizeof(float) * blocks) != cudaSuccess) return DIC_ERR_OOM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    out = DIC_ERR_CUDA;
  } else {
    float best = 0.f;
    for (int rep = 0; rep < 4 && out == DIC_OK; ++rep) {  // first launch warms up
      cudaEventRecord(e0, st);
      if (kind == DIC_PEAK_FP32_FMA)
        fma_probe_kernel<<<blocks, kThreads, 0, st>>>(sink, iters);
      else
        atomic_probe_kernel<<<blocks, kThreads, 0, st>>>(sink, iters);
      cudaEventRecord(e1, st);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        out = DIC_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (out == DIC_OK) {
      const double ops = (double)blocks * kThreads * iters *
                         (kind == DIC_PEAK_FP32_FMA ? 2.0 * kChains : 1.0);
      *rate = ops / (best * 1e-3);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return out;
}
