// FP64 and FP32 FMA throughput of this GPU, measured with CUDA events: the
// denominators of the ALU rooflines of the element kernels (the FP64 pipe
// bounds the FP64 element and update kernels; B300's FP64 rate is a small
// fraction of its FP32 rate).  Touches no clock or power setting.
#include <cuda_runtime.h>

#include "../../include/ipc_b300.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(T* out, int iters, T a, T b) {
  T x[kChains];
  for (int j = 0; j < kChains; ++j) x[j] = T(1) + T(threadIdx.x + j) * T(1e-7);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
  T s = 0;
  for (int j = 0; j < kChains; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <class T>
cudaError_t time_fma(cudaStream_t st, int blocks, int iters, void* scratch, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  T* out = static_cast<T*>(scratch);
  // x -> a x + b with a slightly below 1: values stay near b / (1 - a), finite
  const T a = T(0.9999999), b = T(1e-7);
  k_fma_chain<T><<<blocks, kThreads, 0, st>>>(out, iters / 8, a, b);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_chain<T><<<blocks, kThreads, 0, st>>>(out, iters, a, b);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) {
    const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
  }
  return e;
}

}  // namespace

extern "C" ipc_status ipc_fma_peaks(void* scratch, size_t scratch_bytes, double* fp64_tflops, double* fp32_tflops,
                                    void* stream) {
  if (!scratch || !fp64_tflops || !fp32_tflops) return IPC_EINVAL;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IPC_ECUDA;
  const int blocks = n_sm * 8;
  if (scratch_bytes < (size_t)blocks * kThreads * sizeof(double)) return IPC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (time_fma<double>(st, blocks, 4096, scratch, fp64_tflops) != cudaSuccess) return IPC_ECUDA;
  if (time_fma<float>(st, blocks, 65536, scratch, fp32_tflops) != cudaSuccess) return IPC_ECUDA;
  return IPC_OK;
}
