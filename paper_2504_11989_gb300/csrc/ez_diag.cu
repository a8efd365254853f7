// Diagnostics: sustained FP64 and FP32 FMA rates of the device (independent fma chains,
// every SM busy), timed with CUDA events on the given stream.
#include <cuda_runtime.h>

#include "../../include/ezeta.h"

namespace {
template <typename T>
__global__ void __launch_bounds__(256) fma_loop(T* sink, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
    x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x0 = fma(x0, a, b);
      x1 = fma(x1, a, b);
      x2 = fma(x2, a, b);
      x3 = fma(x3, a, b);
      x4 = fma(x4, a, b);
      x5 = fma(x5, a, b);
      x6 = fma(x6, a, b);
      x7 = fma(x7, a, b);
    }
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)-12345.678) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains live
}

// best of five timed launches of fma_loop<T> over every SM; TFLOP/s (2 flops per FMA)
template <typename T>
int fma_peak(double* tflops, cudaStream_t stream, int iters) {
  if (!tflops) return EZ_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EZ_ECUDA;
  const int blocks = nsm * 4, threads = 256;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * blocks * threads) != cudaSuccess) return EZ_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_loop<T><<<blocks, threads, 0, stream>>>(sink, 10, (T)0.999999, (T)1e-7);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, stream);
    fma_loop<T><<<blocks, threads, 0, stream>>>(sink, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return EZ_ECUDA;
  *tflops = 2.0 * 8 * 16 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return EZ_OK;
}
}  // namespace

extern "C" int ez_diag_fp64_peak(double* tflops, void* stream) {
  return fma_peak<double>(tflops, (cudaStream_t)stream, 200);
}

extern "C" int ez_diag_fp32_peak(double* tflops, void* stream) {
  return fma_peak<float>(tflops, (cudaStream_t)stream, 4000);
}
