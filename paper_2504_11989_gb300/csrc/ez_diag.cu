// Diagnostic: sustained FP64 FMA rate of the device (independent fma chains,
// every SM busy), timed with CUDA events on the given stream.
#include <cuda_runtime.h>

#include "../../include/ezeta.h"

namespace {
__global__ void __launch_bounds__(256) dfma_loop(double* sink, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
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
  const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == -12345.678) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains live
}
}  // namespace

extern "C" int ez_diag_fp64_peak(double* tflops, void* stream_) {
  if (!tflops) return EZ_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EZ_ECUDA;
  const int blocks = nsm * 4, threads = 256, iters = 200;
  double* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks * threads) != cudaSuccess) return EZ_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_loop<<<blocks, threads, 0, stream>>>(sink, 10, 0.999999, 1e-7);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, stream);
    dfma_loop<<<blocks, threads, 0, stream>>>(sink, iters, 0.999999, 1e-7);
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
