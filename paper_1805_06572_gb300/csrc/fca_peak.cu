// Arithmetic peaks of the GPU, measured: the FP32 and FP64 fused multiply-add rates that the
// benchmark's ALU rooflines are stated against. Not part of the method (the paper has no
// counterpart); a short measurement run by the benchmark beside the kernels it rates.
//
// Each thread runs kChains independent FMA recurrences x <- x * a + b (a just below 1, so
// the values stay finite), unrolled, so that every scheduler always has independent FMAs to
// issue; the grid covers every SM several times over. Rate = FMAs * 2 / event time.
#include <cuda_runtime.h>

#include "fca.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345) sink[0] = s;  // keeps the chains live; never true for these values
}

template <typename T>
cudaError_t time_rate(int iters, int blocks, T* sink, double* tflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  fma_chain_kernel<T><<<blocks, kThreads>>>(iters / 8, (T)0.999999, (T)1e-7, sink);  // warm-up
  cudaEventRecord(e0);
  fma_chain_kernel<T><<<blocks, kThreads>>>(iters, (T)0.999999, (T)1e-7, sink);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double fmas = (double)blocks * kThreads * kChains * 16.0 * iters;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace

extern "C" fca_status fca_measure_peaks(double* fp32_tflops, double* fp64_tflops) {
  if (!fp32_tflops || !fp64_tflops) return FCA_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FCA_ERR_CUDA;
  void* sink = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess) return FCA_ERR_NOMEM;
  const int blocks = sms * 8;
  // About 0.1 s of FP32 work and 0.2 s of FP64 work on a GB300-class GPU.
  cudaError_t e = time_rate<float>(80000, blocks, static_cast<float*>(sink), fp32_tflops);
  if (e == cudaSuccess) e = time_rate<double>(2000, blocks, static_cast<double*>(sink), fp64_tflops);
  cudaFree(sink);
  return e == cudaSuccess ? FCA_OK : FCA_ERR_CUDA;
}
