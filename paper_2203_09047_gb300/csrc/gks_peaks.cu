// Measured arithmetic peaks of the current GPU: the denominators of the ALU-bound rooflines of
// the flux kernels (FP32 for the mixed path, FP64 for the FP64 path). Each kernel runs
// independent FMA chains in every thread of a grid that fills every SM several times over, so
// the FMA pipe, not latency, bounds it; the rate counts an FMA as two flops. Timed with CUDA
// events on an internal stream, after one warm-up launch. A utility of this library; the paper
// has no counterpart.
#include <cuda_runtime.h>

#include <string>

#include "gks_internal.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kIters = 4096;   // FMAs per chain
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T a, T b, T* __restrict__ sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 16
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;  // one FMA each
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)12345.678) sink[0] = s;  // keeps the chains live; never true for these inputs
}

template <class T>
cudaError_t run(double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 8;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  T* sink = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(T));
  float ms = 0.f;
  if (e == cudaSuccess) {
    // a and b keep |x| bounded: x -> 0.999 x + 1e-4 converges
    k_fma_peak<T><<<blocks, kThreads, 0, st>>>((T)0.999, (T)1e-4, sink);
    cudaEventRecord(a, st);
    k_fma_peak<T><<<blocks, kThreads, 0, st>>>((T)0.999, (T)1e-4, sink);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess && ms > 0.f)
    *tflops = 2.0 * kChains * kIters * (double)blocks * kThreads / (ms * 1e-3) / 1e12;
  if (sink) cudaFree(sink);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  return e;
}

}  // namespace

extern "C" gks_status gks_alu_peaks(double* fp32_tflops, double* fp64_tflops) {
  if (!fp32_tflops || !fp64_tflops) {
    gks::set_global_error("gks_alu_peaks: invalid argument");
    return GKS_E_INVAL;
  }
  cudaError_t e = run<float>(fp32_tflops);
  if (e == cudaSuccess) e = run<double>(fp64_tflops);
  if (e != cudaSuccess) {
    gks::set_global_error((std::string("gks_alu_peaks: ") + cudaGetErrorString(e)).c_str());
    return GKS_E_CUDA;
  }
  return GKS_OK;
}
