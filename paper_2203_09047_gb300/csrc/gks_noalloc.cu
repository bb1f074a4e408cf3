// Allocation-free CFL time-step bound.
//
// Some callers cannot call cudaMalloc: processes whose device memory is owned by another
// allocator (a framework pool that has reserved the device), or latency-critical loops that must
// not pay for cudaMalloc's implicit device synchronisation. For them this file provides a variant
// of the time-step reduction whose per-block partial minima live in a fixed, file-scope device
// array instead of memory allocated by the solver.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>

#include "gks_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 65536;  // 512 KiB of partial minima
constexpr int64_t kMaxCells = (int64_t)kMaxBlocks * kThreads;  // 16,777,216 cells
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device; it keeps the last call's contents. Every block
// overwrites its own slot before the final reduction reads it, so nothing needs clearing.
static __device__ __align__(256) double g_dt_partial[kMaxBlocks];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void __launch_bounds__(kThreads) k_cfl_partial(int64_t n, const double* __restrict__ Q,
                                                          const double* __restrict__ h,
                                                          double gamma, double mu,
                                                          double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  double best = DBL_MAX;
  if (i < n) {
    const double r = Q[i], mx = Q[n + i], my = Q[2 * n + i], mz = Q[3 * n + i], E = Q[4 * n + i];
    const double u2 = (mx * mx + my * my + mz * mz) / (r * r);
    const double p = (gamma - 1.0) * (E - 0.5 * r * u2);
    // The primitives are tested themselves: rho < 0 with p < 0 gives a positive gamma p / rho,
    // and p = 0 a zero sound speed, so a test of the bound alone would miss both. The negated
    // comparisons also catch NaN.
    if (!(r > 0.0) || !(p > 0.0)) {
      best = -1.0;
    } else {
      const double c = sqrt(gamma * p / r);
      const double hi = h[i];
      best = hi / (sqrt(u2) + c + 2.0 * mu / (r * hi));
      if (!(best >= 0.0)) best = -1.0;  // NaN in the velocity or the cell length
    }
  }
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) partial[blockIdx.x] = best;
  }
}

__global__ void __launch_bounds__(1024) k_cfl_final(const double* __restrict__ partial, int nblocks,
                                                    double cfl, double* __restrict__ out) {
  __shared__ double red[32];
  double best = DBL_MAX;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) best = fmin(best, partial[k]);
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (int)(blockDim.x / 32) ? red[threadIdx.x] : DBL_MAX;
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (threadIdx.x == 0) *out = best < 0.0 ? -1.0 : cfl * best;
  }
}

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dt_partial);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" gks_status gks_cfl_dt_noalloc(int64_t n_cells, const double* Q, const double* h,
                                         double gamma, double mu, double cfl, double* dt,
                                         void* stream) {
  if (n_cells <= 0 || !Q || !h || !dt || !(cfl > 0.0) || !(gamma > 1.0) || !(mu >= 0.0)) {
    gks::set_global_error("gks_cfl_dt_noalloc: invalid argument");
    return GKS_E_INVAL;
  }
  if (n_cells > kMaxCells) {
    gks::set_global_error(("gks_cfl_dt_noalloc: " + std::to_string(n_cells) +
                           " cells exceed the fixed scratch limit of " + std::to_string(kMaxCells))
                              .c_str());
    return GKS_E_INVAL;
  }
  double* scratch = nullptr;
  const cudaError_t se = scratch_for_current_device(&scratch);
  if (se != cudaSuccess) {
    gks::set_global_error((std::string("gks_cfl_dt_noalloc: scratch address lookup failed: ") +
                           cudaGetErrorString(se)).c_str());
    return GKS_E_CUDA;
  }
  const int nblocks = (int)((n_cells + kThreads - 1) / kThreads);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_cfl_partial<<<nblocks, kThreads, 0, st>>>(n_cells, Q, h, gamma, mu, scratch);
  k_cfl_final<<<1, 1024, 0, st>>>(scratch, nblocks, cfl, dt);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    gks::set_global_error((std::string("gks_cfl_dt_noalloc: launch failed: ") +
                           cudaGetErrorString(le)).c_str());
    return GKS_E_CUDA;
  }
  return GKS_OK;
}
