// Integer-throughput microbenchmarks of the GPU the library runs on: the measured
// denominators of the step kernels' integer roofline (the step is bound by the
// integer work of its random numbers, not by memory).  Every kernel here runs a
// fixed number of loop iterations over registers only: no memory traffic beyond
// one store per thread that the results never take, no waits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "../../include/ilg.h"
#include "ilg_device.cuh"
#include "ilg_internal.h"

namespace ilg {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;   // 32 warps per SM: enough to hide every fixed latency
constexpr int kChains = 8;            // independent dependency chains per thread

// kind 0: Philox4x32-10 blocks, kChains independent counters per thread and
// iteration, in the counter layout of the step (a launch-wide word, a per-thread
// word, a constant, a tag); the four output words are folded into one register.
__global__ void __launch_bounds__(kPeakThreads, kPeakBlocksPerSm)
    peak_philox_kernel(uint32_t iters, StepArgs a, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const uint4 b = philox_rk(make_uint4(it, tid * kChains + c, a.replica, kDevTagStep), a.rk);
      acc ^= b.x ^ b.y ^ b.z ^ b.w;
    }
  }
  if (acc == a.key0) sink[tid & 1023] = acc;  // keeps the blocks live; the value is never read
}

__device__ __forceinline__ uint32_t lop3_xor(uint32_t x, uint32_t y, uint32_t z) {
  uint32_t r;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
  return r;
}
__device__ __forceinline__ uint32_t mad_lo(uint32_t x, uint32_t y, uint32_t z) {
  uint32_t r;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(y), "r"(z));
  return r;
}
__device__ __forceinline__ uint64_t mad_wide(uint32_t x, uint32_t y, uint64_t z) {
  uint64_t r;
  asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(x), "r"(y), "l"(z));
  return r;
}

// kinds 1-4: kChains chains per thread, each iteration one operation per chain
// (kind 4: one of each per chain); operands from the neighbouring chain so that no
// chain can be folded away.
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads, kPeakBlocksPerSm)
    peak_int_kernel(uint32_t iters, uint32_t k, uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[kChains];
  uint64_t w[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = tid * 0x9E3779B9u + c;
    w[c] = x[c];
  }
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const uint32_t y = x[(c + 1) % kChains];
      if constexpr (KIND == 1) {
        x[c] = lop3_xor(x[c], y, k);
      } else if constexpr (KIND == 2) {
        x[c] = mad_lo(x[c], k, y);
      } else if constexpr (KIND == 3) {
        w[c] = mad_wide(x[c], k, w[c]);
        x[c] = uint32_t(w[c] >> 32);
      } else {
        x[c] = mad_lo(lop3_xor(x[c], y, k), k, y);
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= x[c];
  if (acc == k) sink[tid & 1023] = acc;
}

// operations one thread performs per loop iteration
double ops_per_iteration(int kind) { return kind == 4 ? 2.0 * kChains : double(kChains); }

cudaError_t launch_peak(int kind, uint32_t iters, int grid, const StepArgs& a, uint32_t* sink, cudaStream_t s) {
  switch (kind) {
    case 0: peak_philox_kernel<<<grid, kPeakThreads, 0, s>>>(iters, a, sink); break;
    case 1: peak_int_kernel<1><<<grid, kPeakThreads, 0, s>>>(iters, 0x5bd1e995u, sink); break;
    case 2: peak_int_kernel<2><<<grid, kPeakThreads, 0, s>>>(iters, 0x5bd1e995u, sink); break;
    case 3: peak_int_kernel<3><<<grid, kPeakThreads, 0, s>>>(iters, 0x5bd1e995u, sink); break;
    default: peak_int_kernel<4><<<grid, kPeakThreads, 0, s>>>(iters, 0x5bd1e995u, sink); break;
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace ilg

extern "C" ilg_status ilg_int_peak(int32_t kind, double seconds, void* stream, double* rate, double* ms) {
  using namespace ilg;
  if (kind < 0 || kind > 4 || !rate || !(seconds >= 0.05 && seconds <= 10.0)) {
    set_context_free_error("ilg_int_peak: kind must lie in 0..4, seconds in [0.05, 10], rate non-NULL");
    return ILG_E_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  uint32_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t) * 1024);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  StepArgs a{};
  a.key0 = 0x243F6A88u;
  a.key1 = 0x85A308D3u;
  a.replica = 7;
  round_keys((uint64_t(a.key1) << 32) | a.key0, a.rk);
  const int grid = sms * kPeakBlocksPerSm;
  const double threads = double(grid) * kPeakThreads;
  float t_ms = 0.f;
  uint32_t iters = 256;
  uint32_t launches = 1;
  // calibrate: grow the iteration count until one launch takes ~1/8 of the region
  for (int k = 0; k < 24 && e == cudaSuccess; ++k) {
    e = launch_peak(kind, iters, grid, a, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_peak(kind, iters, grid, a, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
    if (e != cudaSuccess || t_ms * 8.0 >= seconds * 1e3 || iters >= (1u << 30)) break;
    const double grow = t_ms > 0.f ? (seconds * 1e3 / 8.0) / t_ms : 16.0;
    iters = uint32_t(std::min(double(1u << 30), iters * std::min(16.0, std::max(1.5, grow))));
  }
  if (e == cudaSuccess) launches = uint32_t(std::max(1.0, std::ceil(seconds * 1e3 / std::max(1e-3f, t_ms))));
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (uint32_t k = 0; k < launches && e == cudaSuccess; ++k) e = launch_peak(kind, iters, grid, a, sink, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
  cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_context_free_error(std::string("ilg_int_peak: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ILG_E_OOM : ILG_E_CUDA;
  }
  const double per_launch = kind == 0 ? threads * double(iters) * kChains : threads * double(iters) * ops_per_iteration(kind);
  *rate = per_launch * launches / (double(t_ms) / 1e3);
  if (ms) *ms = t_ms;
  return ILG_OK;
}
