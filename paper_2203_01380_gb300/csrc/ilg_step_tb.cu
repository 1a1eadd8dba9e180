// Temporally blocked D2Q5 step: Tb time steps per round trip through HBM.
//
// A block owns a B x B tile of the output.  It loads the tile with a halo of Tb
// nodes on every side, W = B + 2 Tb wide (global coordinates wrap periodically),
// into shared memory, and runs Tb steps there: step k collides every node of the
// square [k, W-k) of the window and streams into the other buffer, so the square
// with all five inputs valid shrinks by one node per side per step and after Tb
// steps is exactly the tile.  Random numbers are keyed by global node and global
// step, so the result equals Tb single steps bit for bit.  Node updates per tile:
// sum_k (W - 2k)^2 collisions for Tb B^2 useful ones (the halo is recomputed).
#include <cuda_runtime.h>

#include "ilg_device.cuh"
#include "ilg_launch.h"

namespace ilg {

namespace {

constexpr int kTbThreads = 256;
constexpr int kTbExtWords = 8;

__global__ void __launch_bounds__(kTbThreads, 2) step_tb_kernel(StepArgs a, const uint16_t* __restrict__ in,
                                                                uint16_t* __restrict__ out, uint32_t t0,
                                                                uint32_t Tb, uint32_t B,
                                                                unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  uint32_t* tables = reinterpret_cast<uint32_t*>(smem4);
  const uint32_t W = B + 2 * Tb;
  const uint32_t area = W * W;
  uint32_t* xbuf = tables + kDevStagedWords;  // kTbExtWords per thread, interleaved
  uint16_t* bufA = reinterpret_cast<uint16_t*>(xbuf + kTbExtWords * kTbThreads);
  uint16_t* bufB = bufA + 5 * area;
  __shared__ int skip;
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const size_t plane = size_t(Lx) * Ly;
  if (threadIdx.x == 0) skip = (*reinterpret_cast<volatile unsigned long long*>(fail) != ~0ull);
  const uint4* g4 = reinterpret_cast<const uint4*>(a.tables);
#pragma unroll 8
  for (uint32_t i = threadIdx.x; i < kDevStagedWords / 4; i += blockDim.x) smem4[i] = g4[i];
  __syncthreads();
  if (skip) return;

  const uint32_t tiles_x = (Lx + B - 1) / B;
  const uint32_t tiles = tiles_x * ((Ly + B - 1) / B);
  bool bad = false;
  for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint32_t X0 = (tile % tiles_x) * B, Y0 = (tile / tiles_x) * B;
    // window origin in global coordinates, shifted by the halo (wrapped)
    const uint32_t gx0 = (X0 + Lx - (Tb % Lx)) % Lx;
    const uint32_t gy0 = (Y0 + Ly - (Tb % Ly)) % Ly;
    for (uint32_t j = threadIdx.x; j < area; j += blockDim.x) {
      const uint32_t ly = j / W, lx = j - ly * W;
      const uint32_t gx = (gx0 + lx) % Lx, gy = (gy0 + ly) % Ly;
      const size_t at = size_t(gy) * Lx + gx;
#pragma unroll
      for (int i = 0; i < 5; ++i) bufA[i * area + j] = in[i * plane + at];
    }
    __syncthreads();
    uint16_t* src = bufA;
    uint16_t* dst = bufB;
    for (uint32_t k = 0; k < Tb; ++k) {
      const uint32_t lo = k, w = W - 2 * k;   // square [k, W-k) of the window
      for (uint32_t j = threadIdx.x; j < w * w; j += blockDim.x) {
        const uint32_t ry = j / w, rx = j - ry * w;
        const uint32_t lx = lo + rx, ly = lo + ry;
        const uint32_t l = ly * W + lx;
        const uint32_t node = ((gy0 + ly) % Ly) * Lx + (gx0 + lx) % Lx;
        uint32_t n[5], m[5], post[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) n[i] = src[i * area + l];
        m[0] = n[0];
        m[1] = a.flip ? n[2] : n[1];
        m[2] = a.flip ? n[1] : n[2];
        m[3] = a.flip ? n[4] : n[3];
        m[4] = a.flip ? n[3] : n[4];
        if (a.general || !collide_try_fast<5>(a, tables, node, t0 + k, m, post)) {
          collide_general<5, kTbExtWords, kTbThreads>(a, tables, node, t0 + k, m, post, xbuf + threadIdx.x);
#pragma unroll
          for (int i = 0; i < 5; ++i) bad |= post[i] > 65535u;
        }
        // stream inside the window; values leaving it are not needed any more
        dst[l] = uint16_t(post[0]);
        if (lx + 1 < W) dst[area + l + 1] = uint16_t(post[1]);
        if (lx >= 1) dst[2 * area + l - 1] = uint16_t(post[2]);
        if (ly + 1 < W) dst[3 * area + l + W] = uint16_t(post[3]);
        if (ly >= 1) dst[4 * area + l - W] = uint16_t(post[4]);
      }
      __syncthreads();
      uint16_t* tmp = src;
      src = dst;
      dst = tmp;
    }
    // the tile: window square [Tb, Tb + B), clipped to the lattice
    for (uint32_t j = threadIdx.x; j < B * B; j += blockDim.x) {
      const uint32_t ry = j / B, rx = j - ry * B;
      const uint32_t gx = X0 + rx, gy = Y0 + ry;
      if (gx >= Lx || gy >= Ly) continue;
      const uint32_t l = (Tb + ry) * W + (Tb + rx);
      const size_t at = size_t(gy) * Lx + gx;
#pragma unroll
      for (int i = 0; i < 5; ++i) out[i * plane + at] = src[i * area + l];
    }
    __syncthreads();
  }
  if (bad) atomicMin(fail, static_cast<unsigned long long>(t0));
}

}  // namespace

size_t step_tb_smem_bytes(uint32_t B, uint32_t Tb) {
  const size_t W = B + 2 * Tb;
  return sizeof(uint32_t) * (kDevStagedWords + kTbExtWords * kTbThreads) + 2 * 5 * W * W * sizeof(uint16_t);
}

cudaError_t prepare_step_tb_kernel(uint32_t B, uint32_t Tb) {
  return cudaFuncSetAttribute(step_tb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(step_tb_smem_bytes(B, Tb)));
}

cudaError_t launch_step_tb(const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t0, uint32_t Tb,
                           uint32_t B, unsigned long long* fail, int grid, cudaStream_t s) {
  step_tb_kernel<<<grid, kTbThreads, step_tb_smem_bytes(B, Tb), s>>>(a, in, out, t0, Tb, B, fail);
  return cudaGetLastError();
}

}  // namespace ilg
