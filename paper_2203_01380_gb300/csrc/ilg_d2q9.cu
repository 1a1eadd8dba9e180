// D2Q9 time step: the same flip -> collision -> streaming as D1Q3 and D2Q5 on the
// nine-velocity square lattice (rest, four axis and four diagonal velocities;
// weights the products of the D1Q3 weights in x and y); the collision of one node is
// in ilg_d2q9.cuh.  Node-parallel: one thread per node (two neighbouring nodes of a
// row where rows have even length), grid-stride, the three alias tables in shared
// memory.
#include <cuda_runtime.h>

#include "ilg_d2q9.cuh"
#include "ilg_device.cuh"
#include "ilg_launch.h"

namespace ilg {

namespace {

// three alias tables (96 KB) per block: two blocks of twelve warps per SM
constexpr int kD9Threads = 384;
constexpr int kD9BlocksPerSm = 2;

__global__ void __launch_bounds__(kD9Threads, kD9BlocksPerSm) step9_kernel(StepArgs a, const uint16_t* __restrict__ in,
                                                             uint16_t* __restrict__ out, uint32_t t,
                                                             unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  __shared__ int skip;
  uint32_t* s = reinterpret_cast<uint32_t*>(smem4);
  if (threadIdx.x == 0) skip = (*reinterpret_cast<volatile unsigned long long*>(fail) != ~0ull);
  const uint4* g4 = reinterpret_cast<const uint4*>(a.tables);
#pragma unroll 8
  for (uint32_t i = threadIdx.x; i < kDevBlockWords9 / 4; i += blockDim.x) smem4[i] = g4[i];
  __syncthreads();
  if (skip) return;
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const uint32_t nodes = Lx * Ly;
  const size_t plane = nodes;
  bool bad = false;
  for (uint32_t node = blockIdx.x * blockDim.x + threadIdx.x; node < nodes; node += gridDim.x * blockDim.x) {
    const uint32_t y = node / Lx;
    const uint32_t x = node - y * Lx;
    uint32_t n[9], m[9], post[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) n[i] = in[i * plane + node];
    m[0] = n[0];
#pragma unroll
    for (int i = 1; i < 9; i += 2) {  // opposite velocities are neighbours: (1,2) (3,4) (5,6) (7,8)
      m[i] = a.flip ? n[i + 1] : n[i];
      m[i + 1] = a.flip ? n[i] : n[i + 1];
    }
    if (a.particle) {
      collide_particle<9>(a, s, node, t, m, post);
#pragma unroll
      for (int i = 0; i < 9; ++i) bad |= post[i] > 65535u;
    } else if (!collide9_try_fast(a, s, node, t, m, post)) {
      collide9_general(a, s, node, t, m, post);
#pragma unroll
      for (int i = 0; i < 9; ++i) bad |= post[i] > 65535u;
    }
    const uint32_t xp = x + 1 == Lx ? 0 : x + 1, xm = x == 0 ? Lx - 1 : x - 1;
    const uint32_t yp = y + 1 == Ly ? 0 : y + 1, ym = y == 0 ? Ly - 1 : y - 1;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int vx = d9_vx(i), vy = d9_vy(i);
      const uint32_t dx = vx > 0 ? xp : (vx < 0 ? xm : x);
      const uint32_t dy = vy > 0 ? yp : (vy < 0 ? ym : y);
      out[i * plane + size_t(dy) * Lx + dx] = uint16_t(post[i]);
    }
  }
  if (bad) atomicMin(fail, static_cast<unsigned long long>(t));
}

// The same step for rows of even length, two neighbouring nodes of a row per thread:
// one 32-bit load per plane, and one 32-bit store per plane that does not move in x
// (rest, +y, -y); the x-moving planes are stored node by node.
__global__ void __launch_bounds__(kD9Threads, kD9BlocksPerSm) step9_pair_kernel(StepArgs a,
                                                                  const uint16_t* __restrict__ in,
                                                                  uint16_t* __restrict__ out, uint32_t t,
                                                                  unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  __shared__ int skip;
  uint32_t* s = reinterpret_cast<uint32_t*>(smem4);
  if (threadIdx.x == 0) skip = (*reinterpret_cast<volatile unsigned long long*>(fail) != ~0ull);
  const uint4* g4 = reinterpret_cast<const uint4*>(a.tables);
#pragma unroll 8
  for (uint32_t i = threadIdx.x; i < kDevBlockWords9 / 4; i += blockDim.x) smem4[i] = g4[i];
  __syncthreads();
  if (skip) return;
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const uint32_t nodes = Lx * Ly;
  const size_t plane = nodes;  // even, as Lx is: every plane starts on a 32-bit word
  const uint32_t* in32 = reinterpret_cast<const uint32_t*>(in);
  uint32_t* out32 = reinterpret_cast<uint32_t*>(out);
  bool bad = false;
  for (uint32_t pr = blockIdx.x * blockDim.x + threadIdx.x; pr < nodes / 2; pr += gridDim.x * blockDim.x) {
    const uint32_t node0 = 2 * pr;
    const uint32_t y = node0 / Lx;
    const uint32_t x0 = node0 - y * Lx;
    uint32_t w[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) w[i] = in32[(i * plane + node0) >> 1];
    const uint32_t yp = y + 1 == Ly ? 0 : y + 1, ym = y == 0 ? Ly - 1 : y - 1;
    uint32_t keep[3];  // the first node's results of planes 0, 3, 4
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t node = node0 + k, x = x0 + k;
      uint32_t n[9], m[9], post[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) n[i] = (w[i] >> (16 * k)) & 0xFFFFu;
      m[0] = n[0];
#pragma unroll
      for (int i = 1; i < 9; i += 2) {
        m[i] = a.flip ? n[i + 1] : n[i];
        m[i + 1] = a.flip ? n[i] : n[i + 1];
      }
      if (a.particle) {
        collide_particle<9>(a, s, node, t, m, post);
#pragma unroll
        for (int i = 0; i < 9; ++i) bad |= post[i] > 65535u;
      } else if (!collide9_try_fast(a, s, node, t, m, post)) {
        collide9_general(a, s, node, t, m, post);
#pragma unroll
        for (int i = 0; i < 9; ++i) bad |= post[i] > 65535u;
      }
      const uint32_t xp = x + 1 == Lx ? 0 : x + 1, xm = x == 0 ? Lx - 1 : x - 1;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int vx = d9_vx(i), vy = d9_vy(i);
        if (vx == 0) continue;
        const uint32_t dy = vy > 0 ? yp : (vy < 0 ? ym : y);
        out[i * plane + size_t(dy) * Lx + (vx > 0 ? xp : xm)] = uint16_t(post[i]);
      }
      if (k == 0) {
        keep[0] = post[0];
        keep[1] = post[3];
        keep[2] = post[4];
      } else {
        out32[(size_t(y) * Lx + x0) >> 1] = (keep[0] & 0xFFFFu) | (post[0] << 16);
        out32[(3 * plane + size_t(yp) * Lx + x0) >> 1] = (keep[1] & 0xFFFFu) | (post[3] << 16);
        out32[(4 * plane + size_t(ym) * Lx + x0) >> 1] = (keep[2] & 0xFFFFu) | (post[4] << 16);
      }
    }
  }
  if (bad) atomicMin(fail, static_cast<unsigned long long>(t));
}

constexpr size_t kStep9Smem = sizeof(uint32_t) * kDevBlockWords9;

}  // namespace

cudaError_t prepare_step9_kernel() {
  const cudaError_t e = cudaFuncSetAttribute(step9_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStep9Smem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(step9_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStep9Smem));
}

uint32_t step9_threads() { return kD9Threads; }
uint32_t step9_blocks_per_sm() { return kD9BlocksPerSm; }

cudaError_t launch_step9(const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t, unsigned long long* fail,
                         int grid, cudaStream_t s) {
  if (a.Lx % 2 == 0) step9_pair_kernel<<<grid, kD9Threads, kStep9Smem, s>>>(a, in, out, t, fail);
  else step9_kernel<<<grid, kD9Threads, kStep9Smem, s>>>(a, in, out, t, fail);
  return cudaGetLastError();
}

}  // namespace ilg
