// Row-tiled fused step for rows whose length is a multiple of the vector width.
//
// A block walks whole rows (grid-stride over y).  Each row is cut into tiles of
// blockDim vectors; a thread owns one vector of NPT consecutive nodes and moves
// every plane with one NPT*2-byte load and one store.  The rest plane and the
// +-y planes are stored straight back (a +-y shift only changes the row).  The
// +-x planes shift by one node inside the vector: the missing edge value comes
// from the neighbouring thread through shared memory, from the previous tile
// (carried), or — at the two ends of a row, where the lattice wraps — from the
// other end of the same row, so the vectors of the first and last thread are
// held back until that value exists.  Exchange slots are double-buffered by tile
// parity, so one barrier per tile suffices.  A second kernel (step_seg_kernel, below)
// does the same work with warp shuffles and no barrier.
#include <cuda_runtime.h>

#include "ilg_device.cuh"
#include "ilg_launch.h"

namespace ilg {

template <int NPT>
struct Vec {
  uint32_t w[NPT / 2];
};

template <int NPT>
__device__ __forceinline__ Vec<NPT> vload(const uint16_t* p) {
  Vec<NPT> v;
  if constexpr (NPT == 8) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    v.w[0] = q.x; v.w[1] = q.y; v.w[2] = q.z; v.w[3] = q.w;
  } else if constexpr (NPT == 4) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    v.w[0] = q.x; v.w[1] = q.y;
  } else {
    v.w[0] = __ldg(reinterpret_cast<const uint32_t*>(p));
  }
  return v;
}

template <int NPT>
__device__ __forceinline__ void vstore(uint16_t* p, const Vec<NPT>& v) {
  if constexpr (NPT == 8) {
    *reinterpret_cast<uint4*>(p) = make_uint4(v.w[0], v.w[1], v.w[2], v.w[3]);
  } else if constexpr (NPT == 4) {
    *reinterpret_cast<uint2*>(p) = make_uint2(v.w[0], v.w[1]);
  } else {
    *reinterpret_cast<uint32_t*>(p) = v.w[0];
  }
}

__device__ __forceinline__ uint32_t half(const uint32_t* w, int k) {
  return (w[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
}

// +x output: [left, p0 .. p_{NPT-2}]
template <int NPT>
__device__ __forceinline__ Vec<NPT> shift_up(const Vec<NPT>& p, uint32_t left) {
  Vec<NPT> o;
  o.w[0] = __byte_perm(left, p.w[0], 0x5410);
#pragma unroll
  for (int j = 1; j < NPT / 2; ++j) o.w[j] = __byte_perm(p.w[j - 1], p.w[j], 0x5432);
  return o;
}

// -x output: [p1 .. p_{NPT-1}, right]
template <int NPT>
__device__ __forceinline__ Vec<NPT> shift_down(const Vec<NPT>& p, uint32_t right) {
  Vec<NPT> o;
#pragma unroll
  for (int j = 0; j < NPT / 2 - 1; ++j) o.w[j] = __byte_perm(p.w[j], p.w[j + 1], 0x5432);
  o.w[NPT / 2 - 1] = __byte_perm(p.w[NPT / 2 - 1], right, 0x5432);
  return o;
}

constexpr int kVecThreads = 256;

template <int Q>
__device__ __forceinline__ void flip(const StepArgs& a, const uint32_t (&n)[Q], uint32_t (&m)[Q]) {
  m[0] = n[0];
  m[1] = a.flip ? n[2] : n[1];
  m[2] = a.flip ? n[1] : n[2];
  if constexpr (Q == 5) {
    m[3] = a.flip ? n[4] : n[3];
    m[4] = a.flip ? n[3] : n[4];
  }
}

// Flip and collide the NPT nodes of one vector (x0 .. x0+NPT-1 of the row at
// rowoff) into the packed post-collision planes P.  The fast path runs for every
// node; nodes outside its domain (an occupation above 63, more than 63 removed or
// more than 32 moving) are redone with the general collision, reading their input
// again, and overwrite their half-words.  bad is set when a result exceeds 65535.
template <int Q, int NPT>
__device__ __forceinline__ void collide_vector(const StepArgs& a, const uint32_t* s, const uint16_t* __restrict__ in,
                                               size_t plane, size_t rowoff, uint32_t x0, uint32_t t,
                                               Vec<NPT> (&P)[Q], bool& bad) {
  Vec<NPT> N[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) N[i] = vload<NPT>(in + i * plane + rowoff + x0);
  if (a.flip) {
    // the flip F_i(n) = n_{-i} swaps whole opposite planes of the vector
#pragma unroll
    for (int j = 0; j < NPT / 2; ++j) {
      const uint32_t p = N[1].w[j];
      N[1].w[j] = N[2].w[j];
      N[2].w[j] = p;
      if constexpr (Q == 5) {
        const uint32_t q = N[3].w[j];
        N[3].w[j] = N[4].w[j];
        N[4].w[j] = q;
      }
    }
  }
  uint32_t slow = 0;  // nodes that need the general collision
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    uint32_t n[Q], post[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] = half(N[i].w, k);
    if (!collide_try_fast<Q>(a, s, uint32_t(rowoff) + x0 + k, t, n, post)) slow |= 1u << k;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (k & 1) P[i].w[k >> 1] = __byte_perm(P[i].w[k >> 1], post[i], 0x5410);
      else P[i].w[k >> 1] = post[i];
    }
  }
  while (slow) {
    const int k = __ffs(slow) - 1;
    slow &= slow - 1;
    const size_t at = rowoff + x0 + k;
    uint32_t n[Q], m[Q], post[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] = in[i * plane + at];
    flip<Q>(a, n, m);
    collide<Q>(a, s, uint32_t(at), t, m, post);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bad |= post[i] > 65535u;
      const uint32_t v = post[i] & 0xFFFFu;
#pragma unroll
      for (int kk = 0; kk < NPT; ++kk)
        if (kk == k) {
          const uint32_t sh = 16 * (kk & 1);
          P[i].w[kk >> 1] = (P[i].w[kk >> 1] & ~(0xFFFFu << sh)) | (v << sh);
        }
    }
  }
}

// stage the table block, read the overflow word; false when an earlier launch of the
// same call overflowed (this one then does nothing)
__device__ __forceinline__ bool vec_prologue(const StepArgs& a, uint4* smem4, const unsigned long long* fail) {
  __shared__ int skip;
  if (threadIdx.x == 0) skip = (*reinterpret_cast<const volatile unsigned long long*>(fail) != ~0ull);
  const uint4* g4 = reinterpret_cast<const uint4*>(a.tables);
#pragma unroll 8
  for (uint32_t i = threadIdx.x; i < kDevStagedWords / 4; i += blockDim.x) smem4[i] = g4[i];
  __syncthreads();
  return !skip;
}

template <int Q, int NPT, int MINB>
__global__ void __launch_bounds__(kVecThreads, MINB)
    step_vec_kernel(StepArgs a, const uint16_t* __restrict__ in, uint16_t* __restrict__ out, uint32_t t,
                    unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  __shared__ uint32_t xs1[2][kVecThreads];  // +x value of each thread's last node
  __shared__ uint32_t xs2[2][kVecThreads];  // -x value of each thread's first node
  if (!vec_prologue(a, smem4, fail)) return;
  const uint32_t* s = reinterpret_cast<const uint32_t*>(smem4);
  const int tid = threadIdx.x;

  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const size_t plane = size_t(Lx) * Ly;
  const uint32_t vpr = Lx / NPT;                          // vectors per row
  const uint32_t tiles = (vpr + kVecThreads - 1) / kVecThreads;
  const int last_tid = int((vpr - 1) % kVecThreads);       // last active thread of a row's last tile
  bool bad = false;
  int par = 0;

  for (uint32_t y = blockIdx.x; y < Ly; y += gridDim.x) {
    const size_t rowoff = size_t(y) * Lx;
    const uint32_t yp = (Q == 5) ? (y + 1 == Ly ? 0 : y + 1) : 0;
    const uint32_t ym = (Q == 5) ? (y == 0 ? Ly - 1 : y - 1) : 0;
    Vec<NPT> held_px;      // thread 0, tile 0: +x vector waiting for the row's last node
    Vec<NPT> held_mx;      // last thread of a full tile: -x vector waiting for the next tile
    uint32_t first2 = 0;   // -x value of the row's first node
    for (uint32_t tile = 0; tile < tiles; ++tile, par ^= 1) {
      const uint32_t v = tile * kVecThreads + tid;
      const bool active = v < vpr;
      const uint32_t x0 = v * NPT;
      Vec<NPT> P[Q];
      if (active) {
        collide_vector<Q, NPT>(a, s, in, plane, rowoff, x0, t, P, bad);
        vstore<NPT>(out + rowoff + x0, P[0]);
        if constexpr (Q == 5) {
          vstore<NPT>(out + 3 * plane + size_t(yp) * Lx + x0, P[3]);
          vstore<NPT>(out + 4 * plane + size_t(ym) * Lx + x0, P[4]);
        }
        xs1[par][tid] = half(P[1].w, NPT - 1);
        xs2[par][tid] = half(P[2].w, 0);
      }
      __syncthreads();
      if (tile == 0) first2 = xs2[par][0];
      const bool last_tile = tile + 1 == tiles;
      // the -x vector held by the previous tile's last thread gets this tile's first node
      if (tile > 0 && tid == kVecThreads - 1) {
        const size_t xprev = size_t(tile - 1) * kVecThreads * NPT + size_t(kVecThreads - 1) * NPT;
        vstore<NPT>(out + 2 * plane + rowoff + xprev, shift_down<NPT>(held_mx, xs2[par][0]));
      }
      if (active) {
        // +x plane
        if (tid > 0) {
          vstore<NPT>(out + plane + rowoff + x0, shift_up<NPT>(P[1], xs1[par][tid - 1]));
        } else if (tile > 0) {
          vstore<NPT>(out + plane + rowoff + x0, shift_up<NPT>(P[1], xs1[par ^ 1][kVecThreads - 1]));
        } else {
          held_px = P[1];
        }
        // -x plane
        if (last_tile && tid == last_tid) {
          const uint32_t right = (tiles == 1 && tid == 0) ? xs2[par][0] : first2;
          vstore<NPT>(out + 2 * plane + rowoff + x0, shift_down<NPT>(P[2], right));
        } else if (tid < kVecThreads - 1) {
          vstore<NPT>(out + 2 * plane + rowoff + x0, shift_down<NPT>(P[2], xs2[par][tid + 1]));
        } else {
          held_mx = P[2];
        }
      }
      if (last_tile && tid == 0) {
        // the row's first +x vector gets the row's last node
        vstore<NPT>(out + plane + rowoff, shift_up<NPT>(held_px, xs1[par][last_tid]));
      }
    }
  }
  if (bad) atomicMin(fail, static_cast<unsigned long long>(t));
}

// Warp-segment form of the same step: no block-wide exchange.  Each warp takes
// segments of one row in turn (kSegTiles x 32 vectors each, grid-stride over all
// segments of the lattice) and walks its segment left to right, 32 vectors at a
// time.  Neighbouring vectors of a warp tile trade their edge values by shuffles;
// lane 0's left value is carried from the previous tile's lane 31, lane 31's -x
// vector waits in registers for the next tile's first node.  The two values from
// outside the segment (the +x result of the node left of it, the -x result of the
// node right of it, periodic in x) are recomputed by lanes 0 and 1 before the walk:
// every random number is keyed by node and step, so the recomputed node gives the
// same bits as where it is owned.
constexpr uint32_t kSegTiles = 32;  // warp tiles per segment: 1024 vectors

template <int Q, int NPT, int MINB>
__global__ void __launch_bounds__(kVecThreads, MINB)
    step_seg_kernel(StepArgs a, const uint16_t* __restrict__ in, uint16_t* __restrict__ out, uint32_t t,
                    unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  if (!vec_prologue(a, smem4, fail)) return;
  const uint32_t* s = reinterpret_cast<const uint32_t*>(smem4);
  constexpr unsigned kFull = 0xFFFFFFFFu;
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const size_t plane = size_t(Lx) * Ly;
  const uint32_t vpr = Lx / NPT;
  constexpr uint32_t seg_v = 32u * kSegTiles;             // vectors per segment
  const uint32_t segs = (vpr + seg_v - 1) / seg_v;        // segments per row
  const uint32_t units = Ly * segs;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  bool bad = false;

  for (uint32_t u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += nwarps) {
    const uint32_t y = u / segs, g = u - y * segs;
    const uint32_t v0 = g * seg_v;
    const uint32_t v1 = v0 + seg_v < vpr ? v0 + seg_v : vpr;
    const size_t rowoff = size_t(y) * Lx;
    const uint32_t yp = (Q == 5) ? (y + 1 == Ly ? 0 : y + 1) : 0;
    const uint32_t ym = (Q == 5) ? (y == 0 ? Ly - 1 : y - 1) : 0;
    uint32_t edge = 0;
    if (lane < 2) {
      const uint32_t xe = lane == 0 ? (v0 == 0 ? Lx - 1 : v0 * NPT - 1) : (v1 == vpr ? 0 : v1 * NPT);
      const size_t at = rowoff + xe;
      uint32_t n[Q], m[Q], post[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) n[i] = in[i * plane + at];
      flip<Q>(a, n, m);
      if (!collide_try_fast<Q>(a, s, uint32_t(at), t, m, post)) collide<Q>(a, s, uint32_t(at), t, m, post);
      edge = lane == 0 ? post[1] : post[2];
    }
    uint32_t carry = __shfl_sync(kFull, edge, 0);           // left value of the tile's lane 0
    const uint32_t seg_right = __shfl_sync(kFull, edge, 1);  // right value of the segment's last vector
    Vec<NPT> held_mx;                                       // lane 31: -x vector waiting for the next tile
    for (uint32_t vb = v0; vb < v1; vb += 32) {
      const uint32_t v = vb + lane;
      const bool active = v < v1;
      const uint32_t x0 = v * NPT;
      Vec<NPT> P[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < NPT / 2; ++j) P[i].w[j] = 0;
      if (active) {
        collide_vector<Q, NPT>(a, s, in, plane, rowoff, x0, t, P, bad);
        vstore<NPT>(out + rowoff + x0, P[0]);
        if constexpr (Q == 5) {
          vstore<NPT>(out + 3 * plane + size_t(yp) * Lx + x0, P[3]);
          vstore<NPT>(out + 4 * plane + size_t(ym) * Lx + x0, P[4]);
        }
      }
      // +x: the left neighbour's last node
      const uint32_t last_px = half(P[1].w, NPT - 1);
      uint32_t left = __shfl_up_sync(kFull, last_px, 1);
      if (lane == 0) left = carry;
      carry = __shfl_sync(kFull, last_px, 31);
      // -x: the right neighbour's first node
      const uint32_t first_mx = half(P[2].w, 0);
      const uint32_t right = __shfl_down_sync(kFull, first_mx, 1);
      const uint32_t tile_first = __shfl_sync(kFull, first_mx, 0);
      if (lane == 31 && vb > v0)
        vstore<NPT>(out + 2 * plane + rowoff + size_t(vb - 1) * NPT, shift_down<NPT>(held_mx, tile_first));
      if (active) {
        vstore<NPT>(out + plane + rowoff + x0, shift_up<NPT>(P[1], left));
        if (v + 1 == v1) vstore<NPT>(out + 2 * plane + rowoff + x0, shift_down<NPT>(P[2], seg_right));
        else if (lane < 31) vstore<NPT>(out + 2 * plane + rowoff + x0, shift_down<NPT>(P[2], right));
        else held_mx = P[2];
      }
    }
  }
  if (bad) atomicMin(fail, static_cast<unsigned long long>(t));
}

constexpr size_t kVecSmem = sizeof(uint32_t) * kDevStagedWords;
constexpr int kNPT = 8;
constexpr int kMinBlocks = 3;

// second shape for the autotuner: 4 nodes per thread (as many blocks per SM as the
// tables in shared memory allow: 3)
constexpr int kNPT4 = 4;
constexpr int kMinBlocks4 = 3;

template <int Q, int NPT, int MINB>
static cudaError_t vec_attr() {
  cudaError_t e = cudaFuncSetAttribute(step_vec_kernel<Q, NPT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(kVecSmem));
  if constexpr (NPT == kNPT) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(step_seg_kernel<Q, NPT, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(kVecSmem));
  }
  return e;
}

cudaError_t prepare_step_vec_kernels() {
  cudaError_t e = vec_attr<3, kNPT, kMinBlocks>();
  if (e == cudaSuccess) e = vec_attr<5, kNPT, kMinBlocks>();
  if (e == cudaSuccess) e = vec_attr<3, kNPT4, kMinBlocks4>();
  if (e == cudaSuccess) e = vec_attr<5, kNPT4, kMinBlocks4>();
  return e;
}

uint32_t step_vec_width() { return kNPT; }
uint32_t step_vec_blocks_per_sm(int npt) { return npt == kNPT4 ? kMinBlocks4 : kMinBlocks; }

cudaError_t launch_step_vec(int Q, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                            unsigned long long* fail, int grid, cudaStream_t s, int npt) {
  if (npt == kNPT4) {
    if (Q == 3) step_vec_kernel<3, kNPT4, kMinBlocks4><<<grid, kVecThreads, kVecSmem, s>>>(a, in, out, t, fail);
    else step_vec_kernel<5, kNPT4, kMinBlocks4><<<grid, kVecThreads, kVecSmem, s>>>(a, in, out, t, fail);
  } else {
    if (Q == 3) step_vec_kernel<3, kNPT, kMinBlocks><<<grid, kVecThreads, kVecSmem, s>>>(a, in, out, t, fail);
    else step_vec_kernel<5, kNPT, kMinBlocks><<<grid, kVecThreads, kVecSmem, s>>>(a, in, out, t, fail);
  }
  return cudaGetLastError();
}

uint64_t step_seg_units(uint32_t Lx, uint32_t Ly) {
  const uint32_t vpr = Lx / kNPT, seg_v = 32 * kSegTiles;
  return uint64_t(Ly) * ((vpr + seg_v - 1) / seg_v);
}

cudaError_t launch_step_seg(int Q, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                            unsigned long long* fail, int grid, cudaStream_t s) {
  if (Q == 3) step_seg_kernel<3, kNPT, kMinBlocks><<<grid, kVecThreads, kVecSmem, s>>>(a, in, out, t, fail);
  else step_seg_kernel<5, kNPT, kMinBlocks><<<grid, kVecThreads, kVecSmem, s>>>(a, in, out, t, fail);
  return cudaGetLastError();
}

}  // namespace ilg
