// Multi-lattice step: one launch advances every resident lattice of a server by one
// time step.  Work items are runs of about kItemNodes consecutive nodes of one
// lattice (starting at multiples of kItemNodes); blocks pull items one at a time
// from a queue and reload the alias tables only when the lattice changes.  Threads
// walk the nodes (two neighbours at a time on rows of even length): load the Q
// occupations, flip, collide, and scatter n'_i to x + v_i (periodic).  Each lattice keeps its own step
// counter, replica word and two buffers, so its result is the one it would have
// had alone.
#include <cuda_runtime.h>

#include "ilg_device.cuh"
#include "ilg_multi.h"

namespace ilg {

namespace {

// Nodes [node0, node1) of one lattice (row-major): the block's threads walk them
// together, load the Q occupations, flip, collide and scatter n'_i to x + v_i
// (periodic).
template <int Q>
__device__ __forceinline__ void step_nodes(const StepArgs& a, const uint32_t* s, const uint16_t* __restrict__ in,
                                           uint16_t* __restrict__ out, uint32_t node0, uint32_t node1, uint32_t t,
                                           bool& bad, uint32_t* xb) {
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const size_t plane = size_t(Lx) * Ly;
  // (x, y) carried across the block stride instead of a division per node
  const uint32_t sy = blockDim.x / Lx, sx = blockDim.x - sy * Lx;
  uint32_t nd = node0 + threadIdx.x;
  uint32_t y = nd / Lx, x = nd - y * Lx;
  for (; nd < node1; nd += blockDim.x) {
    const size_t row = size_t(y) * Lx;
    const size_t at = row + x;
    uint32_t n[Q], m[Q], post[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) n[k] = in[k * plane + at];
    m[0] = n[0];
    m[1] = a.flip ? n[2] : n[1];
    m[2] = a.flip ? n[1] : n[2];
    if constexpr (Q == 5) {
      m[3] = a.flip ? n[4] : n[3];
      m[4] = a.flip ? n[3] : n[4];
    }
    if (a.general || !collide_try_fast<Q, Alias4>(a, s, uint32_t(at), t, m, post)) {
      collide_general<Q, kExtWords, kMultiThreads, Alias4>(a, s, uint32_t(at), t, m, post, xb);
#pragma unroll
      for (int k = 0; k < Q; ++k) bad |= post[k] > 65535u;
    }
    const uint32_t xp = x + 1 == Lx ? 0 : x + 1;
    const uint32_t xm = x == 0 ? Lx - 1 : x - 1;
    out[at] = uint16_t(post[0]);
    out[plane + row + xp] = uint16_t(post[1]);
    out[2 * plane + row + xm] = uint16_t(post[2]);
    if constexpr (Q == 5) {
      const uint32_t yp = y + 1 == Ly ? 0 : y + 1;
      const uint32_t ym = y == 0 ? Ly - 1 : y - 1;
      out[3 * plane + size_t(yp) * Lx + x] = uint16_t(post[3]);
      out[4 * plane + size_t(ym) * Lx + x] = uint16_t(post[4]);
    }
    x += sx;
    y += sy;
    if (x >= Lx) {
      x -= Lx;
      y += 1;
    }
  }
}

// The same for even Lx (node0, node1 even): each thread takes two neighbouring nodes
// of a row, reads their occupations as 32-bit pairs, collides them one after the
// other and writes the rest and +-y planes as pairs, the +-x planes (shifted by one
// node, so no longer pair-aligned) node by node.
template <int Q>
__device__ __forceinline__ void step_node_pairs(const StepArgs& a, const uint32_t* s, const uint16_t* __restrict__ in,
                                                uint16_t* __restrict__ out, uint32_t node0, uint32_t node1, uint32_t t,
                                                bool& bad, uint32_t* xb) {
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const size_t plane = size_t(Lx) * Ly;
  // (x, y) carried across the block stride (x stays even: Lx and the stride are even)
  const uint32_t sy = 2 * blockDim.x / Lx, sx = 2 * blockDim.x - sy * Lx;
  uint32_t nd = node0 + 2 * threadIdx.x;
  uint32_t y = nd / Lx, x = nd - y * Lx;
  for (; nd < node1; nd += 2 * blockDim.x) {
    const size_t row = size_t(y) * Lx;
    const size_t at = row + x;
    uint32_t w[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) w[k] = __ldg(reinterpret_cast<const uint32_t*>(in + k * plane + at));
    uint32_t post[2][Q];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t n[Q], m[Q];
#pragma unroll
      for (int k = 0; k < Q; ++k) n[k] = (w[k] >> (16 * h)) & 0xFFFFu;
      m[0] = n[0];
      m[1] = a.flip ? n[2] : n[1];
      m[2] = a.flip ? n[1] : n[2];
      if constexpr (Q == 5) {
        m[3] = a.flip ? n[4] : n[3];
        m[4] = a.flip ? n[3] : n[4];
      }
      if (a.general || !collide_try_fast<Q, Alias4>(a, s, uint32_t(at) + h, t, m, post[h])) {
        collide_general<Q, kExtWords, kMultiThreads, Alias4>(a, s, uint32_t(at) + h, t, m, post[h], xb);
#pragma unroll
        for (int k = 0; k < Q; ++k) bad |= post[h][k] > 65535u;
      }
    }
    auto pair = [&](int k) { return __byte_perm(post[0][k], post[1][k], 0x5410); };
    *reinterpret_cast<uint32_t*>(out + at) = pair(0);
    out[plane + row + x + 1] = uint16_t(post[0][1]);
    out[plane + row + (x + 2 == Lx ? 0 : x + 2)] = uint16_t(post[1][1]);
    out[2 * plane + row + (x == 0 ? Lx - 1 : x - 1)] = uint16_t(post[0][2]);
    out[2 * plane + row + x] = uint16_t(post[1][2]);
    if constexpr (Q == 5) {
      const uint32_t yp = y + 1 == Ly ? 0 : y + 1;
      const uint32_t ym = y == 0 ? Ly - 1 : y - 1;
      *reinterpret_cast<uint32_t*>(out + 3 * plane + size_t(yp) * Lx + x) = pair(3);
      *reinterpret_cast<uint32_t*>(out + 4 * plane + size_t(ym) * Lx + x) = pair(4);
    }
    x += sx;
    y += sy;
    if (x >= Lx) {
      x -= Lx;
      y += 1;
    }
  }
}

template <int Q>
__global__ void __launch_bounds__(kMultiThreads, kMultiBlocksPerSm) multi_step_kernel(MultiArgs ma, StepArgs common,
                                                                      uint32_t sub) {
  extern __shared__ uint4 smem4[];
  uint32_t* s = reinterpret_cast<uint32_t*>(smem4);
  __shared__ uint32_t s_item;
  int loaded = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      // skip lattices that overflowed in an earlier sub-step or are done for this round
      uint32_t it = atomicAdd(ma.counter + sub, 1u);
      while (it < ma.n_items &&
             (ma.fail[ma.items[it].lattice] < sub || sub >= ma.lat[ma.items[it].lattice].steps))
        it = atomicAdd(ma.counter + sub, 1u);
      s_item = it;
    }
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= ma.n_items) break;
    const WorkItem w = ma.items[item];
    const LatDesc d = ma.lat[w.lattice];
    if (int(w.lattice) != loaded) {
      stage_tables4(d.tables, s, d.particle != 0);  // packed: room for the extension words
      loaded = int(w.lattice);
    }
    __syncthreads();
    StepArgs a = common;
    a.Lx = d.Lx;
    a.Ly = d.Ly;
    a.flip = d.flip;
    a.omega_mode = d.omega_mode;
    a.rest_mode = d.rest_mode;
    a.replica = d.replica;
    a.general = d.general;
    a.particle = d.particle;
    const uint32_t t = d.t0 + sub;
    const bool odd = ((sub + d.phase) & 1u) != 0;
    const uint16_t* in = odd ? d.buf1 : d.buf0;
    uint16_t* out = odd ? d.buf0 : d.buf1;
    bool bad = false;
    if (d.Lx % 2u == 0) step_node_pairs<Q>(a, s, in, out, w.node0, w.node1, t, bad, s + kDevTableWords4 + threadIdx.x);
    else step_nodes<Q>(a, s, in, out, w.node0, w.node1, t, bad, s + kDevTableWords4 + threadIdx.x);
    if (bad) atomicMin(ma.fail + w.lattice, sub);
    __syncthreads();  // the tables and s_item stay in use until every thread is done
  }
}

}  // namespace

size_t multi_smem_bytes() { return sizeof(uint32_t) * (kDevTableWords4 + kExtWords * kMultiThreads); }

cudaError_t prepare_multi_kernel() {
  return cudaFuncSetAttribute(multi_step_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(multi_smem_bytes()));
}

cudaError_t launch_multi_step(const MultiArgs& ma, const StepArgs& common, uint32_t sub, int grid, cudaStream_t s) {
  multi_step_kernel<5><<<grid, kMultiThreads, multi_smem_bytes(), s>>>(ma, common, sub);
  return cudaGetLastError();
}

}  // namespace ilg
