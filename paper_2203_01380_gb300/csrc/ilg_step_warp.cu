// Warp-segment fused step with 8- or 4-node vectors, shaped for integer issue.
//
// The step's time goes to the integer work of its random numbers (two Philox
// blocks and six alias draws per node), so this kernel spends its registers on the
// independent work of wide vectors in few warps rather than on data in flight:
//  - each lane owns a vector of NPT consecutive nodes (16- or 8-byte accesses; a
//    warp covers 32 NPT nodes of a row per tile); the next tile's occupations are
//    copied into the warp's shared-memory buffer by cp.async while the current tile
//    collides, so the copy holds no registers;
//  - the flip is a compile-time choice of which plane is loaded as which
//    velocity, so it costs nothing;
//  - the fast collision runs branch-free on every node of a vector whose
//    occupations are all below ROWS (64: the rows of the alias tables, staged in
//    shared memory once per SM); the rare node outside that domain is redone by the
//    general collision, out of line (its registers do not weigh on the fast path),
//    which reads the tables from global memory;
//  - warp w takes the w-th of equal shares of the row-major sequence of all
//    vectors (so every warp has the same work to within one vector) and walks it
//    tile by tile, as segments that end at row ends; neighbouring lanes trade
//    edge values by shuffles, and the two values that cross a segment's ends are
//    written as single 16-bit stores by the warp that computes them, so no node is
//    computed twice and no warp waits for another.
// Every random number is keyed by node and step, so the bits equal those of every
// other step kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "ilg_device.cuh"
#include "ilg_launch.h"

namespace ilg {
namespace {

// NPT consecutive nodes of one plane: node k in the low (k even) or high (k odd)
// half of word k / 2
template <int NPT>
struct __align__(2 * NPT < 16 ? 2 * NPT : 16) VN {
  static_assert(NPT == 4 || NPT == 8 || NPT == 16, "vectors of 4, 8 or 16 nodes (8-byte or 16-byte copies)");
  uint32_t w[NPT / 2];
};

template <int NPT>
__device__ __forceinline__ void stv(uint16_t* p, const uint32_t (&w)[NPT / 2]) {
  if constexpr (NPT >= 8) {
#pragma unroll
    for (int j = 0; j < NPT / 8; ++j)
      reinterpret_cast<uint4*>(p)[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
  } else {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  }
}
template <int NPT>
__device__ __forceinline__ uint32_t node_of(const VN<NPT>& v, int k) {
  return (k & 1) ? (v.w[k >> 1] >> 16) : (v.w[k >> 1] & 0xFFFFu);
}

// asynchronous copy of BYTES (8 or 16) global -> shared (zero-filled when !valid: no
// global read)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 16 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the most recent group of this thread's copies have landed
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Binomial(n, P) for n < 64 with one draw u through the alias table A (rows of 64
// columns, column u >> 26): the column's own outcome below its threshold, else its
// alias.
__device__ __forceinline__ uint32_t draw(const uint2* A, uint32_t n, uint32_t u) {
  const uint2 e = A[__funnelshift_l(u, n, 6)];
  return u < e.x ? (u >> 26) : e.y;
}

// Fast collision of one node whose occupations are all below ROWS, branch-free, from
// its slot words W.  Returns nonzero when the node needs the general collision (more than ROWS - 1
// removed, or for ROWS = 64 more than 32 moving particles); out is then garbage,
// but every table index stayed inside the staged rows.
template <int Q, int ROWS>
__device__ __forceinline__ uint32_t fast_draws(const uint2* to, const uint2* tr, const uint32_t (&W)[8],
                                               const uint32_t (&m)[Q], uint32_t (&out)[Q]) {
  uint32_t r[Q];
  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    r[i] = draw(to, m[i], W[i]);
    removed += r[i];
  }
  uint32_t fail = removed >= uint32_t(ROWS) ? 1u : 0u;
  const uint32_t rr = min(removed, uint32_t(ROWS - 1));
  const uint32_t to_rest = draw(tr, rr, W[Q]);
  const uint32_t moving = rr - to_rest;
  if constexpr (ROWS > 33) fail |= moving > 32u ? 1u : 0u;
  const uint32_t mask = __funnelshift_lc(0xFFFFFFFFu, 0u, moving);  // (1 << moving) - 1, moving <= 32
  out[0] = m[0] - r[0] + to_rest;
  if constexpr (Q == 3) {
    const uint32_t minus = __popc(W[Q + 1] & mask);
    out[1] = m[1] - r[1] + (moving - minus);
    out[2] = m[2] - r[2] + minus;
  } else {
    const uint32_t ax = W[Q + 1] & mask, sg = W[Q + 2];
    const uint32_t ny = __popc(ax);                // to +y or -y
    const uint32_t nmy = __popc(ax & sg);          // to -y
    const uint32_t nmx = __popc(sg & mask & ~ax);  // to -x
    out[1] = m[1] - r[1] + (moving - ny - nmx);
    out[2] = m[2] - r[2] + nmx;
    out[3] = m[3] - r[3] + (ny - nmy);
    out[4] = m[4] - r[4] + nmy;
  }
  return fail;
}

// The slot words of a node's step: words 0..7 of its tag-1 stream (two Philox blocks).
__device__ __forceinline__ void slot_words(const StepArgs& a, uint32_t node, uint32_t t, uint32_t (&W)[8]) {
  const uint4 b0 = philox_rk(counter(node, t, a.replica, kDevTagStep | 0u), a.rk);
  const uint4 b1 = philox_rk(counter(node, t, a.replica, kDevTagStep | 1u), a.rk);
  W[0] = b0.x;
  W[1] = b0.y;
  W[2] = b0.z;
  W[3] = b0.w;
  W[4] = b1.x;
  W[5] = b1.y;
  W[6] = b1.z;
  W[7] = b1.w;
}

// The general collision of the nodes of a vector marked in `slow`, out of line; the
// results overwrite their half-words of P.  gt: the full Alias8 tables in global
// memory.  Returns true when a result exceeds 65535.
template <int Q, int NPT>
__device__ __noinline__ bool slow_nodes(const StepArgs& a, const uint32_t* gt, uint32_t node0, uint32_t t,
                                        const VN<NPT>* N, VN<NPT>* P, uint32_t slow) {
  bool bad = false;
  while (slow) {
    const int k = __ffs(slow) - 1;
    slow &= slow - 1;
    uint32_t m[Q], o[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) m[i] = node_of(N[i], k);
    collide<Q>(a, gt, node0 + k, t, m, o);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bad |= o[i] > 65535u;
      const uint32_t v = o[i] & 0xFFFFu;
      uint32_t& w = P[i].w[k >> 1];
      w = (k & 1) ? ((w & 0x0000FFFFu) | (v << 16)) : ((w & 0xFFFF0000u) | v);
    }
  }
  return bad;
}

// Flip and collide the NPT nodes of one vector (first node `node0`) into the packed
// post-collision planes P.  N holds the vector's occupations with the flip already
// applied (plane i loaded from the flipped source).
template <int Q, int ROWS, int NPT>
__device__ __forceinline__ void collide_vec(const StepArgs& a, const uint2* to, const uint2* tr, uint32_t node0,
                                            uint32_t t, VN<NPT> (&N)[Q], VN<NPT> (&P)[Q], bool& bad) {
  constexpr uint32_t kHigh = ROWS == 32 ? 0xFFE0FFE0u : 0xFFC0FFC0u;  // bits of values >= ROWS
  uint32_t any = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i)
#pragma unroll
    for (int j = 0; j < NPT / 2; ++j) any |= N[i].w[j];
  // the fast collision needs both probabilities drawn through their tables
  if (a.omega_mode != kTable || a.rest_mode != kTable) any = 0xFFFFFFFFu;
  uint32_t slow = (any & kHigh) ? (1u << NPT) - 1u : 0u;
#pragma unroll
  for (int i = 0; i < Q; ++i)
#pragma unroll
    for (int j = 0; j < NPT / 2; ++j) P[i].w[j] = 0u;
  if (!slow) {
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      uint32_t m[Q], o[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) m[i] = node_of(N[i], k);
      uint32_t W[8];
      slot_words(a, node0 + k, t, W);
      slow |= fast_draws<Q, ROWS>(to, tr, W, m, o) << k;
      // pack the node's results into its half-words as soon as they exist
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        uint32_t& w = P[i].w[k >> 1];
        w = (k & 1) ? __byte_perm(w, o[i], 0x5410) : o[i];
      }
    }
  }
  if (slow) bad |= slow_nodes<Q, NPT>(a, a.tables, node0, t, N, P, slow);
}

// The segment that starts at vector g of the row-major sequence of all vectors
// (vpr per row) and ends at the end of its row or at end, whichever comes first:
// row y, vectors [v0, v1) of that row.
__device__ __forceinline__ void segment_at(uint32_t g, uint32_t end, uint32_t vpr, uint32_t& y, uint32_t& v0,
                                           uint32_t& v1) {
  y = g / vpr;
  v0 = g - y * vpr;
  v1 = min(vpr, v0 + (end - g));
}

// Queue the copies of one lane's vector (tile row rowoff, vector v) into its slots of
// the warp's tile buffer tb (Q planes of 32 vectors).
template <int Q, bool FLIP, int NPT>
__device__ __forceinline__ void stage_tile(VN<NPT>* tb, const uint16_t* __restrict__ in, size_t plane, size_t rowoff,
                                           uint32_t v, bool active, uint32_t lane) {
  constexpr int kBytes = 2 * NPT < 16 ? 2 * NPT : 16;  // per copy
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    // the flip F_i(n) = n_{-i}: velocity i of the collision reads plane -i
    const int src = !FLIP || i == 0 ? i : (i & 1 ? i + 1 : i - 1);
    const uint16_t* p = active ? in + src * plane + rowoff + size_t(v) * NPT : in;
#pragma unroll
    for (int c = 0; c < 2 * NPT / kBytes; ++c)
      cp_async<kBytes>(reinterpret_cast<char*>(tb + i * 32 + lane) + c * kBytes, active ? p + c * (kBytes / 2) : p,
                       active);
  }
  cp_async_commit();
}

template <int Q, bool FLIP, int ROWS, int NPT, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    step_warp_kernel(const __grid_constant__ StepArgs a, const uint16_t* __restrict__ in,
                     uint16_t* __restrict__ out, uint32_t t, unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  __shared__ int skip;
  if (threadIdx.x == 0) skip = (*reinterpret_cast<const volatile unsigned long long*>(fail) != ~0ull);
  constexpr uint32_t kRow4 = ROWS * kDevAliasCols / 2;  // uint4 per staged table
  {
    // rows 0..ROWS-1 of the thinning and the rest alias tables (uint2 entries, two per uint4)
    const uint4* g4 = reinterpret_cast<const uint4*>(a.tables);
    constexpr uint32_t kTab4 = kDevAliasEntries / 2;  // uint4 per full table
    for (uint32_t i = threadIdx.x; i < 2 * kRow4; i += THREADS) smem4[i] = g4[i < kRow4 ? i : kTab4 + (i - kRow4)];
  }
  __syncthreads();
  if (skip) return;
  const uint2* to = reinterpret_cast<const uint2*>(smem4);
  const uint2* tr = to + ROWS * kDevAliasCols;

  constexpr unsigned kFull = 0xFFFFFFFFu;
  constexpr int H = NPT / 2;  // words per vector
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const size_t plane = size_t(Lx) * Ly;
  const uint32_t vpr = Lx / NPT;
  const uint32_t lane = threadIdx.x & 31u;
  // this warp's two tile buffers (Q planes of 32 vectors each) after the tables
  VN<NPT>* tbuf = reinterpret_cast<VN<NPT>*>(smem4 + 2 * kRow4) + (threadIdx.x >> 5) * (2 * Q * 32);
  // this warp's share of the row-major sequence of all vectors: [g, end)
  const uint64_t total = uint64_t(vpr) * Ly, nwarps = (uint64_t(gridDim.x) * THREADS) >> 5;
  const uint64_t w = (uint64_t(blockIdx.x) * THREADS + threadIdx.x) >> 5;
  const uint32_t end = uint32_t((w + 1) * total / nwarps);
  uint32_t g = uint32_t(w * total / nwarps);
  if (g >= end) return;
  bool bad = false;

  uint32_t y, v0, v1;
  segment_at(g, end, vpr, y, v0, v1);
  uint32_t vb = v0;
  int buf = 0;
  stage_tile<Q, FLIP, NPT>(tbuf, in, plane, size_t(y) * Lx, vb + lane, vb + lane < v1, lane);
  uint32_t carry = 0;  // +x value of the previous tile's lane 31
  VN<NPT> held_mx{};   // lane 31: -x vector waiting for the next tile's first node
  while (true) {
    // the next tile: of this segment, or the first of the segment that follows it;
    // its copies are queued before this tile collides
    const uint32_t g_next = g + (v1 - v0);  // first vector after this segment
    const bool same = vb + 32 < v1;
    const bool more = same || g_next < end;
    uint32_t ny = y, nv0 = v0, nv1 = v1, nvb = vb + 32;
    if (!same && more) {
      segment_at(g_next, end, vpr, ny, nv0, nv1);
      nvb = nv0;
    }
    stage_tile<Q, FLIP, NPT>(tbuf + (buf ^ 1) * (Q * 32), in, plane, size_t(ny) * Lx, nvb + lane,
                             more && nvb + lane < nv1, lane);
    cp_async_wait_prior();
    VN<NPT> cur[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) cur[i] = tbuf[buf * (Q * 32) + i * 32 + lane];

    const size_t rowoff = size_t(y) * Lx;
    const uint32_t v = vb + lane;
    const bool active = v < v1;
    const uint32_t x0 = v * NPT;
    VN<NPT> P[Q];
    collide_vec<Q, ROWS, NPT>(a, to, tr, uint32_t(rowoff) + x0, t, cur, P, bad);
    if (active) {
      stv<NPT>(out + rowoff + x0, P[0].w);
      if constexpr (Q == 5) {
        const uint32_t yp = y + 1 == Ly ? 0 : y + 1;
        const uint32_t ym = y == 0 ? Ly - 1 : y - 1;
        stv<NPT>(out + 3 * plane + size_t(yp) * Lx + x0, P[3].w);
        stv<NPT>(out + 4 * plane + size_t(ym) * Lx + x0, P[4].w);
      }
    }
    // +x: each node's value moves one node right; the left neighbour's last node
    const uint32_t last_px = P[1].w[H - 1] >> 16;
    uint32_t left = __shfl_up_sync(kFull, last_px, 1);
    if (lane == 0) left = carry;
    carry = __shfl_sync(kFull, last_px, 31);
    // -x: one node left; the right neighbour's first node
    const uint32_t first_mx = P[2].w[0] & 0xFFFFu;
    const uint32_t right = __shfl_down_sync(kFull, first_mx, 1);
    const uint32_t tile_first = __shfl_sync(kFull, first_mx, 0);
    uint16_t* const px = out + plane + rowoff;
    uint16_t* const mx = out + 2 * plane + rowoff;
    // [p1 .. p_{NPT-1}, r]: the -x vector with r for its last slot
    auto shift_down = [&](const VN<NPT>& p, uint32_t r) {
      VN<NPT> o;
#pragma unroll
      for (int j = 0; j < H - 1; ++j) o.w[j] = __byte_perm(p.w[j], p.w[j + 1], 0x5432);
      o.w[H - 1] = __byte_perm(p.w[H - 1], r, 0x5432);
      return o;
    };
    if (lane == 31 && vb > v0) stv<NPT>(mx + (vb - 1) * NPT, shift_down(held_mx, tile_first).w);
    if (active) {
      const bool seg_first = v == v0, seg_last = v + 1 == v1;
      if (!seg_first) {
        // [l, p0 .. p_{NPT-2}]
        uint32_t o[H];
        o[0] = __byte_perm(left, P[1].w[0], 0x5410);
#pragma unroll
        for (int j = 1; j < H; ++j) o[j] = __byte_perm(P[1].w[j - 1], P[1].w[j], 0x5432);
        stv<NPT>(px + x0, o);
      } else {
        // the segment's first +x slot belongs to the node left of the segment
        px[x0 + 1] = uint16_t(P[1].w[0]);
#pragma unroll
        for (int j = 1; j < H; ++j)
          *reinterpret_cast<uint32_t*>(px + x0 + 2 * j) = __byte_perm(P[1].w[j - 1], P[1].w[j], 0x5432);
        // and this node's -x value belongs to that node's slot
        mx[x0 == 0 ? Lx - 1 : x0 - 1] = uint16_t(P[2].w[0]);
      }
      if (seg_last) {
        px[x0 + NPT == Lx ? 0 : x0 + NPT] = uint16_t(P[1].w[H - 1] >> 16);
#pragma unroll
        for (int j = 0; j < H - 1; ++j)
          *reinterpret_cast<uint32_t*>(mx + x0 + 2 * j) = __byte_perm(P[2].w[j], P[2].w[j + 1], 0x5432);
        mx[x0 + NPT - 2] = uint16_t(P[2].w[H - 1] >> 16);
      } else if (lane < 31) {
        stv<NPT>(mx + x0, shift_down(P[2], right).w);
      } else {
        held_mx = P[2];
      }
    }
    if (!more) break;
    if (!same) {
      carry = 0;
      g = g_next;
      y = ny;
      v0 = nv0;
      v1 = nv1;
    }
    vb = nvb;
    buf ^= 1;
  }
  cp_async_wait_all();  // the last (empty) group: nothing lands after the warp exits
  if (bad) atomicMin(fail, static_cast<unsigned long long>(t));
}

// Shapes (the autotuner's two candidates): one block per SM, so the 64 staged table
// rows exist once per SM; kNpt nodes per lane, kThreads threads, a multiple of 128 so
// that the four sub-partitions of an SM hold equally many warps.  Few warps with room
// for all their registers beat more warps that spill (measured on the 16384^2
// lattice: 8 nodes per lane, 12 warps at up to 168 registers each, 150 G node
// updates/s; 4 nodes per lane, 24 warps at 80 registers, 135).
constexpr int kRows = 64;
template <int SHAPE>
struct WarpShape;
template <>
struct WarpShape<0> {
  static constexpr int kNpt = 8;
  static constexpr int kThreads = 384;
  static constexpr int kBlocks = 1;
};
template <>
struct WarpShape<1> {
  static constexpr int kNpt = 4;
  static constexpr int kThreads = 768;
  static constexpr int kBlocks = 1;
};

// tables, then two tile buffers of Q planes x 32 vectors per warp
template <int Q, int SHAPE>
constexpr size_t warp_smem() {
  using S = WarpShape<SHAPE>;
  return sizeof(uint2) * 2 * kRows * kDevAliasCols + size_t(S::kThreads / 32) * 2 * Q * 32 * (2 * S::kNpt);
}

template <int Q, bool FLIP, int SHAPE>
constexpr auto warp_kernel() {
  using S = WarpShape<SHAPE>;
  return step_warp_kernel<Q, FLIP, kRows, S::kNpt, S::kThreads, S::kBlocks>;
}

template <int Q, int SHAPE>
cudaError_t warp_attr() {
  cudaError_t e = cudaFuncSetAttribute(warp_kernel<Q, false, SHAPE>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(warp_smem<Q, SHAPE>()));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(warp_kernel<Q, true, SHAPE>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(warp_smem<Q, SHAPE>()));
  return e;
}

template <int Q, int SHAPE>
void warp_launch(const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t, unsigned long long* fail, int grid,
                 cudaStream_t s) {
  constexpr int kThreads = WarpShape<SHAPE>::kThreads;
  if (a.flip) warp_kernel<Q, true, SHAPE>()<<<grid, kThreads, warp_smem<Q, SHAPE>(), s>>>(a, in, out, t, fail);
  else warp_kernel<Q, false, SHAPE>()<<<grid, kThreads, warp_smem<Q, SHAPE>(), s>>>(a, in, out, t, fail);
}

}  // namespace

cudaError_t prepare_step_warp_kernels() {
  cudaError_t e = warp_attr<3, 0>();
  if (e == cudaSuccess) e = warp_attr<3, 1>();
  if (e == cudaSuccess) e = warp_attr<5, 0>();
  if (e == cudaSuccess) e = warp_attr<5, 1>();
  return e;
}

uint32_t step_warp_width(int shape) { return shape == 1 ? WarpShape<1>::kNpt : WarpShape<0>::kNpt; }

// Blocks of a launch: one per SM, or fewer on lattices too small to give each warp
// at least four tiles.
uint32_t step_warp_grid(uint32_t Lx, uint32_t Ly, uint32_t sms, int shape) {
  const int threads = shape == 1 ? WarpShape<1>::kThreads : WarpShape<0>::kThreads;
  const int per_sm = shape == 1 ? WarpShape<1>::kBlocks : WarpShape<0>::kBlocks;
  const uint64_t cap = uint64_t(sms) * per_sm;
  const uint64_t warps = std::max<uint64_t>(1, uint64_t(Lx / step_warp_width(shape)) * Ly / 128);
  return uint32_t(std::min<uint64_t>(cap, (warps + threads / 32 - 1) / (threads / 32)));
}

cudaError_t launch_step_warp(int Q, int shape, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                             unsigned long long* fail, int grid, cudaStream_t s) {
  if (Q == 3) {
    if (shape == 1) warp_launch<3, 1>(a, in, out, t, fail, grid, s);
    else warp_launch<3, 0>(a, in, out, t, fail, grid, s);
  } else {
    if (shape == 1) warp_launch<5, 1>(a, in, out, t, fail, grid, s);
    else warp_launch<5, 0>(a, in, out, t, fail, grid, s);
  }
  return cudaGetLastError();
}

}  // namespace ilg
