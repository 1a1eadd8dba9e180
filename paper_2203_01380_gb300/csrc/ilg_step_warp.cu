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
//    computed twice and no warp waits for another;
//  - D1Q3 and D2Q5 hold a lane's vector and its results in registers; D2Q9 (nine
//    planes, four Philox blocks and eleven draws per node) leaves the vector in the
//    tile buffer and collides it two nodes at a time in place, which frees the
//    registers for more warps.
// Every random number is keyed by node and step, so the bits equal those of every
// other step kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "ilg_d2q9.cuh"
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
// alias.  HI: the column as the high word of u * 64 (a multiply, on the FMA pipe,
// where the ALU pipe is the busier one: D2Q9) instead of a shift.
template <bool HI = false>
__device__ __forceinline__ uint32_t draw(const uint2* A, uint32_t n, uint32_t u) {
  const uint2 e = A[__funnelshift_l(u, n, 6)];
  return u < e.x ? (HI ? __umulhi(u, 64u) : (u >> 26)) : e.y;
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

// D2Q9 fast collision of one node whose occupations are all below ROWS, branch-free
// (the fast path of ilg_d2q9.cuh with the same words and results): thinning W0..W8,
// rest W9, axis share W10, axis particles (A, B) = (W11, W12), diagonal particles
// (X, Y) = (W13, W14).  Nonzero when the node needs the general collision (more than
// ROWS - 1 removed, more than 32 axis or diagonal movers).
template <int ROWS>
__device__ __forceinline__ uint32_t fast_draws9(const uint2* to, const uint2* tr, const uint2* ta,
                                                const uint32_t (&W)[16], const uint32_t (&m)[9], uint32_t (&out)[9]) {
  uint32_t r[9];
  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    r[i] = draw<true>(to, m[i], W[i]);
    removed += r[i];
  }
  uint32_t fail = removed >= uint32_t(ROWS) ? 1u : 0u;
  const uint32_t rr = min(removed, uint32_t(ROWS - 1));
  const uint32_t to_rest = draw<true>(tr, rr, W[9]);
  const uint32_t moving = rr - to_rest;
  const uint32_t axis = draw<true>(ta, moving, W[10]);
  const uint32_t diag = moving - axis;
  fail |= (axis > 32u || diag > 32u) ? 1u : 0u;
  const uint32_t ma = __funnelshift_lc(0xFFFFFFFFu, 0u, axis);  // (1 << c) - 1, c <= 32
  const uint32_t md = __funnelshift_lc(0xFFFFFFFFu, 0u, diag);
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = m[i] - r[i];
  out[0] += to_rest;
  // axis particles: axis bit A (0: x, 1: y), sign bit B (0: +, 1: -)
  const uint32_t A = W[11] & ma, B = W[12] & ma;
  const uint32_t ny = __popc(A), nmy = __popc(A & B), nmx = __popc(B & ~A);
  out[1] += axis - ny - nmx;
  out[2] += nmx;
  out[3] += ny - nmy;
  out[4] += nmy;
  // diagonal particles: x-sign bit X, y-sign bit Y (0: +, 1: -)
  const uint32_t X = W[13] & md, Y = W[14] & md;
  const uint32_t nmm = __popc(X & Y), npm = __popc(Y) - nmm, nmp = __popc(X) - nmm;
  out[5] += diag - nmm - npm - nmp;
  out[6] += nmm;
  out[7] += npm;
  out[8] += nmp;
  return fail;
}

// The general collision of the nodes of a vector marked in `slow`, out of line.  N:
// the lane's slot of the current tile buffer in shared memory (plane i at N[32 i],
// flip applied); node k's results are written to half-word k of R[32 i]: the lane's
// slot of the warp's scratch in shared memory, or the slot itself when the vector is
// collided in place.  Both live in shared memory so that no register array of the
// caller has its address taken (which would keep it in local memory on every tile).
// gt: the full Alias8 tables in global memory.  Returns true when a result exceeds
// 65535.
template <int Q, int NPT>
__device__ __noinline__ bool slow_nodes(const StepArgs& a, const uint32_t* gt, uint32_t node0, uint32_t t,
                                        const VN<NPT>* N, VN<NPT>* R, uint32_t slow) {
  bool bad = false;
  while (slow) {
    const int k = __ffs(slow) - 1;
    slow &= slow - 1;
    uint32_t m[Q], o[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) m[i] = node_of(N[32 * i], k);
    if constexpr (Q == 9) collide9_general(a, gt, node0 + k, t, m, o);
    else collide<Q>(a, gt, node0 + k, t, m, o);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      bad |= o[i] > 65535u;
      reinterpret_cast<uint16_t*>(&R[32 * i])[k] = uint16_t(o[i]);
    }
  }
  return bad;
}

// Flip and collide the NPT nodes of one vector (first node `node0`) into the packed
// post-collision planes P.  N holds the vector's occupations with the flip already
// applied (plane i loaded from the flipped source); slot is where they came from in
// the tile buffer and scratch the lane's slot for the general collision's results
// (both read only by the out-of-line general collision); keys: the launch-wide part
// of every node's slot blocks.
template <int Q, int ROWS, int NPT>
__device__ __forceinline__ void collide_vec(const StepArgs& a, const StepKeys<Q == 9 ? 4 : 2>& keys, const uint2* to,
                                            const uint2* tr, const uint2* ta, uint32_t node0, uint32_t t,
                                            const VN<NPT> (&N)[Q], VN<NPT> (&P)[Q], const VN<NPT>* slot,
                                            VN<NPT>* scratch, bool& bad) {
  constexpr uint32_t kHigh = ROWS == 32 ? 0xFFE0FFE0u : 0xFFC0FFC0u;  // bits of values >= ROWS
  uint32_t any = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i)
#pragma unroll
    for (int j = 0; j < NPT / 2; ++j) any |= N[i].w[j];
  // the fast collision needs every probability drawn through its table
  if (a.omega_mode != kTable || a.rest_mode != kTable || (Q == 9 && a.axis_mode != kTable)) any = 0xFFFFFFFFu;
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
      for (int i = 0; i < Q; ++i) {
        // the odd node is the high half; the even node the word minus it times 2^16,
        // a multiply-add (FMA pipe) where a mask would take the busier ALU pipe
        const uint32_t w = N[i].w[k >> 1], high = w >> 16;
        if (k & 1) {
          m[i] = high;
        } else {
          uint32_t low;
          asm("mad.lo.u32 %0, %1, %2, %3;\n" : "=r"(low) : "r"(high), "r"(0xFFFF0000u), "r"(w));
          m[i] = low;
        }
      }
      if constexpr (Q == 9) {
        uint32_t W[16];
        step_blocks<4>(keys, a.rk, node0 + k, W);
        slow |= fast_draws9<ROWS>(to, tr, ta, W, m, o) << k;
      } else {
        uint32_t W[8];
        step_blocks<2>(keys, a.rk, node0 + k, W);
        slow |= fast_draws<Q, ROWS>(to, tr, W, m, o) << k;
      }
      // pack the node's results into its half-words as soon as they exist: an odd
      // node's by a multiply-add (the FMA pipe: the ALU pipe is the busier one), which
      // is exact because every fast-path result, even a failing node's, lies in
      // [0, 126] (no draw exceeds its trials, and at most min(moving, 32) of the
      // moving particles are sorted), so the even node's high half is zero
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        uint32_t& w = P[i].w[k >> 1];
        if (k & 1) {
          uint32_t packed;
          asm("mad.lo.u32 %0, %1, 65536, %2;\n" : "=r"(packed) : "r"(o[i]), "r"(w));
          w = packed;
        } else {
          w = o[i];
        }
      }
    }
  }
  if (slow) {
    bad |= slow_nodes<Q, NPT>(a, a.tables, node0, t, slot, scratch, slow);
    // take the general collision's half-words for the nodes it redid
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const VN<NPT> r = scratch[32 * i];
#pragma unroll
      for (int j = 0; j < NPT / 2; ++j) {
        const uint32_t mask = ((slow >> (2 * j)) & 1u ? 0x0000FFFFu : 0u) | ((slow >> (2 * j + 1)) & 1u ? 0xFFFF0000u : 0u);
        P[i].w[j] = (P[i].w[j] & ~mask) | (r.w[j] & mask);
      }
    }
  }
}

// 32-bit shared-memory load and store at a shared-window address, kept in program
// order with the other shared accesses of the lane's slots
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}

// collide_vec with the vector left in shared memory: the nodes are taken two at a
// time (one 32-bit word per plane) from the lane's slot of the tile buffer (plane i at
// slot[32 i]), and their packed results replace the occupations they came from, so
// only one pair's occupations and results are held in registers at a time.  A pair is
// written only when both its nodes passed the fast collision; otherwise both are
// redone by the general collision, which still finds their occupations in the slot.
template <int Q, int ROWS, int NPT>
__device__ __forceinline__ void collide_vec_res(const StepArgs& a, const StepKeys<Q == 9 ? 4 : 2>& keys,
                                                const uint2* to, const uint2* tr, const uint2* ta, uint32_t node0,
                                                uint32_t t, VN<NPT>* slot, bool& bad) {
  constexpr uint32_t kHigh = ROWS == 32 ? 0xFFE0FFE0u : 0xFFC0FFC0u;  // bits of values >= ROWS
  constexpr uint32_t kPlane = 32 * sizeof(VN<NPT>);                     // bytes between planes
  const bool tables = a.omega_mode == kTable && a.rest_mode == kTable && (Q != 9 || a.axis_mode == kTable);
  const uint32_t sn = static_cast<uint32_t>(__cvta_generic_to_shared(slot));
  uint32_t slow = 0;
#pragma unroll
  for (int j = 0; j < NPT / 2; ++j) {
    uint32_t w[Q];
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      w[i] = lds32(sn + i * kPlane + 4 * j);
      any |= w[i];
    }
    if (!tables || (any & kHigh)) {
      slow |= 3u << (2 * j);
      continue;
    }
    uint32_t o[2][Q];
    uint32_t f = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t m[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) m[i] = h ? (w[i] >> 16) : (w[i] & 0xFFFFu);
      if constexpr (Q == 9) {
        uint32_t W[16];
        step_blocks<4>(keys, a.rk, node0 + 2 * j + h, W);
        f |= fast_draws9<ROWS>(to, tr, ta, W, m, o[h]) << h;
      } else {
        uint32_t W[8];
        step_blocks<2>(keys, a.rk, node0 + 2 * j + h, W);
        f |= fast_draws<Q, ROWS>(to, tr, W, m, o[h]) << h;
      }
    }
    if (f) {
      slow |= 3u << (2 * j);
      continue;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) sts32(sn + i * kPlane + 4 * j, __byte_perm(o[0][i], o[1][i], 0x5410));
  }
  if (slow) bad |= slow_nodes<Q, NPT>(a, a.tables, node0, t, slot, slot, slow);
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

// Velocity i's displacement (dx, dy) in the storage order of each lattice.
template <int Q>
__device__ __forceinline__ constexpr int vel_dx(int i) {
  return Q == 9 ? ((i == 1 || i == 5 || i == 7) ? 1 : ((i == 2 || i == 6 || i == 8) ? -1 : 0))
                : (i == 1 ? 1 : (i == 2 ? -1 : 0));
}
template <int Q>
__device__ __forceinline__ constexpr int vel_dy(int i) {
  return Q == 9 ? ((i == 3 || i == 5 || i == 8) ? 1 : ((i == 4 || i == 6 || i == 7) ? -1 : 0))
                : (Q == 5 ? (i == 3 ? 1 : (i == 4 ? -1 : 0)) : 0);
}

template <int Q, bool FLIP, int ROWS, int NPT, int THREADS, int MINB, bool RES>
__global__ void __launch_bounds__(THREADS, MINB)
    step_warp_kernel(const __grid_constant__ StepArgs a, const uint16_t* __restrict__ in,
                     uint16_t* __restrict__ out, uint32_t t, unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  __shared__ int skip;
  if (threadIdx.x == 0) skip = (*reinterpret_cast<const volatile unsigned long long*>(fail) != ~0ull);
  constexpr uint32_t kTables = Q == 9 ? 3 : 2;           // thinning, rest (D2Q9: and the axis share)
  constexpr uint32_t kRow4 = ROWS * kDevAliasCols / 2;  // uint4 per staged table
  {
    // rows 0..ROWS-1 of each alias table (uint2 entries, two per uint4)
    const uint4* g4 = reinterpret_cast<const uint4*>(a.tables);
    constexpr uint32_t kTab4 = kDevAliasEntries / 2;  // uint4 per full table
    for (uint32_t i = threadIdx.x; i < kTables * kRow4; i += THREADS)
      smem4[i] = g4[(i / kRow4) * kTab4 + (i % kRow4)];
  }
  __syncthreads();
  if (skip) return;
  const uint2* to = reinterpret_cast<const uint2*>(smem4);
  const uint2* tr = to + ROWS * kDevAliasCols;
  const uint2* ta = tr + ROWS * kDevAliasCols;  // D2Q9 only

  constexpr unsigned kFull = 0xFFFFFFFFu;
  constexpr int H = NPT / 2;  // words per vector
  const uint32_t Lx = a.Lx, Ly = a.Ly;
  const size_t plane = size_t(Lx) * Ly;
  const uint32_t vpr = Lx / NPT;
  const uint32_t lane = threadIdx.x & 31u;
  // this warp's two tile buffers (Q planes of 32 vectors each) after the tables
  VN<NPT>* tbuf = reinterpret_cast<VN<NPT>*>(smem4 + kTables * kRow4) + (threadIdx.x >> 5) * (2 * Q * 32);
  // this lane's slot of the warp's scratch for the general collision's results (after
  // all tile buffers)
  VN<NPT>* const scratch = reinterpret_cast<VN<NPT>*>(smem4 + kTables * kRow4) + (THREADS / 32) * (2 * Q * 32) +
                           (threadIdx.x >> 5) * (Q * 32) + lane;
  // this warp's share of the row-major sequence of all vectors: [g, end)
  const uint64_t total = uint64_t(vpr) * Ly, nwarps = (uint64_t(gridDim.x) * THREADS) >> 5;
  const uint64_t w = (uint64_t(blockIdx.x) * THREADS + threadIdx.x) >> 5;
  const uint32_t end = uint32_t((w + 1) * total / nwarps);
  uint32_t g = uint32_t(w * total / nwarps);
  if (g >= end) return;
  bool bad = false;
  const StepKeys<Q == 9 ? 4 : 2> keys = step_keys<Q == 9 ? 4 : 2>(a, t);  // the launch-uniform Philox rounds

  uint32_t y, v0, v1;
  segment_at(g, end, vpr, y, v0, v1);
  uint32_t vb = v0;
  int buf = 0;
  stage_tile<Q, FLIP, NPT>(tbuf, in, plane, size_t(y) * Lx, vb + lane, vb + lane < v1, lane);
  uint32_t carry[Q];   // +x planes: the value of the previous tile's lane 31
  VN<NPT> held[Q];     // -x planes, lane 31: the vector waiting for the next tile's first node
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    carry[i] = 0;
    held[i] = VN<NPT>{};
  }
  // [p1 .. p_{NPT-1}, r]: a -x vector with r for its last slot
  auto shift_down = [](const VN<NPT>& p, uint32_t r) {
    VN<NPT> o;
#pragma unroll
    for (int j = 0; j < H - 1; ++j) o.w[j] = __byte_perm(p.w[j], p.w[j + 1], 0x5432);
    o.w[H - 1] = __byte_perm(p.w[H - 1], r, 0x5432);
    return o;
  };
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
    const uint32_t v = vb + lane;
    const bool active = v < v1;
    const uint32_t x0 = v * NPT;
    VN<NPT> P[Q];
    if constexpr (RES) {
      VN<NPT>* const slot = tbuf + buf * (Q * 32) + lane;
      collide_vec_res<Q, ROWS, NPT>(a, keys, to, tr, ta, uint32_t(size_t(y) * Lx) + x0, t, slot, bad);
#pragma unroll
      for (int i = 0; i < Q; ++i) P[i] = slot[32 * i];
    } else {
      VN<NPT> cur[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) cur[i] = tbuf[buf * (Q * 32) + i * 32 + lane];
      collide_vec<Q, ROWS, NPT>(a, keys, to, tr, ta, uint32_t(size_t(y) * Lx) + x0, t, cur, P,
                                tbuf + buf * (Q * 32) + lane, scratch, bad);
    }
    const uint32_t yp = y + 1 == Ly ? 0 : y + 1;
    const uint32_t ym = y == 0 ? Ly - 1 : y - 1;
    // streaming: velocity i lands in row y + dy of its plane, shifted by dx within it
    auto row_of = [&](int i) {
      const int dy = vel_dy<Q>(i);
      return out + i * plane + size_t(dy == 0 ? y : (dy > 0 ? yp : ym)) * Lx;
    };
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (vel_dx<Q>(i) == 0) stv<NPT>(row_of(i) + x0, P[i].w);
    }
    // +x planes: each node's value moves one node right (the left neighbour's last
    // node); -x planes: one node left (the right neighbour's first node)
    uint32_t left[Q], right[Q], tile_first[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (vel_dx<Q>(i) > 0) {
        const uint32_t last = P[i].w[H - 1] >> 16;
        left[i] = __shfl_up_sync(kFull, last, 1);
        if (lane == 0) left[i] = carry[i];
        carry[i] = __shfl_sync(kFull, last, 31);
      } else if (vel_dx<Q>(i) < 0) {
        const uint32_t first = P[i].w[0] & 0xFFFFu;
        right[i] = __shfl_down_sync(kFull, first, 1);
        tile_first[i] = __shfl_sync(kFull, first, 0);
      }
    }
    if (lane == 31 && vb > v0) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (vel_dx<Q>(i) < 0) stv<NPT>(row_of(i) + (vb - 1) * NPT, shift_down(held[i], tile_first[i]).w);
    }
    if (active) {
      const bool seg_first = v == v0, seg_last = v + 1 == v1;
      if (!seg_first) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (vel_dx<Q>(i) > 0) {
            // [l, p0 .. p_{NPT-2}]
            uint32_t o[H];
            o[0] = __byte_perm(left[i], P[i].w[0], 0x5410);
#pragma unroll
            for (int j = 1; j < H; ++j) o[j] = __byte_perm(P[i].w[j - 1], P[i].w[j], 0x5432);
            stv<NPT>(row_of(i) + x0, o);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          uint16_t* const row = row_of(i);
          if (vel_dx<Q>(i) > 0) {
            // the segment's first +x slot belongs to the node left of the segment
            row[x0 + 1] = uint16_t(P[i].w[0]);
#pragma unroll
            for (int j = 1; j < H; ++j)
              *reinterpret_cast<uint32_t*>(row + x0 + 2 * j) = __byte_perm(P[i].w[j - 1], P[i].w[j], 0x5432);
          } else if (vel_dx<Q>(i) < 0) {
            // and this node's -x value belongs to that node's slot
            row[x0 == 0 ? Lx - 1 : x0 - 1] = uint16_t(P[i].w[0]);
          }
        }
      }
      if (seg_last) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          uint16_t* const row = row_of(i);
          if (vel_dx<Q>(i) > 0) {
            // the segment's last +x value belongs to the first slot of the next segment
            row[x0 + NPT == Lx ? 0 : x0 + NPT] = uint16_t(P[i].w[H - 1] >> 16);
          } else if (vel_dx<Q>(i) < 0) {
            // [p1 .. p_{NPT-1}]: the last -x slot belongs to the node right of the segment
#pragma unroll
            for (int j = 0; j < H - 1; ++j)
              *reinterpret_cast<uint32_t*>(row + x0 + 2 * j) = __byte_perm(P[i].w[j], P[i].w[j + 1], 0x5432);
            row[x0 + NPT - 2] = uint16_t(P[i].w[H - 1] >> 16);
          }
        }
      } else if (lane < 31) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (vel_dx<Q>(i) < 0) stv<NPT>(row_of(i) + x0, shift_down(P[i], right[i]).w);
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i)
          if (vel_dx<Q>(i) < 0) held[i] = P[i];
      }
    }
    if (!more) break;
    if (!same) {
#pragma unroll
      for (int i = 0; i < Q; ++i) carry[i] = 0;
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
// for all their registers beat more warps that spill (measured on the 16384^2 D2Q5
// lattice: 8 nodes per lane, 12 warps at up to 168 registers each, 158 G node
// updates/s; 8 nodes per lane in 16 warps at 128 registers (spills), 153; 4 nodes per
// lane, 20 warps at up to 96 registers, 142).
constexpr int kRows = 64;
template <int SHAPE>
struct WarpShape;
template <>
struct WarpShape<0> {
  static constexpr int kNpt = 8;
  static constexpr int kThreads = 384;
  static constexpr int kBlocks = 1;
  static constexpr bool kRes = false;
};
template <>
struct WarpShape<1> {
  static constexpr int kNpt = 4;
  static constexpr int kThreads = 640;
  static constexpr int kBlocks = 1;
  static constexpr bool kRes = false;
};

// D2Q9 (nine planes, four Philox blocks and eleven draws per node): 4 nodes per lane
// left in shared memory and collided two at a time (nine planes of vectors in
// registers would cost 36 of them), 512 or 640 threads (measured on the 16384^2
// lattice: 72.6 and 68.9 G node updates/s; with the vectors in registers, 512
// threads: 62.9 before the launch-wide Philox rounds were split off)
template <int Q, int SHAPE>
struct WarpShapeQ : WarpShape<SHAPE> {};
template <>
struct WarpShapeQ<9, 0> {
  static constexpr int kNpt = 4;
  static constexpr int kThreads = 512;
  static constexpr int kBlocks = 1;
  static constexpr bool kRes = true;
};
template <>
struct WarpShapeQ<9, 1> {
  static constexpr int kNpt = 4;
  static constexpr int kThreads = 640;
  static constexpr int kBlocks = 1;
  static constexpr bool kRes = true;
};

// tables, then two tile buffers of Q planes x 32 vectors per warp, then (vectors in
// registers only) one scratch buffer of the same shape per warp
template <int Q, int SHAPE>
constexpr size_t warp_smem() {
  using S = WarpShapeQ<Q, SHAPE>;
  return sizeof(uint2) * (Q == 9 ? 3 : 2) * kRows * kDevAliasCols +
         size_t(S::kThreads / 32) * (S::kRes ? 2 : 3) * Q * 32 * (2 * S::kNpt);
}

template <int Q, bool FLIP, int SHAPE>
constexpr auto warp_kernel() {
  using S = WarpShapeQ<Q, SHAPE>;
  return step_warp_kernel<Q, FLIP, kRows, S::kNpt, S::kThreads, S::kBlocks, S::kRes>;
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
  constexpr int kThreads = WarpShapeQ<Q, SHAPE>::kThreads;
  if (a.flip) warp_kernel<Q, true, SHAPE>()<<<grid, kThreads, warp_smem<Q, SHAPE>(), s>>>(a, in, out, t, fail);
  else warp_kernel<Q, false, SHAPE>()<<<grid, kThreads, warp_smem<Q, SHAPE>(), s>>>(a, in, out, t, fail);
}

template <int Q>
void shape_of(int shape, uint32_t* npt, uint32_t* threads, uint32_t* per_sm) {
  if (shape == 1) {
    *npt = WarpShapeQ<Q, 1>::kNpt;
    *threads = WarpShapeQ<Q, 1>::kThreads;
    *per_sm = WarpShapeQ<Q, 1>::kBlocks;
  } else {
    *npt = WarpShapeQ<Q, 0>::kNpt;
    *threads = WarpShapeQ<Q, 0>::kThreads;
    *per_sm = WarpShapeQ<Q, 0>::kBlocks;
  }
}

void shape_of(int Q, int shape, uint32_t* npt, uint32_t* threads, uint32_t* per_sm) {
  if (Q == 9) shape_of<9>(shape, npt, threads, per_sm);
  else shape_of<5>(shape, npt, threads, per_sm);
}

}  // namespace

cudaError_t prepare_step_warp_kernels() {
  cudaError_t e = warp_attr<3, 0>();
  if (e == cudaSuccess) e = warp_attr<3, 1>();
  if (e == cudaSuccess) e = warp_attr<5, 0>();
  if (e == cudaSuccess) e = warp_attr<5, 1>();
  if (e == cudaSuccess) e = warp_attr<9, 0>();
  if (e == cudaSuccess) e = warp_attr<9, 1>();
  return e;
}

uint32_t step_warp_width(int Q, int shape) {
  uint32_t npt, threads, per_sm;
  shape_of(Q, shape, &npt, &threads, &per_sm);
  return npt;
}

// Blocks of a launch: one per SM, or fewer on lattices too small to give each warp
// at least four tiles.
uint32_t step_warp_grid(int Q, uint32_t Lx, uint32_t Ly, uint32_t sms, int shape) {
  uint32_t npt, threads, per_sm;
  shape_of(Q, shape, &npt, &threads, &per_sm);
  const uint64_t cap = uint64_t(sms) * per_sm;
  const uint64_t warps = std::max<uint64_t>(1, uint64_t(Lx / npt) * Ly / 128);
  return uint32_t(std::min<uint64_t>(cap, (warps + threads / 32 - 1) / (threads / 32)));
}

cudaError_t launch_step_warp(int Q, int shape, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                             unsigned long long* fail, int grid, cudaStream_t s) {
  if (Q == 3) {
    if (shape == 1) warp_launch<3, 1>(a, in, out, t, fail, grid, s);
    else warp_launch<3, 0>(a, in, out, t, fail, grid, s);
  } else if (Q == 5) {
    if (shape == 1) warp_launch<5, 1>(a, in, out, t, fail, grid, s);
    else warp_launch<5, 0>(a, in, out, t, fail, grid, s);
  } else {
    if (shape == 1) warp_launch<9, 1>(a, in, out, t, fail, grid, s);
    else warp_launch<9, 0>(a, in, out, t, fail, grid, s);
  }
  return cudaGetLastError();
}

}  // namespace ilg
