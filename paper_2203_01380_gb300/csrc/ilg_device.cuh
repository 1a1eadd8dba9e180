// Device building blocks of the lattice-gas step: Philox4x32-10 and the
// sampling collision of one node (flip, binomial thinning, multinomial
// redistribution), in integer arithmetic only.
#pragma once

#include <cstdint>

namespace ilg {

constexpr uint32_t kDevNmax = 64;
constexpr uint32_t kDevTableWords = kDevNmax * (kDevNmax + 1) / 2;
constexpr uint32_t kDevTagStep = 1u << 24;
constexpr uint32_t kDevTagExt = 2u << 24;
constexpr uint32_t kDevTagInit = 3u << 24;

// How a probability P/2^32 is drawn: never (P = 0), by table (0 < P < 2^32),
// always (P = 2^32).
enum : uint32_t { kNever = 0, kTable = 1, kAlways = 2 };

struct StepArgs {
  uint32_t Lx, Ly;
  uint32_t flip;
  uint32_t omega_mode;   // kNever / kTable / kAlways for the thinning probability
  uint32_t rest_mode;    // same for the rest weight w_0
  uint32_t key0, key1;   // Philox key = seed
  uint32_t replica;
  const uint32_t* T_omega;  // device, kDevTableWords entries
  const uint32_t* T_rest;
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies, the high halves xored with the other counter words and the round key,
// the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint32_t lane_of(const uint4& b, uint32_t i) {
  return i == 0 ? b.x : (i == 1 ? b.y : (i == 2 ? b.z : b.w));
}

// Sequential reader of the extension words of one node and step (tag 2 stream).
struct ExtStream {
  uint32_t node, t, next, cached;
  uint4 blk;
};

__device__ __forceinline__ uint32_t ext_word(const StepArgs& a, ExtStream& e) {
  const uint32_t b = e.next >> 2;
  if (b != e.cached) {
    e.blk = philox(make_uint4(e.node, e.t, a.replica, kDevTagExt | b), a.key0, a.key1);
    e.cached = b;
  }
  const uint32_t w = lane_of(e.blk, e.next & 3u);
  e.next += 1;
  return w;
}

// Binomial(n, P) for n <= 64 by inversion of the integer CDF row n.
__device__ __forceinline__ uint32_t binomial_row(const uint32_t* T, uint32_t n, uint32_t u) {
  const uint32_t* row = T + n * (n - 1) / 2;
  uint32_t k = 0;
  while (k < n && u >= row[k]) ++k;
  return k;
}

// Binomial(m, P): chunks of 64 trials, the first with the slot word, every further
// chunk with the next extension word.
__device__ __forceinline__ uint32_t binomial(uint32_t mode, const uint32_t* T, uint32_t m,
                                             uint32_t slot, const StepArgs& a, ExtStream& e) {
  if (mode == kNever) return 0;
  if (mode == kAlways) return m;
  if (m <= kDevNmax) return m ? binomial_row(T, m, slot) : 0;
  uint32_t r = binomial_row(T, kDevNmax, slot);
  uint32_t left = m - kDevNmax;
  while (left > 0) {
    const uint32_t c = left < kDevNmax ? left : kDevNmax;
    r += binomial_row(T, c, ext_word(a, e));
    left -= c;
  }
  return r;
}

// The collision of one node.  m = occupations after the flip; out = n'.
// Tables sTo (thinning) and sTr (rest weight) are usually in shared memory.
template <int Q>
__device__ __forceinline__ void collide(const StepArgs& a, const uint32_t* sTo, const uint32_t* sTr,
                                        uint32_t node, uint32_t t, const uint32_t (&m)[Q],
                                        uint32_t (&out)[Q]) {
  const uint4 b0 = philox(make_uint4(node, t, a.replica, kDevTagStep | 0u), a.key0, a.key1);
  const uint4 b1 = philox(make_uint4(node, t, a.replica, kDevTagStep | 1u), a.key0, a.key1);
  const uint32_t W[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
  ExtStream e{node, t, 0u, 0xFFFFFFFFu, make_uint4(0, 0, 0, 0)};

  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const uint32_t r = binomial(a.omega_mode, sTo, m[i], W[i], a, e);
    out[i] = m[i] - r;
    removed += r;
  }
  const uint32_t to_rest = binomial(a.rest_mode, sTr, removed, W[Q], a, e);
  out[0] += to_rest;
  uint32_t moving = removed - to_rest;
  bool first = true;
  while (moving > 0) {
    const uint32_t c = moving < 32 ? moving : 32;
    const uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
    if constexpr (Q == 3) {
      const uint32_t s = first ? W[Q + 1] : ext_word(a, e);
      const uint32_t plus = __popc(~s & mask);
      out[1] += plus;
      out[2] += c - plus;
    } else {
      const uint32_t ax = first ? W[Q + 1] : ext_word(a, e);
      const uint32_t sg = first ? W[Q + 2] : ext_word(a, e);
      out[1] += __popc(~ax & ~sg & mask);
      out[2] += __popc(~ax & sg & mask);
      out[3] += __popc(ax & ~sg & mask);
      out[4] += __popc(ax & sg & mask);
    }
    moving -= c;
    first = false;
  }
}

}  // namespace ilg
