// Device building blocks of the lattice-gas step: Philox4x32-10 and the
// sampling collision of one node (binomial thinning, multinomial
// redistribution), in integer arithmetic only.
#pragma once

#include <cstdint>

namespace ilg {

constexpr uint32_t kDevNmax = 63;                                  // trials per alias row
constexpr uint32_t kDevAliasCols = 64;                             // columns per row: u >> 26
constexpr uint32_t kDevAliasEntries = (kDevNmax + 1) * kDevAliasCols;  // rows n = 0..63
// table block: alias table (thinning) | alias table (rest), one uint2 {thr, alias} per
// column (kDevStagedWords words, what most kernels stage), then for D1Q3 / D2Q5 the
// same two tables packed one word per column (Alias4, kDevTableWords4 words);
// D2Q9 lattices have the alias table of the axis share as a third and no packed form
constexpr uint32_t kDevStagedWords = 2 * kDevAliasEntries * 2;
constexpr uint32_t kDevTableWords4 = 2 * kDevAliasEntries;
constexpr uint32_t kDevBlockWords = kDevStagedWords + kDevTableWords4;
constexpr uint32_t kDevBlockWords9 = 3 * kDevAliasEntries * 2;
static_assert(kDevStagedWords % 4 == 0 && kDevBlockWords % 4 == 0 && kDevBlockWords9 % 4 == 0,
              "table blocks are staged as uint4");
constexpr uint32_t kDevTagStep = 1u << 24;
constexpr uint32_t kDevTagExt = 2u << 24;
constexpr uint32_t kDevTagInit = 3u << 24;
constexpr uint32_t kDevTagParticle = 4u << 24;
constexpr int kExtWords = 20;        // extension words per thread held in shared memory

// How a probability P/2^32 is drawn: never (P = 0), by table (0 < P < 2^32),
// always (P = 2^32).
enum : uint32_t { kNever = 0, kTable = 1, kAlways = 2 };

struct StepArgs {
  uint32_t Lx, Ly;
  uint32_t flip;
  uint32_t omega_mode;   // kNever / kTable / kAlways for the thinning probability
  uint32_t rest_mode;    // same for the rest weight w_0
  uint32_t general;      // 1: skip the fast path (occupations so high that it would mostly
                         //    fail, or the particle sampler)
  uint32_t particle;     // 1: particle sampler (one word per particle, tag-4 stream); the
                         //    table block then holds the boundaries B_0..B_Q (uint64)
  uint32_t axis_mode;    // D2Q9: kNever / kTable / kAlways for the axis share
  uint32_t key0, key1;   // Philox key = seed
  uint32_t replica;
  const uint32_t* tables;   // device, kDevBlockWords words (layout above)
  uint32_t rk[20];          // round keys (key0 + r W0, key1 + r W1), r = 0..9
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

// Same function with the ten round keys precomputed (rk[2r], rk[2r+1]); the keys
// then come straight from the kernel's parameter bank.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = uint64_t(0xD2511F53u) * c.x;
    const uint64_t p1 = uint64_t(0xCD9E8D57u) * c.z;
    c = make_uint4(uint32_t(p1 >> 32) ^ c.y ^ rk[2 * r], uint32_t(p1), uint32_t(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                   uint32_t(p0));
  }
  return c;
}

// Counter of block `tagblock` (purpose tag << 24 | block index) of the random stream
// of a node at step t.  The step leads and the node follows: the first round then
// multiplies words that are the same across a launch, and the two step blocks of a
// node share their second- and third-round multiplies.
__device__ __forceinline__ uint4 counter(uint32_t node, uint32_t t, uint32_t replica, uint32_t tagblock) {
  return make_uint4(t, node, replica, tagblock);
}

// The slot blocks b = 0..NB-1 of a node at step t, split into the part that is the
// same for every node of a launch (StepKeys, computed once) and the rest (step_blocks).
// With the counter (t, node, replica, tag | b), round 1 multiplies t and the replica;
// round 2 multiplies node-dependent x0 (shared by the blocks) and a block-dependent but
// node-independent x2; round 3 multiplies a node-independent x0 and a node-dependent x2
// shared by the blocks.  Writing those rounds out, a node's blocks enter round 4 as
//   (hi(R2) ^ H_b, lo(R2), lo(P1) ^ I_b, J_b),  P1 = M0 (node ^ A),
//   R2 = M1 (hi(P1) ^ G),
// with A, G, H_b, I_b, J_b fixed by t, the replica and the keys: two wide products
// per node for rounds 1-3 instead of six per block, the same words as philox_rk.
template <int NB>
struct StepKeys {
  uint32_t A, G, H[NB], I[NB], J[NB];
};

template <int NB>
__device__ __forceinline__ StepKeys<NB> step_keys(const StepArgs& a, uint32_t t) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  StepKeys<NB> k;
  const uint64_t P = uint64_t(M0) * t, R = uint64_t(M1) * a.replica;
  k.A = uint32_t(R >> 32) ^ a.rk[0];
  k.G = uint32_t(P) ^ a.rk[3];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const uint32_t C = uint32_t(P >> 32) ^ (kDevTagStep | uint32_t(b)) ^ a.rk[1];  // round 2's x2
    const uint64_t R1 = uint64_t(M1) * C;
    const uint32_t E = uint32_t(R1 >> 32) ^ uint32_t(R) ^ a.rk[2];                  // round 3's x0
    const uint64_t P2 = uint64_t(M0) * E;
    k.H[b] = uint32_t(R1) ^ a.rk[4];
    k.I[b] = uint32_t(P2 >> 32) ^ a.rk[5];
    k.J[b] = uint32_t(P2);
  }
  return k;
}

// Words 0..4 NB - 1 of a node's tag-1 stream at the step its keys were made for.
template <int NB>
__device__ __forceinline__ void step_blocks(const StepKeys<NB>& k, const uint32_t (&rk)[20], uint32_t node,
                                            uint32_t (&W)[4 * NB]) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint64_t P1 = uint64_t(M0) * (node ^ k.A);
  const uint64_t R2 = uint64_t(M1) * (uint32_t(P1 >> 32) ^ k.G);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    uint4 c = make_uint4(uint32_t(R2 >> 32) ^ k.H[b], uint32_t(R2), uint32_t(P1) ^ k.I[b], k.J[b]);
#pragma unroll
    for (int r = 3; r < 10; ++r) {
      const uint64_t p0 = uint64_t(M0) * c.x;
      const uint64_t p1 = uint64_t(M1) * c.z;
      c = make_uint4(uint32_t(p1 >> 32) ^ c.y ^ rk[2 * r], uint32_t(p1), uint32_t(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                     uint32_t(p0));
    }
    W[4 * b] = c.x;
    W[4 * b + 1] = c.y;
    W[4 * b + 2] = c.z;
    W[4 * b + 3] = c.w;
  }
}

// A node's eight slot words (two blocks): from its launch's StepKeys where the caller
// made them, else from the full rounds.
__device__ __forceinline__ void slot_words8(const StepArgs& a, const StepKeys<2>* keys, uint32_t node, uint32_t t,
                                            uint32_t (&W)[8]) {
  if (keys) {
    step_blocks<2>(*keys, a.rk, node, W);
  } else {
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
    e.blk = philox_rk(counter(e.node, e.t, a.replica, kDevTagExt | b), a.rk);
    e.cached = b;
  }
  const uint32_t w = lane_of(e.blk, e.next & 3u);
  e.next += 1;
  return w;
}

// Word e of a node's extension stream, computed alone and out of line: the rare
// word beyond a thread's shared-memory buffer, kept out of the loops that read the
// buffer (inlined there, its Philox rounds weigh on every iteration).
static __device__ __noinline__ uint32_t ext_word_at(const StepArgs& a, uint32_t node, uint32_t t, uint32_t e) {
  const uint4 b = philox_rk(counter(node, t, a.replica, kDevTagExt | (e >> 2)), a.rk);
  return lane_of(b, e & 3u);
}

// The two alias tables of the block (shared memory).
__device__ __forceinline__ const uint2* thinning_table(const uint32_t* s) {
  return reinterpret_cast<const uint2*>(s);
}
__device__ __forceinline__ const uint2* rest_table(const uint32_t* s) {
  return reinterpret_cast<const uint2*>(s) + kDevAliasEntries;
}

// Binomial(n, P/2^32) for 0 <= n <= 63 with one draw u: column j = u >> 26 of row n
// (entries 64 n ..), entry 64 n + j = (n << 6) | (u >> 26) in one funnel shift;
// j if u is below the column's threshold, else its alias.
__device__ __forceinline__ uint32_t binomial_alias(const uint2* A, uint32_t n, uint32_t u) {
  const uint32_t idx = __funnelshift_l(u, n, 6);
  const uint2 e = A[idx];
  return u < e.x ? (idx & (kDevAliasCols - 1)) : e.y;
}

// Views of one alias table of the table block, called as draw(n, u).
// Alias8: the {threshold, alias} pairs as the host builds them (binomial_alias).
// Alias4: the same table packed into one word per column, for kernels short of
//   shared memory: (thr - j 2^26) << 6 | alias, or j for a full column.  The draw
//   compares u's offset within its column, shifted up over six one bits, with the
//   packed word: below it exactly when the offset is below the column's share
//   (thr - j 2^26 < 2^26), so the outcome is the same as binomial_alias's.
struct Alias8 {
  const uint2* A;
  __device__ __forceinline__ static Alias8 of(const uint32_t* s, uint32_t which) {
    return Alias8{reinterpret_cast<const uint2*>(s) + which * kDevAliasEntries};
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t n, uint32_t u) const { return binomial_alias(A, n, u); }
};
struct Alias4 {
  const uint32_t* A;
  __device__ __forceinline__ static Alias4 of(const uint32_t* s, uint32_t which) {
    return Alias4{s + which * kDevAliasEntries};
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t n, uint32_t u) const {
    const uint32_t e = A[__funnelshift_l(u, n, 6)];
    return __funnelshift_l(0xFFFFFFFFu, u, 6) < e ? (u >> 26) : (e & (kDevAliasCols - 1));
  }
};

// Stage a D1Q3 / D2Q5 lattice's table block (global memory) into shared memory as
// kDevTableWords4 words: its packed alias tables, or, for the particle sampler, the
// block's first words (they hold the boundaries B_0..B_Q).  The caller synchronises
// the block afterwards.
__device__ __forceinline__ void stage_tables4(const uint32_t* __restrict__ g, uint32_t* s, bool particle) {
  const uint4* g4 = reinterpret_cast<const uint4*>(particle ? g : g + kDevStagedWords);
#pragma unroll 8
  for (uint32_t i = threadIdx.x; i < kDevTableWords4 / 4; i += blockDim.x) reinterpret_cast<uint4*>(s)[i] = g4[i];
}

// Binomial(m, P) for any m: chunks of 63 trials, the first with the slot word,
// every further chunk with the next extension word.
__device__ __forceinline__ uint32_t binomial(uint32_t mode, const uint2* A, uint32_t m, uint32_t slot,
                                             const StepArgs& a, ExtStream& e) {
  if (mode == kNever || m == 0) return 0;
  if (mode == kAlways) return m;
  if (m <= kDevNmax) return binomial_alias(A, m, slot);
  uint32_t r = binomial_alias(A, kDevNmax, slot);
  uint32_t left = m - kDevNmax;
  while (left > 0) {
    const uint32_t c = left < kDevNmax ? left : kDevNmax;
    r += binomial_alias(A, c, ext_word(a, e));
    left -= c;
  }
  return r;
}

// The general collision of one node (any occupations).  m = occupations after
// the flip; out = n'.  s = the table block (usually in shared memory).
template <int Q>
__device__ __forceinline__ void collide(const StepArgs& a, const uint32_t* s, uint32_t node, uint32_t t,
                                        const uint32_t (&m)[Q], uint32_t (&out)[Q]) {
  const uint2* to = thinning_table(s);
  const uint2* tr = rest_table(s);
  const uint4 b0 = philox_rk(counter(node, t, a.replica, kDevTagStep | 0u), a.rk);
  const uint4 b1 = philox_rk(counter(node, t, a.replica, kDevTagStep | 1u), a.rk);
  const uint32_t W[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
  ExtStream e{node, t, 0u, 0xFFFFFFFFu, make_uint4(0, 0, 0, 0)};

  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const uint32_t r = binomial(a.omega_mode, to, m[i], W[i], a, e);
    out[i] = m[i] - r;
    removed += r;
  }
  const uint32_t to_rest = binomial(a.rest_mode, tr, removed, W[Q], a, e);
  out[0] += to_rest;
  uint32_t moving = removed - to_rest;
  bool first = true;
  while (moving > 0) {
    const uint32_t c = moving < 32 ? moving : 32;
    const uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
    if constexpr (Q == 3) {
      const uint32_t sw = first ? W[Q + 1] : ext_word(a, e);
      const uint32_t plus = __popc(~sw & mask);
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

// The general collision of one node (any occupations), in the same word order as
// collide(): the extension words [0, K) of the node are generated before the
// phase that first needs them (thinning chunks, then rest chunks, then moving
// groups), a whole Philox block at a time, into this thread's shared-memory
// buffer (word e at xb[e * S]; threads interleaved with stride S, so a warp's
// accesses hit distinct banks), so a warp runs its blocks together; words beyond K
// are read lazily, inline, or with OOL one at a time out of line (which keeps the
// loops that read the buffer small, where a kernel has registers for the call).  A
// probability of 0 or 2^32 draws nothing.
template <int Q, int K, int S, class Tab = Alias8, bool OOL = false>
__device__ __forceinline__ void collide_buffered(const StepArgs& a, const uint32_t* s, uint32_t node, uint32_t t,
                                                 const uint32_t (&m)[Q], uint32_t (&out)[Q], uint32_t* xb,
                                                 const StepKeys<2>* keys = nullptr) {
  static_assert(K % 4 == 0, "whole Philox blocks");
  const Tab to = Tab::of(s, 0);
  const Tab tr = Tab::of(s, 1);
  auto extra = [](uint32_t mode, uint32_t x) -> uint32_t { return mode == kTable && x > kDevNmax ? (x - 1) / kDevNmax : 0u; };
  uint32_t need = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) need += extra(a.omega_mode, m[i]);
  uint32_t W[8];
  slot_words8(a, keys, node, t, W);
  uint32_t filled = 0;
  auto gen = [&](uint32_t upto) {
    upto = upto < uint32_t(K) ? upto : uint32_t(K);
    for (; filled < upto; filled += 4) {
      const uint4 b = philox_rk(counter(node, t, a.replica, kDevTagExt | (filled >> 2)), a.rk);
      uint32_t* p = xb + filled * S;
      p[0] = b.x;
      p[S] = b.y;
      p[2 * S] = b.z;
      p[3 * S] = b.w;
    }
  };
  ExtStream lazy{node, t, 0u, 0xFFFFFFFFu, make_uint4(0, 0, 0, 0)};
  auto word = [&](uint32_t e) -> uint32_t {
    if (e < uint32_t(K)) return xb[e * S];
    if constexpr (OOL) return ext_word_at(a, node, t, e);
    lazy.next = e;
    return ext_word(a, lazy);
  };
  uint32_t e = 0;
  // Binomial(x, P) in chunks of 63 trials: the first with the slot word, the others
  // with the next extension words
  auto draw = [&](uint32_t mode, const Tab& A, uint32_t x, uint32_t slot) -> uint32_t {
    if (mode == kNever) return 0u;
    if (mode == kAlways) return x;
    uint32_t r = A(x < kDevNmax ? x : kDevNmax, slot);
    for (uint32_t left = x > kDevNmax ? x - kDevNmax : 0u; left > 0; left -= (left < kDevNmax ? left : kDevNmax))
      r += A(left < kDevNmax ? left : kDevNmax, word(e++));
    return r;
  };
  gen(need);
  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const uint32_t r = draw(a.omega_mode, to, m[i], W[i]);
    out[i] = m[i] - r;
    removed += r;
  }
  need += extra(a.rest_mode, removed);
  gen(need);
  const uint32_t to_rest = draw(a.rest_mode, tr, removed, W[Q]);
  out[0] += to_rest;
  const uint32_t moving = removed - to_rest;
  const uint32_t groups = (moving + 31) >> 5;
  need += groups > 1 ? (groups - 1) * (Q == 5 ? 2u : 1u) : 0u;
  gen(need);
  // groups of 32 moving particles: D1Q3 one sign word, D2Q5 an axis and a sign word
  uint32_t left = moving;
  uint32_t A = W[Q + 1], Bw = Q == 5 ? W[Q + 2] : 0u;
  while (left > 0) {
    const uint32_t c = left < 32 ? left : 32;
    const uint32_t mask = __funnelshift_lc(0xFFFFFFFFu, 0u, c);
    if constexpr (Q == 3) {
      const uint32_t minus = __popc(A & mask);
      out[1] += c - minus;
      out[2] += minus;
    } else {
      const uint32_t ax = A & mask, sg = Bw & mask;
      const uint32_t ny = __popc(ax), nmy = __popc(ax & sg), nmx = __popc(sg & ~ax);
      out[1] += c - ny - nmx;
      out[2] += nmx;
      out[3] += ny - nmy;
      out[4] += nmy;
    }
    left -= c;
    if (left > 0) {
      A = word(e++);
      if constexpr (Q == 5) Bw = word(e++);
    }
  }
}

// The collision of one node with the particle sampler: particle k of velocity i
// (in the order i = 0..Q-1, k = 0..m_i-1) takes word d (its running index) of the
// tag-4 stream and stays when u < B_0, otherwise goes to the velocity j with
// B_j <= u < B_{j+1}.  s holds B_0..B_Q as 64-bit integers (B_Q = 2^32).
// The loop runs over whole Philox blocks, so a warp computes its blocks together;
// a word's velocity follows from the prefix sums of m, and counts of picked
// particles at or above each prefix sum (each boundary) give the removals (the
// arrivals) without a dynamically indexed array.
template <int Q>
__device__ void collide_particle(const StepArgs& a, const uint32_t* s, uint32_t node, uint32_t t,
                                 const uint32_t (&m)[Q], uint32_t (&out)[Q]) {
  // D1Q3 / D2Q5 keep the boundaries in registers; D2Q9 reads them from shared memory
  // per comparison to spare registers
  const unsigned long long* B = reinterpret_cast<const unsigned long long*>(s);
  unsigned long long breg[Q <= 5 ? Q : 1];
#pragma unroll
  for (int k = 0; k < (Q <= 5 ? Q : 1); ++k) breg[k] = B[k];
  auto bound = [&](int k) -> unsigned long long { if constexpr (Q <= 5) return breg[k]; else return B[k]; };
  uint32_t start[Q];  // start[k]: running index of the first particle of velocity k
  uint32_t N = 0;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    start[k] = N;
    N += m[k];
  }
  uint32_t ge[Q];     // ge[0]: picked particles; ge[j]: picked ones with u >= B_j
  uint32_t from[Q];   // from[0]: picked particles; from[k]: picked ones of velocity >= k
#pragma unroll
  for (int k = 0; k < Q; ++k) ge[k] = from[k] = 0;
  if (bound(0) < (1ull << 32)) {  // B_0 = 2^32: every particle stays, the words are not needed
    for (uint32_t b = 0; 4 * b < N; ++b) {
      const uint4 blk = philox_rk(counter(node, t, a.replica, kDevTagParticle | b), a.rk);
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t d = 4 * b + q;
        const unsigned long long u = lane_of(blk, q);
        if (d < N && u >= bound(0)) {
          ge[0] += 1;
          from[0] += 1;
#pragma unroll
          for (int j = 1; j < Q; ++j) {
            ge[j] += u >= bound(j) ? 1u : 0u;
            from[j] += d >= start[j] ? 1u : 0u;
          }
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    const uint32_t removed = from[j] - (j + 1 < Q ? from[j + 1] : 0u);
    const uint32_t arrived = ge[j] - (j + 1 < Q ? ge[j + 1] : 0u);
    out[j] = m[j] - removed + arrived;
  }
}

// The general collision in whichever sampler the lattice uses.
template <int Q, int K, int S, class Tab = Alias8, bool OOL = false>
__device__ __forceinline__ void collide_general(const StepArgs& a, const uint32_t* s, uint32_t node, uint32_t t,
                                                const uint32_t (&m)[Q], uint32_t (&out)[Q], uint32_t* xb,
                                                const StepKeys<2>* keys = nullptr) {
  if (a.particle) collide_particle<Q>(a, s, node, t, m, out);
  else collide_buffered<Q, K, S, Tab, OOL>(a, s, node, t, m, out, xb, keys);
}

// The collision of one node, fast path: every occupation <= 63, at most 63
// removed and at most 32 moving particles, so no extension word is needed, and
// both probabilities drawn through their tables (0 < P < 2^32).  Returns false
// (out undefined) when the node falls outside that domain; the caller then runs
// collide().  Same result as collide() wherever it returns true.  No result can
// exceed 65535 here (mass is conserved and at most 5 * 63).
template <int Q, class Tab = Alias8>
__device__ __forceinline__ bool collide_try_fast(const StepArgs& a, const uint32_t* s, uint32_t node,
                                                 uint32_t t, const uint32_t (&m)[Q], uint32_t (&out)[Q],
                                                 const StepKeys<2>* keys = nullptr) {
  const Tab to = Tab::of(s, 0);
  const Tab tr = Tab::of(s, 1);
  if (a.omega_mode != kTable || a.rest_mode != kTable) return false;
  uint32_t any = m[0];
#pragma unroll
  for (int i = 1; i < Q; ++i) any |= m[i];
  if (any >> 6) return false;
  // slot words: thinning 0..Q-1, rest Q, moving Q+1 (and Q+2)
  uint32_t W[8];
  slot_words8(a, keys, node, t, W);
  uint32_t r[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) r[i] = to(m[i], W[i]);
  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) removed += r[i];
  if (removed >> 6) return false;
  const uint32_t to_rest = tr(removed, W[Q]);
  const uint32_t moving = removed - to_rest;
  if (moving > 32) return false;
  const uint32_t mask = moving == 32 ? 0xFFFFFFFFu : ((1u << moving) - 1u);
  out[0] = m[0] - r[0] + to_rest;
  if constexpr (Q == 3) {
    const uint32_t minus = __popc(W[Q + 1] & mask);
    out[1] = m[1] - r[1] + (moving - minus);
    out[2] = m[2] - r[2] + minus;
  } else {
    const uint32_t ax = W[Q + 1] & mask, sg = W[Q + 2] & mask;
    const uint32_t ny = __popc(ax);          // to +y or -y
    const uint32_t nmy = __popc(ax & sg);    // to -y
    const uint32_t nmx = __popc(sg & ~ax);   // to -x
    out[1] = m[1] - r[1] + (moving - ny - nmx);
    out[2] = m[2] - r[2] + nmx;
    out[3] = m[3] - r[3] + (ny - nmy);
    out[4] = m[4] - r[4] + nmy;
  }
  return true;
}

}  // namespace ilg
