// D2Q9 collision of one node (shared by the node-parallel D2Q9 kernels and the
// staged warp kernel): the collision thins every velocity, sends a binomial share of
// the removed particles to rest, splits the moving ones binomially into axis and
// diagonal particles, and gives each axis particle an axis bit and a sign bit and
// each diagonal particle an x-sign and a y-sign bit (slot words 11/12 and 13/14 for
// the first group of 32).  The table block holds the thinning, rest and axis-share
// alias tables, one after the other.
#pragma once

#include <cstdint>

#include "ilg_device.cuh"

namespace ilg {

// velocity order: rest, +x, -x, +y, -y, (+1,+1), (-1,-1), (+1,-1), (-1,+1)
__device__ __forceinline__ int d9_vx(int i) { return (i == 1 || i == 5 || i == 7) ? 1 : ((i == 2 || i == 6 || i == 8) ? -1 : 0); }
__device__ __forceinline__ int d9_vy(int i) { return (i == 3 || i == 5 || i == 8) ? 1 : ((i == 4 || i == 6 || i == 7) ? -1 : 0); }

__device__ __forceinline__ const uint2* axis_table(const uint32_t* s) {
  return reinterpret_cast<const uint2*>(s) + 2 * kDevAliasEntries;
}

// axis particles (c <= 32): axis word A, sign word B, as on D2Q5
__device__ __forceinline__ void add_axis(uint32_t c, uint32_t A, uint32_t Bw, uint32_t (&out)[9]) {
  const uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
  A &= mask;
  Bw &= mask;
  const uint32_t ny = __popc(A), nmy = __popc(A & Bw), nmx = __popc(Bw & ~A);
  out[1] += c - ny - nmx;
  out[2] += nmx;
  out[3] += ny - nmy;
  out[4] += nmy;
}

// diagonal particles (c <= 32): x-sign word X, y-sign word Y
__device__ __forceinline__ void add_diag(uint32_t c, uint32_t X, uint32_t Y, uint32_t (&out)[9]) {
  const uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
  X &= mask;
  Y &= mask;
  const uint32_t nmm = __popc(X & Y);        // (-1,-1)
  const uint32_t npm = __popc(Y) - nmm;      // (+1,-1)
  const uint32_t nmp = __popc(X) - nmm;      // (-1,+1)
  out[5] += c - nmm - npm - nmp;
  out[6] += nmm;
  out[7] += npm;
  out[8] += nmp;
}

// Fast path: every occupation <= 63, at most 63 removed, at most 32 axis and 32
// diagonal movers, all three probabilities drawn through tables.  False outside.
__device__ __forceinline__ bool collide9_try_fast(const StepArgs& a, const uint32_t* s, uint32_t node, uint32_t t,
                                                  const uint32_t (&m)[9], uint32_t (&out)[9]) {
  if (a.omega_mode != kTable || a.rest_mode != kTable || a.axis_mode != kTable) return false;
  uint32_t any = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) any |= m[i];
  if (any >> 6) return false;
  uint32_t W[16];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint4 w = philox_rk(counter(node, t, a.replica, kDevTagStep | uint32_t(b)), a.rk);
    W[4 * b] = w.x;
    W[4 * b + 1] = w.y;
    W[4 * b + 2] = w.z;
    W[4 * b + 3] = w.w;
  }
  const uint2* to = thinning_table(s);
  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const uint32_t r = binomial_alias(to, m[i], W[i]);
    out[i] = m[i] - r;
    removed += r;
  }
  if (removed >> 6) return false;
  const uint32_t to_rest = binomial_alias(rest_table(s), removed, W[9]);
  const uint32_t moving = removed - to_rest;
  const uint32_t axis = binomial_alias(axis_table(s), moving, W[10]);
  const uint32_t diag = moving - axis;
  if (axis > 32 || diag > 32) return false;
  out[0] += to_rest;
  add_axis(axis, W[11], W[12], out);
  add_diag(diag, W[13], W[14], out);
  return true;
}

// General path: any occupations, extension words read lazily in the order
// thinning chunks, rest chunks, axis-share chunks, axis groups, diagonal groups.
__device__ __forceinline__ void collide9_general(const StepArgs& a, const uint32_t* s, uint32_t node, uint32_t t,
                                 const uint32_t (&m)[9], uint32_t (&out)[9]) {
  uint32_t W[16];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint4 w = philox_rk(counter(node, t, a.replica, kDevTagStep | uint32_t(b)), a.rk);
    W[4 * b] = w.x;
    W[4 * b + 1] = w.y;
    W[4 * b + 2] = w.z;
    W[4 * b + 3] = w.w;
  }
  ExtStream e{node, t, 0u, 0xFFFFFFFFu, make_uint4(0, 0, 0, 0)};
  const uint2* to = thinning_table(s);
  uint32_t removed = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const uint32_t r = binomial(a.omega_mode, to, m[i], W[i], a, e);
    out[i] = m[i] - r;
    removed += r;
  }
  const uint32_t to_rest = binomial(a.rest_mode, rest_table(s), removed, W[9], a, e);
  out[0] += to_rest;
  const uint32_t moving = removed - to_rest;
  uint32_t axis = binomial(a.axis_mode, axis_table(s), moving, W[10], a, e);
  uint32_t diag = moving - axis;
  bool first = true;
  while (axis > 0) {
    const uint32_t c = axis < 32 ? axis : 32;
    const uint32_t A = first ? W[11] : ext_word(a, e);
    const uint32_t Bw = first ? W[12] : ext_word(a, e);
    add_axis(c, A, Bw, out);
    axis -= c;
    first = false;
  }
  first = true;
  while (diag > 0) {
    const uint32_t c = diag < 32 ? diag : 32;
    const uint32_t X = first ? W[13] : ext_word(a, e);
    const uint32_t Y = first ? W[14] : ext_word(a, e);
    add_diag(c, X, Y, out);
    diag -= c;
    first = false;
  }
}

}  // namespace ilg
