/*
 * Plain CPU oracle for the over-relaxed diffusive integer lattice gas
 * (Strand & Wagner, "Over-Relaxation in Diffusive Integer Lattice Gas").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table generator or constant generator with the CUDA path; both
 * implement the same written definition independently.
 *
 * Everything here is single-threaded, slow and written to be checked by eye:
 * one node at a time, one decision at a time, linear searches.
 *
 * What it computes, one time step t -> t+1, for every node x:
 *   1. m_i = n_i(x,t), or m_i = n_{-i}(x,t) when flipping is on
 *      (flip operator F_i(n) = n_{-i}, Sec. III, Eq. (flip); applied before the
 *      collision as in the flipped evolution equation, Sec. III).
 *   2. sampling collision with collision fraction omega* (Sec. II: a fraction
 *      of the particles is picked at random and redistributed with
 *      probabilities w_i):
 *        r_i  = Binomial(m_i, omega*)     particles removed from velocity i
 *        R    = sum_i r_i
 *        R_0  = Binomial(R, w_0)          removed particles sent to rest
 *        the other R - R_0 pick one of the moving velocities uniformly
 *        (all moving weights are equal, w = theta/2 each)
 *        n'_i = m_i - r_i + (particles received by i)
 *      Mass sum_i n'_i = sum_i m_i is conserved exactly (Sec. II, Eq. 2).
 *   3. streaming n_i(x + v_i, t+1) = n'_i(x), periodic (Sec. II, Eq. ilgeq).
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written here
 * from its published round function.  Counter = (t, node id, replica,
 * tag<<24 | block), key = (seed lo, seed hi); word d of a stream is lane d&3 of
 * block d>>2.  Binomial draws go through an alias table built in integers from
 * a pmf that is defined by an integer Pascal recurrence (below), so both
 * implementations produce the same bits without floating point.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NMAX 63u      /* largest binomial trial count taken by one table row */
#define OR_ALIAS_COLS 64u /* columns of every alias row; column j covers u >> 26 == j */
#define OR_TAG_STEP 1u
#define OR_TAG_EXT 2u
#define OR_TAG_INIT 3u
#define OR_TAG_PARTICLE 4u
#define OR_POISSON_KMAX 4096u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* word d of the stream (t, node, replica, tag) under key seed */
static uint32_t stream_word(uint64_t seed, uint32_t node, uint32_t t, uint32_t replica,
                            uint32_t tag, uint32_t d) {
  uint32_t ctr[4] = {t, node, replica, (tag << 24) | (d >> 2)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  oracle_philox(ctr, key, out);
  return out[d & 3u];
}

/* ------------------------------------------------------------------------ */
/* Binomial CDF table                                                        */
/* ------------------------------------------------------------------------ */
/*
 * Probability p = P / 2^32, 0 < P < 2^32, q = (2^32 - P) / 2^32.
 * pmf rows in fixed point with 1.0 = 2^63:
 *   f_0(0) = 2^63
 *   f_n(k) = floor(f_{n-1}(k) * (2^32-P) / 2^32) + floor(f_{n-1}(k-1) * P / 2^32)
 *            (terms with k-1 < 0 or k > n-1 are zero)
 * CDF row n (1 <= n <= nmax), k = 0..n-1:
 *   T[n][k] = floor( (f_n(0) + ... + f_n(k)) / 2^31 )
 * stored at T[n(n-1)/2 + k].  Every entry lies in [0, 2^32 - 1].
 */
void oracle_binomial_table(uint64_t P, uint32_t nmax, uint32_t *T) {
  uint64_t *f = (uint64_t *)calloc(nmax + 2, sizeof(uint64_t));
  uint64_t *g = (uint64_t *)calloc(nmax + 2, sizeof(uint64_t));
  uint64_t Q = ((uint64_t)1 << 32) - P;
  f[0] = (uint64_t)1 << 63;
  for (uint32_t n = 1; n <= nmax; ++n) {
    for (uint32_t k = 0; k <= n; ++k) {
      unsigned __int128 stay = 0, move = 0;
      if (k <= n - 1) stay = ((unsigned __int128)f[k] * Q) >> 32;
      if (k >= 1) move = ((unsigned __int128)f[k - 1] * P) >> 32;
      g[k] = (uint64_t)(stay + move);
    }
    for (uint32_t k = 0; k <= n; ++k) f[k] = g[k];
    uint64_t cum = 0;
    for (uint32_t k = 0; k < n; ++k) {
      cum += f[k];
      T[n * (n - 1) / 2 + k] = (uint32_t)(cum >> 31);
    }
  }
  free(f);
  free(g);
}

/*
 * Alias table (Walker's method, Vose's construction in integers) over the same
 * integer pmf.  Row n (0 <= n <= nmax <= 63) has 64 columns j of 2^26 draws
 * each (column j covers j 2^26 <= u < (j+1) 2^26), stored at offset 64 n.
 * Outcome weights: W_0 = T[n][0], W_k = T[n][k] - T[n][k-1] (0 < k < n),
 * W_n = 2^32 - T[n][n-1] (W_0 = 2^32 for n = 0), W_k = 0 for n < k < 64; they
 * sum to 2^32.  A draw u picks column j = u >> 26 and yields j if u < thr[j],
 * else alias[j].
 * Construction: columns with W_j = 2^26 are full (alias = j); the others go on a
 * "small" (W_j < 2^26) or "large" (W_j > 2^26) stack, pushed in increasing j.
 * While both stacks are non-empty: pop l (small) and g (large) from their tops;
 * column l gives its first W_l draws to l (thr[l] = l 2^26 + W_l) and the rest
 * to g (alias[l] = g); W_g drops by 2^26 - W_l and g is pushed back on the stack
 * its new weight belongs to (or is full).  Every outcome's weight is realised
 * exactly; columns of the zero-weight outcomes k > n go wholly to their alias.
 */
void oracle_alias_table(uint64_t P, uint32_t nmax, uint32_t *thr, uint8_t *alias) {
  const uint64_t s = (uint64_t)1 << 26; /* draws per column */
  if (nmax >= OR_ALIAS_COLS) return;     /* a row holds at most 64 outcomes */
  uint32_t *T = (uint32_t *)malloc(sizeof(uint32_t) * (nmax * (nmax + 1) / 2 + 1));
  uint64_t W[OR_ALIAS_COLS];
  uint32_t small[OR_ALIAS_COLS], large[OR_ALIAS_COLS];
  oracle_binomial_table(P, nmax, T);
  for (uint32_t n = 0; n <= nmax; ++n) {
    const uint32_t *row = T + (n ? n * (n - 1) / 2 : 0);
    uint32_t *th = thr + OR_ALIAS_COLS * n;
    uint8_t *al = alias + OR_ALIAS_COLS * n;
    uint64_t prev = 0;
    for (uint32_t k = 0; k < OR_ALIAS_COLS; ++k) W[k] = 0;
    for (uint32_t k = 0; k < n; ++k) {
      W[k] = (uint64_t)row[k] - prev;
      prev = row[k];
    }
    W[n] = ((uint64_t)1 << 32) - prev;
    uint32_t ns = 0, nl = 0;
    for (uint32_t j = 0; j < OR_ALIAS_COLS; ++j) {
      th[j] = 0;
      al[j] = (uint8_t)j;
      if (W[j] < s) small[ns++] = j;
      else if (W[j] > s) large[nl++] = j;
    }
    while (ns > 0 && nl > 0) {
      uint32_t l = small[--ns];
      uint32_t g = large[--nl];
      th[l] = (uint32_t)((uint64_t)l * s + W[l]);
      al[l] = (uint8_t)g;
      W[g] -= s - W[l];
      if (W[g] < s) small[ns++] = g;
      else if (W[g] > s) large[nl++] = g;
    }
  }
  free(T);
}

/* Binomial(n, P/2^32) for n <= OR_NMAX: one draw through row n of the alias table */
static uint32_t binomial_draw(const uint32_t *thr, const uint8_t *alias, uint32_t n, uint32_t u) {
  uint32_t off = OR_ALIAS_COLS * n;
  uint32_t j = u >> 26;
  return u < thr[off + j] ? j : alias[off + j];
}

/* ------------------------------------------------------------------------ */
/* Parameters                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t lattice;    /* 1 = D1Q3, 2 = D2Q5 */
  uint32_t Lx, Ly;    /* Ly = 1 for D1Q3 */
  int32_t flip;       /* 1 when omega_eff > 1 */
  uint64_t P_omega;   /* round(omega* * 2^32) in [0, 2^32] */
  uint64_t P_rest;    /* round(w_0 * 2^32) in [0, 2^32] */
  uint64_t seed;
  uint32_t replica;
  const uint32_t *thr_omega; /* alias table of P_omega (unused if P_omega is 0 or 2^32) */
  const uint8_t *alias_omega;
  const uint32_t *thr_rest;  /* alias table of P_rest (unused if P_rest is 0 or 2^32) */
  const uint8_t *alias_rest;
  int32_t sampler;           /* 0: binomial draws (collide_node); 1: one word per particle */
  uint64_t P_axis;           /* D2Q9: round(4 w_axis / (1 - w_0) * 2^32), share of the axis velocities */
  const uint32_t *thr_axis;  /* alias table of P_axis (D2Q9 only) */
  const uint8_t *alias_axis;
} oracle_step_params;

static int num_vel(int32_t lattice) { return lattice == 1 ? 3 : (lattice == 2 ? 5 : 9); }

/* velocity sets, rest first: D1Q3 {0, +1, -1}; D2Q5 {0, +x, -x, +y, -y} */
static const int VX3[3] = {0, 1, -1};
static const int VX5[5] = {0, 1, -1, 0, 0};
static const int VY5[5] = {0, 0, 0, 1, -1};
static const int OPP3[3] = {0, 2, 1};
static const int OPP5[5] = {0, 2, 1, 4, 3};
/* D2Q9: rest, +x, -x, +y, -y, (+1,+1), (-1,-1), (+1,-1), (-1,+1) */
static const int VX9[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
static const int VY9[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
static const int OPP9[9] = {0, 2, 1, 4, 3, 6, 5, 8, 7};

/* sequential reader of the extension stream of one node and step */
typedef struct {
  const oracle_step_params *p;
  uint32_t node, t, next;
} ext_reader;

static uint32_t ext_next(ext_reader *e) {
  uint32_t w = stream_word(e->p->seed, e->node, e->t, e->p->replica, OR_TAG_EXT, e->next);
  e->next += 1;
  return w;
}

/* Binomial(m, P/2^32): chunks of at most OR_NMAX trials; the first chunk uses
 * the word of its fixed slot, every further chunk the next extension word. */
static uint32_t binomial_chunked(uint64_t P, const uint32_t *thr, const uint8_t *alias, uint32_t m,
                                 uint32_t slot_word, ext_reader *ext) {
  if (P == 0) return 0;
  if (P == ((uint64_t)1 << 32)) return m;
  uint32_t r = 0, left = m;
  int first = 1;
  while (left > 0) {
    uint32_t c = left < OR_NMAX ? left : OR_NMAX;
    uint32_t u = first ? slot_word : ext_next(ext);
    first = 0;
    r += binomial_draw(thr, alias, c, u);
    left -= c;
  }
  return r;
}

static uint32_t popcount32(uint32_t v) {
  uint32_t c = 0;
  while (v) { c += v & 1u; v >>= 1; }
  return c;
}

/* The collision of one node.  m[] is the (already flipped) occupation,
 * out[] receives n'.  Slot words W[0..7] are words 0..7 of the step stream. */
static void collide_node(const oracle_step_params *p, uint32_t node, uint32_t t,
                         const uint32_t *m, uint32_t *out) {
  int Q = num_vel(p->lattice);
  uint32_t W[16];
  for (uint32_t d = 0; d < 16; ++d) W[d] = stream_word(p->seed, node, t, p->replica, OR_TAG_STEP, d);
  ext_reader ext = {p, node, t, 0};

  /* thinning: r_i = Binomial(m_i, omega*), slot word i */
  uint32_t removed_total = 0;
  for (int i = 0; i < Q; ++i) {
    uint32_t r = binomial_chunked(p->P_omega, p->thr_omega, p->alias_omega, m[i], W[i], &ext);
    out[i] = m[i] - r;
    removed_total += r;
  }
  /* rest share: R_0 = Binomial(R, w_0), slot word Q */
  uint32_t to_rest = binomial_chunked(p->P_rest, p->thr_rest, p->alias_rest, removed_total, W[Q], &ext);
  out[0] += to_rest;
  uint32_t moving = removed_total - to_rest;

  if (Q == 9) {
    /* D2Q9: the moving particles split into axis and diagonal ones, R_a =
     * Binomial(moving, 4 w_axis / (1 - w_0)) with slot word 10; then per group of 32
     * axis particles an axis word A and a sign word B (slot words 11, 12 for the
     * first group) as on D2Q5, and per group of 32 diagonal particles an x-sign word
     * X and a y-sign word Y (slot words 13, 14 for the first group): (0,0) -> (+1,+1),
     * (1,1) -> (-1,-1), (0,1) -> (+1,-1), (1,0) -> (-1,+1).  Later groups take
     * extension words, two per group, axis groups before diagonal groups. */
    uint32_t axis = binomial_chunked(p->P_axis, p->thr_axis, p->alias_axis, moving, W[10], &ext);
    uint32_t diag = moving - axis;
    uint32_t group = 0;
    while (axis > 0) {
      uint32_t c = axis < 32 ? axis : 32;
      uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
      uint32_t a = group == 0 ? W[11] : ext_next(&ext);
      uint32_t b = group == 0 ? W[12] : ext_next(&ext);
      out[1] += popcount32(~a & ~b & mask);
      out[2] += popcount32(~a & b & mask);
      out[3] += popcount32(a & ~b & mask);
      out[4] += popcount32(a & b & mask);
      axis -= c;
      group += 1;
    }
    group = 0;
    while (diag > 0) {
      uint32_t c = diag < 32 ? diag : 32;
      uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
      uint32_t x = group == 0 ? W[13] : ext_next(&ext);
      uint32_t y = group == 0 ? W[14] : ext_next(&ext);
      out[5] += popcount32(~x & ~y & mask);
      out[6] += popcount32(x & y & mask);
      out[7] += popcount32(~x & y & mask);
      out[8] += popcount32(x & ~y & mask);
      diag -= c;
      group += 1;
    }
    return;
  }

  /* uniform choice among the moving velocities, groups of 32 particles */
  uint32_t group = 0;
  while (moving > 0) {
    uint32_t c = moving < 32 ? moving : 32;
    uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
    if (Q == 3) {
      uint32_t s = group == 0 ? W[Q + 1] : ext_next(&ext);
      /* bit 0 -> +1 (index 1), bit 1 -> -1 (index 2) */
      uint32_t plus = popcount32(~s & mask);
      out[1] += plus;
      out[2] += c - plus;
    } else {
      uint32_t a = group == 0 ? W[Q + 1] : ext_next(&ext); /* axis bit: 0 = x, 1 = y */
      uint32_t b = group == 0 ? W[Q + 2] : ext_next(&ext); /* sign bit: 0 = +, 1 = - */
      out[1] += popcount32(~a & ~b & mask);
      out[2] += popcount32(~a & b & mask);
      out[3] += popcount32(a & ~b & mask);
      out[4] += popcount32(a & b & mask);
    }
    moving -= c;
    group += 1;
  }
}

/* ------------------------------------------------------------------------ */
/* Particle sampler: every particle decides on its own word                  */
/* ------------------------------------------------------------------------ */
/*
 * The same law as above, drawn the plain way (Sec. II: each particle is picked
 * with probability omega* and a picked particle goes to velocity j with
 * probability w_j).  One 32-bit word u per particle, from the tag-4 stream of
 * the node, in particle order (velocity 0..Q-1 of the flipped occupation, then
 * particle 0..m_i-1).  The word is compared with integer boundaries
 *   B_0     = 2^32 - P_omega                      (below: the particle stays)
 *   B_{j+1} = B_0 + floor(P_omega (P_rest (Q-1) + j (2^32 - P_rest)) / ((Q-1) 2^32))
 * for j = 0..Q-1 (B_Q = 2^32): a particle with B_j <= u < B_{j+1} goes to
 * velocity j.  Picked with probability P_omega / 2^32; then rest with P_rest / 2^32
 * and each moving velocity with an equal share of the remainder (to within one
 * unit of 2^-32 per boundary).
 */
static void particle_bounds(int Q, uint64_t P_omega, uint64_t P_rest, uint64_t P_axis, uint64_t *B) {
  const unsigned __int128 two32 = (unsigned __int128)1 << 32;
  B[0] = (uint64_t)(two32 - P_omega);
  if (Q == 9) {
    /* shares of a picked particle, in units of 1 / (4 2^64): rest 4 P_rest 2^32, each axis
     * velocity (2^32 - P_rest) P_axis, each diagonal (2^32 - P_rest) (2^32 - P_axis) */
    unsigned __int128 cum = (unsigned __int128)4 * P_rest * two32;
    const unsigned __int128 den = (unsigned __int128)4 << 64;
    for (int j = 0; j < 9; ++j) {
      if (j >= 1 && j <= 4) cum += (two32 - P_rest) * (unsigned __int128)P_axis;
      if (j >= 5) cum += (two32 - P_rest) * (two32 - P_axis);
      /* P_omega * cum <= 2^32 * 2^66 fits in 128 bits */
      B[j + 1] = B[0] + (uint64_t)(((unsigned __int128)P_omega * cum) / den);
    }
    return;
  }
  for (int j = 0; j < Q; ++j) {
    unsigned __int128 num = (unsigned __int128)P_omega *
                            ((unsigned __int128)P_rest * (unsigned)(Q - 1) + (unsigned __int128)j * (two32 - P_rest));
    unsigned __int128 den = (unsigned __int128)(unsigned)(Q - 1) << 32;
    B[j + 1] = B[0] + (uint64_t)(num / den);
  }
}

static void collide_node_particle(const oracle_step_params *p, uint32_t node, uint32_t t,
                                  const uint32_t *m, uint32_t *out) {
  int Q = num_vel(p->lattice);
  uint64_t B[10];
  particle_bounds(Q, p->P_omega, p->P_rest, p->P_axis, B);
  for (int i = 0; i < Q; ++i) out[i] = 0;
  uint32_t d = 0;
  for (int i = 0; i < Q; ++i) {
    for (uint32_t k = 0; k < m[i]; ++k) {
      uint64_t u = stream_word(p->seed, node, t, p->replica, OR_TAG_PARTICLE, d);
      d += 1;
      if (u < B[0]) {
        out[i] += 1;
      } else {
        int j = 0;
        while (u >= B[j + 1]) j += 1;
        out[j] += 1;
      }
    }
  }
}

static void collide_any(const oracle_step_params *p, uint32_t node, uint32_t t, const uint32_t *m,
                        uint32_t *out) {
  if (p->sampler == 1) collide_node_particle(p, node, t, m, out);
  else collide_node(p, node, t, m, out);
}

/* exported for the tests: the boundaries B_0..B_Q */
void oracle_particle_bounds(int32_t lattice, uint64_t P_omega, uint64_t P_rest, uint64_t P_axis, uint64_t *B) {
  particle_bounds(num_vel(lattice), P_omega, P_rest, P_axis, B);
}

/* ------------------------------------------------------------------------ */
/* Time step over a rectangular region                                       */
/* ------------------------------------------------------------------------ */
/*
 * in/out hold a w x h patch whose lower corner sits at global node (x0, y0)
 * of the Lx x Ly periodic lattice, as planes [Q][h][w], x fastest.  Global
 * coordinates (taken modulo Lx, Ly) name the random streams.
 * periodic != 0 requires the patch to be the whole lattice and wraps streaming;
 * otherwise particles that leave the patch are dropped and cells fed from
 * outside the patch are left at 0 (they are invalid: callers crop one layer
 * per step).  Returns 0, or 3 when some n'_i exceeds 65535 (out is then
 * incomplete).
 */
int oracle_step_region(const oracle_step_params *p, const uint16_t *in, uint16_t *out,
                       uint32_t x0, uint32_t y0, uint32_t w, uint32_t h, int periodic,
                       uint32_t t) {
  int Q = num_vel(p->lattice);
  const int *VX = Q == 3 ? VX3 : (Q == 5 ? VX5 : VX9);
  const int *VY = Q == 3 ? VX3 : (Q == 5 ? VY5 : VY9); /* unused for D1Q3 */
  const int *OPP = Q == 3 ? OPP3 : (Q == 5 ? OPP5 : OPP9);
  size_t plane = (size_t)w * h;
  memset(out, 0, sizeof(uint16_t) * plane * Q);
  for (uint32_t j = 0; j < h; ++j) {
    for (uint32_t i = 0; i < w; ++i) {
      uint32_t gx = (x0 + i) % p->Lx, gy = (y0 + j) % p->Ly;
      uint32_t node = gx + p->Lx * gy;
      uint32_t n[9], m[9], post[9];
      for (int v = 0; v < Q; ++v) n[v] = in[v * plane + (size_t)j * w + i];
      for (int v = 0; v < Q; ++v) m[v] = p->flip ? n[OPP[v]] : n[v];
      collide_any(p, node, t, m, post);
      for (int v = 0; v < Q; ++v) {
        if (post[v] > 65535u) return 3;
        long di = (long)i + VX[v];
        long dj = (long)j + (Q == 3 ? 0 : VY[v]);
        if (periodic) {
          di = (di + (long)w) % (long)w;
          dj = (dj + (long)h) % (long)h;
        } else if (di < 0 || dj < 0 || di >= (long)w || dj >= (long)h) {
          continue;
        }
        out[v * plane + (size_t)dj * w + (size_t)di] = (uint16_t)post[v];
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Poisson initial state (Sec. V: Poisson numbers with mean w_i P(rho))      */
/* ------------------------------------------------------------------------ */
/*
 * CDF table of Poisson(lambda) in double precision, then quantised:
 *   p_0 = exp(-lambda); c_0 = p_0; p_k = p_{k-1} * lambda / k; c_k = c_{k-1} + p_k
 *   T[k] = min(floor(c_k * 2^32), 2^32 - 1), stopping at the first k with
 *   T[k] = 2^32 - 1 (K = k + 1 entries).
 * A draw u gives the number of j < K-1 with u >= T[j].
 * Returns K, or 0 when K would exceed kmax.
 */
uint32_t oracle_poisson_table(double lambda, uint32_t *T, uint32_t kmax) {
  double pk = exp(-lambda);
  double c = pk;
  for (uint32_t k = 0; k < kmax; ++k) {
    if (k > 0) {
      pk = pk * lambda / (double)k;
      c = c + pk;
    }
    double scaled = floor(c * 4294967296.0);
    uint32_t v = scaled >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)scaled;
    T[k] = v;
    if (v == 0xFFFFFFFFu) return k + 1;
  }
  return 0;
}

typedef struct {
  int32_t lattice;
  uint32_t Lx, Ly;
  double n0, amp;
  int32_t mode_mx, mode_my;
  int32_t init_weighted;
  double theta;
  uint64_t seed;
  uint32_t replica;
} oracle_init_params;

/* mean of velocity v at global node (gx, gy), as the initial condition states */
double oracle_init_lambda(const oracle_init_params *p, uint32_t gx, uint32_t gy, int v) {
  int Q = num_vel(p->lattice);
  double s = 0.0;
  if (p->mode_mx != 0) {
    uint32_t mx = (uint32_t)(((int64_t)p->mode_mx % (int64_t)p->Lx + (int64_t)p->Lx) % (int64_t)p->Lx);
    uint32_t r = (uint32_t)(((uint64_t)mx * gx) % p->Lx);
    s = sin((6.283185307179586 * (double)r) / (double)p->Lx);
  } else if (p->mode_my != 0) {
    uint32_t my = (uint32_t)(((int64_t)p->mode_my % (int64_t)p->Ly + (int64_t)p->Ly) % (int64_t)p->Ly);
    uint32_t r = (uint32_t)(((uint64_t)my * gy) % p->Ly);
    s = sin((6.283185307179586 * (double)r) / (double)p->Ly);
  }
  if (p->init_weighted) {
    double w;
    if (Q == 3) w = v == 0 ? 1.0 - p->theta : p->theta / 2.0;
    else if (Q == 5) w = v == 0 ? 1.0 - 2.0 * p->theta : p->theta / 2.0;
    else w = v == 0 ? (1.0 - p->theta) * (1.0 - p->theta)
                    : (v <= 4 ? (p->theta * (1.0 - p->theta)) / 2.0 : (p->theta * p->theta) / 4.0);
    return w * ((double)Q * p->n0 + p->amp * s);
  }
  return p->n0 + (p->amp * s) / (double)Q;
}

/* Fill a w x h patch at (x0, y0) with the Poisson initial state.
 * Returns 0, or 1 if some mean is negative or its table exceeds the cap. */
int oracle_init_region(const oracle_init_params *p, uint16_t *out, uint32_t x0, uint32_t y0,
                       uint32_t w, uint32_t h) {
  int Q = num_vel(p->lattice);
  size_t plane = (size_t)w * h;
  uint32_t *T = (uint32_t *)malloc(sizeof(uint32_t) * OR_POISSON_KMAX);
  double cached = -1.0;
  uint32_t K = 0;
  for (uint32_t j = 0; j < h; ++j) {
    for (uint32_t i = 0; i < w; ++i) {
      uint32_t gx = (x0 + i) % p->Lx, gy = (y0 + j) % p->Ly;
      uint32_t node = gx + p->Lx * gy;
      for (int v = 0; v < Q; ++v) {
        double lam = oracle_init_lambda(p, gx, gy, v);
        if (!(lam >= 0.0)) { free(T); return 1; }
        if (lam != cached) {
          K = oracle_poisson_table(lam, T, OR_POISSON_KMAX);
          if (K == 0) { free(T); return 1; }
          cached = lam;
        }
        uint32_t u = stream_word(p->seed, node, 0u, p->replica, OR_TAG_INIT, (uint32_t)v);
        uint32_t x = 0;
        while (x < K - 1 && u >= T[x]) ++x;
        out[v * plane + (size_t)j * w + i] = (uint16_t)x;
      }
    }
  }
  free(T);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Integer observables                                                       */
/* ------------------------------------------------------------------------ */
/* N(x,y) = sum_i n_i; column sums C(x) = sum_y N; row sums R(y) = sum_x N;
 * mass M = sum N (Sec. V: the measured amplitude sums N(x,t)). */
void oracle_sums(int32_t lattice, uint32_t Lx, uint32_t Ly, const uint16_t *state,
                 int64_t *col, int64_t *row, uint64_t *mass) {
  int Q = num_vel(lattice);
  size_t plane = (size_t)Lx * Ly;
  uint64_t M = 0;
  for (uint32_t x = 0; x < Lx; ++x) col[x] = 0;
  for (uint32_t y = 0; y < Ly; ++y) row[y] = 0;
  for (uint32_t y = 0; y < Ly; ++y)
    for (uint32_t x = 0; x < Lx; ++x) {
      int64_t N = 0;
      for (int v = 0; v < Q; ++v) N += state[v * plane + (size_t)y * Lx + x];
      col[x] += N;
      row[y] += N;
      M += (uint64_t)N;
    }
  *mass = M;
}

/* ------------------------------------------------------------------------ */
/* Single-node collision, for distribution tests                             */
/* ------------------------------------------------------------------------ */
/* Collide the same occupation m[] (already flipped if wanted) at nodes
 * node0 .. node0+count-1 of step t; out[k*Q + i] = n'_i of the k-th node. */
void oracle_collide_many(const oracle_step_params *p, const uint32_t *m, uint32_t t,
                         uint32_t node0, uint32_t count, uint32_t *out) {
  int Q = num_vel(p->lattice);
  for (uint32_t k = 0; k < count; ++k) collide_any(p, node0 + k, t, m, out + (size_t)k * Q);
}
