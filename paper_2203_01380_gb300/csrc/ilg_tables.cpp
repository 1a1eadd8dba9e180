// Host-side construction of the integer tables the kernels read.
//
// Compiled with -ffp-contract=off: the Poisson tables and the initial means are
// defined by a fixed sequence of IEEE double operations and libm calls, and must
// come out the same on every host.
#include <algorithm>
#include <atomic>

#include "ilg_internal.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace ilg {

// Integer CDF rows of Binomial(n, P/2^32), n = 1..kNmax.  The pmf of n trials is
// carried in fixed point with one = 2^63; each row follows from the previous one
// by Pascal's rule with the two products floored, and the CDF entry of (n, k) is
// the running pmf sum shifted down to 32 fractional bits.
void build_binomial_table(uint64_t P, uint32_t* T) {
  const uint64_t Pq = (uint64_t(1) << 32) - P;
  uint64_t pmf[kNmax + 2];
  uint64_t next[kNmax + 2];
  std::memset(pmf, 0, sizeof(pmf));
  pmf[0] = uint64_t(1) << 63;
  for (uint32_t n = 1; n <= kNmax; ++n) {
    next[0] = uint64_t((static_cast<unsigned __int128>(pmf[0]) * Pq) >> 32);
    for (uint32_t k = 1; k < n; ++k) {
      unsigned __int128 a = (static_cast<unsigned __int128>(pmf[k]) * Pq) >> 32;
      unsigned __int128 b = (static_cast<unsigned __int128>(pmf[k - 1]) * P) >> 32;
      next[k] = uint64_t(a + b);
    }
    next[n] = uint64_t((static_cast<unsigned __int128>(pmf[n - 1]) * P) >> 32);
    std::memcpy(pmf, next, sizeof(uint64_t) * (n + 1));
    uint32_t* row = T + n * (n - 1) / 2;
    uint64_t run = 0;
    for (uint32_t k = 0; k < n; ++k) {
      run += pmf[k];
      row[k] = uint32_t(run >> 31);
    }
  }
}

// Alias tables (Walker; Vose's construction carried out in integers) realising
// the integer pmf of each CDF row exactly.  Row n (0..kNmax) has kAliasCols = 64
// columns at entry offset 64 n; column j owns the 2^26 draws u with u >> 26 = j.
// Outcomes n+1..63 have weight zero, so their columns go wholly to an alias.  The
// draw yields j when u is below the column's threshold, its alias otherwise.
void build_alias_table(uint64_t P, AliasEntry* out) {
  constexpr uint64_t kColumn = uint64_t(1) << 26;  // draws per column
  std::vector<uint32_t> cdf(kTableWords);
  build_binomial_table(P, cdf.data());
  std::vector<uint64_t> weight(kAliasCols);
  std::vector<uint32_t> under, over;
  for (uint32_t n = 0; n <= kNmax; ++n) {
    AliasEntry* row = out + n * kAliasCols;
    std::fill(weight.begin(), weight.end(), 0);
    uint64_t below = 0;
    for (uint32_t k = 0; k < n; ++k) {
      const uint64_t c = cdf[n * (n - 1) / 2 + k];
      weight[k] = c - below;
      below = c;
    }
    weight[n] = (uint64_t(1) << 32) - below;
    under.clear();
    over.clear();
    for (uint32_t j = 0; j < kAliasCols; ++j) {
      row[j].thr = 0;
      row[j].alias = j;
      if (weight[j] < kColumn) under.push_back(j);
      else if (weight[j] > kColumn) over.push_back(j);
    }
    while (!under.empty() && !over.empty()) {
      const uint32_t l = under.back();
      under.pop_back();
      const uint32_t g = over.back();
      over.pop_back();
      row[l].thr = uint32_t(uint64_t(l) * kColumn + weight[l]);
      row[l].alias = g;
      weight[g] -= kColumn - weight[l];
      if (weight[g] < kColumn) under.push_back(g);
      else if (weight[g] > kColumn) over.push_back(g);
    }
  }
}

// Poisson(lambda) CDF scaled to 2^32, floored, saturating at 2^32 - 1, up to and
// including the first saturated entry.  Returns the entry count, 0 if above cap.
uint32_t build_poisson_table(double lambda, uint32_t* T, uint32_t cap) {
  double term = std::exp(-lambda);
  double cdf = term;
  for (uint32_t k = 0; k < cap; ++k) {
    if (k != 0) {
      term = term * lambda / static_cast<double>(k);
      cdf = cdf + term;
    }
    const double s = std::floor(cdf * 4294967296.0);
    const uint32_t v = (s >= 4294967295.0) ? 0xFFFFFFFFu : static_cast<uint32_t>(s);
    T[k] = v;
    if (v == 0xFFFFFFFFu) return k + 1;
  }
  return 0;
}

// The fast collision path needs at most 63 removed and 32 moving particles per
// node; with about omega* Q m removed on average (m = mean occupation per
// velocity), above ~40 it would mostly fail and the general path is taken at once.
// Either path gives the same result.
// Particle sampler boundaries: B_0 = 2^32 - P_omega (below: the particle stays),
// B_{j+1} = B_0 + floor(P_omega (P_rest (Q-1) + j (2^32 - P_rest)) / ((Q-1) 2^32))
// for j = 0..Q-1, so a picked particle goes to rest with P_rest / 2^32 and to each
// moving velocity with an equal share of the rest; B_Q = 2^32.
void build_particle_bounds(int Q, uint64_t P_omega, uint64_t P_rest, uint64_t P_axis, uint64_t* B) {
  typedef unsigned __int128 u128;
  const u128 two32 = u128(1) << 32;
  B[0] = uint64_t(two32 - P_omega);
  if (Q == 9) {
    // D2Q9: a picked particle goes to rest with P_rest / 2^32, to each axis velocity
    // with (1 - P_rest / 2^32) (P_axis / 2^32) / 4 and to each diagonal one with
    // (1 - P_rest / 2^32) (1 - P_axis / 2^32) / 4; cumulative shares in units of
    // 1 / (4 2^64)
    const u128 den = u128(4) << 64;
    u128 cum = u128(4) * P_rest * two32;
    for (int j = 0; j < 9; ++j) {
      if (j >= 1 && j <= 4) cum += (two32 - P_rest) * u128(P_axis);
      if (j >= 5) cum += (two32 - P_rest) * (two32 - P_axis);
      B[j + 1] = B[0] + uint64_t((u128(P_omega) * cum) / den);
    }
    return;
  }
  const u128 den = u128(uint32_t(Q - 1)) << 32;
  for (int j = 0; j < Q; ++j) {
    const u128 num = u128(P_omega) * (u128(P_rest) * uint32_t(Q - 1) + u128(uint32_t(j)) * (two32 - P_rest));
    B[j + 1] = B[0] + uint64_t(num / den);
  }
}

// The device table block of a lattice: the two alias tables (binomial sampler),
// followed for D1Q3 / D2Q5 by the same two tables packed one word per column for
// kernels short of shared memory; or the particle boundaries.
void build_table_block(int Q, uint32_t sampler, uint64_t P_omega, uint64_t P_rest, uint64_t P_axis,
                       uint32_t* block) {
  std::fill(block, block + (Q == 9 ? kBlockWords9 : kBlockWords), 0u);
  if (sampler == ILG_SAMPLER_PARTICLE) {
    uint64_t B[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    build_particle_bounds(Q, P_omega, P_rest, P_axis, B);
    std::memcpy(block, B, sizeof(B));
    return;
  }
  const uint64_t two32 = uint64_t(1) << 32;
  AliasEntry* al = reinterpret_cast<AliasEntry*>(block);
  if (P_omega > 0 && P_omega < two32) build_alias_table(P_omega, al);
  if (P_rest > 0 && P_rest < two32) build_alias_table(P_rest, al + kAliasEntries);
  if (Q == 9 && P_axis > 0 && P_axis < two32) build_alias_table(P_axis, al + 2 * kAliasEntries);
  if (Q == 9) return;
  // packed entry of column j: (thr - j 2^26) << 6 | alias, or j for a full column
  // (alias j); the draw then compares u's offset in its column, shifted up over six
  // one bits, with the word
  uint32_t* packed = block + kPackedOffset;
  for (uint32_t i = 0; i < 2 * kAliasEntries; ++i) {
    const uint32_t j = i % kAliasCols;
    packed[i] = al[i].alias == j ? j : (((al[i].thr - (j << 26)) << 6) | al[i].alias);
  }
}

double axis_share(double theta) {
  double w[9];
  weights(ILG_D2Q9, theta, w);
  return (4.0 * w[1]) / (1.0 - w[0]);
}

namespace {
// P(X >= k) for X ~ Poisson(lambda); 1 where the terms would underflow (lambda that
// large fails the fast collision anyway)
double poisson_tail(double lambda, int k) {
  if (lambda <= 0.0) return 0.0;
  if (lambda > 700.0) return 1.0;
  double term = std::exp(-lambda), below = 0.0;
  for (int j = 0; j < k; ++j) {
    below += term;
    term *= lambda / double(j + 1);
  }
  return below >= 1.0 ? 0.0 : 1.0 - below;
}
}  // namespace

// The fast collision needs every occupation below 64, at most 63 removed and at most 32
// moving particles (D2Q9: 32 axis and 32 diagonal).  With Poisson occupations of the
// given mean, removals and movers are thinned Poisson counts; the lattice goes straight
// to the general collision when the expected share of nodes that fail the fast one is
// above kGeneralShare, or, where sync_nodes nodes wait for one another every step (a
// batched ring and its block barrier), when one of them is expected to fail in more
// than about one step in three: trying the fast collision first then costs more than it
// saves, since the warp or block that holds a failing node runs both collisions.
uint32_t general_path(int lattice, double theta, double omega_star, double mean_occupation, uint32_t sync_nodes) {
  constexpr double kGeneralShare = 0.02;
  const double share = std::min(kGeneralShare, 0.3 / double(std::max<uint32_t>(sync_nodes, 1)));
  double w[9];
  weights(lattice, theta, w);
  const int Q = lattice == ILG_D1Q3 ? 3 : (lattice == ILG_D2Q9 ? 9 : 5);
  const double removed = omega_star * Q * mean_occupation, moving = removed * (1.0 - w[0]);
  double fail = Q * poisson_tail(mean_occupation, 64) + poisson_tail(removed, 64);
  if (lattice == ILG_D2Q9) {
    const double a = axis_share(theta);
    fail += poisson_tail(moving * a, 33) + poisson_tail(moving * (1.0 - a), 33);
  } else {
    fail += poisson_tail(moving, 33);
  }
  return fail > share ? 1u : 0u;
}

uint64_t quantise_probability(double p) {
  double v = std::floor(p * 4294967296.0 + 0.5);
  if (v <= 0.0) return 0;
  if (v >= 4294967296.0) return uint64_t(1) << 32;
  return static_cast<uint64_t>(v);
}

void weights(int lattice, double theta, double* w) {
  if (lattice == ILG_D1Q3) {
    w[0] = 1.0 - theta;
    w[1] = w[2] = theta / 2.0;
  } else if (lattice == ILG_D2Q9) {
    // products of the D1Q3 weights in x and y: rest, four axis, four diagonal
    w[0] = (1.0 - theta) * (1.0 - theta);
    w[1] = w[2] = w[3] = w[4] = (theta * (1.0 - theta)) / 2.0;
    w[5] = w[6] = w[7] = w[8] = (theta * theta) / 4.0;
  } else {
    w[0] = 1.0 - 2.0 * theta;
    w[1] = w[2] = w[3] = w[4] = theta / 2.0;
  }
}

// Sine value of the initial profile for phase residue r of a mode of period L.
static double profile_sine(uint32_t r, uint32_t L) {
  return std::sin((6.283185307179586 * static_cast<double>(r)) / static_cast<double>(L));
}

// Initial mean of velocity class c (0 = rest, 1 = moving; only class 0 when the
// means are not weighted) at phase residue r.
double initial_mean(const ilg_params& p, int Q, int cls, uint32_t r, uint32_t L) {
  const double s = (p.amp != 0.0 && L != 0) ? profile_sine(r, L) : 0.0;
  if (p.init_weighted) {
    double w[9];
    weights(p.lattice, p.theta, w);
    const double wc = cls == 0 ? w[0] : (cls == 1 ? w[1] : w[5]);
    return wc * (static_cast<double>(Q) * p.n0 + p.amp * s);
  }
  return p.n0 + (p.amp * s) / static_cast<double>(Q);
}

uint32_t initial_period(const ilg_params& p) {
  if (p.amp != 0.0 && p.mode_mx != 0) return p.Lx;
  if (p.amp != 0.0 && p.mode_my != 0) return (p.lattice == ILG_D1Q3) ? 1 : p.Ly;
  return 1;
}

bool build_init_tables(const ilg_params& p, int Q, InitTables* out, std::string* err) {
  const uint32_t L = initial_period(p);  // period of the phase residue
  const int classes = p.init_weighted ? (Q == 9 ? 3 : 2) : 1;
  out->period = L;
  out->classes = classes;
  out->offset.assign(size_t(classes) * L, 0);
  out->count.assign(size_t(classes) * L, 0);
  out->table.clear();
  std::vector<uint32_t> buf(kPoissonCap);
  for (int c = 0; c < classes; ++c) {
    for (uint32_t r = 0; r < L; ++r) {
      const double lam = initial_mean(p, Q, c, r, L);
      if (!(lam >= 0.0) || lam > kMaxMean) {
        *err = "initial mean " + std::to_string(lam) + " outside [0, 700]";
        return false;
      }
      const uint32_t K = build_poisson_table(lam, buf.data(), kPoissonCap);
      if (K == 0) {
        *err = "Poisson table of mean " + std::to_string(lam) + " exceeds its cap";
        return false;
      }
      out->offset[size_t(c) * L + r] = static_cast<uint32_t>(out->table.size());
      out->count[size_t(c) * L + r] = K;
      out->table.insert(out->table.end(), buf.begin(), buf.begin() + K);
    }
  }
  return true;
}

namespace {
// allocations still to succeed before the injected failure; negative: none injected
std::atomic<int64_t> g_alloc_countdown{-1};
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  int64_t left = g_alloc_countdown.load();
  while (left >= 0) {
    // take one allocation off the countdown; the one that finds it at 0 fails
    if (g_alloc_countdown.compare_exchange_weak(left, left - 1)) {
      if (left == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

}  // namespace ilg

extern "C" ilg_status ilg_inject_alloc_failure(int64_t after) {
  ilg::g_alloc_countdown.store(after < 0 ? -1 : after);
  return ILG_OK;
}

