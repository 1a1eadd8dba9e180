// Internal declarations shared by the sources of libilg.so (host side).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ilg.h"

namespace ilg {

constexpr uint32_t kNmax = 63;                              // trials per binomial table row
constexpr uint32_t kTableWords = kNmax * (kNmax + 1) / 2;   // 2016 entries
constexpr uint32_t kPoissonCap = 4096;                       // entries per Poisson table
constexpr double kMaxMean = 700.0;                           // largest initial mean
constexpr uint32_t kMaxTbDepth = 8;                          // temporal blocking: steps per launch
constexpr uint32_t kTbWindow = 44;                           // temporal blocking: tile + halo per side
// temporal blocking: output tile side at depth Tb (the window with its halo stays 44
// nodes wide, so two blocks fit on an SM beside their alias tables)
constexpr uint32_t tb_tile(uint32_t depth) { return kTbWindow - 2 * depth; }

// Philox purpose tags (top 8 bits of the fourth counter word).
constexpr uint32_t kTagStep = 1;
constexpr uint32_t kTagExt = 2;
constexpr uint32_t kTagInit = 3;

constexpr uint32_t kAliasCols = 64;                                // columns per alias row
constexpr uint32_t kAliasEntries = (kNmax + 1) * kAliasCols;       // rows n = 0..63
struct AliasEntry {
  uint32_t thr;    // draws below the threshold keep the column's own outcome
  uint32_t alias;  // outcome of the other draws of the column
};
// device table block: alias(thinning) | alias(rest), AliasEntry each, then the same
// two tables packed one word per entry (D1Q3, D2Q5)
constexpr uint32_t kPackedOffset = 2 * kAliasEntries * 2;
constexpr uint32_t kBlockWords = kPackedOffset + 2 * kAliasEntries;
// D2Q9: alias(thinning) | alias(rest) | alias(axis share)
constexpr uint32_t kBlockWords9 = 3 * kAliasEntries * 2;

void build_binomial_table(uint64_t P, uint32_t* T);
void build_alias_table(uint64_t P, AliasEntry* out);
uint32_t build_poisson_table(double lambda, uint32_t* T, uint32_t cap);
uint64_t quantise_probability(double p);
// 1 when a lattice of this velocity set, theta, omega* and mean occupation per velocity
// should skip the fast collision (too many of its nodes would fail it); sync_nodes: the
// nodes that wait for one another every step (a warp's 32, or a batched ring's length)
uint32_t general_path(int lattice, double theta, double omega_star, double mean_occupation,
                      uint32_t sync_nodes = 32);
void build_particle_bounds(int Q, uint64_t P_omega, uint64_t P_rest, uint64_t P_axis, uint64_t* B);
// table block of a lattice (kBlockWords words, kBlockWords9 for D2Q9)
void build_table_block(int Q, uint32_t sampler, uint64_t P_omega, uint64_t P_rest, uint64_t P_axis,
                       uint32_t* block);
// D2Q9: probability that a moving particle takes an axis velocity, 4 w_axis / (1 - w_0)
double axis_share(double theta);
void weights(int lattice, double theta, double* w);

// Poisson tables of the initial state, one per (velocity class, phase residue).
struct InitTables {
  uint32_t period = 1;              // number of phase residues
  int classes = 1;                  // 2 when means are weighted (rest, moving)
  std::vector<uint32_t> offset;     // [classes * period] start in table
  std::vector<uint32_t> count;      // [classes * period] entries
  std::vector<uint32_t> table;      // concatenated CDF entries
};
bool build_init_tables(const ilg_params& p, int Q, InitTables* out, std::string* err);
// Initial Poisson mean of velocity class cls (0 rest, 1 moving; only 0 when the
// means are not weighted) at phase residue r of period L, and that period.
double initial_mean(const ilg_params& p, int Q, int cls, uint32_t r, uint32_t L);
uint32_t initial_period(const ilg_params& p);

void set_context_free_error(const std::string& msg);

// NVTX range for the duration of a scope (step, observables, batch run, server
// round): visible in Nsight timelines, free when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device allocations of the library go through here: cudaMalloc, unless a failure
// has been injected (ilg_inject_alloc_failure), in which case the allocation
// reports cudaErrorMemoryAllocation without calling the allocator.
cudaError_t dev_malloc(void** p, size_t bytes);
template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
std::string validate_params(const ilg_params& p);   // empty when valid
void round_keys(uint64_t seed, uint32_t* rk);        // Philox round keys, 20 words

}  // namespace ilg
