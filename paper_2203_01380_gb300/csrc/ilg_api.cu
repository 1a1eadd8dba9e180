// C ABI of libilg.so: contexts, validation, scheduling of the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ilg_internal.h"
#include "ilg_launch.h"

using namespace ilg;

struct ilg_ctx {
  ilg_params p{};
  int Q = 0;
  uint32_t flip = 0;
  uint64_t P_omega = 0, P_rest = 0, P_axis = 0;  // P_axis: D2Q9 axis share
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  size_t nodes = 0;
  uint16_t* buf[2] = {nullptr, nullptr};
  int cur = 0;
  uint64_t t = 0;
  bool has_state = false;
  uint32_t* d_tables = nullptr;            // thinning table, rest table
  unsigned long long* d_fail = nullptr;    // first failing step, ~0 if none
  unsigned long long* d_col = nullptr;     // Lx
  unsigned long long* d_row = nullptr;     // Ly
  unsigned long long* d_mass = nullptr;
  int32_t* d_modes = nullptr;
  double* d_res = nullptr;
  uint32_t mode_cap = 0;
  uint32_t tb_depth = 0;                   // temporal blocking: steps per launch (0: off)
  uint32_t general = 0;                    // too many nodes would fail the fast collision: general at once
  int kernel_choice = -1;                  // single-step kernel chosen by ilg_autotune (-1: default)
  double omega_star = 0;
  unsigned long long* h_word = nullptr;    // pinned 8-byte readback
  std::string err;
};

namespace {

thread_local std::string g_create_error;

ilg_status fail(ilg_ctx* c, ilg_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

ilg_status cuda_fail(ilg_ctx* c, cudaError_t e, const char* what) {
  const ilg_status s = (e == cudaErrorMemoryAllocation) ? ILG_E_OOM : ILG_E_CUDA;
  return fail(c, s, std::string(what) + ": " + cudaGetErrorString(e));
}

#define ILG_CUDA(c, call, what)                        \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

int num_vel(int lattice) { return lattice == ILG_D1Q3 ? 3 : (lattice == ILG_D2Q5 ? 5 : 9); }

uint32_t prob_mode(uint64_t P) {
  if (P == 0) return kNever;
  if (P == (uint64_t(1) << 32)) return kAlways;
  return kTable;
}

}  // namespace

namespace ilg {
std::string validate_params(const ilg_params& p) {
  if (p.lattice != ILG_D1Q3 && p.lattice != ILG_D2Q5 && p.lattice != ILG_D2Q9)
    return "lattice must be ILG_D1Q3, ILG_D2Q5 or ILG_D2Q9";
  if (p.sampler != ILG_SAMPLER_BINOMIAL && p.sampler != ILG_SAMPLER_PARTICLE)
    return "sampler must be ILG_SAMPLER_BINOMIAL or ILG_SAMPLER_PARTICLE";
  const uint64_t Ly = p.lattice == ILG_D1Q3 ? 1 : p.Ly;
  if (p.Lx < 3) return "Lx must be >= 3";
  if (p.lattice != ILG_D1Q3 && p.Ly < 3) return "Ly must be >= 3";
  if (uint64_t(p.Lx) * Ly >= (uint64_t(1) << 32)) return "Lx * Ly must be below 2^32";
  if (!(p.omega_eff > 0.0 && p.omega_eff <= 2.0)) return "omega_eff must lie in (0, 2]";
  if (p.lattice == ILG_D1Q3 && !(p.theta > 0.0 && p.theta < 1.0)) return "theta must lie in (0, 1) on D1Q3";
  if (p.lattice == ILG_D2Q5 && !(p.theta > 0.0 && p.theta <= 0.5)) return "theta must lie in (0, 1/2] on D2Q5";
  if (p.lattice == ILG_D2Q9 && !(p.theta > 0.0 && p.theta < 1.0)) return "theta must lie in (0, 1) on D2Q9";
  if (!(p.n0 >= 0.0) || !std::isfinite(p.n0)) return "n0 must be finite and >= 0";
  if (!std::isfinite(p.amp)) return "amp must be finite";
  if (p.mode_mx != 0 && p.mode_my != 0) return "the initial sine must be an axis mode";
  if (p.lattice == ILG_D1Q3 && p.mode_my != 0) return "D1Q3 has no y mode";
  return "";
}

void round_keys(uint64_t seed, uint32_t* rk) {
  uint32_t k0 = uint32_t(seed), k1 = uint32_t(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0;
    rk[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}
}  // namespace ilg

namespace {
using ilg::validate_params;

// node-parallel kernels: `per_sm` resident blocks of `threads` threads on every SM
int step_grid(const ilg_ctx* c, size_t per_sm, size_t threads = 256) {
  const size_t blocks = (c->nodes + threads - 1) / threads;
  const size_t cap = size_t(c->sms) * per_sm;
  return int(blocks < cap ? blocks : cap);
}

// row-tiled step: one block per row at a time, per_sm blocks per SM
int vec_grid(const ilg_ctx* c, size_t per_sm) {
  const size_t rows = c->p.Ly;
  const size_t cap = size_t(c->sms) * per_sm;
  return int(rows < cap ? rows : cap);
}

StepArgs step_args(const ilg_ctx* c) {
  StepArgs a{};
  a.Lx = c->p.Lx;
  a.Ly = c->Q == 3 ? 1 : c->p.Ly;
  a.flip = c->flip;
  a.omega_mode = prob_mode(c->P_omega);
  a.rest_mode = prob_mode(c->P_rest);
  a.axis_mode = prob_mode(c->P_axis);
  a.particle = c->p.sampler == ILG_SAMPLER_PARTICLE ? 1u : 0u;
  a.general = c->general | a.particle;
  a.key0 = uint32_t(c->p.seed);
  a.key1 = uint32_t(c->p.seed >> 32);
  a.replica = c->p.replica;
  a.tables = c->d_tables;
  ilg::round_keys(c->p.seed, a.rk);
  return a;
}

void free_ctx(ilg_ctx* c) {
  cudaFree(c->buf[0]);
  cudaFree(c->buf[1]);
  cudaFree(c->d_tables);
  cudaFree(c->d_fail);
  cudaFree(c->d_col);
  cudaFree(c->d_row);
  cudaFree(c->d_mass);
  cudaFree(c->d_modes);
  cudaFree(c->d_res);
  if (c->h_word) cudaFreeHost(c->h_word);
}

}  // namespace

namespace ilg {
// message for ilg_last_error(NULL), set by entry points that have no context
void set_context_free_error(const std::string& msg) { g_create_error = msg; }
}  // namespace ilg

extern "C" {

const char* ilg_last_error(const ilg_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

ilg_status ilg_create(const ilg_params* params, void* stream, ilg_ctx** out) {
  if (!out) return fail(nullptr, ILG_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!params) return fail(nullptr, ILG_E_INVALID, "params is NULL");
  const std::string bad = validate_params(*params);
  if (!bad.empty()) return fail(nullptr, ILG_E_INVALID, bad);
  ilg_ctx* c = new (std::nothrow) ilg_ctx();
  if (!c) return fail(nullptr, ILG_E_OOM, "host allocation failed");
  c->p = *params;
  if (c->p.lattice == ILG_D1Q3) c->p.Ly = 1;
  c->Q = num_vel(c->p.lattice);
  c->stream = static_cast<cudaStream_t>(stream);
  double w[9];
  weights(c->p.lattice, c->p.theta, w);
  double omega_star = c->p.omega_eff;
  if (c->p.omega_eff > 1.0) {
    c->flip = 1;
    omega_star = 2.0 - c->p.omega_eff;
  }
  c->omega_star = omega_star;
  c->P_omega = quantise_probability(omega_star);
  c->P_rest = quantise_probability(w[0]);
  c->P_axis = c->Q == 9 ? quantise_probability(axis_share(c->p.theta)) : 0;
  c->nodes = size_t(c->p.Lx) * c->p.Ly;

  auto bail = [&](cudaError_t e, const char* what) {
    cuda_fail(nullptr, e, what);
    free_ctx(c);
    delete c;
    return (e == cudaErrorMemoryAllocation) ? ILG_E_OOM : ILG_E_CUDA;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return bail(e, "cudaDeviceGetAttribute");
  const size_t state_bytes = sizeof(uint16_t) * c->nodes * c->Q;
  for (int b = 0; b < 2; ++b) {
    e = dev_alloc(&c->buf[b], state_bytes);
    if (e != cudaSuccess) return bail(e, "cudaMalloc state");
  }
  static_assert(kBlockWords == kDevBlockWords && kBlockWords9 == kDevBlockWords9, "table block layout");
  const size_t block_words = c->Q == 9 ? kBlockWords9 : kBlockWords;
  if ((e = dev_alloc(&c->d_tables, sizeof(uint32_t) * block_words)) != cudaSuccess) return bail(e, "cudaMalloc tables");
  if ((e = dev_alloc(&c->d_fail, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "cudaMalloc flag");
  if ((e = dev_alloc(&c->d_col, sizeof(unsigned long long) * c->p.Lx)) != cudaSuccess) return bail(e, "cudaMalloc sums");
  if ((e = dev_alloc(&c->d_row, sizeof(unsigned long long) * c->p.Ly)) != cudaSuccess) return bail(e, "cudaMalloc sums");
  if ((e = dev_alloc(&c->d_mass, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "cudaMalloc mass");
  if ((e = cudaMallocHost(&c->h_word, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "cudaMallocHost");

  std::vector<uint32_t> tables(block_words, 0u);
  build_table_block(c->Q, c->p.sampler, c->P_omega, c->P_rest, c->P_axis, tables.data());
  if ((e = prepare_step9_kernel()) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  if ((e = prepare_step_kernels()) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  if ((e = prepare_step_vec_kernels()) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  if ((e = prepare_step_warp_kernels()) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  e = cudaMemcpyAsync(c->d_tables, tables.data(), sizeof(uint32_t) * tables.size(), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return bail(e, "copy tables");
  e = cudaMemsetAsync(c->d_fail, 0xFF, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return bail(e, "reset flag");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return bail(e, "cudaStreamSynchronize");
  *out = c;
  return ILG_OK;
}

ilg_status ilg_destroy(ilg_ctx* c) {
  if (!c) return ILG_OK;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
  delete c;
  return ILG_OK;
}

ilg_status ilg_init(ilg_ctx* c) {
  if (!c) return ILG_E_INVALID;
  InitTables it;
  std::string msg;
  if (!build_init_tables(c->p, c->Q, &it, &msg)) return fail(c, ILG_E_INVALID, msg);
  uint32_t *d_off = nullptr, *d_cnt = nullptr, *d_tab = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_off);
    cudaFree(d_cnt);
    cudaFree(d_tab);
  };
  cudaError_t e;
  if ((e = dev_alloc(&d_off, sizeof(uint32_t) * it.offset.size())) != cudaSuccess ||
      (e = dev_alloc(&d_cnt, sizeof(uint32_t) * it.count.size())) != cudaSuccess ||
      (e = dev_alloc(&d_tab, sizeof(uint32_t) * it.table.size())) != cudaSuccess) {
    cleanup();
    return cuda_fail(c, e, "cudaMalloc init tables");
  }
  if ((e = cudaMemcpyAsync(d_off, it.offset.data(), sizeof(uint32_t) * it.offset.size(), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_cnt, it.count.data(), sizeof(uint32_t) * it.count.size(), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_tab, it.table.data(), sizeof(uint32_t) * it.table.size(), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess) {
    cleanup();
    return cuda_fail(c, e, "copy init tables");
  }
  InitArgs a{};
  a.Lx = c->p.Lx;
  a.Ly = c->p.Ly;
  a.period = it.period;
  a.axis = 0;
  a.mode = 0;
  if (it.period > 1) {
    const bool along_x = c->p.mode_mx != 0;
    const int64_t L = it.period;
    const int64_t mraw = along_x ? c->p.mode_mx : c->p.mode_my;
    a.axis = along_x ? 1 : 2;
    a.mode = uint32_t(((mraw % L) + L) % L);
  }
  a.weighted = c->p.init_weighted ? 1 : 0;
  a.key0 = uint32_t(c->p.seed);
  a.key1 = uint32_t(c->p.seed >> 32);
  a.replica = c->p.replica;
  a.offset = d_off;
  a.count = d_cnt;
  a.table = d_tab;
  if ((e = launch_init(c->Q, a, c->buf[c->cur], step_grid(c, 4), c->stream)) != cudaSuccess) {
    cleanup();
    return cuda_fail(c, e, "init kernel");
  }
  e = cudaStreamSynchronize(c->stream);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  c->t = 0;
  c->has_state = true;
  c->general = general_path(c->p.lattice, c->p.theta, c->omega_star, c->p.n0);
  return ILG_OK;
}

// mean occupation of the current state decides between the collision paths
static ilg_status update_path_choice(ilg_ctx* c) {
  const uint32_t Lx = c->p.Lx, Ly = c->p.Ly;
  ILG_CUDA(c, cudaMemsetAsync(c->d_col, 0, sizeof(unsigned long long) * Lx, c->stream), "clear sums");
  ILG_CUDA(c, launch_sums(c->Q, c->buf[c->cur], Lx, Ly, c->d_col, c->d_row, 0, c->stream), "sums kernel");
  ILG_CUDA(c, launch_project(c->d_col, c->d_row, Lx, Ly, nullptr, 0, nullptr, c->d_mass, c->stream), "mass kernel");
  ILG_CUDA(c, cudaMemcpyAsync(c->h_word, c->d_mass, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream),
           "read mass");
  ILG_CUDA(c, cudaStreamSynchronize(c->stream), "read mass");
  c->general = general_path(c->p.lattice, c->p.theta, c->omega_star, double(*c->h_word) / (double(c->nodes) * c->Q));
  return ILG_OK;
}

static ilg_status set_state_impl(ilg_ctx* c, const uint16_t* src, size_t n, uint64_t t, cudaMemcpyKind kind) {
  if (!c || !src) return ILG_E_INVALID;
  if (n != c->nodes * c->Q) return fail(c, ILG_E_INVALID, "state size must be Q * Lx * Ly");
  if (t >= (uint64_t(1) << 32)) return fail(c, ILG_E_INVALID, "t must be below 2^32");
  ILG_CUDA(c, cudaMemcpyAsync(c->buf[c->cur], src, sizeof(uint16_t) * n, kind, c->stream), "copy state in");
  ILG_CUDA(c, cudaStreamSynchronize(c->stream), "copy state in");
  c->t = t;
  c->has_state = true;
  return update_path_choice(c);
}

static ilg_status get_state_impl(ilg_ctx* c, uint16_t* dst, size_t n, uint64_t* t, cudaMemcpyKind kind) {
  if (!c || !dst) return ILG_E_INVALID;
  if (!c->has_state) return fail(c, ILG_E_STATE, "no state: call ilg_init or ilg_set_state first");
  if (n != c->nodes * c->Q) return fail(c, ILG_E_INVALID, "state size must be Q * Lx * Ly");
  ILG_CUDA(c, cudaMemcpyAsync(dst, c->buf[c->cur], sizeof(uint16_t) * n, kind, c->stream), "copy state out");
  ILG_CUDA(c, cudaStreamSynchronize(c->stream), "copy state out");
  if (t) *t = c->t;
  return ILG_OK;
}

ilg_status ilg_set_state(ilg_ctx* c, const uint16_t* host, size_t n, uint64_t t) {
  return set_state_impl(c, host, n, t, cudaMemcpyHostToDevice);
}
ilg_status ilg_set_state_device(ilg_ctx* c, const uint16_t* dev, size_t n, uint64_t t) {
  return set_state_impl(c, dev, n, t, cudaMemcpyDeviceToDevice);
}
ilg_status ilg_get_state(ilg_ctx* c, uint16_t* host, size_t n, uint64_t* t) {
  return get_state_impl(c, host, n, t, cudaMemcpyDeviceToHost);
}
ilg_status ilg_get_state_device(ilg_ctx* c, uint16_t* dev, size_t n, uint64_t* t) {
  return get_state_impl(c, dev, n, t, cudaMemcpyDeviceToDevice);
}

ilg_status ilg_set_temporal_blocking(ilg_ctx* c, uint32_t depth) {
  if (!c) return ILG_E_INVALID;
  if (depth > kMaxTbDepth) return fail(c, ILG_E_INVALID, "temporal blocking depth above 8");
  if (depth >= 2 && c->Q != 5) return fail(c, ILG_E_INVALID, "temporal blocking is for D2Q5 lattices");
  if (depth >= 2) ILG_CUDA(c, prepare_step_tb_kernel(tb_tile(depth), depth), "cudaFuncSetAttribute");
  c->tb_depth = depth >= 2 ? depth : 0;
  return ILG_OK;
}

namespace {

// Single-step kernels, numbered as the autotuner's candidates (3 and 4 are the
// temporal-blocking depths).
enum : int { kKernelVec8 = 0, kKernelVec4 = 1, kKernelNode = 2, kKernelSeg = 5, kKernelWarp8 = 6, kKernelWarp4 = 7 };
constexpr int kCandidates = 8;

bool is_single_step(int cand) { return cand <= kKernelNode || (cand >= kKernelSeg && cand < kCandidates); }

bool kernel_applies(const ilg_ctx* c, const StepArgs& a, int kind) {
  if (kind == kKernelNode) return true;
  if (a.general) return false;  // the general path runs node-parallel
  if (kind == kKernelWarp8 || kind == kKernelWarp4) {
    // whole vectors per row; the fast collision draws every probability through its
    // table (D2Q9: the axis share too)
    return c->p.Lx % step_warp_width(c->Q, kind == kKernelWarp4 ? 1 : 0) == 0 && a.omega_mode == kTable &&
           a.rest_mode == kTable && (c->Q != 9 || a.axis_mode == kTable);
  }
  if (c->Q == 9) return false;  // the row-tiled register kernels: D1Q3 and D2Q5 only
  return c->p.Lx % (kind == kKernelVec4 ? 4u : 8u) == 0;
}

// resident warps of the row-tiled kernels (3 blocks of 8 warps per SM)
uint64_t vec_warps(const ilg_ctx* c) { return uint64_t(c->sms) * 3 * 8; }

// the kernel a step runs: the tuned one while it applies to the current state, else
// the default: the shared-memory-staged warp kernel with 8-node, else 4-node vectors
// where the rows and probabilities allow; else 8-node row tiles where the rows allow;
// node-parallel otherwise
int pick_kernel(const ilg_ctx* c, const StepArgs& a) {
  if (c->kernel_choice >= 0 && kernel_applies(c, a, c->kernel_choice)) return c->kernel_choice;
  if (kernel_applies(c, a, kKernelWarp8)) return kKernelWarp8;
  if (kernel_applies(c, a, kKernelWarp4)) return kKernelWarp4;
  if (!kernel_applies(c, a, kKernelVec8)) return kKernelNode;
  return step_seg_units(c->p.Lx, c->p.Ly) >= 2 * vec_warps(c) ? kKernelSeg : kKernelVec8;
}

cudaError_t launch_single(const ilg_ctx* c, int kind, const StepArgs& a, const uint16_t* in, uint16_t* out,
                          uint64_t t, unsigned long long* fail_word) {
  if (c->Q == 9 && kind != kKernelWarp8 && kind != kKernelWarp4) {
    // rows of even length run two neighbouring nodes per thread (launch_step9)
    const size_t work = c->p.Lx % 2 == 0 ? c->nodes / 2 : c->nodes;
    const size_t blocks = (work + step9_threads() - 1) / step9_threads();
    const size_t cap = size_t(c->sms) * step9_blocks_per_sm();
    return launch_step9(a, in, out, uint32_t(t), fail_word, int(blocks < cap ? blocks : cap), c->stream);
  }
  if (kind == kKernelVec8)
    return launch_step_vec(c->Q, a, in, out, uint32_t(t), fail_word, vec_grid(c, step_vec_blocks_per_sm(8)), c->stream,
                           8);
  if (kind == kKernelVec4)
    return launch_step_vec(c->Q, a, in, out, uint32_t(t), fail_word, vec_grid(c, step_vec_blocks_per_sm(4)), c->stream,
                           4);
  if (kind == kKernelSeg) {
    const uint64_t blocks = (step_seg_units(c->p.Lx, c->p.Ly) + 7) / 8, cap = vec_warps(c) / 8;
    return launch_step_seg(c->Q, a, in, out, uint32_t(t), fail_word, int(blocks < cap ? blocks : cap), c->stream);
  }
  if (kind == kKernelWarp8 || kind == kKernelWarp4) {
    const int shape = kind == kKernelWarp4 ? 1 : 0;
    const uint32_t Ly = c->Q == 3 ? 1u : c->p.Ly;
    return launch_step_warp(c->Q, shape, a, in, out, uint32_t(t), fail_word,
                            int(step_warp_grid(c->Q, c->p.Lx, Ly, uint32_t(c->sms), shape)), c->stream);
  }
  return launch_step(c->Q, a, in, out, uint32_t(t), fail_word,
                     step_grid(c, step_kernel_blocks_per_sm(), step_kernel_threads()), c->stream);
}

int tb_grid(const ilg_ctx* c, uint32_t depth) {
  const uint32_t B = tb_tile(depth);
  const size_t tiles = size_t((c->p.Lx + B - 1) / B) * ((c->p.Ly + B - 1) / B);
  return int(std::min<size_t>(tiles, size_t(c->sms) * 2));
}

}  // namespace

ilg_status ilg_step(ilg_ctx* c, uint32_t T) {
  if (!c) return ILG_E_INVALID;
  NvtxRange nvtx("ilg_step");
  if (!c->has_state) return fail(c, ILG_E_STATE, "no state: call ilg_init or ilg_set_state first");
  if (c->t + T >= (uint64_t(1) << 32)) return fail(c, ILG_E_INVALID, "step counter would reach 2^32");
  if (T == 0) return ILG_OK;
  const StepArgs a = step_args(c);
  // high occupations and the particle sampler go straight to the general collision
  // (node-parallel kernel)
  const int kind = pick_kernel(c, a);
  const int cur0 = c->cur;
  const uint64_t t0 = c->t;
  // launches: blocks of tb_depth steps (temporal blocking), then single steps;
  // launch_t[k] is the step a launch starts from, its input is buffer cur0 ^ (k & 1)
  std::vector<uint64_t> launch_t;
  int cur = cur0;
  uint64_t t = t0;
  const uint32_t tb = c->tb_depth;
  if (tb >= 2) {
    const int tgrid = tb_grid(c, tb);
    for (uint32_t k = 0; k + tb <= T; k += tb) {
      cudaError_t e = launch_step_tb(a, c->buf[cur], c->buf[cur ^ 1], uint32_t(t), tb, tb_tile(tb), c->d_fail, tgrid,
                                     c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "temporal blocking kernel");
      launch_t.push_back(t);
      t += tb;
      cur ^= 1;
    }
  }
  while (t < t0 + T) {
    cudaError_t e = launch_single(c, kind, a, c->buf[cur], c->buf[cur ^ 1], t, c->d_fail);
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
    launch_t.push_back(t);
    t += 1;
    cur ^= 1;
  }
  ILG_CUDA(c, cudaMemcpyAsync(c->h_word, c->d_fail, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream),
           "read overflow word");
  ILG_CUDA(c, cudaStreamSynchronize(c->stream), "step");
  const unsigned long long f = *c->h_word;
  if (f != ~0ull) {
    // the launch that started at step f failed: its input buffer still holds the state at f
    size_t k = 0;
    while (k < launch_t.size() && launch_t[k] != f) ++k;
    c->cur = cur0 ^ int(k & 1u);
    c->t = f;
    ILG_CUDA(c, cudaMemsetAsync(c->d_fail, 0xFF, sizeof(unsigned long long), c->stream), "reset flag");
    ILG_CUDA(c, cudaStreamSynchronize(c->stream), "reset flag");
    char buf[160];
    std::snprintf(buf, sizeof(buf), "occupation above 65535 in the launch from step %llu; state kept at t = %llu", f, f);
    return fail(c, ILG_E_OVERFLOW, buf);
  }
  c->cur = cur;
  c->t = t0 + T;
  return ILG_OK;
}

ilg_status ilg_set_step_kernel(ilg_ctx* c, int32_t candidate) {
  if (!c) return ILG_E_INVALID;
  if (candidate < -1 || (candidate >= 0 && !is_single_step(candidate)))
    return fail(c, ILG_E_INVALID, "candidate must be -1, 0, 1, 2, 5, 6 or 7");
  c->kernel_choice = candidate;
  return ILG_OK;
}

ilg_status ilg_autotune(ilg_ctx* c, uint32_t trial_steps, ilg_tuning* out) {
  if (!c) return ILG_E_INVALID;
  if (!c->has_state) return fail(c, ILG_E_STATE, "no state: call ilg_init or ilg_set_state first");
  if (trial_steps == 0) trial_steps = 20;
  if (trial_steps > 1000) return fail(c, ILG_E_INVALID, "at most 1000 trial steps");
  if (c->t + 2ull * trial_steps + 16 >= (uint64_t(1) << 32))
    return fail(c, ILG_E_INVALID, "step counter would reach 2^32 in the trials");
  const StepArgs a = step_args(c);
  // trials on a copy of the state (two scratch buffers and their own overflow word);
  // every candidate gives the same bits, only the time is kept
  const size_t bytes = sizeof(uint16_t) * c->nodes * c->Q;
  uint16_t* s[2] = {nullptr, nullptr};
  unsigned long long* fw = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    cudaFree(s[0]);
    cudaFree(s[1]);
    cudaFree(fw);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  cudaError_t e = dev_alloc(&s[0], bytes);
  if (e == cudaSuccess) e = dev_alloc(&s[1], bytes);
  if (e == cudaSuccess) e = dev_alloc(&fw, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s[0], c->buf[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "autotune scratch");
  }
  // candidates: 0 8-node vectors, 1 4-node vectors, 2 node-parallel, 3 / 4 temporal
  // blocking of depth 2 / 4 (D2Q5), 5 warp segments of 8-node vectors, 6 / 7 the
  // shared-memory-staged warp kernel with 8 / 4 nodes per lane
  ilg_tuning res{};
  res.n = kCandidates;
  for (int k = 0; k < 8; ++k) res.ms_per_step[k] = -1.0;
  auto trial = [&](int cand, double* ms_per_step) -> cudaError_t {
    const uint32_t depth = cand == 3 ? 2u : (cand == 4 ? 4u : 1u);
    const uint32_t launches = std::max<uint32_t>(1, trial_steps / depth);
    uint64_t t = c->t;
    int cur = 0;
    auto one = [&]() -> cudaError_t {
      cudaError_t r = depth > 1 ? launch_step_tb(a, s[cur], s[cur ^ 1], uint32_t(t), depth, tb_tile(depth), fw, tb_grid(c, depth),
                                                 c->stream)
                                : launch_single(c, cand, a, s[cur], s[cur ^ 1], t, fw);
      t += depth;
      cur ^= 1;
      return r;
    };
    cudaError_t r = cudaMemsetAsync(fw, 0xFF, sizeof(unsigned long long), c->stream);
    if (r == cudaSuccess) r = one();  // warm-up launch
    if (r == cudaSuccess) r = cudaEventRecord(e0, c->stream);
    for (uint32_t k = 0; k < launches && r == cudaSuccess; ++k) r = one();
    if (r == cudaSuccess) r = cudaEventRecord(e1, c->stream);
    if (r == cudaSuccess) r = cudaMemcpyAsync(c->h_word, fw, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(c->stream);
    float ms = 0.f;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
    // a trial that overflowed skipped work after the overflow: its time is not kept
    if (r == cudaSuccess && *c->h_word == ~0ull) *ms_per_step = double(ms) / (double(launches) * depth);
    return r;
  };
  for (int cand = 0; cand < kCandidates && e == cudaSuccess; ++cand) {
    if (is_single_step(cand) && !kernel_applies(c, a, cand)) continue;
    if (!is_single_step(cand)) {
      if (c->Q != 5) continue;
      const uint32_t depth = cand == 3 ? 2u : 4u;
      if ((e = prepare_step_tb_kernel(tb_tile(depth), depth)) != cudaSuccess) break;
    }
    e = trial(cand, &res.ms_per_step[cand]);
  }
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune trial");
  int best = -1;
  for (int k = 0; k < kCandidates; ++k)
    if (res.ms_per_step[k] >= 0.0 && (best < 0 || res.ms_per_step[k] < res.ms_per_step[best])) best = k;
  if (best < 0) return fail(c, ILG_E_OVERFLOW, "every trial overflowed: no choice made");
  if (!is_single_step(best)) {
    // temporal blocking; the remaining single steps take the fastest single-step kernel
    int single = -1;
    for (int k = 0; k < kCandidates; ++k)
      if (is_single_step(k) && res.ms_per_step[k] >= 0.0 &&
          (single < 0 || res.ms_per_step[k] < res.ms_per_step[single]))
        single = k;
    c->kernel_choice = single;
    c->tb_depth = best == 3 ? 2u : 4u;
    ILG_CUDA(c, prepare_step_tb_kernel(tb_tile(c->tb_depth), c->tb_depth), "cudaFuncSetAttribute");
  } else {
    c->kernel_choice = best;
    c->tb_depth = 0;
  }
  res.choice = uint32_t(best);
  res.tb_depth = c->tb_depth;
  res.threads = 256;
  if (out) *out = res;
  return ILG_OK;
}

ilg_status ilg_observables(ilg_ctx* c, const int32_t* modes, uint32_t nmodes, uint64_t* t, uint64_t* mass,
                           double* re, double* im, double* amp, double* Sk, int64_t* col_sums,
                           int64_t* row_sums) {
  if (!c) return ILG_E_INVALID;
  NvtxRange nvtx("ilg_observables");
  if (!c->has_state) return fail(c, ILG_E_STATE, "no state: call ilg_init or ilg_set_state first");
  if (nmodes && !modes) return fail(c, ILG_E_INVALID, "modes is NULL");
  bool want_rows = row_sums != nullptr;
  for (uint32_t i = 0; i < nmodes; ++i) {
    const int32_t mx = modes[2 * i], my = modes[2 * i + 1];
    if ((mx == 0) == (my == 0)) return fail(c, ILG_E_INVALID, "each mode must have exactly one nonzero component");
    if (my != 0 && c->Q == 3) return fail(c, ILG_E_INVALID, "D1Q3 has no y modes");
    if (my != 0) want_rows = true;
  }
  if (nmodes > c->mode_cap) {
    cudaFree(c->d_modes);
    cudaFree(c->d_res);
    c->d_modes = nullptr;
    c->d_res = nullptr;
    c->mode_cap = 0;
    ILG_CUDA(c, dev_alloc(&c->d_modes, sizeof(int32_t) * 2 * nmodes), "cudaMalloc modes");
    ILG_CUDA(c, dev_alloc(&c->d_res, sizeof(double) * 4 * nmodes), "cudaMalloc modes");
    c->mode_cap = nmodes;
  }
  const uint32_t Lx = c->p.Lx, Ly = c->p.Ly;
  ILG_CUDA(c, cudaMemsetAsync(c->d_col, 0, sizeof(unsigned long long) * Lx, c->stream), "clear sums");
  if (want_rows) ILG_CUDA(c, cudaMemsetAsync(c->d_row, 0, sizeof(unsigned long long) * Ly, c->stream), "clear sums");
  if (nmodes)
    ILG_CUDA(c, cudaMemcpyAsync(c->d_modes, modes, sizeof(int32_t) * 2 * nmodes, cudaMemcpyHostToDevice, c->stream),
             "copy modes");
  ILG_CUDA(c, launch_sums(c->Q, c->buf[c->cur], Lx, Ly, c->d_col, c->d_row, want_rows ? 1 : 0, c->stream), "sums kernel");
  ILG_CUDA(c, launch_project(c->d_col, c->d_row, Lx, Ly, c->d_modes, nmodes, c->d_res, c->d_mass, c->stream),
           "projection kernel");
  std::vector<double> res(size_t(4) * nmodes);
  unsigned long long M = 0;
  if (nmodes)
    ILG_CUDA(c, cudaMemcpyAsync(res.data(), c->d_res, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, c->stream),
             "copy results");
  ILG_CUDA(c, cudaMemcpyAsync(&M, c->d_mass, sizeof(M), cudaMemcpyDeviceToHost, c->stream), "copy mass");
  if (col_sums)
    ILG_CUDA(c, cudaMemcpyAsync(col_sums, c->d_col, sizeof(int64_t) * Lx, cudaMemcpyDeviceToHost, c->stream), "copy sums");
  if (row_sums)
    ILG_CUDA(c, cudaMemcpyAsync(row_sums, c->d_row, sizeof(int64_t) * Ly, cudaMemcpyDeviceToHost, c->stream), "copy sums");
  ILG_CUDA(c, cudaStreamSynchronize(c->stream), "observables");
  if (t) *t = c->t;
  if (mass) *mass = M;
  for (uint32_t i = 0; i < nmodes; ++i) {
    if (re) re[i] = res[4 * i + 0];
    if (im) im[i] = res[4 * i + 1];
    if (amp) amp[i] = res[4 * i + 2];
    if (Sk) Sk[i] = res[4 * i + 3];
  }
  return ILG_OK;
}

ilg_status ilg_philox(const uint32_t* ctr, uint64_t seed, uint32_t* out, size_t n, void* stream) {
  if (!ctr || !out) return fail(nullptr, ILG_E_INVALID, "NULL argument");
  if (n == 0) return ILG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t *d_c = nullptr, *d_o = nullptr;
  cudaError_t e = dev_alloc(&d_c, sizeof(uint32_t) * 4 * n);
  if (e == cudaSuccess) e = dev_alloc(&d_o, sizeof(uint32_t) * 4 * n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_c, ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_philox(d_c, uint32_t(seed), uint32_t(seed >> 32), d_o, n, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_o, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_c);
  cudaFree(d_o);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox probe");
  return ILG_OK;
}

ilg_status ilg_binomial_table(uint64_t P, uint32_t* out) {
  if (!out || P == 0 || P >= (uint64_t(1) << 32)) return fail(nullptr, ILG_E_INVALID, "P must lie in (0, 2^32)");
  build_binomial_table(P, out);
  return ILG_OK;
}

ilg_status ilg_alias_table(uint64_t P, uint32_t* thr, uint32_t* alias) {
  if (!thr || !alias || P == 0 || P >= (uint64_t(1) << 32)) return fail(nullptr, ILG_E_INVALID, "P must lie in (0, 2^32)");
  std::vector<AliasEntry> t(kAliasEntries);
  build_alias_table(P, t.data());
  for (uint32_t i = 0; i < kAliasEntries; ++i) {
    thr[i] = t[i].thr;
    alias[i] = t[i].alias;
  }
  return ILG_OK;
}

ilg_status ilg_poisson_table(double lambda, uint32_t* out, uint32_t cap, uint32_t* K) {
  if (!out || !K || !(lambda >= 0.0) || lambda > kMaxMean) return fail(nullptr, ILG_E_INVALID, "bad argument");
  std::vector<uint32_t> buf(kPoissonCap);
  const uint32_t k = build_poisson_table(lambda, buf.data(), kPoissonCap);
  if (k == 0 || k > cap) return fail(nullptr, ILG_E_INVALID, "table longer than cap");
  std::memcpy(out, buf.data(), sizeof(uint32_t) * k);
  *K = k;
  return ILG_OK;
}

}  // extern "C"
