// C ABI of the batched D1Q3 mode (ilg_batch_*): many independent rings advanced
// together by one persistent kernel launch, captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "ilg_batch.h"
#include "ilg_internal.h"
#include "ilg_launch.h"

using namespace ilg;

struct ilg_batch {
  uint32_t n = 0;
  std::vector<ilg_params> p;
  std::vector<ReplicaDesc> desc;      // host mirror (t updated after each run)
  cudaStream_t stream = nullptr;
  bool own_stream = false;            // created here: a capture needs a non-legacy stream
  int sms = 0;
  uint32_t Lmax = 0;
  int threads = 0;                    // block shape of the batch kernel (default or autotuned)
  size_t total = 0;                   // uint16 words of state
  uint16_t* d_state = nullptr;
  ReplicaDesc* d_desc = nullptr;
  uint32_t* d_tables = nullptr;
  uint32_t* d_order = nullptr;
  unsigned int* d_counter = nullptr;
  uint32_t* d_failed = nullptr;
  long long* d_record = nullptr;      // raw 128-bit amplitude sums, n x (T + 1) x 4
  size_t record_cap = 0;
  double* d_rec = nullptr;            // the same as (re, im) doubles, n x (T + 1) x 2
  size_t rec_cap = 0;
  double* d_out = nullptr;            // amplitude record or ensemble statistics
  size_t out_cap = 0;
  uint16_t* d_states = nullptr;       // per-step states (ilg_batch_run_record), T x total
  size_t states_cap = 0;
  longlong2* d_trig = nullptr;        // fixed-point trigonometric table of the recorded mode
  size_t trig_cap = 0;                 // entries (one per node of the batch)
  unsigned long long* d_mass = nullptr;
  double* d_amp = nullptr;
  StepArgs common{};
  cudaGraphExec_t graph = nullptr;
  uint32_t graph_T = 0;
  bool graph_rec = false;
  bool graph_trig = false;
  bool graph_states = false;
  int32_t graph_mode = 0;
  std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

ilg_status bfail(ilg_batch* b, ilg_status s, const std::string& msg) {
  if (b) b->err = msg;
  else g_batch_create_error = msg;
  return s;
}

ilg_status bcuda(ilg_batch* b, cudaError_t e, const char* what) {
  return bfail(b, e == cudaErrorMemoryAllocation ? ILG_E_OOM : ILG_E_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCUDA(b, call, what)                           \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return bcuda(b, e_, what);  \
  } while (0)

uint32_t mode_of(uint64_t P) {
  if (P == 0) return kNever;
  if (P == (uint64_t(1) << 32)) return kAlways;
  return kTable;
}

void free_batch(ilg_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->d_state);
  cudaFree(b->d_desc);
  cudaFree(b->d_tables);
  cudaFree(b->d_order);
  cudaFree(b->d_counter);
  cudaFree(b->d_failed);
  cudaFree(b->d_record);
  cudaFree(b->d_rec);
  cudaFree(b->d_out);
  cudaFree(b->d_states);
  cudaFree(b->d_trig);
  cudaFree(b->d_mass);
  cudaFree(b->d_amp);
  if (b->own_stream) cudaStreamDestroy(b->stream);
}

}  // namespace

extern "C" {

const char* ilg_batch_last_error(const ilg_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

ilg_status ilg_batch_create(const ilg_params* params, uint32_t n, void* stream, ilg_batch** out) {
  if (!out) return bfail(nullptr, ILG_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!params || n == 0) return bfail(nullptr, ILG_E_INVALID, "need at least one replica");
  for (uint32_t i = 0; i < n; ++i) {
    const std::string bad = validate_params(params[i]);
    if (!bad.empty()) return bfail(nullptr, ILG_E_INVALID, "replica " + std::to_string(i) + ": " + bad);
    if (params[i].lattice != ILG_D1Q3) return bfail(nullptr, ILG_E_INVALID, "batches hold D1Q3 rings");
    if (params[i].seed != params[0].seed) return bfail(nullptr, ILG_E_INVALID, "all replicas of a batch share one seed");
    if (params[i].Lx > kBatchMaxL) return bfail(nullptr, ILG_E_INVALID, "ring longer than 10240");
  }
  ilg_batch* b = new (std::nothrow) ilg_batch();
  if (!b) return bfail(nullptr, ILG_E_OOM, "host allocation failed");
  b->n = n;
  b->p.assign(params, params + n);
  b->stream = static_cast<cudaStream_t>(stream);
  auto bail = [&](cudaError_t e, const char* what) {
    bcuda(nullptr, e, what);
    free_batch(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? ILG_E_OOM : ILG_E_CUDA;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bail(e, "device query");
  if (!b->stream) {
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "cudaStreamCreate");
    b->own_stream = true;
  }
  b->desc.resize(n);
  std::vector<uint32_t> tables(size_t(n) * kBlockWords, 0u);
  for (uint32_t i = 0; i < n; ++i) {
    const ilg_params& q = b->p[i];
    ReplicaDesc& d = b->desc[i];
    double w[9];
    weights(ILG_D1Q3, q.theta, w);
    const double omega_star = q.omega_eff > 1.0 ? 2.0 - q.omega_eff : q.omega_eff;
    const uint64_t Po = quantise_probability(omega_star), Pr = quantise_probability(w[0]);
    d.L = q.Lx;
    d.flip = q.omega_eff > 1.0 ? 1u : 0u;
    d.omega_mode = mode_of(Po);
    d.rest_mode = mode_of(Pr);
    d.replica = q.replica;
    d.t = 0;
    d.particle = q.sampler == ILG_SAMPLER_PARTICLE ? 1u : 0u;
    d.general = general_path(ILG_D1Q3, q.theta, omega_star, q.n0, q.Lx) | d.particle;
    d.state_off = b->total;
    b->total += 3 * size_t(q.Lx);
    b->Lmax = std::max(b->Lmax, q.Lx);
    build_table_block(3, q.sampler, Po, Pr, 0, tables.data() + size_t(i) * kBlockWords);
  }
  // longest rings first
  std::vector<uint32_t> order(n);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return b->desc[x].L > b->desc[y].L; });

  if ((e = dev_alloc(&b->d_state, sizeof(uint16_t) * b->total)) != cudaSuccess) return bail(e, "cudaMalloc state");
  if ((e = dev_alloc(&b->d_desc, sizeof(ReplicaDesc) * n)) != cudaSuccess) return bail(e, "cudaMalloc desc");
  if ((e = dev_alloc(&b->d_tables, sizeof(uint32_t) * tables.size())) != cudaSuccess) return bail(e, "cudaMalloc tables");
  if ((e = dev_alloc(&b->d_order, sizeof(uint32_t) * n)) != cudaSuccess) return bail(e, "cudaMalloc order");
  if ((e = dev_alloc(&b->d_counter, sizeof(unsigned int))) != cudaSuccess) return bail(e, "cudaMalloc counter");
  if ((e = dev_alloc(&b->d_failed, sizeof(uint32_t) * n)) != cudaSuccess) return bail(e, "cudaMalloc flags");
  if ((e = dev_alloc(&b->d_mass, sizeof(unsigned long long) * n)) != cudaSuccess) return bail(e, "cudaMalloc mass");
  if ((e = dev_alloc(&b->d_amp, sizeof(double) * n)) != cudaSuccess) return bail(e, "cudaMalloc amp");
  if ((e = cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(ReplicaDesc) * n, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_tables, tables.data(), sizeof(uint32_t) * tables.size(), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(b->d_state, 0, sizeof(uint16_t) * b->total, b->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
    return bail(e, "upload");
  b->threads = int(batch_default_threads(b->Lmax));
  if ((e = prepare_batch_kernel(b->Lmax, b->threads)) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  round_keys(params[0].seed, b->common.rk);
  b->common.key0 = uint32_t(params[0].seed);
  b->common.key1 = uint32_t(params[0].seed >> 32);
  *out = b;
  return ILG_OK;
}

ilg_status ilg_batch_destroy(ilg_batch* b) {
  if (!b) return ILG_OK;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
  return ILG_OK;
}

ilg_status ilg_batch_init(ilg_batch* b) {
  if (!b) return ILG_E_INVALID;
  // every replica's Poisson tables in one upload, then one init launch per replica
  std::vector<InitTables> its(b->n);
  std::vector<uint32_t> all;
  std::vector<size_t> base(b->n);
  for (uint32_t i = 0; i < b->n; ++i) {
    std::string msg;
    if (!build_init_tables(b->p[i], 3, &its[i], &msg)) return bfail(b, ILG_E_INVALID, "replica " + std::to_string(i) + ": " + msg);
    base[i] = all.size();
    all.insert(all.end(), its[i].offset.begin(), its[i].offset.end());
    all.insert(all.end(), its[i].count.begin(), its[i].count.end());
    all.insert(all.end(), its[i].table.begin(), its[i].table.end());
  }
  uint32_t* d_all = nullptr;
  BCUDA(b, dev_alloc(&d_all, sizeof(uint32_t) * all.size()), "cudaMalloc init tables");
  cudaError_t e = cudaMemcpyAsync(d_all, all.data(), sizeof(uint32_t) * all.size(), cudaMemcpyHostToDevice, b->stream);
  for (uint32_t i = 0; i < b->n && e == cudaSuccess; ++i) {
    const ilg_params& q = b->p[i];
    InitArgs a{};
    a.Lx = q.Lx;
    a.Ly = 1;
    a.period = its[i].period;
    a.axis = its[i].period > 1 ? 1u : 0u;
    a.mode = its[i].period > 1 ? uint32_t(((int64_t(q.mode_mx) % int64_t(q.Lx)) + q.Lx) % q.Lx) : 0u;
    a.weighted = q.init_weighted ? 1u : 0u;
    a.key0 = uint32_t(q.seed);
    a.key1 = uint32_t(q.seed >> 32);
    a.replica = q.replica;
    const size_t cells = its[i].offset.size();
    a.offset = d_all + base[i];
    a.count = d_all + base[i] + cells;
    a.table = d_all + base[i] + 2 * cells;
    const int grid = int(std::min<size_t>((q.Lx + 255) / 256, size_t(b->sms) * 4));
    e = launch_init(3, a, b->d_state + b->desc[i].state_off, grid, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(d_all);
  if (e != cudaSuccess) return bcuda(b, e, "batch init");
  for (auto& d : b->desc) d.t = 0;
  BCUDA(b, cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(ReplicaDesc) * b->n, cudaMemcpyHostToDevice, b->stream),
        "upload desc");
  BCUDA(b, cudaStreamSynchronize(b->stream), "batch init");
  return ILG_OK;
}

ilg_status ilg_batch_set_state(ilg_batch* b, uint32_t i, const uint16_t* host, size_t n, uint64_t t) {
  if (!b || !host || i >= b->n) return ILG_E_INVALID;
  if (n != 3 * size_t(b->desc[i].L)) return bfail(b, ILG_E_INVALID, "state size must be 3 * L");
  if (t >= (uint64_t(1) << 32)) return bfail(b, ILG_E_INVALID, "t must be below 2^32");
  b->desc[i].t = uint32_t(t);
  uint64_t mass = 0;
  for (size_t k = 0; k < n; ++k) mass += host[k];
  const double om = b->p[i].omega_eff > 1.0 ? 2.0 - b->p[i].omega_eff : b->p[i].omega_eff;
  b->desc[i].general = general_path(ILG_D1Q3, b->p[i].theta, om, double(mass) / double(n), b->p[i].Lx) | b->desc[i].particle;
  BCUDA(b, cudaMemcpyAsync(b->d_state + b->desc[i].state_off, host, sizeof(uint16_t) * n, cudaMemcpyHostToDevice, b->stream),
        "copy state in");
  BCUDA(b, cudaMemcpyAsync(b->d_desc + i, &b->desc[i], sizeof(ReplicaDesc), cudaMemcpyHostToDevice, b->stream), "copy desc");
  BCUDA(b, cudaStreamSynchronize(b->stream), "copy state in");
  return ILG_OK;
}

ilg_status ilg_batch_get_state(ilg_batch* b, uint32_t i, uint16_t* host, size_t n, uint64_t* t) {
  if (!b || !host || i >= b->n) return ILG_E_INVALID;
  if (n != 3 * size_t(b->desc[i].L)) return bfail(b, ILG_E_INVALID, "state size must be 3 * L");
  BCUDA(b, cudaMemcpyAsync(host, b->d_state + b->desc[i].state_off, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost, b->stream),
        "copy state out");
  BCUDA(b, cudaStreamSynchronize(b->stream), "copy state out");
  if (t) *t = b->desc[i].t;
  return ILG_OK;
}

namespace {

// Queue one persistent launch of T steps (graph-captured, re-captured when T, the
// record flag or the mode change) and the read-back of the per-ring flags and
// descriptors.  With rec the complex amplitude of record_mode is recorded at the
// start and after every step (n x (T + 1) x 4 raw 128-bit sums in d_record).
ilg_status batch_launch(ilg_batch* b, uint32_t T, int32_t record_mode, bool rec, bool trig,
                        std::vector<uint32_t>& failed, bool states = false) {
  for (const auto& d : b->desc)
    if (uint64_t(d.t) + T >= (uint64_t(1) << 32)) return bfail(b, ILG_E_INVALID, "step counter would reach 2^32");
  const size_t need = size_t(b->n) * (size_t(T) + 1) * 4;
  if (rec && b->record_cap < need) {
    cudaFree(b->d_record);
    b->d_record = nullptr;
    b->record_cap = 0;
    BCUDA(b, dev_alloc(&b->d_record, sizeof(long long) * need), "cudaMalloc record");
    b->record_cap = need;
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  if (trig) {
    // every ring's values of the recorded mode at its nodes' place, rebuilt each call
    // (the fixed-point cos and sin take double-precision sincospi: once per node here
    // instead of once per node and step in the kernel)
    const size_t nodes = b->total / 3;
    if (b->trig_cap < nodes) {
      cudaFree(b->d_trig);
      b->d_trig = nullptr;
      b->trig_cap = 0;
      BCUDA(b, dev_alloc(&b->d_trig, sizeof(longlong2) * nodes), "cudaMalloc trig");
      b->trig_cap = nodes;
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
    }
    BCUDA(b, launch_batch_trig_rings(b->d_desc, b->n, record_mode, b->d_trig, b->stream), "trig table");
  }
  if (states && b->states_cap < size_t(T) * b->total) {
    cudaFree(b->d_states);
    b->d_states = nullptr;
    b->states_cap = 0;
    BCUDA(b, dev_alloc(&b->d_states, sizeof(uint16_t) * size_t(T) * b->total), "cudaMalloc state record");
    b->states_cap = size_t(T) * b->total;
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  if (!b->graph || b->graph_T != T || b->graph_rec != rec || b->graph_mode != record_mode || b->graph_trig != trig ||
      b->graph_states != states) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    BatchArgs a{};
    a.n = b->n;
    a.T = T;
    a.Lmax = b->Lmax;
    a.record_mode = record_mode;
    a.order = b->d_order;
    a.desc = b->d_desc;
    a.tables = b->d_tables;
    a.state = b->d_state;
    a.counter = b->d_counter;
    a.failed = b->d_failed;
    a.record = rec ? b->d_record : nullptr;
    a.trig = trig ? b->d_trig : nullptr;
    a.states = states ? b->d_states : nullptr;
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_failed, 0, sizeof(uint32_t) * b->n, b->stream);
    if (e == cudaSuccess) e = launch_batch(a, b->common, b->sms, b->stream, b->threads);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bcuda(b, e != cudaSuccess ? e : e2, "capture batch launch");
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(b, e, "instantiate batch graph");
    b->graph_T = T;
    b->graph_rec = rec;
    b->graph_mode = record_mode;
    b->graph_trig = trig;
    b->graph_states = states;
  }
  BCUDA(b, cudaGraphLaunch(b->graph, b->stream), "batch launch");
  failed.assign(b->n, 0);
  BCUDA(b, cudaMemcpyAsync(failed.data(), b->d_failed, sizeof(uint32_t) * b->n, cudaMemcpyDeviceToHost, b->stream), "read flags");
  BCUDA(b, cudaMemcpyAsync(b->desc.data(), b->d_desc, sizeof(ReplicaDesc) * b->n, cudaMemcpyDeviceToHost, b->stream), "read desc");
  return ILG_OK;
}

// Wait for the queued work; ILG_E_OVERFLOW if a ring stopped.
ilg_status batch_finish(ilg_batch* b, const std::vector<uint32_t>& failed) {
  BCUDA(b, cudaStreamSynchronize(b->stream), "batch run");
  uint32_t nf = 0, first = 0;
  for (uint32_t i = 0; i < b->n; ++i)
    if (failed[i]) {
      if (!nf) first = i;
      ++nf;
    }
  if (nf) {
    char buf[200];
    std::snprintf(buf, sizeof(buf), "%u replica(s) stopped on an occupation above 65535 (first: %u at t = %u)", nf, first,
                  b->desc[first].t);
    return bfail(b, ILG_E_OVERFLOW, buf);
  }
  return ILG_OK;
}

ilg_status ensure_doubles(ilg_batch* b, double** buf, size_t* cap, size_t need) {
  if (*cap >= need) return ILG_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  BCUDA(b, dev_alloc(buf, sizeof(double) * need), "cudaMalloc");
  *cap = need;
  return ILG_OK;
}

}  // namespace

ilg_status ilg_batch_run_record(ilg_batch* b, uint32_t T, int32_t record_mode, double* amp_record,
                                uint16_t* state_record) {
  if (!b) return ILG_E_INVALID;
  NvtxRange nvtx("ilg_batch_run");
  if (T == 0) return ILG_OK;
  const bool rec = amp_record != nullptr;
  const bool states = state_record != nullptr;
  std::vector<uint32_t> failed;
  if (rec) {
    ilg_status st = ensure_doubles(b, &b->d_out, &b->out_cap, size_t(b->n) * T);
    if (st == ILG_OK) st = ensure_doubles(b, &b->d_rec, &b->rec_cap, size_t(b->n) * (size_t(T) + 1) * 2);
    if (st != ILG_OK) return st;
  }
  ilg_status st = batch_launch(b, T, record_mode, rec, rec, failed, states);
  if (st != ILG_OK) return st;
  if (rec) {
    BCUDA(b, launch_batch_convert(b->d_desc, b->d_record, b->n, T, b->d_rec, b->stream), "convert record");
    BCUDA(b, launch_batch_amp(b->d_desc, b->d_rec, b->n, T, b->d_out, b->stream), "amplitude record");
    BCUDA(b, cudaMemcpyAsync(amp_record, b->d_out, sizeof(double) * b->n * size_t(T), cudaMemcpyDeviceToHost, b->stream),
          "read record");
  }
  if (states)
    BCUDA(b, cudaMemcpyAsync(state_record, b->d_states, sizeof(uint16_t) * size_t(T) * b->total,
                             cudaMemcpyDeviceToHost, b->stream),
          "read state record");
  return batch_finish(b, failed);
}

ilg_status ilg_batch_run(ilg_batch* b, uint32_t T, int32_t record_mode, double* amp_record) {
  return ilg_batch_run_record(b, T, record_mode, amp_record, nullptr);
}

ilg_status ilg_batch_ensemble(ilg_batch* b, uint32_t T, int32_t mode, double* stats, double* record) {
  if (!b) return ILG_E_INVALID;
  NvtxRange nvtx("ilg_batch_ensemble");
  if (!stats) return bfail(b, ILG_E_INVALID, "stats is NULL");
  if (b->n < 2) return bfail(b, ILG_E_INVALID, "an ensemble needs at least two rings");
  for (const auto& d : b->desc)
    if (d.L != b->desc[0].L) return bfail(b, ILG_E_INVALID, "ensemble statistics need rings of one length");
  if (mode % int64_t(b->desc[0].L) == 0) return bfail(b, ILG_E_INVALID, "the mode must not be a multiple of L");
  ilg_status st = ensure_doubles(b, &b->d_out, &b->out_cap, 6 * (size_t(T) + 1));
  if (st == ILG_OK) st = ensure_doubles(b, &b->d_rec, &b->rec_cap, size_t(b->n) * (size_t(T) + 1) * 2);
  if (st != ILG_OK) return st;
  std::vector<uint32_t> failed;
  st = batch_launch(b, T, mode, true, true, failed);
  if (st != ILG_OK) return st;
  BCUDA(b, launch_batch_convert(b->d_desc, b->d_record, b->n, T, b->d_rec, b->stream), "convert record");
  BCUDA(b, launch_batch_ensemble(b->d_rec, b->n, T, b->d_out, b->stream), "ensemble statistics");
  BCUDA(b, cudaMemcpyAsync(stats, b->d_out, sizeof(double) * 6 * (size_t(T) + 1), cudaMemcpyDeviceToHost, b->stream),
        "read statistics");
  if (record)
    BCUDA(b, cudaMemcpyAsync(record, b->d_rec, sizeof(double) * 2 * b->n * (size_t(T) + 1), cudaMemcpyDeviceToHost,
                             b->stream),
          "read record");
  return batch_finish(b, failed);
}

ilg_status ilg_batch_autotune(ilg_batch* b, uint32_t trial_steps, ilg_tuning* out) {
  if (!b) return ILG_E_INVALID;
  if (trial_steps == 0) trial_steps = 50;
  if (trial_steps > 10000) return bfail(b, ILG_E_INVALID, "at most 10000 trial steps");
  for (const auto& d : b->desc)
    if (uint64_t(d.t) + 8ull * trial_steps >= (uint64_t(1) << 32))
      return bfail(b, ILG_E_INVALID, "step counter would reach 2^32 in the trials");
  // the trials run on copies of the rings and descriptors; results are discarded
  uint16_t* s_state = nullptr;
  ReplicaDesc* s_desc = nullptr;
  unsigned int* s_counter = nullptr;
  uint32_t* s_failed = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    cudaFree(s_state);
    cudaFree(s_desc);
    cudaFree(s_counter);
    cudaFree(s_failed);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  cudaError_t e = dev_alloc(&s_state, sizeof(uint16_t) * b->total);
  if (e == cudaSuccess) e = dev_alloc(&s_desc, sizeof(ReplicaDesc) * b->n);
  if (e == cudaSuccess) e = dev_alloc(&s_counter, sizeof(unsigned int));
  if (e == cudaSuccess) e = dev_alloc(&s_failed, sizeof(uint32_t) * b->n);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s_state, b->d_state, sizeof(uint16_t) * b->total, cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s_desc, b->d_desc, sizeof(ReplicaDesc) * b->n, cudaMemcpyDeviceToDevice, b->stream);
  if (e != cudaSuccess) {
    release();
    return bcuda(b, e, "autotune scratch");
  }
  static const int kShapes[3] = {256, 512, 1024};
  ilg_tuning res{};
  res.n = 3;
  for (int k = 0; k < 8; ++k) res.ms_per_step[k] = -1.0;
  int best = -1;
  for (int k = 0; k < 3; ++k) {
    const int threads = kShapes[k];
    if (prepare_batch_kernel(b->Lmax, threads) != cudaSuccess) {  // the rings do not fit this shape
      cudaGetLastError();
      continue;
    }
    BatchArgs a{};
    a.n = b->n;
    a.T = trial_steps;
    a.Lmax = b->Lmax;
    a.order = b->d_order;
    a.desc = s_desc;
    a.tables = b->d_tables;
    a.state = s_state;
    a.counter = s_counter;
    a.failed = s_failed;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
      e = cudaMemsetAsync(s_counter, 0, sizeof(unsigned int), b->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s_failed, 0, sizeof(uint32_t) * b->n, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = launch_batch(a, b->common, b->sms, b->stream, threads);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e != cudaSuccess) {
      release();
      prepare_batch_kernel(b->Lmax, b->threads);
      return bcuda(b, e, "autotune trial");
    }
    res.ms_per_step[k] = double(ms) / trial_steps;
    if (best < 0 || res.ms_per_step[k] < res.ms_per_step[best]) best = k;
  }
  release();
  if (best < 0) return bfail(b, ILG_E_INVALID, "no block shape fits the rings");
  b->threads = kShapes[best];
  BCUDA(b, prepare_batch_kernel(b->Lmax, b->threads), "cudaFuncSetAttribute");
  if (b->graph) {  // the next run captures the chosen shape
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  res.choice = uint32_t(best);
  res.threads = uint32_t(b->threads);
  if (out) *out = res;
  return ILG_OK;
}

ilg_status ilg_batch_observables(ilg_batch* b, int32_t mode, uint64_t* mass, double* amp) {
  if (!b) return ILG_E_INVALID;
  BCUDA(b, launch_batch_obs(b->d_desc, b->d_state, b->n, mode, b->d_mass, b->d_amp, b->stream), "batch observables");
  if (mass)
    BCUDA(b, cudaMemcpyAsync(mass, b->d_mass, sizeof(uint64_t) * b->n, cudaMemcpyDeviceToHost, b->stream), "copy mass");
  if (amp) BCUDA(b, cudaMemcpyAsync(amp, b->d_amp, sizeof(double) * b->n, cudaMemcpyDeviceToHost, b->stream), "copy amp");
  BCUDA(b, cudaStreamSynchronize(b->stream), "batch observables");
  return ILG_OK;
}

}  // extern "C"
