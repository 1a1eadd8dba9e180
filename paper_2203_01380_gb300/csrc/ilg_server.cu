// Serving loop (ilg_server_*): a worker thread admits D2Q5 lattice requests into a
// preallocated device arena while memory and slots allow, keeps every admitted
// lattice resident, and advances all of them together — one multi-lattice launch
// per time step, a quantum of steps per round — so requests that arrive while
// others run join the next round (continuous batching).  A finished request's
// observables (and, if asked, its final state) are copied out, its memory goes back
// to the arena, and waiting requests are admitted.  Every random number is keyed by
// the request's replica word, so results do not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ilg_internal.h"
#include "ilg_launch.h"
#include "ilg_multi.h"

using namespace ilg;

namespace {

constexpr uint32_t kServerMaxSide = 32768;
constexpr size_t kAlign = 256;

struct Request {
  uint64_t id;
  ilg_params p;
  uint32_t steps;
  uint16_t* final_state;  // caller's host buffer or NULL
  double t_submit;
};

struct Resident {
  Request rq;
  size_t off_state = 0, state_bytes = 0;  // two buffers
  size_t off_tab = 0;
  uint32_t t = 0, remaining = 0, phase = 0;
  uint32_t flip = 0, omega_mode = 0, rest_mode = 0, general = 0, particle = 0;
  double t_admit = 0;
  int status = ILG_OK;
};

// First-fit allocator over one device allocation.
class Arena {
 public:
  void reset(size_t bytes) {
    free_.clear();
    if (bytes) free_[0] = bytes;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
 private:
  std::map<size_t, size_t> free_;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

uint32_t mode_of(uint64_t P) {
  if (P == 0) return kNever;
  if (P == (uint64_t(1) << 32)) return kAlways;
  return kTable;
}

}  // namespace

struct ilg_server {
  uint64_t seed = 0;
  uint32_t max_slots = 0, quantum = 0;
  int32_t policy = ILG_ADMIT_FIFO;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 0;
  uint8_t* d_arena = nullptr;
  size_t arena_bytes = 0;
  Arena arena;
  LatDesc* d_lat = nullptr;
  WorkItem* d_items = nullptr;
  size_t items_cap = 0;
  unsigned int* d_counters = nullptr;
  uint32_t* d_fail = nullptr;
  unsigned long long* d_col = nullptr;
  unsigned long long* d_row = nullptr;
  unsigned long long* d_mass = nullptr;
  int32_t* d_modes = nullptr;
  double* d_res = nullptr;
  StepArgs common{};
  std::chrono::steady_clock::time_point t0;
  // admissions: a newcomer's tables and Poisson initial state are written on their own
  // stream; the serving stream waits on the event before the next round, and the
  // arena memory of its initial-state tables returns once the event has completed
  cudaStream_t init_stream = nullptr;
  struct PendingInit {
    cudaEvent_t ev;
    size_t off, bytes;
  };
  std::vector<PendingInit> inits;
  cudaEvent_t round_ev = nullptr;   // end of a round's launches and its flag read-back
  uint32_t* h_fail = nullptr;       // pinned: per-lattice overflow flags of a round

  std::thread worker;
  std::mutex mu;
  std::condition_variable cv, idle_cv;
  bool stop = false;
  std::deque<Request> pending;
  std::vector<Resident> resident;
  std::vector<ilg_result> done;
  size_t in_flight = 0;  // submitted and not yet finished
  std::string err;
  int fatal = ILG_OK;
  double busy_s = 0, node_updates = 0;
  uint32_t peak_resident = 0;
};

namespace {

thread_local std::string g_server_create_error;

void free_server(ilg_server* s) {
  for (auto& pi : s->inits) cudaEventDestroy(pi.ev);
  s->inits.clear();
  if (s->round_ev) cudaEventDestroy(s->round_ev);
  if (s->h_fail) cudaFreeHost(s->h_fail);
  if (s->init_stream) cudaStreamDestroy(s->init_stream);
  cudaFree(s->d_arena);
  cudaFree(s->d_lat);
  cudaFree(s->d_items);
  cudaFree(s->d_counters);
  cudaFree(s->d_fail);
  cudaFree(s->d_col);
  cudaFree(s->d_row);
  cudaFree(s->d_mass);
  cudaFree(s->d_modes);
  cudaFree(s->d_res);
  if (s->own_stream) cudaStreamDestroy(s->stream);
}

size_t state_bytes_of(const ilg_params& p) { return sizeof(uint16_t) * 5 * size_t(p.Lx) * p.Ly; }

// Admit one request: arena memory for two state buffers and its tables, Poisson
// initial state.  Returns false (nothing changed) when the arena cannot hold it.
bool admit(ilg_server* s, const Request& rq, Resident* out, cudaError_t* cerr, std::string* msg) {
  *cerr = cudaSuccess;
  Resident r;
  r.rq = rq;
  const size_t tab_bytes = sizeof(uint32_t) * kBlockWords;
  InitTables it;
  if (!build_init_tables(rq.p, 5, &it, msg)) {
    r.status = ILG_E_INVALID;  // no memory held: reported as invalid when it finishes
    *out = r;
    return true;
  }
  const size_t init_words = it.offset.size() + it.count.size() + it.table.size();
  size_t off_init = 0;
  r.state_bytes = state_bytes_of(rq.p);
  if (!s->arena.alloc(2 * r.state_bytes, &r.off_state)) return false;
  if (!s->arena.alloc(tab_bytes, &r.off_tab)) {
    s->arena.release(r.off_state, 2 * r.state_bytes);
    return false;
  }
  if (!s->arena.alloc(sizeof(uint32_t) * init_words, &off_init)) {
    s->arena.release(r.off_state, 2 * r.state_bytes);
    s->arena.release(r.off_tab, tab_bytes);
    return false;
  }
  double w[9];
  weights(ILG_D2Q5, rq.p.theta, w);
  const double omega_star = rq.p.omega_eff > 1.0 ? 2.0 - rq.p.omega_eff : rq.p.omega_eff;
  const uint64_t Po = quantise_probability(omega_star), Pr = quantise_probability(w[0]);
  r.flip = rq.p.omega_eff > 1.0 ? 1u : 0u;
  r.particle = rq.p.sampler == ILG_SAMPLER_PARTICLE ? 1u : 0u;
  r.general = general_path(ILG_D2Q5, rq.p.theta, omega_star, rq.p.n0) | r.particle;
  r.omega_mode = mode_of(Po);
  r.rest_mode = mode_of(Pr);
  std::vector<uint32_t> tables(kBlockWords, 0u);
  build_table_block(5, rq.p.sampler, Po, Pr, 0, tables.data());
  std::vector<uint32_t> init(init_words);
  std::copy(it.offset.begin(), it.offset.end(), init.begin());
  std::copy(it.count.begin(), it.count.end(), init.begin() + it.offset.size());
  std::copy(it.table.begin(), it.table.end(), init.begin() + it.offset.size() + it.count.size());
  uint32_t* d_init = reinterpret_cast<uint32_t*>(s->d_arena + off_init);
  // (copies from pageable host memory: the source is consumed before the call returns)
  cudaError_t e =
      cudaMemcpyAsync(s->d_arena + r.off_tab, tables.data(), tab_bytes, cudaMemcpyHostToDevice, s->init_stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_init, init.data(), sizeof(uint32_t) * init_words, cudaMemcpyHostToDevice, s->init_stream);
  if (e == cudaSuccess) {
    InitArgs a{};
    a.Lx = rq.p.Lx;
    a.Ly = rq.p.Ly;
    a.period = it.period;
    a.axis = it.period > 1 ? (rq.p.mode_mx != 0 ? 1u : 2u) : 0u;
    const int64_t L = it.period;
    const int64_t mraw = rq.p.mode_mx != 0 ? rq.p.mode_mx : rq.p.mode_my;
    a.mode = it.period > 1 ? uint32_t(((mraw % L) + L) % L) : 0u;
    a.weighted = rq.p.init_weighted ? 1u : 0u;
    a.key0 = uint32_t(rq.p.seed);
    a.key1 = uint32_t(rq.p.seed >> 32);
    a.replica = rq.p.replica;
    a.offset = d_init;
    a.count = d_init + it.offset.size();
    a.table = d_init + it.offset.size() + it.count.size();
    const size_t nodes = size_t(rq.p.Lx) * rq.p.Ly;
    const int grid = int(std::min<size_t>((nodes + 255) / 256, size_t(s->sms) * 4));
    e = launch_init(5, a, reinterpret_cast<uint16_t*>(s->d_arena + r.off_state), grid, s->init_stream);
  }
  cudaEvent_t ev = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, s->init_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, ev, 0);
  if (e != cudaSuccess) {
    *cerr = e;
    if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(s->init_stream);
    s->arena.release(off_init, sizeof(uint32_t) * init_words);
    s->arena.release(r.off_state, 2 * r.state_bytes);
    s->arena.release(r.off_tab, tab_bytes);
    return false;
  }
  s->inits.push_back(ilg_server::PendingInit{ev, off_init, sizeof(uint32_t) * init_words});
  r.t = 0;
  r.remaining = rq.steps;
  r.phase = 0;
  *out = r;
  return true;
}

// Observables and (optionally) the final state of a finished request, then its
// memory goes back to the arena.
cudaError_t finish(ilg_server* s, Resident& r, ilg_result* res) {
  std::memset(res, 0, sizeof(*res));
  res->id = r.rq.id;
  res->status = r.status;
  res->t = r.t;
  res->t_submit = r.rq.t_submit;
  res->t_admit = r.t_admit;
  cudaError_t e = cudaSuccess;
  if (r.status == ILG_OK || r.status == ILG_E_OVERFLOW) {
    const uint16_t* st = reinterpret_cast<const uint16_t*>(s->d_arena + r.off_state + (r.phase ? r.state_bytes : 0));
    const uint32_t Lx = r.rq.p.Lx, Ly = r.rq.p.Ly;
    e = cudaMemsetAsync(s->d_col, 0, sizeof(unsigned long long) * Lx, s->stream);
    if (e == cudaSuccess) e = launch_sums(5, st, Lx, Ly, s->d_col, s->d_row, 0, s->stream);
    if (e == cudaSuccess) e = launch_project(s->d_col, s->d_row, Lx, Ly, s->d_modes, 1, s->d_res, s->d_mass, s->stream);
    double h[4] = {0, 0, 0, 0};
    unsigned long long M = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, s->d_res, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&M, s->d_mass, sizeof(M), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && r.rq.final_state)
      e = cudaMemcpyAsync(r.rq.final_state, st, r.state_bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    res->mass = M;
    res->amp = h[2];
    res->Sk = h[3];
  }
  if (r.state_bytes) {
    s->arena.release(r.off_state, 2 * r.state_bytes);
    s->arena.release(r.off_tab, sizeof(uint32_t) * kBlockWords);
  }
  res->t_done = now_s(s->t0);
  return e;
}

// Initial states whose event has completed give their tables' arena memory back.
cudaError_t release_inits(ilg_server* s) {
  size_t k = 0;
  for (size_t i = 0; i < s->inits.size(); ++i) {
    const cudaError_t q = cudaEventQuery(s->inits[i].ev);
    if (q == cudaSuccess) {
      cudaEventDestroy(s->inits[i].ev);
      s->arena.release(s->inits[i].off, s->inits[i].bytes);
    } else if (q == cudaErrorNotReady) {
      s->inits[k++] = s->inits[i];
    } else {
      return q;
    }
  }
  s->inits.resize(k);
  return cudaSuccess;
}

// Admission: in arrival order (or least work first) while slots and arena memory
// allow; every admitted request's initial state is queued on the admission stream.
void admit_pending(ilg_server* s, cudaError_t& e) {
  e = release_inits(s);
  if (e != cudaSuccess) return;
  for (;;) {
    Request rq;
    size_t pick = 0;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->pending.empty() || s->resident.size() >= s->max_slots) break;
      if (s->policy == ILG_ADMIT_SMALLEST) {
        // least work (node updates) first
        double best = -1.0;
        for (size_t k = 0; k < s->pending.size(); ++k) {
          const Request& q = s->pending[k];
          const double w = double(q.p.Lx) * q.p.Ly * q.steps;
          if (best < 0.0 || w < best) {
            best = w;
            pick = k;
          }
        }
      }
      rq = s->pending[pick];
    }
    Resident r;
    std::string msg;
    if (!admit(s, rq, &r, &e, &msg)) {
      if (e != cudaSuccess) break;
      break;  // wait for memory to come back
    }
    r.t_admit = now_s(s->t0);
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.erase(s->pending.begin() + long(pick));
    s->resident.push_back(r);
    s->peak_resident = std::max<uint32_t>(s->peak_resident, uint32_t(s->resident.size()));
  }
}

void worker_main(ilg_server* s) {
  cudaError_t e = cudaSuccess;
  std::vector<LatDesc> lat;
  std::vector<WorkItem> items;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || !s->pending.empty() || !s->resident.empty(); });
      if (s->stop && s->resident.empty() && s->pending.empty()) break;
      if (s->stop) {
        // shutting down: drop what is queued
        s->in_flight -= s->pending.size();
        s->pending.clear();
      }
    }
    const double t_round = now_s(s->t0);
    NvtxRange nvtx("ilg_server round");
    admit_pending(s, e);
    double round_updates = 0;
    if (e != cudaSuccess) break;
    // one round: up to `quantum` steps, each lattice taking min(quantum, remaining)
    uint32_t q = 0;
    for (auto& r : s->resident)
      if (r.status == ILG_OK) q = std::max(q, std::min(s->quantum, r.remaining));
    lat.clear();
    items.clear();
    std::vector<size_t> which;
    for (size_t k = 0; k < s->resident.size(); ++k) {
      Resident& r = s->resident[k];
      if (r.status != ILG_OK || r.remaining == 0) continue;
      LatDesc d{};
      d.Lx = r.rq.p.Lx;
      d.Ly = r.rq.p.Ly;
      d.t0 = r.t;
      d.phase = r.phase;
      d.replica = r.rq.p.replica;
      d.flip = r.flip;
      d.omega_mode = r.omega_mode;
      d.rest_mode = r.rest_mode;
      d.steps = std::min(q, r.remaining);
      d.general = r.general;
      d.particle = r.particle;
      d.buf0 = reinterpret_cast<uint16_t*>(s->d_arena + r.off_state);
      d.buf1 = reinterpret_cast<uint16_t*>(s->d_arena + r.off_state + r.state_bytes);
      d.tables = reinterpret_cast<const uint32_t*>(s->d_arena + r.off_tab);
      const uint32_t li = uint32_t(lat.size());
      lat.push_back(d);
      which.push_back(k);
      const uint32_t nodes = d.Lx * d.Ly;
      for (uint32_t n0 = 0; n0 < nodes; n0 += kItemNodes) items.push_back(WorkItem{li, n0, std::min(nodes, n0 + kItemNodes)});
    }
    if (!lat.empty() && q > 0) {
      if (items.size() > s->items_cap) {
        cudaFree(s->d_items);
        s->d_items = nullptr;
        e = dev_alloc(&s->d_items, sizeof(WorkItem) * items.size() * 2);
        if (e != cudaSuccess) break;
        s->items_cap = items.size() * 2;
      }
      e = cudaMemcpyAsync(s->d_lat, lat.data(), sizeof(LatDesc) * lat.size(), cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->d_counters, 0, sizeof(unsigned int) * q, s->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->d_fail, 0xFF, sizeof(uint32_t) * lat.size(), s->stream);
      MultiArgs ma{};
      ma.lat = s->d_lat;
      ma.items = s->d_items;
      ma.n_items = uint32_t(items.size());
      ma.counter = s->d_counters;
      ma.fail = s->d_fail;
      // persistent blocks: as many as are resident at once (3 per SM at this register count)
      const int grid = int(std::min<size_t>(items.size(), size_t(s->sms) * kMultiBlocksPerSm));
      for (uint32_t sub = 0; sub < q && e == cudaSuccess; ++sub) e = launch_multi_step(ma, s->common, sub, grid, s->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_fail, s->d_fail, sizeof(uint32_t) * lat.size(), cudaMemcpyDeviceToHost, s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(s->round_ev, s->stream);
      // while the round runs, requests that arrive are admitted (their initial states
      // queued on the admission stream, for the next round)
      while (e == cudaSuccess) {
        const cudaError_t q_ = cudaEventQuery(s->round_ev);
        if (q_ == cudaSuccess) break;
        if (q_ != cudaErrorNotReady) {
          e = q_;
          break;
        }
        admit_pending(s, e);
        if (e == cudaSuccess) std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
      if (e != cudaSuccess) break;
      const uint32_t* fail = s->h_fail;
      for (size_t j = 0; j < which.size(); ++j) {
        Resident& r = s->resident[which[j]];
        const uint32_t done = fail[j] == 0xFFFFFFFFu ? lat[j].steps : fail[j];
        round_updates += double(r.rq.p.Lx) * r.rq.p.Ly * done;
        r.t += done;
        r.remaining -= done;
        r.phase ^= (done & 1u);
        if (fail[j] != 0xFFFFFFFFu) r.status = ILG_E_OVERFLOW;
      }
    }
    // finished requests
    std::vector<ilg_result> out;
    std::vector<Resident> keep;
    for (auto& r : s->resident) {
      if (r.status == ILG_OK && r.remaining > 0) {
        keep.push_back(r);
        continue;
      }
      ilg_result res;
      e = finish(s, r, &res);
      if (e != cudaSuccess) break;
      out.push_back(res);
    }
    if (e != cudaSuccess) break;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->busy_s += now_s(s->t0) - t_round;
      s->node_updates += round_updates;
      s->resident.swap(keep);
      for (auto& r : out) s->done.push_back(r);
      s->in_flight -= out.size();
      if (s->in_flight == 0) s->idle_cv.notify_all();
    }
  }
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fatal = ILG_E_CUDA;
    s->err = std::string("server worker: ") + cudaGetErrorString(e);
    s->idle_cv.notify_all();
  }
}

}  // namespace

extern "C" {

const char* ilg_server_last_error(const ilg_server* s) { return s ? s->err.c_str() : g_server_create_error.c_str(); }

ilg_status ilg_server_create(uint64_t seed, uint64_t hbm_bytes, uint32_t max_slots, uint32_t quantum, void* stream,
                             ilg_server** out) {
  if (!out) return ILG_E_INVALID;
  *out = nullptr;
  if (max_slots == 0 || quantum == 0 || hbm_bytes < (1u << 20)) {
    g_server_create_error = "need max_slots > 0, quantum > 0 and at least 1 MiB of arena";
    return ILG_E_INVALID;
  }
  ilg_server* s = new (std::nothrow) ilg_server();
  if (!s) return ILG_E_OOM;
  s->seed = seed;
  s->max_slots = max_slots;
  s->quantum = quantum;
  s->stream = static_cast<cudaStream_t>(stream);
  s->t0 = std::chrono::steady_clock::now();
  auto bail = [&](cudaError_t e, const char* what) {
    g_server_create_error = std::string(what) + ": " + cudaGetErrorString(e);
    free_server(s);
    delete s;
    return e == cudaErrorMemoryAllocation ? ILG_E_OOM : ILG_E_CUDA;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bail(e, "device query");
  if (!s->stream) {
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "cudaStreamCreate");
    s->own_stream = true;
  }
  if ((e = dev_alloc(&s->d_arena, hbm_bytes)) != cudaSuccess) return bail(e, "cudaMalloc arena");
  s->arena_bytes = hbm_bytes;
  s->arena.reset(hbm_bytes);
  if ((e = dev_alloc(&s->d_lat, sizeof(LatDesc) * max_slots)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dev_alloc(&s->d_counters, sizeof(unsigned int) * quantum)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dev_alloc(&s->d_fail, sizeof(uint32_t) * max_slots)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dev_alloc(&s->d_col, sizeof(unsigned long long) * kServerMaxSide)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dev_alloc(&s->d_row, sizeof(unsigned long long) * kServerMaxSide)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dev_alloc(&s->d_mass, sizeof(unsigned long long))) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dev_alloc(&s->d_modes, sizeof(int32_t) * 2)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dev_alloc(&s->d_res, sizeof(double) * 4)) != cudaSuccess) return bail(e, "cudaMalloc");
  const int32_t mode1[2] = {1, 0};
  if ((e = cudaMemcpy(s->d_modes, mode1, sizeof(mode1), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e, "upload");
  if ((e = prepare_multi_kernel()) != cudaSuccess) return bail(e, "cudaFuncSetAttribute");
  if ((e = cudaStreamCreateWithFlags(&s->init_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "cudaStreamCreate");
  if ((e = cudaEventCreateWithFlags(&s->round_ev, cudaEventDisableTiming)) != cudaSuccess)
    return bail(e, "cudaEventCreate");
  if ((e = cudaMallocHost(&s->h_fail, sizeof(uint32_t) * max_slots)) != cudaSuccess) return bail(e, "cudaMallocHost");
  round_keys(seed, s->common.rk);
  s->common.key0 = uint32_t(seed);
  s->common.key1 = uint32_t(seed >> 32);
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    g_server_create_error = "cannot start the worker thread";
    free_server(s);
    delete s;
    return ILG_E_OOM;
  }
  *out = s;
  return ILG_OK;
}

ilg_status ilg_server_submit(ilg_server* s, uint64_t id, const ilg_params* p, uint32_t steps, uint16_t* final_state) {
  if (!s || !p) return ILG_E_INVALID;
  const std::string bad = validate_params(*p);
  std::lock_guard<std::mutex> lk(s->mu);
  if (!bad.empty()) {
    s->err = bad;
    return ILG_E_INVALID;
  }
  if (p->lattice != ILG_D2Q5) {
    s->err = "the server runs D2Q5 lattices";
    return ILG_E_INVALID;
  }
  if (p->seed != s->seed) {
    s->err = "a request's seed must be the server's";
    return ILG_E_INVALID;
  }
  if (p->Lx > kServerMaxSide || p->Ly > kServerMaxSide) {
    s->err = "side above 32768";
    return ILG_E_INVALID;
  }
  if (2 * state_bytes_of(*p) + sizeof(uint32_t) * kBlockWords + (1u << 20) > s->arena_bytes) {
    s->err = "request larger than the server's device arena";
    return ILG_E_OOM;
  }
  if (s->fatal != ILG_OK) return ilg_status(s->fatal);
  if (uint64_t(steps) >= (uint64_t(1) << 32)) return ILG_E_INVALID;
  s->pending.push_back(Request{id, *p, steps, final_state, now_s(s->t0)});
  ++s->in_flight;
  s->cv.notify_one();
  return ILG_OK;
}

ilg_status ilg_server_set_policy(ilg_server* s, int32_t policy) {
  if (!s || (policy != ILG_ADMIT_FIFO && policy != ILG_ADMIT_SMALLEST)) return ILG_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  s->policy = policy;
  return ILG_OK;
}

ilg_status ilg_server_poll(ilg_server* s, ilg_result* out, uint32_t cap, uint32_t* n) {
  if (!s || !n || (cap && !out)) return ILG_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  const uint32_t k = uint32_t(std::min<size_t>(cap, s->done.size()));
  for (uint32_t i = 0; i < k; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *n = k;
  return s->fatal != ILG_OK ? ilg_status(s->fatal) : ILG_OK;
}

ilg_status ilg_server_wait_idle(ilg_server* s, double timeout_s) {
  if (!s) return ILG_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->idle_cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] { return s->in_flight == 0 || s->fatal != ILG_OK; });
  if (s->fatal != ILG_OK) return ilg_status(s->fatal);
  if (!ok) {
    s->err = "requests still running at the timeout";
    return ILG_E_TIMEOUT;
  }
  return ILG_OK;
}

ilg_status ilg_server_stats(ilg_server* s, double* busy_s, double* node_updates, uint32_t* peak_resident) {
  if (!s) return ILG_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (busy_s) *busy_s = s->busy_s;
  if (node_updates) *node_updates = s->node_updates;
  if (peak_resident) *peak_resident = s->peak_resident;
  return ILG_OK;
}

ilg_status ilg_server_destroy(ilg_server* s) {
  if (!s) return ILG_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaStreamSynchronize(s->stream);
  if (s->init_stream) cudaStreamSynchronize(s->init_stream);
  free_server(s);
  delete s;
  return ILG_OK;
}

}  // extern "C"
