// Observables of a caller-held device state without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// observables: applications whose device memory already belongs to their own
// pool (a framework's caching allocator that holds the free HBM, so cudaMalloc
// would fail), and real-time loops that must not wait on the allocator's locks or
// on the device-wide synchronisation that freeing memory implies.
// ilg_observables_noalloc serves them: it runs the same reduction and projection
// kernels as ilg_observables, but its scratch (column and row sums, mass, modes,
// results) is the file-scope array below, which every GPU that loads the library
// holds until the process exits.  The call still synchronises its stream to
// return the results.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ilg_internal.h"
#include "ilg_launch.h"

namespace {

constexpr uint32_t kMaxSide = 32768;   // largest Lx and Ly
constexpr uint32_t kMaxModes = 256;    // largest number of modes per call
constexpr int kMaxDevices = 64;

// scratch layout, in 8-byte words: col[kMaxSide] | row[kMaxSide] | mass | res[4 kMaxModes] | modes
constexpr size_t kColOff = 0;
constexpr size_t kRowOff = kColOff + kMaxSide;
constexpr size_t kMassOff = kRowOff + kMaxSide;
constexpr size_t kResOff = kMassOff + 1;
constexpr size_t kModesOff = kResOff + 4 * kMaxModes;
constexpr size_t kScratchWords = kModesOff + kMaxModes;  // modes: kMaxModes int32 pairs

static __device__ __align__(256) unsigned long long noalloc_scratch[kScratchWords];

std::mutex g_setup_mutex;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};

ilg_status context_free_fail(ilg_status s, const std::string& msg) {
  ilg::set_context_free_error(msg);
  return s;
}

}  // namespace

extern "C" ilg_status ilg_observables_noalloc(int32_t lattice, uint32_t Lx, uint32_t Ly, const uint16_t* state,
                                              const int32_t* modes, uint32_t nmodes, void* stream,
                                              uint64_t* mass, double* re, double* im, double* amp,
                                              double* Sk) {
  if (lattice != ILG_D1Q3 && lattice != ILG_D2Q5 && lattice != ILG_D2Q9)
    return context_free_fail(ILG_E_INVALID, "bad lattice");
  if (lattice == ILG_D1Q3) Ly = 1;
  if (!state) return context_free_fail(ILG_E_INVALID, "state is NULL");
  if (Lx < 3 || (lattice != ILG_D1Q3 && Ly < 3)) return context_free_fail(ILG_E_INVALID, "Lx and Ly must be >= 3");
  if (Lx > kMaxSide || Ly > kMaxSide)
    return context_free_fail(ILG_E_INVALID, "ilg_observables_noalloc: Lx and Ly are limited to 32768 by its static scratch");
  if (nmodes > kMaxModes)
    return context_free_fail(ILG_E_INVALID, "ilg_observables_noalloc: at most 256 modes per call (static scratch)");
  if (nmodes && !modes) return context_free_fail(ILG_E_INVALID, "modes is NULL");
  bool rows = false;
  for (uint32_t i = 0; i < nmodes; ++i) {
    const int32_t mx = modes[2 * i], my = modes[2 * i + 1];
    if ((mx == 0) == (my == 0)) return context_free_fail(ILG_E_INVALID, "each mode must have exactly one nonzero component");
    if (my != 0 && lattice == ILG_D1Q3) return context_free_fail(ILG_E_INVALID, "D1Q3 has no y modes");
    rows |= my != 0;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return context_free_fail(ILG_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return context_free_fail(ILG_E_INVALID, "device ordinal out of range");
  unsigned long long* base = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&g_scratch_ptr[dev]), noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        return context_free_fail(ILG_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    base = g_scratch_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int Q = lattice == ILG_D1Q3 ? 3 : (lattice == ILG_D2Q5 ? 5 : 9);
  unsigned long long* col = base + kColOff;
  unsigned long long* row = base + kRowOff;
  unsigned long long* d_mass = base + kMassOff;
  double* res = reinterpret_cast<double*>(base + kResOff);
  int32_t* d_modes = reinterpret_cast<int32_t*>(base + kModesOff);
  // the array keeps the previous call's contents: clear the sums that accumulate
  e = cudaMemsetAsync(col, 0, sizeof(unsigned long long) * Lx, s);
  if (e == cudaSuccess && rows) e = cudaMemsetAsync(row, 0, sizeof(unsigned long long) * Ly, s);
  if (e == cudaSuccess && nmodes)
    e = cudaMemcpyAsync(d_modes, modes, sizeof(int32_t) * 2 * nmodes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = ilg::launch_sums(Q, state, Lx, Ly, col, row, rows ? 1 : 0, s);
  if (e == cudaSuccess) e = ilg::launch_project(col, row, Lx, Ly, d_modes, nmodes, res, d_mass, s);
  double h_res[4 * kMaxModes];
  unsigned long long h_mass = 0;
  if (e == cudaSuccess && nmodes)
    e = cudaMemcpyAsync(h_res, res, sizeof(double) * 4 * nmodes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_mass, d_mass, sizeof(h_mass), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return context_free_fail(ILG_E_CUDA, std::string("ilg_observables_noalloc: ") + cudaGetErrorString(e));
  if (mass) *mass = h_mass;
  for (uint32_t i = 0; i < nmodes; ++i) {
    if (re) re[i] = h_res[4 * i + 0];
    if (im) im[i] = h_res[4 * i + 1];
    if (amp) amp[i] = h_res[4 * i + 2];
    if (Sk) Sk[i] = h_res[4 * i + 3];
  }
  return ILG_OK;
}
