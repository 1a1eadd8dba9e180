// Kernels of the lattice-gas path: the fused flip + collision + streaming step,
// the Poisson initial state, the integer sums and the double-precision
// projections of the observables, and a Philox probe.
#include <cuda_runtime.h>

#include <type_traits>

#include "ilg_device.cuh"
#include "ilg_launch.h"

namespace ilg {

// --------------------------------------------------------------------------
// step: one thread per node, any extent.  Loads the Q occupations of its node,
// flips, collides and scatters n'_i to the neighbour x + v_i (periodic).
// The lattice's two alias tables (packed one word per column, or as {threshold,
// alias} pairs) are staged in shared memory once per block, beside 20 extension
// words per thread for the general collision.  A block returns without work when an
// earlier launch recorded an overflow.
// --------------------------------------------------------------------------
constexpr int kStepThreads = 256;
constexpr int kStepBlocksPerSm = 4;
// packed tables (32 KB, one word per column) leave room for four blocks per SM; the
// pair form (64 KB) saves two instructions per draw
constexpr bool kStepPairTables = false;
using StepTab = std::conditional_t<kStepPairTables, Alias8, Alias4>;
constexpr uint32_t kStepTableWords = kStepPairTables ? kDevStagedWords : kDevTableWords4;

template <int Q>
__global__ void __launch_bounds__(kStepThreads, kStepBlocksPerSm) step_kernel(StepArgs a, const uint16_t* __restrict__ in,
                                                      uint16_t* __restrict__ out, uint32_t t,
                                                      unsigned long long* __restrict__ fail) {
  extern __shared__ uint4 smem4[];
  __shared__ int skip;
  uint32_t* s = reinterpret_cast<uint32_t*>(smem4);
  uint32_t* xb = s + kStepTableWords + threadIdx.x;  // this thread's extension words
  if (threadIdx.x == 0) skip = (*reinterpret_cast<volatile unsigned long long*>(fail) != ~0ull);
  if constexpr (kStepPairTables) {
    // the block's first words: the pair tables, or the particle sampler's boundaries
    const uint4* g4 = reinterpret_cast<const uint4*>(a.tables);
    for (uint32_t i = threadIdx.x; i < kDevStagedWords / 4; i += blockDim.x) smem4[i] = g4[i];
  } else {
    stage_tables4(a.tables, s, a.particle != 0);
  }
  __syncthreads();
  if (skip) return;

  const uint32_t nodes = a.Lx * a.Ly;
  const size_t plane = nodes;
  bool bad = false;
  // (x, y) of the node, advanced by the grid stride (stride_y rows and stride_x
  // nodes) with a carry instead of a division per node
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t stride_y = stride / a.Lx, stride_x = stride - stride_y * a.Lx;
  uint32_t node = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t y = node / a.Lx, x = node - y * a.Lx;
  const StepKeys<2> keys = step_keys<2>(a, t);  // the launch-wide Philox rounds of the slot blocks
  for (; node < nodes; node += stride) {
    uint32_t n[Q], m[Q], post[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] = in[i * plane + node];
    if constexpr (Q == 3) {
      m[0] = n[0];
      m[1] = a.flip ? n[2] : n[1];
      m[2] = a.flip ? n[1] : n[2];
    } else {
      m[0] = n[0];
      m[1] = a.flip ? n[2] : n[1];
      m[2] = a.flip ? n[1] : n[2];
      m[3] = a.flip ? n[4] : n[3];
      m[4] = a.flip ? n[3] : n[4];
    }
    if (a.general || !collide_try_fast<Q, StepTab>(a, s, node, t, m, post, &keys)) {
      collide_general<Q, kExtWords, kStepThreads, StepTab, true>(a, s, node, t, m, post, xb, &keys);
#pragma unroll
      for (int i = 0; i < Q; ++i) bad |= post[i] > 65535u;
    }
    const uint32_t xp = x + 1 == a.Lx ? 0 : x + 1;
    const uint32_t xm = x == 0 ? a.Lx - 1 : x - 1;
    const size_t row = size_t(y) * a.Lx;
    out[node] = uint16_t(post[0]);
    out[plane + row + xp] = uint16_t(post[1]);
    out[2 * plane + row + xm] = uint16_t(post[2]);
    if constexpr (Q == 5) {
      const uint32_t yp = y + 1 == a.Ly ? 0 : y + 1;
      const uint32_t ym = y == 0 ? a.Ly - 1 : y - 1;
      out[3 * plane + size_t(yp) * a.Lx + x] = uint16_t(post[3]);
      out[4 * plane + size_t(ym) * a.Lx + x] = uint16_t(post[4]);
    }
    x += stride_x;
    y += stride_y;
    if (x >= a.Lx) {
      x -= a.Lx;
      y += 1;
    }
  }
  if (bad) atomicMin(fail, static_cast<unsigned long long>(t));
}

constexpr size_t kStepSmem = sizeof(uint32_t) * (kStepTableWords + kExtWords * kStepThreads);

cudaError_t prepare_step_kernels() {
  cudaError_t e = cudaFuncSetAttribute(step_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStepSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(step_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStepSmem));
}

uint32_t step_kernel_threads() { return kStepThreads; }
uint32_t step_kernel_blocks_per_sm() { return kStepBlocksPerSm; }

cudaError_t launch_step(int Q, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                        unsigned long long* fail, int grid, cudaStream_t s) {
  if (Q == 3) step_kernel<3><<<grid, kStepThreads, kStepSmem, s>>>(a, in, out, t, fail);
  else step_kernel<5><<<grid, kStepThreads, kStepSmem, s>>>(a, in, out, t, fail);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// initial state: n_i = number of table entries T[j], j < K-1, with u >= T[j]
// (binary search), u = word i of the init stream of the node.
// --------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(256) init_kernel(InitArgs a, uint16_t* __restrict__ out) {
  const uint32_t nodes = a.Lx * a.Ly;
  const size_t plane = nodes;
  for (uint32_t node = blockIdx.x * blockDim.x + threadIdx.x; node < nodes;
       node += gridDim.x * blockDim.x) {
    const uint32_t y = node / a.Lx;
    const uint32_t x = node - y * a.Lx;
    uint32_t r = 0;
    if (a.axis == 1) r = uint32_t((uint64_t(a.mode) * x) % a.period);
    else if (a.axis == 2) r = uint32_t((uint64_t(a.mode) * y) % a.period);
    uint32_t W[(Q + 3) / 4 * 4];
#pragma unroll
    for (int b = 0; b < (Q + 3) / 4; ++b) {
      const uint4 w = philox(counter(node, 0u, a.replica, kDevTagInit | uint32_t(b)), a.key0, a.key1);
      W[4 * b] = w.x;
      W[4 * b + 1] = w.y;
      W[4 * b + 2] = w.z;
      W[4 * b + 3] = w.w;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      // weight class of the velocity: rest, moving (D2Q9: axis, diagonal)
      const uint32_t cls = !a.weighted || i == 0 ? 0u : (Q == 9 && i > 4 ? 2u : 1u);
      const uint32_t idx = cls * a.period + r;
      const uint32_t* T = a.table + a.offset[idx];
      const uint32_t K = a.count[idx];
      const uint32_t u = W[i];
      // first j in [0, K-1) with T[j] > u, i.e. the count of entries <= u
      uint32_t lo = 0, hi = K - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (u >= T[mid]) lo = mid + 1;
        else hi = mid;
      }
      out[i * plane + node] = uint16_t(lo);
    }
  }
}

cudaError_t launch_init(int Q, const InitArgs& a, uint16_t* out, int grid, cudaStream_t s) {
  if (Q == 3) init_kernel<3><<<grid, 256, 0, s>>>(a, out);
  else if (Q == 5) init_kernel<5><<<grid, 256, 0, s>>>(a, out);
  else init_kernel<9><<<grid, 256, 0, s>>>(a, out);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// integer sums: N(x,y) = sum_i n_i; column sums C(x) over a block of rows, one
// 64-bit atomic per column and block; row sums R(y) by warp shuffles, one
// atomic per warp and row.
// --------------------------------------------------------------------------
constexpr int kSumRows = 64;

template <int Q>
__global__ void __launch_bounds__(256) sums_kernel(const uint16_t* __restrict__ in, uint32_t Lx, uint32_t Ly,
                                                   unsigned long long* __restrict__ col,
                                                   unsigned long long* __restrict__ row, int want_rows) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y0 = blockIdx.y * kSumRows;
  const uint32_t y1 = min(Ly, y0 + kSumRows);
  const size_t plane = size_t(Lx) * Ly;
  uint64_t acc = 0;
  for (uint32_t y = y0; y < y1; ++y) {
    uint32_t N = 0;
    if (x < Lx) {
      const size_t at = size_t(y) * Lx + x;
#pragma unroll
      for (int i = 0; i < Q; ++i) N += in[i * plane + at];
    }
    acc += N;
    if (want_rows) {
      uint64_t v = N;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(row + y, static_cast<unsigned long long>(v));
    }
  }
  if (x < Lx && acc) atomicAdd(col + x, static_cast<unsigned long long>(acc));
}

cudaError_t launch_sums(int Q, const uint16_t* in, uint32_t Lx, uint32_t Ly, unsigned long long* col,
                        unsigned long long* row, int want_rows, cudaStream_t s) {
  dim3 grid((Lx + 255) / 256, (Ly + kSumRows - 1) / kSumRows);
  if (Q == 9) sums_kernel<9><<<grid, 256, 0, s>>>(in, Lx, Ly, col, row, want_rows);
  else if (Q == 3) sums_kernel<3><<<grid, 256, 0, s>>>(in, Lx, Ly, col, row, want_rows);
  else sums_kernel<5><<<grid, 256, 0, s>>>(in, Lx, Ly, col, row, want_rows);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// projections: one block per mode.  D(x) = L*S(x) - M in exact int64, then
// compensated dot products (Ogita, Rump & Oishi 2005: error-free TwoProduct by
// FMA, TwoSum) with cos and sin of 2 pi r / L, r = (m*x) mod L.
// --------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct Dot2 {
  double s, c;
  __device__ void add_product(double a, double b) {
    const double p = a * b;
    const double pe = fma(a, b, -p);
    double q;
    two_sum(s, p, s, q);
    c += q + pe;
  }
  __device__ void merge(const Dot2& o) {
    double q;
    two_sum(s, o.s, s, q);
    c += o.c + q;
  }
};

__global__ void __launch_bounds__(256) project_kernel(const unsigned long long* __restrict__ colsum,
                                                      const unsigned long long* __restrict__ rowsum,
                                                      uint32_t Lx, uint32_t Ly, const int32_t* __restrict__ modes,
                                                      double* __restrict__ res, unsigned long long* __restrict__ mass) {
  __shared__ long long sM[8];
  __shared__ double sv[4][8];
  const int mi = blockIdx.x;
  const int32_t mx = modes[2 * mi], my = modes[2 * mi + 1];
  const bool along_x = (my == 0);
  const unsigned long long* S = along_x ? colsum : rowsum;
  const uint32_t L = along_x ? Lx : Ly;
  const int64_t mraw = along_x ? mx : my;
  const uint64_t m = uint64_t(((mraw % int64_t(L)) + int64_t(L)) % int64_t(L));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  long long part = 0;
  for (uint32_t x = threadIdx.x; x < L; x += blockDim.x) part += static_cast<long long>(S[x]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, o);
  if (lane == 0) sM[warp] = part;
  __syncthreads();
  long long M = 0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) M += sM[w];

  Dot2 re{0.0, 0.0}, im{0.0, 0.0};
  for (uint32_t x = threadIdx.x; x < L; x += blockDim.x) {
    const long long D = static_cast<long long>(L) * static_cast<long long>(S[x]) - M;
    const uint32_t r = uint32_t((m * x) % L);
    double sn, cs;
    sincospi(2.0 * double(r) / double(L), &sn, &cs);
    re.add_product(cs, double(D));
    im.add_product(sn, double(D));
  }
  // tree over the block: warp shuffles, then the warps' partial pairs
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Dot2 ore{__shfl_down_sync(0xFFFFFFFFu, re.s, o), __shfl_down_sync(0xFFFFFFFFu, re.c, o)};
    Dot2 oim{__shfl_down_sync(0xFFFFFFFFu, im.s, o), __shfl_down_sync(0xFFFFFFFFu, im.c, o)};
    re.merge(ore);
    im.merge(oim);
  }
  if (lane == 0) {
    sv[0][warp] = re.s; sv[1][warp] = re.c; sv[2][warp] = im.s; sv[3][warp] = im.c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Dot2 R{sv[0][0], sv[1][0]}, I{sv[2][0], sv[3][0]};
    for (int w = 1; w < int(blockDim.x >> 5); ++w) {
      R.merge(Dot2{sv[0][w], sv[1][w]});
      I.merge(Dot2{sv[2][w], sv[3][w]});
    }
    const double vre = (R.s + R.c) / double(L);
    const double vim = (I.s + I.c) / double(L);
    const double K = double(Lx) * double(Ly);
    res[4 * mi + 0] = vre;
    res[4 * mi + 1] = vim;
    res[4 * mi + 2] = vim / (K / 2.0);
    res[4 * mi + 3] = (vre * vre + vim * vim) / K;
    if (mi == 0) *mass = static_cast<unsigned long long>(M);
  }
}

// mass alone (no modes requested)
__global__ void mass_kernel(const unsigned long long* __restrict__ colsum, uint32_t Lx,
                            unsigned long long* __restrict__ mass) {
  __shared__ unsigned long long sM[8];
  unsigned long long part = 0;
  for (uint32_t x = threadIdx.x; x < Lx; x += blockDim.x) part += colsum[x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xFFFFFFFFu, part, o);
  if ((threadIdx.x & 31) == 0) sM[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long M = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) M += sM[w];
    *mass = M;
  }
}

cudaError_t launch_project(const unsigned long long* col, const unsigned long long* row, uint32_t Lx,
                           uint32_t Ly, const int32_t* modes, uint32_t nmodes, double* res,
                           unsigned long long* mass, cudaStream_t s) {
  if (nmodes == 0) mass_kernel<<<1, 256, 0, s>>>(col, Lx, mass);
  else project_kernel<<<nmodes, 256, 0, s>>>(col, row, Lx, Ly, modes, res, mass);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Philox probe
// --------------------------------------------------------------------------
__global__ void philox_kernel(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, uint4* __restrict__ out,
                              size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = philox(ctr[i], k0, k1);
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, size_t n,
                          cudaStream_t s) {
  const int grid = int(n < 65536 * 256 ? (n + 255) / 256 : 65536);
  philox_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), k0, k1,
                                                     reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

}  // namespace ilg
