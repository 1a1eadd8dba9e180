// Batched D1Q3 replicas: one persistent launch advances every ring of a batch by T
// steps.  Blocks pull replicas from a queue ordered by decreasing ring length
// (longest processing time first); a block copies its replica's ring and alias
// tables into shared memory, runs all T steps there (flip, collision, streaming,
// two buffers, one barrier per step) and writes the ring back.  Random numbers are
// keyed by the replica's own id, so a replica's result does not depend on which
// block ran it or on the other replicas of the batch.
#include <cuda_runtime.h>

#include "ilg_batch.h"
#include "ilg_device.cuh"

namespace ilg {

namespace {

// Compensated double-precision sum (Ogita, Rump & Oishi 2005), per thread and
// merged across the block.
__device__ __forceinline__ void two_sum_b(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <int THREADS>
__device__ double block_dot2(double s, double c, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double os = __shfl_down_sync(0xFFFFFFFFu, s, o);
    const double oc = __shfl_down_sync(0xFFFFFFFFu, c, o);
    double q;
    two_sum_b(s, os, s, q);
    c += oc + q;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[2 * warp] = s;
    red[2 * warp + 1] = c;
  }
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    double S = red[0], C = red[1];
    for (int w = 1; w < THREADS / 32; ++w) {
      double q;
      two_sum_b(S, red[2 * w], S, q);
      C += red[2 * w + 1] + q;
    }
    r = S + C;
  }
  return r;  // valid in thread 0
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) batch_d1q3_kernel(BatchArgs b, StepArgs common) {
  extern __shared__ uint4 smem4[];
  uint32_t* tables = reinterpret_cast<uint32_t*>(smem4);                     // kDevBlockWords words
  uint32_t* xbuf = tables + kDevBlockWords;                                   // kBatchExtWords x THREADS
  uint16_t* ring = reinterpret_cast<uint16_t*>(xbuf + kBatchExtWords * THREADS);  // 2 x 3 x Lmax
  __shared__ uint32_t s_task;
  __shared__ int s_fail;
  __shared__ unsigned long long s_mass;
  __shared__ double s_red[2 * (THREADS / 32)];
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) {
      s_task = atomicAdd(b.counter, 1u);
      s_fail = -1;
      s_mass = 0ull;
    }
    __syncthreads();
    const uint32_t task = s_task;
    if (task >= b.n) break;
    const uint32_t r = b.order[task];
    const ReplicaDesc d = b.desc[r];
    const uint32_t L = d.L;
    StepArgs a = common;
    a.Lx = L;
    a.Ly = 1;
    a.flip = d.flip;
    a.omega_mode = d.omega_mode;
    a.rest_mode = d.rest_mode;
    a.replica = d.replica;
    a.general = d.general;

    // tables and ring into shared memory
    const uint4* gt = reinterpret_cast<const uint4*>(b.tables + size_t(r) * kDevBlockWords);
    for (uint32_t i = tid; i < kDevBlockWords / 4; i += THREADS) smem4[i] = gt[i];
    const uint16_t* gs = b.state + d.state_off;
    uint16_t* buf0 = ring;
    uint16_t* buf1 = ring + 3 * b.Lmax;
    for (uint32_t i = tid; i < 3 * L; i += THREADS) buf0[(i / L) * b.Lmax + (i % L)] = gs[i];
    __syncthreads();

    // mass and mode phases for the amplitude record (integers, exact)
    uint64_t mass = 0;
    const bool rec = b.record != nullptr;
    const uint32_t mrec = rec ? uint32_t(((int64_t(b.record_mode) % int64_t(L)) + L) % L) : 0u;
    if (rec) {
      unsigned long long part = 0;
      for (uint32_t x = tid; x < L; x += THREADS)
        part += (unsigned long long)buf0[x] + buf0[b.Lmax + x] + buf0[2 * b.Lmax + x];
      if (part) atomicAdd(&s_mass, part);
      __syncthreads();
      mass = s_mass;
    }

    uint16_t* src = buf0;
    uint16_t* dst = buf1;
    uint32_t steps_done = 0;
    for (uint32_t s = 0; s < b.T; ++s) {
      const uint32_t t = d.t + s;
      bool bad = false;
      for (uint32_t x = tid; x < L; x += THREADS) {
        const uint32_t n[3] = {src[x], src[b.Lmax + x], src[2 * b.Lmax + x]};
        uint32_t m[3], post[3];
        m[0] = n[0];
        m[1] = a.flip ? n[2] : n[1];
        m[2] = a.flip ? n[1] : n[2];
        if (a.general || !collide_try_fast<3>(a, tables, x, t, m, post)) {
          collide_phased<3, kBatchExtWords, THREADS>(a, tables, x, t, m, post, xbuf + tid);
          bad |= post[0] > 65535u || post[1] > 65535u || post[2] > 65535u;
        }
        const uint32_t xp = x + 1 == L ? 0 : x + 1;
        const uint32_t xm = x == 0 ? L - 1 : x - 1;
        dst[x] = uint16_t(post[0]);
        dst[b.Lmax + xp] = uint16_t(post[1]);
        dst[2 * b.Lmax + xm] = uint16_t(post[2]);
      }
      if (bad) atomicMax(&s_fail, 0);
      __syncthreads();
      if (s_fail >= 0) break;  // src still holds the state at step t: keep it
      uint16_t* tmp = src;
      src = dst;
      dst = tmp;
      steps_done = s + 1;
      if (rec) {
        // amplitude projection of the new state (t + 1): sum_x s(x) (L N(x) - M) / L
        double ps = 0.0, pc = 0.0;
        for (uint32_t x = tid; x < L; x += THREADS) {
          const long long N = (long long)src[x] + src[b.Lmax + x] + src[2 * b.Lmax + x];
          const long long D = (long long)L * N - (long long)mass;
          const uint32_t rr = uint32_t((uint64_t(mrec) * x) % L);
          double sn, cs;
          sincospi(2.0 * double(rr) / double(L), &sn, &cs);
          const double p = sn * double(D);
          const double pe = fma(sn, double(D), -p);
          double q;
          two_sum_b(ps, p, ps, q);
          pc += q + pe;
        }
        const double im = block_dot2<THREADS>(ps, pc, s_red) / double(L);
        if (tid == 0) b.record[size_t(r) * b.T + s] = im / (double(L) / 2.0);
        __syncthreads();
      }
    }
    // ring back to global memory; the replica's step counter moves on
    uint16_t* gd = b.state + d.state_off;
    for (uint32_t i = tid; i < 3 * L; i += THREADS) gd[i] = src[(i / L) * b.Lmax + (i % L)];
    if (tid == 0) {
      b.desc[r].t = d.t + steps_done;
      if (s_fail >= 0) b.failed[r] = 1u;
    }
    __syncthreads();
  }
}

}  // namespace

constexpr int kBatchThreads = 1024;

size_t batch_smem_bytes(uint32_t Lmax) {
  return sizeof(uint32_t) * (kDevBlockWords + size_t(kBatchExtWords) * kBatchThreads) +
         sizeof(uint16_t) * 2 * 3 * size_t(Lmax);
}

cudaError_t prepare_batch_kernel(uint32_t Lmax) {
  return cudaFuncSetAttribute(batch_d1q3_kernel<kBatchThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(batch_smem_bytes(Lmax)));
}

cudaError_t launch_batch(const BatchArgs& b, const StepArgs& common, int grid, cudaStream_t s) {
  batch_d1q3_kernel<kBatchThreads><<<grid, kBatchThreads, batch_smem_bytes(b.Lmax), s>>>(b, common);
  return cudaGetLastError();
}

}  // namespace ilg

namespace ilg {
namespace {

// Per replica: mass and the amplitude A^LG of one mode (one block per replica).
__global__ void __launch_bounds__(256) batch_obs_kernel(const ReplicaDesc* __restrict__ desc,
                                                        const uint16_t* __restrict__ state, int32_t mode,
                                                        unsigned long long* __restrict__ mass_out,
                                                        double* __restrict__ amp_out) {
  __shared__ unsigned long long s_mass;
  __shared__ double s_red[2 * 8];
  const ReplicaDesc d = desc[blockIdx.x];
  const uint32_t L = d.L;
  const uint16_t* s = state + d.state_off;
  if (threadIdx.x == 0) s_mass = 0ull;
  __syncthreads();
  unsigned long long part = 0;
  for (uint32_t x = threadIdx.x; x < L; x += blockDim.x) part += (unsigned long long)s[x] + s[L + x] + s[2 * L + x];
  if (part) atomicAdd(&s_mass, part);
  __syncthreads();
  const long long M = (long long)s_mass;
  const uint32_t m = uint32_t(((int64_t(mode) % int64_t(L)) + L) % L);
  double ps = 0.0, pc = 0.0;
  for (uint32_t x = threadIdx.x; x < L; x += blockDim.x) {
    const long long N = (long long)s[x] + s[L + x] + s[2 * L + x];
    const long long D = (long long)L * N - M;
    const uint32_t rr = uint32_t((uint64_t(m) * x) % L);
    double sn, cs;
    sincospi(2.0 * double(rr) / double(L), &sn, &cs);
    const double p = sn * double(D);
    const double pe = fma(sn, double(D), -p);
    double q;
    two_sum_b(ps, p, ps, q);
    pc += q + pe;
  }
  const double im = block_dot2<256>(ps, pc, s_red) / double(L);
  if (threadIdx.x == 0) {
    mass_out[blockIdx.x] = (unsigned long long)M;
    amp_out[blockIdx.x] = im / (double(L) / 2.0);
  }
}

}  // namespace

cudaError_t launch_batch_obs(const ReplicaDesc* desc, const uint16_t* state, uint32_t n, int32_t mode,
                             unsigned long long* mass, double* amp, cudaStream_t s) {
  batch_obs_kernel<<<n, 256, 0, s>>>(desc, state, mode, mass, amp);
  return cudaGetLastError();
}

}  // namespace ilg
