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

// Exact 128-bit integer accumulator of products of int64 values.
struct I128 {
  unsigned long long lo = 0;
  long long hi = 0;
  __device__ __forceinline__ void add(unsigned long long l, long long h) {
    const unsigned long long n = lo + l;
    hi += h + (n < lo ? 1 : 0);
    lo = n;
  }
  __device__ __forceinline__ void add_product(long long a, long long b) {
    add((unsigned long long)(a * b), __mul64hi(a, b));
  }
};

// v * 2^-62 rounded once to double (round to nearest even).
__device__ double i128_to_double_2m62(I128 v) {
  const bool neg = v.hi < 0;
  unsigned long long lo = v.lo, hi = (unsigned long long)v.hi;
  if (neg) {  // two's complement negation
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0 ? 1ull : 0ull);
  }
  double mag;
  if (hi == 0) {
    mag = __ull2double_rn(lo);
  } else {
    // keep the top 64 bits, fold the rest into a sticky bit: one correct rounding
    const int k = 64 - __clzll((long long)hi);  // significant bits of hi, 1..64
    unsigned long long m = k == 64 ? hi : ((hi << (64 - k)) | (lo >> k));
    const unsigned long long dropped = k == 64 ? lo : (lo << (64 - k));
    if (dropped) m |= 1ull;
    mag = ldexp(__ull2double_rn(m), k);
  }
  const double r = ldexp(mag, -62);
  return neg ? -r : r;
}

// Fixed-point (2^-62) cosine and sine of 2 pi r / L.
__device__ __forceinline__ longlong2 trig_fixed(uint32_t r, uint32_t L) {
  double sn, cs;
  sincospi(2.0 * double(r) / double(L), &sn, &cs);
  return make_longlong2(__double2ll_rn(ldexp(cs, 62)), __double2ll_rn(ldexp(sn, 62)));
}

// Complex amplitude of axis mode m of a ring held in shared memory (buf, planes
// Lmax apart): with D(x) = L N(x) - M and r = (m x) mod L,
//   re = sum_x cos(2 pi r / L) D(x) / L,  im = sum_x sin(2 pi r / L) D(x) / L.
// The trigonometric values enter as 2^-62 fixed-point integers (from trig, indexed
// by x, when given) and the sums are exact in 128-bit integers, so they do not
// depend on the summation order.  ring_partials: every warp reduces its nodes and
// its lane 0 stores (re.lo, re.hi, im.lo, im.hi) at red[4 warp ..]; no barrier.
template <int THREADS>
__device__ void ring_partials(const uint16_t* buf, uint32_t L, uint32_t Lmax, uint64_t mass, uint32_t m,
                              const longlong2* trig, unsigned long long* red) {
  I128 ac, as;
  for (uint32_t x = threadIdx.x; x < L; x += THREADS) {
    const long long N = (long long)buf[x] + buf[Lmax + x] + buf[2 * Lmax + x];
    const long long D = (long long)L * N - (long long)mass;
    const longlong2 cs = trig ? trig[x] : trig_fixed(uint32_t((uint64_t(m) * x) % L), L);
    ac.add_product(cs.x, D);
    as.add_product(cs.y, D);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long cl = __shfl_down_sync(0xFFFFFFFFu, ac.lo, o);
    const long long ch = __shfl_down_sync(0xFFFFFFFFu, ac.hi, o);
    const unsigned long long sl = __shfl_down_sync(0xFFFFFFFFu, as.lo, o);
    const long long sh = __shfl_down_sync(0xFFFFFFFFu, as.hi, o);
    ac.add(cl, ch);
    as.add(sl, sh);
  }
  if ((threadIdx.x & 31) == 0) {
    const int w = threadIdx.x >> 5;
    red[4 * w + 0] = ac.lo;
    red[4 * w + 1] = (unsigned long long)ac.hi;
    red[4 * w + 2] = as.lo;
    red[4 * w + 3] = (unsigned long long)as.hi;
  }
}

// Sum of the warps' partials (one thread): the raw 128-bit sums of re and im
// (times L 2^62) go to out[0..3].
template <int THREADS>
__device__ void ring_finalise(const unsigned long long* red, long long* out) {
  I128 c, s;
  for (int w = 0; w < THREADS / 32; ++w) {
    c.add(red[4 * w + 0], (long long)red[4 * w + 1]);
    s.add(red[4 * w + 2], (long long)red[4 * w + 3]);
  }
  out[0] = (long long)c.lo;
  out[1] = c.hi;
  out[2] = (long long)s.lo;
  out[3] = s.hi;
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) batch_d1q3_kernel(BatchArgs b, StepArgs common) {
  extern __shared__ uint4 smem4[];
  uint32_t* tables = reinterpret_cast<uint32_t*>(smem4);                     // kBatchTableWords words
  uint32_t* xbuf = tables + kBatchTableWords;                                 // kBatchExtWords x THREADS
  uint16_t* ring = reinterpret_cast<uint16_t*>(xbuf + kBatchExtWords * THREADS);  // 2 x 3 x Lmax
  __shared__ uint32_t s_task;
  __shared__ int s_fail;
  __shared__ unsigned long long s_mass;
  __shared__ unsigned long long s_red[2][4 * (THREADS / 32)];   // projection partials, by state parity
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
    a.particle = d.particle;

    // tables (the two alias tables packed one word per column; the particle
    // sampler's boundaries as they are) and ring into shared memory
    stage_tables4(b.tables + size_t(r) * kDevBlockWords, tables, a.particle != 0);
    const uint16_t* gs = b.state + d.state_off;
    uint16_t* buf0 = ring;
    uint16_t* buf1 = ring + 3 * b.Lmax;
    for (uint32_t i = tid; i < 3 * L; i += THREADS) buf0[(i / L) * b.Lmax + (i % L)] = gs[i];
    __syncthreads();

    // mass and mode phases for the amplitude record (integers, exact)
    uint64_t mass = 0;
    const bool rec = b.record != nullptr;
    const uint32_t mrec = rec ? uint32_t(((int64_t(b.record_mode) % int64_t(L)) + L) % L) : 0u;
    const longlong2* trig = b.trig ? b.trig + d.state_off / 3 : nullptr;  // this ring's values
    if (rec) {
      unsigned long long part = 0;
      for (uint32_t x = tid; x < L; x += THREADS)
        part += (unsigned long long)buf0[x] + buf0[b.Lmax + x] + buf0[2 * b.Lmax + x];
      if (part) atomicAdd(&s_mass, part);
      __syncthreads();
      mass = s_mass;
      // partials of state 0 into slot 0 (finalised after the first step's barrier)
      ring_partials<THREADS>(buf0, L, b.Lmax, mass, mrec, trig, s_red[0]);
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
        if (a.general || !collide_try_fast<3, Alias4>(a, tables, x, t, m, post)) {
          collide_general<3, kBatchExtWords, THREADS, Alias4>(a, tables, x, t, m, post, xbuf + tid);
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
      if (b.states) {
        // the state after this step, planes rest, +1, -1 as the batch buffer holds them
        uint16_t* rs = b.states + d.state_off * b.T + size_t(s) * 3 * L;
        for (uint32_t i = tid; i < 3 * L; i += THREADS) {
          const uint32_t pl = i >= 2 * L ? 2u : (i >= L ? 1u : 0u);
          rs[i] = src[pl * b.Lmax + (i - pl * L)];
        }
      }
      if (rec) {
        // state s was reduced into slot s & 1 before this step's barrier: finalise
        // it; then the warps reduce the new state s + 1 into the other slot
        if (tid == 0) ring_finalise<THREADS>(s_red[s & 1], b.record + (size_t(r) * (b.T + 1) + s) * 4);
        ring_partials<THREADS>(src, L, b.Lmax, mass, mrec, trig, s_red[(s + 1) & 1]);
      }
    }
    if (rec && s_fail < 0) {
      __syncthreads();
      if (tid == 0) ring_finalise<THREADS>(s_red[b.T & 1], b.record + (size_t(r) * (b.T + 1) + b.T) * 4);
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

// Default shape: batches whose rings all have at most kBatchSmallL nodes run on
// 256-thread blocks, several per SM; others on 1024-thread blocks, or 512 where the
// longest ring does not fit beside 1024 threads' buffers.  The autotuner
// (ilg_batch_autotune) may pick 256, 512 or 1024 threads instead.
constexpr int kBatchThreads = 1024;
constexpr int kBatchSmallThreads = 256;
constexpr uint32_t kBatchSmallL = 1024;

size_t batch_smem_bytes(uint32_t Lmax, int threads) {
  return sizeof(uint32_t) * (kBatchTableWords + size_t(kBatchExtWords) * threads) +
         sizeof(uint16_t) * 2 * 3 * size_t(Lmax);
}

// largest dynamic shared memory a shape may ask for (the 227 KB a block may opt into,
// less room for the kernel's static shared memory)
constexpr size_t kBatchSmemCap = 223 * 1024;

bool batch_shape_fits(uint32_t Lmax, int threads) { return batch_smem_bytes(Lmax, threads) <= kBatchSmemCap; }

uint32_t batch_default_threads(uint32_t Lmax) {
  if (Lmax <= kBatchSmallL) return kBatchSmallThreads;
  return batch_shape_fits(Lmax, kBatchThreads) ? kBatchThreads : kBatchThreads / 2;
}

template <int THREADS>
static cudaError_t batch_attr(uint32_t Lmax) {
  return cudaFuncSetAttribute(batch_d1q3_kernel<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(batch_smem_bytes(Lmax, THREADS)));
}

cudaError_t prepare_batch_kernel(uint32_t Lmax, int threads) {
  if (!batch_shape_fits(Lmax, threads)) return cudaErrorInvalidValue;
  if (threads == 256) return batch_attr<256>(Lmax);
  if (threads == 512) return batch_attr<512>(Lmax);
  if (threads == 1024) return batch_attr<1024>(Lmax);
  return cudaErrorInvalidValue;
}

// Persistent grid: as many blocks as fit on every SM (shared memory and registers
// decide), at most one per ring.
template <int THREADS>
static cudaError_t launch_shape(const BatchArgs& b, const StepArgs& common, int sms, cudaStream_t s) {
  const size_t smem = batch_smem_bytes(b.Lmax, THREADS);
  int per_sm = 1;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_d1q3_kernel<THREADS>, THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint32_t cap = uint32_t(per_sm) * uint32_t(sms);
  const int grid = int(b.n < cap ? b.n : cap);
  batch_d1q3_kernel<THREADS><<<grid, THREADS, smem, s>>>(b, common);
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs& b, const StepArgs& common, int sms, cudaStream_t s, int threads) {
  if (threads == 0) threads = int(batch_default_threads(b.Lmax));
  if (threads == 256) return launch_shape<256>(b, common, sms, s);
  if (threads == 512) return launch_shape<512>(b, common, sms, s);
  return launch_shape<1024>(b, common, sms, s);
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

// ring r's trig[state_off_r / 3 + x] = fixed-point (cos, sin) of 2 pi ((m_r x) mod L_r) / L_r,
// m_r the mode reduced modulo L_r: the values ring_partials would compute per node
__global__ void batch_trig_rings_kernel(const ReplicaDesc* __restrict__ desc, uint32_t n, int32_t mode,
                                        longlong2* __restrict__ trig) {
  for (uint32_t r = blockIdx.x; r < n; r += gridDim.x) {
    const uint32_t L = desc[r].L;
    const uint32_t m = uint32_t(((int64_t(mode) % int64_t(L)) + L) % L);
    longlong2* out = trig + desc[r].state_off / 3;
    for (uint32_t x = threadIdx.x; x < L; x += blockDim.x) out[x] = trig_fixed(uint32_t((uint64_t(m) * x) % L), L);
  }
}

// Raw 128-bit sums (L 2^62 re, L 2^62 im) -> (re, im) in double, rounded once and
// divided by L.
__global__ void batch_convert_kernel(const ReplicaDesc* __restrict__ desc, const long long* __restrict__ raw,
                                     uint32_t n, uint32_t T, double* __restrict__ rec) {
  const size_t total = size_t(n) * (T + 1);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
    const double L = double(desc[i / (T + 1)].L);
    const long long* v = raw + 4 * i;
    I128 re, im;
    re.lo = (unsigned long long)v[0];
    re.hi = v[1];
    im.lo = (unsigned long long)v[2];
    im.hi = v[3];
    rec[2 * i] = i128_to_double_2m62(re) / L;
    rec[2 * i + 1] = i128_to_double_2m62(im) / L;
  }
}

// amp[r T + s] = im / (L_r / 2) of the record entry after step s.
__global__ void batch_amp_kernel(const ReplicaDesc* __restrict__ desc, const double* __restrict__ record,
                                 uint32_t n, uint32_t T, double* __restrict__ amp) {
  const size_t total = size_t(n) * T;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
    const size_t r = i / T, s = i - r * T;
    amp[i] = record[(r * (T + 1) + s + 1) * 2 + 1] / (double(desc[r].L) / 2.0);
  }
}

// Ensemble statistics over the n rings of the record, one block per time index t:
// means of re and im, sample variances (divisor n - 1) and the connected
// correlation with t = 0 of a = re + i im:  cov = sum (a(t) - <a(t)>) conj(a(0) - <a(0)>) / (n - 1).
// Fixed-order sums (deterministic); two passes (means, then deviations).
__global__ void __launch_bounds__(256) batch_ensemble_kernel(const double* __restrict__ record, uint32_t n,
                                                             uint32_t T, double* __restrict__ out) {
  __shared__ double red[4][256];
  const uint32_t t = blockIdx.x;
  const size_t stride = size_t(T + 1) * 2;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double* o = record + r * stride;
    v[0] += o[2 * t];
    v[1] += o[2 * t + 1];
    v[2] += o[0];
    v[3] += o[1];
  }
  auto reduce4 = [&](double (&w)[4]) {
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = w[k];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (int(threadIdx.x) < h)
        for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
      __syncthreads();
    }
    for (int k = 0; k < 4; ++k) w[k] = red[k][0];
    __syncthreads();
  };
  reduce4(v);
  const double mre = v[0] / n, mim = v[1] / n, m0re = v[2] / n, m0im = v[3] / n;
  double w[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double* o = record + r * stride;
    const double dre = o[2 * t] - mre, dim = o[2 * t + 1] - mim;
    const double d0re = o[0] - m0re, d0im = o[1] - m0im;
    w[0] += dre * dre;
    w[1] += dim * dim;
    w[2] += dre * d0re + dim * d0im;
    w[3] += dim * d0re - dre * d0im;
  }
  reduce4(w);
  if (threadIdx.x == 0) {
    const size_t P = T + 1;
    const double dn = double(n) - 1.0;
    out[0 * P + t] = mre;
    out[1 * P + t] = mim;
    out[2 * P + t] = w[0] / dn;
    out[3 * P + t] = w[1] / dn;
    out[4 * P + t] = w[2] / dn;
    out[5 * P + t] = w[3] / dn;
  }
}

}  // namespace

cudaError_t launch_batch_obs(const ReplicaDesc* desc, const uint16_t* state, uint32_t n, int32_t mode,
                             unsigned long long* mass, double* amp, cudaStream_t s) {
  batch_obs_kernel<<<n, 256, 0, s>>>(desc, state, mode, mass, amp);
  return cudaGetLastError();
}

cudaError_t launch_batch_amp(const ReplicaDesc* desc, const double* record, uint32_t n, uint32_t T, double* amp,
                             cudaStream_t s) {
  const size_t total = size_t(n) * T;
  const int grid = int(total / 256 + 1 < 4096 ? total / 256 + 1 : 4096);
  batch_amp_kernel<<<grid, 256, 0, s>>>(desc, record, n, T, amp);
  return cudaGetLastError();
}

cudaError_t launch_batch_convert(const ReplicaDesc* desc, const long long* raw, uint32_t n, uint32_t T, double* rec,
                                 cudaStream_t s) {
  const size_t total = size_t(n) * (T + 1);
  const int grid = int(total / 256 + 1 < 4096 ? total / 256 + 1 : 4096);
  batch_convert_kernel<<<grid, 256, 0, s>>>(desc, raw, n, T, rec);
  return cudaGetLastError();
}

cudaError_t launch_batch_trig_rings(const ReplicaDesc* desc, uint32_t n, int32_t mode, longlong2* trig, cudaStream_t s) {
  batch_trig_rings_kernel<<<n < 1024u ? n : 1024u, 256, 0, s>>>(desc, n, mode, trig);
  return cudaGetLastError();
}

cudaError_t launch_batch_ensemble(const double* record, uint32_t n, uint32_t T, double* out, cudaStream_t s) {
  batch_ensemble_kernel<<<T + 1, 256, 0, s>>>(record, n, T, out);
  return cudaGetLastError();
}

}  // namespace ilg
