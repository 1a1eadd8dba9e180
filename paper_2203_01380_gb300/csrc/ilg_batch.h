// Batched D1Q3 replicas: device descriptors and the persistent kernel's launcher.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ilg_device.cuh"

namespace ilg {

constexpr uint32_t kBatchMaxL = 10240;  // longest ring (the ring and its copy live in shared memory)
constexpr int kBatchExtWords = 16;      // extension words per thread in shared memory
// the ring's alias tables in shared memory, one word per column (Alias4)
constexpr uint32_t kBatchTableWords = kDevTableWords4;

struct ReplicaDesc {
  uint32_t L;           // ring length
  uint32_t flip;
  uint32_t omega_mode;  // kNever / kTable / kAlways
  uint32_t rest_mode;
  uint32_t replica;     // replica word of the Philox counter
  uint32_t t;           // step counter (advanced by the kernel)
  uint32_t general;     // 1: skip the fast path (high occupation or particle sampler)
  uint32_t particle;    // 1: particle sampler
  uint64_t state_off;   // first of the replica's 3 L occupations in the batch buffer
};

struct BatchArgs {
  uint32_t n;              // replicas
  uint32_t T;              // steps per launch
  uint32_t Lmax;           // longest ring
  int32_t record_mode;     // wave number of the recorded amplitude (record != NULL)
  const uint32_t* order;   // replica ids, longest first
  ReplicaDesc* desc;
  const uint32_t* tables;  // kDevBlockWords words per replica
  uint16_t* state;
  unsigned int* counter;   // work queue head, 0 at launch
  uint32_t* failed;        // per replica: 1 when a step would exceed 65535
  long long* record;       // n x (T + 1) x 4: exact sums (L 2^62 re, L 2^62 im) as 128-bit
                           // (lo, hi) pairs of the recorded mode at the launch's start, then
                           // after every step; or NULL
  const longlong2* trig;   // fixed-point (cos, sin) of the recorded mode, ring r's values at
                           // x + state_off / 3 (its nodes' place in the batch); or NULL
                           // (computed per node and step)
  uint16_t* states;        // state of every ring after every step, or NULL: ring r's
                           // T x 3 L_r occupations at T * state_off, step s at s * 3 L_r
};

size_t batch_smem_bytes(uint32_t Lmax, int threads);
bool batch_shape_fits(uint32_t Lmax, int threads);
// block shapes: 256, 512 or 1024 threads (ceil(L / threads) nodes per thread and step)
uint32_t batch_default_threads(uint32_t Lmax);
cudaError_t prepare_batch_kernel(uint32_t Lmax, int threads);
// threads 0: the default shape for Lmax
cudaError_t launch_batch(const BatchArgs& b, const StepArgs& common, int sms, cudaStream_t s, int threads = 0);
cudaError_t launch_batch_obs(const ReplicaDesc* desc, const uint16_t* state, uint32_t n, int32_t mode,
                             unsigned long long* mass, double* amp, cudaStream_t s);
cudaError_t launch_batch_amp(const ReplicaDesc* desc, const double* record, uint32_t n, uint32_t T, double* amp,
                             cudaStream_t s);
cudaError_t launch_batch_convert(const ReplicaDesc* desc, const long long* raw, uint32_t n, uint32_t T, double* rec,
                                 cudaStream_t s);
// every ring's table of the recorded mode at its nodes' place in the batch (desc on the
// device, n rings)
cudaError_t launch_batch_trig_rings(const ReplicaDesc* desc, uint32_t n, int32_t mode, longlong2* trig, cudaStream_t s);
cudaError_t launch_batch_ensemble(const double* record, uint32_t n, uint32_t T, double* out, cudaStream_t s);

}  // namespace ilg
