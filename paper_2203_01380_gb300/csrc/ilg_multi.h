// Multi-lattice step used by the server: descriptors, work items, launcher.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ilg_device.cuh"

namespace ilg {

constexpr int kMultiThreads = 256;
constexpr uint32_t kItemNodes = 1024;  // nodes per work item (a run of consecutive nodes of one lattice)

struct LatDesc {
  uint32_t Lx, Ly;
  uint32_t t0;          // step counter at the start of the quantum
  uint32_t phase;       // 0: buf0 holds the state at t0, 1: buf1 does
  uint32_t replica;
  uint32_t flip, omega_mode, rest_mode;
  uint32_t steps;       // sub-steps this lattice takes in the round (it idles after)
  uint32_t general;     // 1: skip the fast path (high occupation or particle sampler)
  uint32_t particle;    // 1: particle sampler
  uint32_t pad;
  uint16_t* buf0;
  uint16_t* buf1;
  const uint32_t* tables;  // kDevBlockWords words
};

constexpr int kMultiBlocksPerSm = 4;   // resident blocks per SM (the kernel's launch bounds)

struct WorkItem {
  uint32_t lattice, node0, node1;  // nodes [node0, node1) of the lattice, row-major
};

struct MultiArgs {
  const LatDesc* lat;
  const WorkItem* items;
  uint32_t n_items;
  unsigned int* counter;  // one work-queue head per sub-step of the quantum, 0 at start
  uint32_t* fail;         // per lattice: first sub-step that would exceed 65535, ~0 if none
};

size_t multi_smem_bytes();
cudaError_t prepare_multi_kernel();
cudaError_t launch_multi_step(const MultiArgs& ma, const StepArgs& common, uint32_t sub, int grid, cudaStream_t s);

}  // namespace ilg
