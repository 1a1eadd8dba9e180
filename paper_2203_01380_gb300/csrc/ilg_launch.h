// Kernel launchers of libilg.so (implemented in ilg_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ilg_device.cuh"

namespace ilg {

struct InitArgs {
  uint32_t Lx, Ly;
  uint32_t axis;      // 0 no sine mode, 1 along x, 2 along y
  uint32_t mode;      // wave number reduced to [0, period)
  uint32_t period;    // Lx, Ly, or 1
  uint32_t weighted;  // 1: classes rest / moving (D2Q9: rest / axis / diagonal)
  uint32_t key0, key1, replica;
  const uint32_t* offset;  // [classes * period]
  const uint32_t* count;   // [classes * period]
  const uint32_t* table;
};

cudaError_t prepare_step_kernels();  // opt in to the table block's shared memory
uint32_t step_kernel_threads();       // block shape of the node-parallel step
uint32_t step_kernel_blocks_per_sm();
cudaError_t launch_step(int Q, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                        unsigned long long* fail, int grid, cudaStream_t s);
cudaError_t prepare_step_vec_kernels();
uint32_t step_vec_width();  // nodes per thread of the default row-tiled step (rows must be a multiple)
uint32_t step_vec_blocks_per_sm(int npt);
// npt: nodes per thread, 8 (default) or 4 (rows a multiple of npt)
cudaError_t launch_step_vec(int Q, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                            unsigned long long* fail, int grid, cudaStream_t s, int npt = 8);
// warp-segment form of the 8-node row-tiled step (segments of 8192 nodes of a row,
// one warp each): step_seg_units = the number of segments of a lattice
uint64_t step_seg_units(uint32_t Lx, uint32_t Ly);
cudaError_t launch_step_seg(int Q, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                            unsigned long long* fail, int grid, cudaStream_t s);
// warp segments of staged vectors (ilg_step_warp.cu): rows a multiple of the width,
// every probability drawn through its table; D1Q3 and D2Q5: shape 0 = 8 nodes per
// lane, one block of 384 threads per SM, shape 1 = 4 nodes per lane, 640 threads;
// D2Q9: 4 nodes per lane collided in shared memory, 512 (shape 0) or 640 (shape 1)
// threads; step_warp_grid =
// blocks of a launch
cudaError_t prepare_step_warp_kernels();
uint32_t step_warp_width(int Q, int shape);  // nodes per lane (rows must be a multiple)
uint32_t step_warp_grid(int Q, uint32_t Lx, uint32_t Ly, uint32_t sms, int shape);
cudaError_t launch_step_warp(int Q, int shape, const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t,
                             unsigned long long* fail, int grid, cudaStream_t s);
size_t step_tb_smem_bytes(uint32_t B, uint32_t Tb);
cudaError_t prepare_step_tb_kernel(uint32_t B, uint32_t Tb);
cudaError_t launch_step_tb(const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t0, uint32_t Tb,
                           uint32_t B, unsigned long long* fail, int grid, cudaStream_t s);
cudaError_t launch_init(int Q, const InitArgs& a, uint16_t* out, int grid, cudaStream_t s);
cudaError_t prepare_step9_kernel();  // D2Q9 (ilg_d2q9.cu)
uint32_t step9_threads();
uint32_t step9_blocks_per_sm();
cudaError_t launch_step9(const StepArgs& a, const uint16_t* in, uint16_t* out, uint32_t t, unsigned long long* fail,
                         int grid, cudaStream_t s);
cudaError_t launch_sums(int Q, const uint16_t* in, uint32_t Lx, uint32_t Ly, unsigned long long* col,
                        unsigned long long* row, int want_rows, cudaStream_t s);
cudaError_t launch_project(const unsigned long long* col, const unsigned long long* row, uint32_t Lx,
                           uint32_t Ly, const int32_t* modes, uint32_t nmodes, double* res,
                           unsigned long long* mass, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, size_t n,
                          cudaStream_t s);

}  // namespace ilg
