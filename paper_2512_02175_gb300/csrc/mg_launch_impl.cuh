// mg_launch_impl.cuh -- host-side launch helpers of the fused EM-Step kernels
// for one kernel mode (a precision mode, plus kVarSigma for graphs with
// position-dependent diffusion); included by the units that instantiate them.
#pragma once
#include "mg_em_step.cuh"
#include "mg_launch.h"

namespace mg {

template <int kMode>
void set_smem_attributes_t() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(em_step_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(em_range_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(em_batch_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    done = true;
  }
}

// a.range > kBlock: the range kernel; else the tile kernel, a.range
// particles per block
template <int kMode>
cudaError_t launch_step_t(const SimArgs& a, const Keys& k, size_t smem, cudaStream_t st) {
  set_smem_attributes_t<kMode>();
  const int64_t grid = (a.n + a.range - 1) / a.range;
  if (a.range > kBlock) em_range_kernel<kMode><<<(unsigned)grid, kBlock, smem, st>>>(a, k);
  else em_step_kernel<kMode><<<(unsigned)grid, kBlock, smem, st>>>(a, k);
  return cudaGetLastError();
}

template <int kMode>
int step_blocks_per_sm_t(size_t smem) {
  set_smem_attributes_t<kMode>();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, em_step_kernel<kMode>, kBlock, smem);
  return nb;
}

template <int kMode>
int range_blocks_per_sm_t(size_t smem) {
  set_smem_attributes_t<kMode>();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, em_range_kernel<kMode>, kBlock, smem);
  return nb;
}

template <int kMode>
cudaError_t launch_batch_t(const SimArgs* insts, const BatchItem* items, int32_t n_items,
                           uint32_t* head, const Keys& k, size_t smem, int blocks,
                           cudaStream_t st) {
  set_smem_attributes_t<kMode>();
  em_batch_kernel<kMode><<<blocks, kBlock, smem, st>>>(insts, items, n_items, head, k);
  return cudaGetLastError();
}

template <int kMode>
int batch_blocks_per_sm_t(size_t smem) {
  set_smem_attributes_t<kMode>();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, em_batch_kernel<kMode>, kBlock, smem);
  return nb;
}

}  // namespace mg
