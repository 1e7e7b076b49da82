// em_step_f64.cu -- binary64 instantiation of the fused EM-Step kernel and of
// the histogram kernel.  Built without floating-point contraction
// (--fmad=false) so that every binary64 operation rounds exactly as written,
// in the same order as the plain CPU reference of the scheme.
#include "mg_em_step.cuh"
#include "mg_histogram.cuh"
#include "mg_launch.h"

namespace mg {

static void set_smem_attributes() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(em_step_kernel<kModeF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(em_range_kernel<kModeF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(em_batch_kernel<kModeF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    done = true;
  }
}

cudaError_t launch_em_step_f64(const SimArgs& a, const Keys& k, size_t smem, cudaStream_t st) {
  set_smem_attributes();
  const int64_t grid = (a.n + a.range - 1) / a.range;
  if (a.range > kBlock) em_range_kernel<kModeF64><<<(unsigned)grid, kBlock, smem, st>>>(a, k);
  else em_step_kernel<kModeF64><<<(unsigned)grid, kBlock, smem, st>>>(a, k);
  return cudaGetLastError();
}

int em_step_blocks_per_sm_f64(size_t smem) {
  set_smem_attributes();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, em_step_kernel<kModeF64>, kBlock, smem);
  return nb;
}

int em_range_blocks_per_sm_f64(size_t smem) {
  set_smem_attributes();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, em_range_kernel<kModeF64>, kBlock, smem);
  return nb;
}

cudaError_t launch_em_batch_f64(const SimArgs* insts, const BatchItem* items, int32_t n_items,
                                uint32_t* head, const Keys& k, size_t smem, int blocks,
                                cudaStream_t st) {
  set_smem_attributes();
  em_batch_kernel<kModeF64><<<blocks, kBlock, smem, st>>>(insts, items, n_items, head, k);
  return cudaGetLastError();
}

int em_batch_blocks_per_sm_f64(size_t smem) {
  set_smem_attributes();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, em_batch_kernel<kModeF64>, kBlock, smem);
  return nb;
}

cudaError_t launch_histogram_f64(const GraphView& g, const int32_t* edge, const void* x, int64_t n,
                                 int32_t bins, uint32_t* out, bool smem, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + kBlock - 1) / kBlock;
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  if (grid < 1) grid = 1;
  const size_t sh = smem ? align16((size_t)g.E * bins * 4) : 0;
  if (sh > 48 * 1024)
    cudaFuncSetAttribute(histogram_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sh);
  histogram_kernel<double><<<(unsigned)grid, kBlock, sh, st>>>(g, edge, x, n, bins, out, smem ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_histogram_binned_f64(const int32_t* edge, const void* x, int64_t n,
                                        const int32_t* off, const double* up, int32_t n_bins,
                                        uint32_t* out, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + kBlock - 1) / kBlock;
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  if (grid < 1) grid = 1;
  const bool smem = (size_t)n_bins * 4 <= 96 * 1024;
  const size_t sh = smem ? align16((size_t)n_bins * 4) : 0;
  if (sh > 48 * 1024)
    cudaFuncSetAttribute(histogram_binned_kernel<double>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  histogram_binned_kernel<double><<<(unsigned)grid, kBlock, sh, st>>>(edge, x, n, off, up, n_bins,
                                                                      out, smem ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace mg
