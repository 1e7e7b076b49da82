// em_step_f64.cu -- binary64 instantiations of the fused EM-Step kernels
// (constant and position-dependent diffusion) and of the histogram kernels.  Built without floating-point contraction
// (--fmad=false) so that every binary64 operation rounds exactly as written,
// in the same order as the plain CPU reference of the scheme.
#include "mg_em_step.cuh"
#include "mg_histogram.cuh"
#include "mg_launch.h"
#include "mg_launch_impl.cuh"

namespace mg {

// Modes of this unit: binary64 with constant or position-dependent
// (kVarSigma) diffusion.
constexpr int kF64Var = kModeF64 | kVarSigma;

cudaError_t launch_em_step_f64(int mode, const SimArgs& a, const Keys& k, size_t smem,
                               cudaStream_t st) {
  return var_sigma(mode) ? launch_step_t<kF64Var>(a, k, smem, st)
                         : launch_step_t<kModeF64>(a, k, smem, st);
}

int em_step_blocks_per_sm_f64(int mode, size_t smem) {
  return var_sigma(mode) ? step_blocks_per_sm_t<kF64Var>(smem)
                         : step_blocks_per_sm_t<kModeF64>(smem);
}

int em_range_blocks_per_sm_f64(int mode, size_t smem) {
  return var_sigma(mode) ? range_blocks_per_sm_t<kF64Var>(smem)
                         : range_blocks_per_sm_t<kModeF64>(smem);
}

cudaError_t launch_em_batch_f64(int mode, const SimArgs* insts, const BatchItem* items,
                                int32_t n_items, uint32_t* head, const Keys& k, size_t smem,
                                int blocks, cudaStream_t st) {
  return var_sigma(mode)
             ? launch_batch_t<kF64Var>(insts, items, n_items, head, k, smem, blocks, st)
             : launch_batch_t<kModeF64>(insts, items, n_items, head, k, smem, blocks, st);
}

int em_batch_blocks_per_sm_f64(int mode, size_t smem) {
  return var_sigma(mode) ? batch_blocks_per_sm_t<kF64Var>(smem)
                         : batch_blocks_per_sm_t<kModeF64>(smem);
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
