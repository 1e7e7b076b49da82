// em_step_f64.cu -- binary64 instantiation of the fused EM-Step kernel and of
// the histogram kernel.  Built without floating-point contraction
// (--fmad=false) so that every binary64 operation rounds exactly as written,
// in the same order as the plain CPU reference of the scheme.
#include "mg_em_step.cuh"
#include "mg_launch.h"

namespace mg {

cudaError_t launch_em_step_f64(const SimArgs& a, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(em_step_kernel<kModeF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr = true;
  }
  const int64_t grid = (a.n + kBlock - 1) / kBlock;
  em_step_kernel<kModeF64><<<(unsigned)grid, kBlock, smem, st>>>(a);
  return cudaGetLastError();
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

}  // namespace mg
