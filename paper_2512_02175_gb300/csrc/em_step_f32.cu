// em_step_f32.cu -- binary32-mixed and binary32 instantiations of the fused
// EM-Step kernel, the binary32 histogram kernel and the state initialisation
// kernels.
#include "mg_em_step.cuh"
#include "mg_histogram.cuh"
#include "mg_launch.h"
#include "mg_launch_impl.cuh"

namespace mg {

// Modes of this unit: FP32-mixed and FP32, each with constant or
// position-dependent (kVarSigma) diffusion.
cudaError_t launch_em_step_f32x(int mode, const SimArgs& a, const Keys& k, size_t smem,
                                cudaStream_t st) {
  switch (mode) {
    case kModeMixed: return launch_step_t<kModeMixed>(a, k, smem, st);
    case kModeF32: return launch_step_t<kModeF32>(a, k, smem, st);
    case kModeMixed | kVarSigma: return launch_step_t<kModeMixed | kVarSigma>(a, k, smem, st);
    case kModeF32 | kVarSigma: return launch_step_t<kModeF32 | kVarSigma>(a, k, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

int em_step_blocks_per_sm_f32x(int mode, size_t smem) {
  switch (mode) {
    case kModeMixed: return step_blocks_per_sm_t<kModeMixed>(smem);
    case kModeF32: return step_blocks_per_sm_t<kModeF32>(smem);
    case kModeMixed | kVarSigma: return step_blocks_per_sm_t<kModeMixed | kVarSigma>(smem);
    case kModeF32 | kVarSigma: return step_blocks_per_sm_t<kModeF32 | kVarSigma>(smem);
    default: return 0;
  }
}

int em_step_blocks_per_sm(int mode, size_t smem) {
  return prec_of(mode) == kModeF64 ? em_step_blocks_per_sm_f64(mode, smem)
                                   : em_step_blocks_per_sm_f32x(mode, smem);
}

int em_range_blocks_per_sm_f32x(int mode, size_t smem) {
  switch (mode) {
    case kModeMixed: return range_blocks_per_sm_t<kModeMixed>(smem);
    case kModeF32: return range_blocks_per_sm_t<kModeF32>(smem);
    case kModeMixed | kVarSigma: return range_blocks_per_sm_t<kModeMixed | kVarSigma>(smem);
    case kModeF32 | kVarSigma: return range_blocks_per_sm_t<kModeF32 | kVarSigma>(smem);
    default: return 0;
  }
}

int em_range_blocks_per_sm(int mode, size_t smem) {
  return prec_of(mode) == kModeF64 ? em_range_blocks_per_sm_f64(mode, smem)
                                   : em_range_blocks_per_sm_f32x(mode, smem);
}

cudaError_t launch_em_batch_f32x(int mode, const SimArgs* insts, const BatchItem* items,
                                 int32_t n_items, uint32_t* head, const Keys& k, size_t smem,
                                 int blocks, cudaStream_t st) {
  switch (mode) {
    case kModeMixed:
      return launch_batch_t<kModeMixed>(insts, items, n_items, head, k, smem, blocks, st);
    case kModeF32:
      return launch_batch_t<kModeF32>(insts, items, n_items, head, k, smem, blocks, st);
    case kModeMixed | kVarSigma:
      return launch_batch_t<kModeMixed | kVarSigma>(insts, items, n_items, head, k, smem, blocks,
                                                    st);
    case kModeF32 | kVarSigma:
      return launch_batch_t<kModeF32 | kVarSigma>(insts, items, n_items, head, k, smem, blocks,
                                                  st);
    default: return cudaErrorInvalidValue;
  }
}

int em_batch_blocks_per_sm_f32x(int mode, size_t smem) {
  switch (mode) {
    case kModeMixed: return batch_blocks_per_sm_t<kModeMixed>(smem);
    case kModeF32: return batch_blocks_per_sm_t<kModeF32>(smem);
    case kModeMixed | kVarSigma: return batch_blocks_per_sm_t<kModeMixed | kVarSigma>(smem);
    case kModeF32 | kVarSigma: return batch_blocks_per_sm_t<kModeF32 | kVarSigma>(smem);
    default: return 0;
  }
}

cudaError_t launch_em_step(int mode, const SimArgs& a, const Keys& k, size_t smem,
                           cudaStream_t st) {
  return prec_of(mode) == kModeF64 ? launch_em_step_f64(mode, a, k, smem, st)
                                   : launch_em_step_f32x(mode, a, k, smem, st);
}

cudaError_t launch_em_batch(int mode, const SimArgs* insts, const BatchItem* items, int32_t n_items,
                            uint32_t* head, const Keys& k, size_t smem, int blocks,
                            cudaStream_t st) {
  return prec_of(mode) == kModeF64
             ? launch_em_batch_f64(mode, insts, items, n_items, head, k, smem, blocks, st)
             : launch_em_batch_f32x(mode, insts, items, n_items, head, k, smem, blocks, st);
}

int em_batch_blocks_per_sm(int mode, size_t smem) {
  return prec_of(mode) == kModeF64 ? em_batch_blocks_per_sm_f64(mode, smem)
                                   : em_batch_blocks_per_sm_f32x(mode, smem);
}

cudaError_t launch_histogram_f32(const GraphView& g, const int32_t* edge, const void* x, int64_t n,
                                 int32_t bins, uint32_t* out, bool smem, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + kBlock - 1) / kBlock;
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  if (grid < 1) grid = 1;
  const size_t sh = smem ? align16((size_t)g.E * bins * 4) : 0;
  if (sh > 48 * 1024)
    cudaFuncSetAttribute(histogram_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sh);
  histogram_kernel<float><<<(unsigned)grid, kBlock, sh, st>>>(g, edge, x, n, bins, out, smem ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_histogram_binned_f32(const int32_t* edge, const void* x, int64_t n,
                                        const int32_t* off, const float* up, int32_t n_bins,
                                        uint32_t* out, cudaStream_t st);
cudaError_t launch_histogram_binned_f64(const int32_t* edge, const void* x, int64_t n,
                                        const int32_t* off, const double* up, int32_t n_bins,
                                        uint32_t* out, cudaStream_t st);

cudaError_t launch_histogram_binned(bool f64, const int32_t* edge, const void* x, int64_t n,
                                    const int32_t* off, const void* up, int32_t n_bins,
                                    uint32_t* out, cudaStream_t st) {
  return f64 ? launch_histogram_binned_f64(edge, x, n, off, static_cast<const double*>(up), n_bins,
                                           out, st)
             : launch_histogram_binned_f32(edge, x, n, off, static_cast<const float*>(up), n_bins,
                                           out, st);
}

cudaError_t launch_histogram_binned_f32(const int32_t* edge, const void* x, int64_t n,
                                        const int32_t* off, const float* up, int32_t n_bins,
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
    cudaFuncSetAttribute(histogram_binned_kernel<float>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  histogram_binned_kernel<float><<<(unsigned)grid, kBlock, sh, st>>>(edge, x, n, off, up, n_bins,
                                                                     out, smem ? 1 : 0);
  return cudaGetLastError();
}

__global__ void init_state_kernel(GraphView g, const int32_t* __restrict__ edge0,
                                  const double* x0, int64_t n, int32_t f64, StateView s,
                                  uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = edge0[i];
    const double x = x0[i];
    uint32_t bad = 0;
    if (e < kDead || e >= g.E) bad |= kErrBadEdge;
    else if (e >= 0 && !(x >= 0.0 && x <= g.e64[e].L && isfinite(x))) bad |= kErrNan;
    if (bad) atomicOr(err, bad);
    s.edge[i] = e;
    if (f64) reinterpret_cast<double*>(s.x)[i] = x;
    else reinterpret_cast<float*>(s.x)[i] = (float)x;  // x <= l_e rounds to <= (float)l_e
  }
}

__global__ void zero_counters_kernel(StateView s, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    s.n_draw[i] = 0u;
    s.hits[i] = 0u;
    s.first_hits[i] = 0u;
    s.flags[i] = 0u;
  }
}

cudaError_t launch_init_state(const GraphView& g, const int32_t* edge0, const double* x0, int64_t n,
                              bool f64, StateView s, uint32_t* err, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + kBlock - 1) / kBlock;
  if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
  if (grid < 1) grid = 1;
  // x0 may live in the hits/first_hits storage: convert everything first,
  // then zero the counters in a second, stream-ordered kernel.
  init_state_kernel<<<(unsigned)grid, kBlock, 0, st>>>(g, edge0, x0, n, f64 ? 1 : 0, s, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  zero_counters_kernel<<<(unsigned)grid, kBlock, 0, st>>>(s, n);
  return cudaGetLastError();
}

// The hitting-fraction root of n coefficient triples by the device function
// of precision mode `mode` (mg_hit_root).
__global__ void hit_root_kernel(int32_t mode, int64_t n, const float* __restrict__ A,
                                const float* __restrict__ B, const float* __restrict__ C,
                                double* __restrict__ s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float a = A[i], b = B[i], c = C[i];
    double r;
    if (mode == kModeF32) {
      r = widen_f32(hit_root_fast(a, b, c));
    } else if (mode == kModeMixed) {
      r = hit_root_f64_eft(a, b, c);
    } else {
      r = hit_root_f64_closed(a, b, c);
    }
    s[i] = r;
  }
}

cudaError_t launch_hit_root(int32_t mode, int64_t n, const float* A, const float* B,
                            const float* C, double* s, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + kBlock - 1) / kBlock;
  if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
  if (grid < 1) grid = 1;
  hit_root_kernel<<<(unsigned)grid, kBlock, 0, st>>>(mode, n, A, B, C, s);
  return cudaGetLastError();
}

}  // namespace mg
