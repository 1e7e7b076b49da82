// mg_histogram.cuh -- standalone snapshot histograms of a particle set
// (uniform bins per edge, and bins of any width per edge), the counterparts
// of the histogram fused into the EM-Step kernel's tail.
#pragma once
#include "mg_em_step.cuh"

namespace mg {

// Snapshot histogram of the living particles (no stepping).
template <typename R>
__global__ void __launch_bounds__(256) histogram_kernel(GraphView g, const int32_t* __restrict__ edge,
                                                        const void* __restrict__ xv, int64_t n,
                                                        int32_t bins, uint32_t* __restrict__ out,
                                                        int32_t use_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* sh = reinterpret_cast<uint32_t*>(smem);
  const int32_t len = g.E * bins;
  if (use_smem) {
    block_zero(sh, len);
    __syncthreads();
  }
  const R* x = reinterpret_cast<const R*>(xv);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = edge[i];
    if (e < 0 || e >= g.E) continue;
    const int32_t key = e * bins + hist_bin<R>(x[i], g.range[e], bins);
    if (use_smem) atomicAdd(&sh[key], 1u);
    else atomicAdd(&out[key], 1u);
  }
  if (use_smem) {
    __syncthreads();
    for (int32_t k = threadIdx.x; k < len; k += blockDim.x)
      if (sh[k]) atomicAdd(&out[k], sh[k]);
  }
}

// Snapshot histogram with bins of any width per edge: bins off[e] ..
// off[e+1]-1 of edge e with upper boundaries up[j] (increasing within the
// edge; in the state's precision, binary32 boundaries rounded up so that
// x < up[j] decides exactly as in binary64); a living particle counts in the
// first bin j of its edge with x < up[j], else in the edge's last bin.
template <typename R>
__global__ void __launch_bounds__(256) histogram_binned_kernel(
    const int32_t* __restrict__ edge, const void* __restrict__ xv, int64_t n,
    const int32_t* __restrict__ off, const R* __restrict__ up, int32_t n_bins,
    uint32_t* __restrict__ out, int32_t use_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* sh = reinterpret_cast<uint32_t*>(smem);
  if (use_smem) {
    block_zero(sh, n_bins);
    __syncthreads();
  }
  const R* x = reinterpret_cast<const R*>(xv);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = edge[i];
    if (e < 0) continue;
    int32_t lo = off[e], hi = off[e + 1] - 1;  // search [lo, hi]; hi is the catch-all
    if (hi < lo) continue;
    const R xi = x[i];
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (xi < up[mid]) hi = mid;
      else lo = mid + 1;
    }
    if (use_smem) atomicAdd(&sh[lo], 1u);
    else atomicAdd(&out[lo], 1u);
  }
  if (use_smem) {
    __syncthreads();
    for (int32_t k = threadIdx.x; k < n_bins; k += blockDim.x)
      if (sh[k]) atomicAdd(&out[k], sh[k]);
  }
}

}  // namespace mg
