// mg_launch.h -- host-side launchers of the kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "mg_types.h"

namespace mg {

constexpr int kBlock = kThreads;

// Fused EM-Step kernel over one particle set, by kernel mode: a precision
// mode, plus kVarSigma for a graph with position-dependent diffusion
// (binary64 modes in em_step_f64.cu, the binary32 ones in em_step_f32.cu).
cudaError_t launch_em_step(int mode, const SimArgs& a, const Keys& k, size_t smem,
                           cudaStream_t st);
cudaError_t launch_em_step_f64(int mode, const SimArgs& a, const Keys& k, size_t smem,
                               cudaStream_t st);
cudaError_t launch_em_step_f32x(int mode, const SimArgs& a, const Keys& k, size_t smem,
                                cudaStream_t st);
// (a.range > 256 launches the range kernel: lanes claim particles of their
// block's range; a.range <= 256 the tile kernel, a.range particles per
// block.)  Resident blocks per SM of either kernel at `smem` bytes of dynamic
// shared memory.
int em_step_blocks_per_sm(int mode, size_t smem);
int em_step_blocks_per_sm_f64(int mode, size_t smem);
int em_step_blocks_per_sm_f32x(int mode, size_t smem);
int em_range_blocks_per_sm(int mode, size_t smem);
int em_range_blocks_per_sm_f64(int mode, size_t smem);
int em_range_blocks_per_sm_f32x(int mode, size_t smem);

// The batched persistent kernel: `blocks` blocks pop the n_items work items
// (head must be zero at launch).  blocks_per_sm: resident blocks per SM at
// `smem` bytes of dynamic shared memory.
cudaError_t launch_em_batch(int mode, const SimArgs* insts, const BatchItem* items, int32_t n_items,
                            uint32_t* head, const Keys& k, size_t smem, int blocks,
                            cudaStream_t st);
cudaError_t launch_em_batch_f64(int mode, const SimArgs* insts, const BatchItem* items,
                                int32_t n_items, uint32_t* head, const Keys& k, size_t smem,
                                int blocks, cudaStream_t st);
cudaError_t launch_em_batch_f32x(int mode, const SimArgs* insts, const BatchItem* items,
                                 int32_t n_items, uint32_t* head, const Keys& k, size_t smem,
                                 int blocks, cudaStream_t st);
int em_batch_blocks_per_sm(int mode, size_t smem);
int em_batch_blocks_per_sm_f64(int mode, size_t smem);
int em_batch_blocks_per_sm_f32x(int mode, size_t smem);

// Snapshot histogram of the living particles (adds into out); x is binary32
// or binary64.
cudaError_t launch_histogram_f32(const GraphView& g, const int32_t* edge, const void* x, int64_t n,
                                 int32_t bins, uint32_t* out, bool smem, cudaStream_t st);
cudaError_t launch_histogram_f64(const GraphView& g, const int32_t* edge, const void* x, int64_t n,
                                 int32_t bins, uint32_t* out, bool smem, cudaStream_t st);

// Snapshot histogram with variable-width bins (adds into out[n_bins]): off
// [E+1] and the upper boundaries up (binary32 for binary32 states, binary64
// otherwise) on the device.
cudaError_t launch_histogram_binned(bool f64, const int32_t* edge, const void* x, int64_t n,
                                    const int32_t* off, const void* up, int32_t n_bins,
                                    uint32_t* out, cudaStream_t st);

// Initialise a particle state from binary64 positions x0 (device) and edges
// edge0 (device): copies the edges, converts x to the state's precision,
// zeroes n_draw / hits / first_hits / flags, and sets kErrBadEdge / kErrNan in
// *err for an edge out of range or x outside [0, l_e].  x0 may alias the hits
// and first_hits arrays (all of x0 is read before they are zeroed).
cudaError_t launch_init_state(const GraphView& g, const int32_t* edge0, const double* x0, int64_t n,
                              bool f64, StateView s, uint32_t* err, cudaStream_t st);

// The first root s in [0, 1] of A s^2 + B s + C = 0 (binary32 coefficients,
// device arrays) by the device function precision mode `mode` uses in a
// split; s (device) in binary64.
cudaError_t launch_hit_root(int32_t mode, int64_t n, const float* A, const float* B,
                            const float* C, double* s, cudaStream_t st);

}  // namespace mg
