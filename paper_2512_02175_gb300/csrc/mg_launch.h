// mg_launch.h -- host-side launchers of the kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "mg_types.h"

namespace mg {

constexpr int kBlock = kThreads;

// Fused EM-Step kernel: binary64 (em_step_f64.cu), binary32-mixed and
// binary32 (em_step_f32.cu).
cudaError_t launch_em_step_f64(const SimArgs& a, size_t smem, cudaStream_t st);
cudaError_t launch_em_step_mixed(const SimArgs& a, size_t smem, cudaStream_t st);
cudaError_t launch_em_step_f32(const SimArgs& a, size_t smem, cudaStream_t st);

// Snapshot histogram of the living particles (adds into out); x is binary32
// or binary64.
cudaError_t launch_histogram_f32(const GraphView& g, const int32_t* edge, const void* x, int64_t n,
                                 int32_t bins, uint32_t* out, bool smem, cudaStream_t st);
cudaError_t launch_histogram_f64(const GraphView& g, const int32_t* edge, const void* x, int64_t n,
                                 int32_t bins, uint32_t* out, bool smem, cudaStream_t st);

// Initialise a particle state from binary64 positions x0 (device) and edges
// edge0 (device): copies the edges, converts x to the state's precision,
// zeroes n_draw / hits / first_hits / flags, and sets kErrBadEdge / kErrNan in
// *err for an edge out of range or x outside [0, l_e].  x0 may alias the hits
// and first_hits arrays (all of x0 is read before they are zeroed).
cudaError_t launch_init_state(const GraphView& g, const int32_t* edge0, const double* x0, int64_t n,
                              bool f64, StateView s, uint32_t* err, cudaStream_t st);

}  // namespace mg
