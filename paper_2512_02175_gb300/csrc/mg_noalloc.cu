// mg_noalloc.cu -- mg_histogram_static: the occupancy histogram of a particle
// set, copied to host memory, without allocating any device memory.
//
// mg_histogram with a host output stages the counts in a device buffer that
// it allocates (once per set).  Some callers cannot let a library allocate:
// code that runs with a fixed, pre-reserved memory budget (the allocation
// could fail or take memory another part of the program counts on), code that
// must not synchronise the device (cudaMalloc and cudaFree can), and code that
// hands the library a custom allocator which is not safe to call from every
// place a histogram is read.  This entry point stages the counts in a
// file-scope device array instead, of fixed size: at most kMaxStaticBins
// counts (n_edges x bins), 4 MiB, held by every GPU that loads the library's
// device code until the process exits.  Under CUDA's lazy module loading that
// code (and the array) is loaded on a device by the first kernel or symbol
// lookup there, which can synchronise: the first call on a device belongs in
// set-up.  The array's device address is looked up once per device and kept;
// cudaDeviceReset frees the array, so a caller that resets a device must not
// call this entry point on it again in the same process.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "mg.h"
#include "mg_em_step.cuh"
#include "mg_launch.h"

bool mg_particles_view(mg_particles p, mg::GraphView* g, const int32_t** edge, const void** x,
                       int64_t* n, int* precision);
mg_status mg_fail_message(mg_status st, const char* msg);

namespace {

constexpr int64_t kMaxStaticBins = 1 << 20;
constexpr int kMaxDevices = 64;

// The staging counts.  In host code this name is only a stand-in for the
// device symbol, not a device address: the address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) uint32_t g_static_hist[kMaxStaticBins];

std::mutex g_mu;
uint32_t* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_hist on the current device (set up on the first
// call for that device).
mg_status static_hist_ptr(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mg_fail_message(MG_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return mg_fail_message(MG_ERR_INVALID_ARG, "mg_histogram_static: device ordinal >= 64");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_hist);
    if (e != cudaSuccess) {
      char msg[256];
      snprintf(msg, sizeof msg, "mg_histogram_static: cudaGetSymbolAddress: %s",
               cudaGetErrorString(e));
      return mg_fail_message(MG_ERR_CUDA, msg);
    }
    g_static_ptr[dev] = static_cast<uint32_t*>(ptr);
  }
  *out = g_static_ptr[dev];
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_histogram_static(mg_particles p, int32_t bins, uint32_t* out,
                                         void* stream) {
  mg::GraphView g;
  const int32_t* edge = nullptr;
  const void* x = nullptr;
  int64_t n = 0;
  int prec = 0;
  if (!out || !mg_particles_view(p, &g, &edge, &x, &n, &prec))
    return mg_fail_message(MG_ERR_INVALID_ARG, "mg_histogram_static: NULL argument");
  if (bins < 1) return mg_fail_message(MG_ERR_INVALID_ARG, "mg_histogram_static: bins must be >= 1");
  {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess) (void)cudaGetLastError();
    else if (at.type == cudaMemoryTypeDevice)
      return mg_fail_message(MG_ERR_INVALID_ARG,
                             "mg_histogram_static: out must be host memory, not device memory");
  }
  const int64_t len = (int64_t)g.E * bins;
  if (len > kMaxStaticBins) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "mg_histogram_static: n_edges x bins = %lld exceeds the static limit of %lld counts",
             (long long)len, (long long)kMaxStaticBins);
    return mg_fail_message(MG_ERR_INVALID_ARG, msg);
  }
  uint32_t* scratch = nullptr;
  mg_status s = static_hist_ptr(&scratch);
  if (s != MG_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)len * 4;
  // the array keeps the previous call's counts: clear the part this call uses
  cudaError_t e = cudaMemsetAsync(scratch, 0, bytes, st);
  if (e == cudaSuccess) {
    const bool sm = bytes <= 96 * 1024;
    e = (prec == MG_FP64) ? mg::launch_histogram_f64(g, edge, x, n, bins, scratch, sm, st)
                          : mg::launch_histogram_f32(g, edge, x, n, bins, scratch, sm, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, scratch, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return mg_fail_message(MG_ERR_CUDA, cudaGetErrorString(e));
  return MG_OK;
}
