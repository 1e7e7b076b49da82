// mg_api.cpp -- the C ABI of libmetricgraph (declared in include/mg.h):
// validation, graph tables, particle-set memory and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "mg.h"
#include "mg_launch.h"
#include "mg_types.h"

static_assert(MG_DEVERR_BAD_EDGE == mg::kErrBadEdge, "device error bits");
static_assert(MG_DEVERR_NAN == mg::kErrNan, "device error bits");
static_assert(MG_DEVERR_STREAM == mg::kErrStream, "device error bits");
static_assert(MG_DEVERR_STUCK == mg::kErrStuck, "device error bits");
static_assert((int)MG_FP64 == (int)mg::kModeF64 && (int)MG_FP32_MIXED == (int)mg::kModeMixed &&
                  (int)MG_FP32 == (int)mg::kModeF32,
              "precision modes");

namespace {

thread_local std::string g_err;

mg_status fail(mg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

mg_status cuda_fail(cudaError_t e, const char* what) {
  return fail(MG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MG_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Where a caller's pointer points, as CUDA sees it.  A kernel of the current
// device may use its device memory, managed memory and mapped pinned host
// memory; ordinary host memory (an address CUDA does not know) or another
// device's memory would fault it, so such "device" arguments are rejected.  A
// "host" argument read or written by the CPU must not be device memory.
enum class Mem { kHost, kDevice };

mg_status check_memory(const void* ptr, Mem want, const char* what) {
  if (!ptr) return MG_OK;  // NULL is the caller's check
  cudaPointerAttributes at{};
  cudaError_t ce = cudaPointerGetAttributes(&at, ptr);
  if (ce != cudaSuccess) {
    (void)cudaGetLastError();
    // without a usable device nothing is device memory
    return want == Mem::kHost ? MG_OK : cuda_fail(ce, what);
  }
  if (want == Mem::kDevice) {
    if (at.type == cudaMemoryTypeUnregistered)
      return fail(MG_ERR_INVALID_ARG, "%s must be device memory, not ordinary host memory", what);
    if (at.type == cudaMemoryTypeDevice) {
      int dev = 0;
      MG_CUDA(cudaGetDevice(&dev));
      if (at.device != dev)
        return fail(MG_ERR_INVALID_ARG, "%s is memory of device %d, the current device is %d", what,
                    at.device, dev);
    }
  } else if (at.type == cudaMemoryTypeDevice) {
    return fail(MG_ERR_INVALID_ARG, "%s must be host memory, not device memory", what);
  }
  return MG_OK;
}

mg_status check_host(std::initializer_list<std::pair<const void*, const char*>> ptrs) {
  for (const auto& q : ptrs) {
    mg_status s = check_memory(q.first, Mem::kHost, q.second);
    if (s != MG_OK) return s;
  }
  return MG_OK;
}

// Pinned host memory of the calling thread for results copied to the host
// (grown as needed, up to kStageMax, and kept for the thread's life): a copy
// into it runs at DMA speed, one into ordinary host memory goes through the
// driver's own staging, several times slower for megabytes (a vascular
// graph's histogram and counters).  Null if pinned memory cannot be had.
constexpr size_t kStageMax = 64u << 20;

struct PinnedStage {
  void* p = nullptr;
  size_t bytes = 0;
  ~PinnedStage() {
    if (p) (void)cudaFreeHost(p);  // may run after the runtime has unloaded
  }
  void* get(size_t n) {
    if (n > kStageMax) return nullptr;
    if (n > bytes) {
      if (p) (void)cudaFreeHost(p);
      p = nullptr;
      bytes = 0;
      const size_t want = std::max(n, (size_t)1 << 20);
      if (cudaMallocHost(&p, want) != cudaSuccess) {
        (void)cudaGetLastError();
        p = nullptr;
        return nullptr;
      }
      bytes = want;
    }
    return p;
  }
};
thread_local PinnedStage g_stage;

// Device-to-host copy of `bytes` through the pinned stage (then a host
// copy), or straight into dst; returns after the copy has completed.
cudaError_t copy_to_host(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  void* stage = g_stage.get(bytes);
  cudaError_t e = cudaMemcpyAsync(stage ? stage : dst, src, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && stage) memcpy(dst, stage, bytes);
  return e;
}

// ---------------------------------------------------------------- memory

std::mutex g_alloc_mu;
mg_alloc_fn g_alloc = nullptr;
mg_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  mg_free_fn free_fn = nullptr;  // hooks that allocated it (nullptr: cudaFree)
  void* ctx = nullptr;
};

mg_status dev_alloc(DevBuf& b, size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  b.bytes = bytes;
  if (g_alloc) {
    b.p = g_alloc(bytes, (void*)st, g_alloc_ctx);
    b.free_fn = g_free;
    b.ctx = g_alloc_ctx;
    if (!b.p) return fail(MG_ERR_OUT_OF_MEMORY, "allocator hook returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      b.p = nullptr;
      cudaGetLastError();
      return fail(MG_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  return MG_OK;
}

void dev_free(DevBuf& b, cudaStream_t st) {
  if (!b.p) return;
  if (b.free_fn) b.free_fn(b.p, (void*)st, b.ctx);
  else cudaFree(b.p);
  b.p = nullptr;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// ------------------------------------------------------------------ graph

struct mg_graph_s {
  int32_t V = 0, E = 0, S = 0;
  // host copies
  std::vector<int32_t> src, dst, vtx_off, slot_edge, slot_of_end;
  std::vector<uint8_t> slot_end, kind;
  bool has_absorbing = false;  // particles can die
  bool var_sigma = false;      // some edge has a nonzero diffusion slope
  std::vector<uint64_t> slot_T;
  std::vector<double> length, range;
  // device tables (one allocation)
  DevBuf buf;
  mg::GraphView view{};
  size_t table_bytes32 = 0, table_bytes64 = 0;
  std::atomic<int> refs{0};
};

namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

extern "C" mg_status mg_set_allocator(mg_alloc_fn alloc, mg_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(MG_ERR_INVALID_ARG, "mg_set_allocator: give both hooks or neither");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return MG_OK;
}

extern "C" mg_status mg_graph_create(const mg_graph_desc* d, mg_graph* out) {
  if (!d || !out) return fail(MG_ERR_INVALID_ARG, "mg_graph_create: NULL argument");
  *out = nullptr;
  const int32_t V = d->n_vertices, E = d->n_edges;
  if (V < 1 || E < 1) return fail(MG_ERR_INVALID_ARG, "need n_vertices >= 1 and n_edges >= 1");
  if (!d->edge_src || !d->edge_dst || !d->length || !d->drift_c0 || !d->drift_c1 || !d->sigma ||
      !d->weight_init || !d->weight_term)
    return fail(MG_ERR_INVALID_ARG, "mg_graph_create: a required array is NULL");
  {
    mg_status s = check_host({{d->edge_src, "edge_src"}, {d->edge_dst, "edge_dst"},
                              {d->length, "length"}, {d->drift_c0, "drift_c0"},
                              {d->drift_c1, "drift_c1"}, {d->sigma, "sigma"},
                              {d->weight_init, "weight_init"}, {d->weight_term, "weight_term"},
                              {d->hist_range, "hist_range"}, {d->vertex_kind, "vertex_kind"},
                              {d->sigma_slope, "sigma_slope"}});
    if (s != MG_OK) return s;
  }
  for (int32_t e = 0; e < E; ++e) {
    const int32_t s = d->edge_src[e], t = d->edge_dst[e];
    if (s < 0 || s >= V) return fail(MG_ERR_INVALID_ARG, "edge %d: src %d out of range", e, s);
    if (t < -1 || t >= V) return fail(MG_ERR_INVALID_ARG, "edge %d: dst %d out of range", e, t);
    const double L = d->length[e];
    if (t == -1) {
      if (!(std::isinf(L) && L > 0))
        return fail(MG_ERR_INVALID_ARG, "edge %d: a semi-infinite edge needs length +inf", e);
    } else if (!finite_pos(L)) {
      return fail(MG_ERR_INVALID_ARG, "edge %d: length must be finite and > 0", e);
    }
    if (!finite_pos(d->sigma[e])) return fail(MG_ERR_INVALID_ARG, "edge %d: sigma must be > 0", e);
    if (!std::isfinite(d->drift_c0[e]) || !std::isfinite(d->drift_c1[e]))
      return fail(MG_ERR_INVALID_ARG, "edge %d: drift must be finite", e);
    if (!(std::isfinite(d->weight_init[e]) && d->weight_init[e] >= 0.0))
      return fail(MG_ERR_INVALID_ARG, "edge %d: weight_init must be >= 0", e);
    if (t >= 0 && !(std::isfinite(d->weight_term[e]) && d->weight_term[e] >= 0.0))
      return fail(MG_ERR_INVALID_ARG, "edge %d: weight_term must be >= 0", e);
    if (d->hist_range && !finite_pos(d->hist_range[e]))
      return fail(MG_ERR_INVALID_ARG, "edge %d: hist_range must be finite and > 0", e);
    if (d->sigma_slope) {
      const double k = d->sigma_slope[e];
      if (!std::isfinite(k))
        return fail(MG_ERR_INVALID_ARG, "edge %d: sigma_slope must be finite", e);
      if (t == -1 ? !(k >= 0.0) : !(d->sigma[e] + k * L > 0.0))
        return fail(MG_ERR_INVALID_ARG, "edge %d: sigma_e(x) = sigma + sigma_slope x must stay "
                    "> 0 on the edge", e);
    }
  }
  if (d->vertex_kind)
    for (int32_t v = 0; v < V; ++v)
      if (d->vertex_kind[v] > MG_VERTEX_ABSORBING)
        return fail(MG_ERR_INVALID_ARG, "vertex %d: unknown kind %d", v, d->vertex_kind[v]);

  mg_graph g = new mg_graph_s();
  g->V = V;
  g->E = E;
  g->src.assign(d->edge_src, d->edge_src + E);
  g->dst.assign(d->edge_dst, d->edge_dst + E);
  g->length.assign(d->length, d->length + E);
  g->range.resize(E);
  for (int32_t e = 0; e < E; ++e)
    g->range[e] = d->hist_range ? d->hist_range[e] : (g->dst[e] >= 0 ? g->length[e] : 1.0);
  g->kind.assign(V, 0);
  if (d->vertex_kind) g->kind.assign(d->vertex_kind, d->vertex_kind + V);
  for (int32_t v = 0; v < V; ++v)
    if (g->kind[v] == MG_VERTEX_ABSORBING) g->has_absorbing = true;
  std::vector<double> s1_64(E, 0.0);
  std::vector<float> s1_32(E, 0.0f);
  if (d->sigma_slope)
    for (int32_t e = 0; e < E; ++e) {
      s1_64[e] = d->sigma_slope[e];
      s1_32[e] = (float)d->sigma_slope[e];
      if (s1_64[e] != 0.0) g->var_sigma = true;
    }

  // Slots by counting sort on the vertex: each edge contributes its init end
  // then its term end, edges in id order, so within a vertex the slots are
  // ordered by (edge id, init before term).
  std::vector<int32_t> deg(V + 1, 0);
  for (int32_t e = 0; e < E; ++e) {
    deg[g->src[e]]++;
    if (g->dst[e] >= 0) deg[g->dst[e]]++;
  }
  g->vtx_off.assign(V + 1, 0);
  for (int32_t v = 0; v < V; ++v) g->vtx_off[v + 1] = g->vtx_off[v] + deg[v];
  const int32_t S = g->vtx_off[V];
  g->S = S;
  g->slot_edge.assign(S, 0);
  g->slot_end.assign(S, 0);
  g->slot_T.assign(S, 0);
  g->slot_of_end.assign(2 * (size_t)E, -1);
  std::vector<double> w(S, 0.0);
  std::vector<int32_t> fill(g->vtx_off.begin(), g->vtx_off.end() - 1);
  for (int32_t e = 0; e < E; ++e) {
    int32_t j = fill[g->src[e]]++;
    g->slot_edge[j] = e;
    g->slot_end[j] = mg::kEndInit;
    w[j] = d->weight_init[e];
    g->slot_of_end[2 * (size_t)e] = j;
    if (g->dst[e] >= 0) {
      j = fill[g->dst[e]]++;
      g->slot_edge[j] = e;
      g->slot_end[j] = mg::kEndTerm;
      w[j] = d->weight_term[e];
      g->slot_of_end[2 * (size_t)e + 1] = j;
    }
  }
  // Integer thresholds of b_v: T_j = min(floor(2^32 C_j), 2^32) with C_j the
  // binary64 running sum of v's weights divided by their binary64 total; the
  // last slot of v gets 2^32.
  for (int32_t v = 0; v < V; ++v) {
    const int32_t lo = g->vtx_off[v], hi = g->vtx_off[v + 1];
    if (lo == hi) continue;
    double tot = 0.0;
    for (int32_t j = lo; j < hi; ++j) tot += w[j];
    if (g->kind[v] == MG_VERTEX_STANDARD && !(tot > 0.0)) {
      delete g;
      return fail(MG_ERR_INVALID_ARG, "vertex %d: jump weights sum to 0", v);
    }
    double cum = 0.0;
    for (int32_t j = lo; j < hi; ++j) {
      cum += w[j];
      const double c = (tot > 0.0) ? cum / tot : 1.0;
      const double f = std::floor(c * 4294967296.0);
      g->slot_T[j] = (f >= 4294967296.0) ? 4294967296ull : (uint64_t)f;
    }
    g->slot_T[hi - 1] = 4294967296ull;
  }

  // device tables
  std::vector<mg::EdgeRec32> e32(E);
  std::vector<mg::EdgeRec64> e64(E);
  for (int32_t e = 0; e < E; ++e) {
    const double L = g->length[e];
    e64[e] = {L, d->drift_c0[e], d->drift_c1[e], d->sigma[e], g->src[e], g->dst[e],
              g->slot_of_end[2 * (size_t)e], g->slot_of_end[2 * (size_t)e + 1]};
    e32[e] = {(float)L, (float)d->drift_c0[e], (float)d->drift_c1[e], (float)d->sigma[e],
              g->src[e], g->dst[e], g->slot_of_end[2 * (size_t)e],
              g->slot_of_end[2 * (size_t)e + 1]};
  }
  std::vector<mg::SlotRec> slots(S);
  for (int32_t j = 0; j < S; ++j)
    slots[j] = {g->slot_T[j] ? (uint32_t)(g->slot_T[j] - 1u) : 0u, g->slot_edge[j],
                g->slot_end[j], 0};
  // Guide tables: vertex v with d slots gets 2^gb entries (2^gb >= d); entry
  // k is the first slot whose threshold exceeds k 2^(32 - gb).  Thresholds are
  // non-decreasing and the last is 2^32, so every entry is a slot of v.
  std::vector<mg::VtxRec> vtx(V);
  std::vector<int32_t> guide;
  for (int32_t v = 0; v < V; ++v) {
    const int32_t lo = g->vtx_off[v], hi = g->vtx_off[v + 1];
    int gb = 0;
    while ((1 << gb) < hi - lo) ++gb;
    vtx[v] = {lo, hi, g->kind[v], (int32_t)guide.size()};
    int32_t j = lo;
    for (int64_t k = 0; k < (int64_t(1) << gb); ++k) {
      const uint64_t bucket_lo = (uint64_t)k << (32 - gb);
      while (j < hi - 1 && g->slot_T[j] <= bucket_lo) ++j;
      guide.push_back(j);
    }
  }
  const int32_t G = (int32_t)guide.size();

  const size_t o32 = 0, o64 = a256(o32 + E * sizeof(mg::EdgeRec32));
  const size_t os = a256(o64 + E * sizeof(mg::EdgeRec64));
  const size_t ov = a256(os + S * sizeof(mg::SlotRec));
  const size_t og = a256(ov + V * sizeof(mg::VtxRec));
  const size_t orr = a256(og + (size_t)G * sizeof(int32_t));
  const size_t os32 = a256(orr + E * sizeof(double));
  const size_t os64 = a256(os32 + E * sizeof(float));
  const size_t total = a256(os64 + E * sizeof(double));
  mg_status st = dev_alloc(g->buf, total, nullptr);
  if (st != MG_OK) {
    delete g;
    return st;
  }
  std::vector<unsigned char> host(total, 0);
  memcpy(host.data() + o32, e32.data(), E * sizeof(mg::EdgeRec32));
  memcpy(host.data() + o64, e64.data(), E * sizeof(mg::EdgeRec64));
  memcpy(host.data() + os, slots.data(), S * sizeof(mg::SlotRec));
  memcpy(host.data() + ov, vtx.data(), V * sizeof(mg::VtxRec));
  memcpy(host.data() + og, guide.data(), (size_t)G * sizeof(int32_t));
  memcpy(host.data() + orr, g->range.data(), E * sizeof(double));
  memcpy(host.data() + os32, s1_32.data(), E * sizeof(float));
  memcpy(host.data() + os64, s1_64.data(), E * sizeof(double));
  cudaError_t ce = cudaMemcpy(g->buf.p, host.data(), total, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    dev_free(g->buf, nullptr);
    delete g;
    return cuda_fail(ce, "mg_graph_create: upload");
  }
  unsigned char* base = static_cast<unsigned char*>(g->buf.p);
  g->view.V = V;
  g->view.E = E;
  g->view.S = S;
  g->view.e32 = reinterpret_cast<const mg::EdgeRec32*>(base + o32);
  g->view.e64 = reinterpret_cast<const mg::EdgeRec64*>(base + o64);
  g->view.slot = reinterpret_cast<const mg::SlotRec*>(base + os);
  g->view.vtx = reinterpret_cast<const mg::VtxRec*>(base + ov);
  g->view.G = G;
  g->view.guide = reinterpret_cast<const int32_t*>(base + og);
  g->view.range = reinterpret_cast<const double*>(base + orr);
  g->view.s1_32 = reinterpret_cast<const float*>(base + os32);
  g->view.s1_64 = reinterpret_cast<const double*>(base + os64);
  *out = g;
  return MG_OK;
}

extern "C" mg_status mg_graph_destroy(mg_graph g) {
  if (!g) return MG_OK;
  if (g->refs.load() > 0)
    return fail(MG_ERR_BUSY, "mg_graph_destroy: %d particle sets still use the graph",
                g->refs.load());
  dev_free(g->buf, nullptr);
  delete g;
  return MG_OK;
}

extern "C" mg_status mg_graph_info(mg_graph g, int32_t* V, int32_t* E, int32_t* S) {
  if (!g) return fail(MG_ERR_INVALID_ARG, "mg_graph_info: NULL graph");
  if (V) *V = g->V;
  if (E) *E = g->E;
  if (S) *S = g->S;
  return MG_OK;
}

extern "C" mg_status mg_graph_slots(mg_graph g, int32_t* vtx_off, int32_t* slot_edge,
                                    uint8_t* slot_end, uint64_t* slot_threshold) {
  if (!g) return fail(MG_ERR_INVALID_ARG, "mg_graph_slots: NULL graph");
  mg_status s = check_host({{vtx_off, "vtx_off"}, {slot_edge, "slot_edge"}, {slot_end, "slot_end"},
                            {slot_threshold, "slot_threshold"}});
  if (s != MG_OK) return s;
  if (vtx_off) memcpy(vtx_off, g->vtx_off.data(), (g->V + 1) * sizeof(int32_t));
  if (slot_edge) memcpy(slot_edge, g->slot_edge.data(), g->S * sizeof(int32_t));
  if (slot_end) memcpy(slot_end, g->slot_end.data(), g->S);
  if (slot_threshold) memcpy(slot_threshold, g->slot_T.data(), g->S * sizeof(uint64_t));
  return MG_OK;
}

// -------------------------------------------------------------- particles

struct mg_particles_s {
  mg_graph g = nullptr;
  int64_t n = 0;
  uint32_t pid_base = 0;
  uint64_t seed = 0;
  uint32_t instance = 0;
  mg_precision prec = MG_FP64;
  uint64_t step = 0;
  int32_t split_batch = 0;       // 0: the library's default for the mode
  int64_t steps_per_launch = 0;  // 0: as many as fit one launch
  int32_t max_blocks = 0;        // range kernel: most blocks per launch (0: resident)
  DevBuf state;      // edge | x | n_draw | hits | first_hits | flags
  DevBuf counters;   // exits[S] | absorbed[V] | trunc | psteps | err
  DevBuf hist_tmp;   // histogram staging for host output
  DevBuf bins_tmp;   // variable-width bin tables (offsets | boundaries)
  mg::StateView sv{};
  mg::CounterView cv{};
  cudaStream_t last_stream = nullptr;
};

namespace {

size_t xbytes(const mg_particles_s* p) { return p->prec == MG_FP64 ? 8 : 4; }

void state_layout(mg_particles_s* p) {
  const int64_t n = p->n;
  unsigned char* b = static_cast<unsigned char*>(p->state.p);
  size_t o = 0;
  p->sv.edge = reinterpret_cast<int32_t*>(b + o);
  o = a256(o + 4 * (size_t)n);
  p->sv.x = b + o;
  o = a256(o + xbytes(p) * (size_t)n);
  p->sv.n_draw = reinterpret_cast<uint32_t*>(b + o);
  o = a256(o + 4 * (size_t)n);
  // hits and first_hits are adjacent: 8n contiguous bytes, 8-byte aligned,
  // reused as the binary64 staging area of host positions at initialisation
  p->sv.hits = reinterpret_cast<uint32_t*>(b + o);
  p->sv.first_hits = p->sv.hits + n;
  o = a256(o + 8 * (size_t)n);
  p->sv.flags = reinterpret_cast<uint32_t*>(b + o);
}

size_t state_bytes(int64_t n, size_t xb) {
  return a256(4 * (size_t)n) + a256(xb * (size_t)n) + a256(4 * (size_t)n) + a256(8 * (size_t)n) +
         a256(4 * (size_t)n);
}

void counter_layout(mg_particles_s* p) {
  unsigned char* b = static_cast<unsigned char*>(p->counters.p);
  size_t o = 0;
  p->cv.exits = reinterpret_cast<unsigned long long*>(b + o);
  o += 8 * (size_t)p->g->S;
  p->cv.absorbed = reinterpret_cast<unsigned long long*>(b + o);
  o += 8 * (size_t)p->g->V;
  p->cv.trunc = reinterpret_cast<unsigned long long*>(b + o);
  o += 8;
  p->cv.psteps = reinterpret_cast<unsigned long long*>(b + o);
  o += 8;
  p->cv.err = reinterpret_cast<uint32_t*>(b + o);
}

size_t counter_bytes(const mg_graph g) { return 8 * ((size_t)g->S + g->V + 2) + 16; }

// First index i in [0, n) with bad(i), or n.  Large ranges are split over
// the host's cores (checking 2^24 starting positions on one core takes about
// 15 ms, 4% of a 10^4-step launch); if threads cannot be had, one core.
template <class F>
int64_t first_bad(int64_t n, const F& bad) {
  constexpr int64_t kPerThread = 1 << 18;
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t T = std::min<int64_t>(std::min<int64_t>(hw ? hw : 1, 32), n / kPerThread);
  if (T > 1) {
    std::vector<int64_t> found((size_t)T, n);
    std::vector<std::thread> pool;
    bool ok = true;
    try {
      for (int64_t t = 0; t < T; ++t)
        pool.emplace_back([&, t] {
          const int64_t lo = n * t / T, hi = n * (t + 1) / T;
          for (int64_t i = lo; i < hi; ++i)
            if (bad(i)) {
              found[(size_t)t] = i;
              return;
            }
        });
    } catch (...) {
      ok = false;  // fewer threads than asked: finish on this one
    }
    for (auto& th : pool) th.join();
    if (ok) return *std::min_element(found.begin(), found.end());
  }
  for (int64_t i = 0; i < n; ++i)
    if (bad(i)) return i;
  return n;
}

// Starting edges and positions given in host memory are checked here (those
// in device memory by the init kernel, which sets the device error word).
mg_status check_positions(mg_particles p, const int32_t* edge0, const double* x0, int on_device) {
  if (!edge0 || !x0) return fail(MG_ERR_INVALID_ARG, "edge0 and x0 are required");
  const Mem want = on_device ? Mem::kDevice : Mem::kHost;
  mg_status s = check_memory(edge0, want, "edge0");
  if (s == MG_OK) s = check_memory(x0, want, "x0");
  if (s != MG_OK || on_device) return s;
  const mg_graph g = p->g;
  const double* len = g->length.data();
  const int32_t E = g->E;
  const int64_t i = first_bad(p->n, [&](int64_t k) {
    const int32_t e = edge0[k];
    if (e < 0 || e >= E) return true;
    const double x = x0[k];
    return !(x >= 0.0 && x <= len[e] && std::isfinite(x));
  });
  if (i == p->n) return MG_OK;
  const int32_t e = edge0[i];
  if (e < 0 || e >= E)
    return fail(MG_ERR_INVALID_ARG, "particle %lld: edge %d out of range", (long long)i, e);
  return fail(MG_ERR_INVALID_ARG, "particle %lld: x0 outside [0, l_e] or not finite",
              (long long)i);
}

// Uploads checked starting positions and launches the init kernels.  Host
// arrays have been copied when this returns (they may be pinned memory, which
// an asynchronous copy would still read later).
mg_status load_positions(mg_particles p, const int32_t* edge0, const double* x0, int on_device,
                         cudaStream_t st) {
  const int64_t n = p->n;
  const mg_graph g = p->g;
  const int32_t* dedge = edge0;
  const double* dx = x0;
  if (!on_device) {
    // edges straight into place; positions into the 8n bytes of hits and
    // first_hits (binary64 staging), converted by the init kernel
    MG_CUDA(cudaMemcpyAsync(p->sv.edge, edge0, 4 * (size_t)n, cudaMemcpyHostToDevice, st));
    MG_CUDA(cudaMemcpyAsync(p->sv.hits, x0, 8 * (size_t)n, cudaMemcpyHostToDevice, st));
    dedge = p->sv.edge;
    dx = reinterpret_cast<const double*>(p->sv.hits);
  }
  MG_CUDA(mg::launch_init_state(g->view, dedge, dx, n, p->prec == MG_FP64, p->sv, p->cv.err, st));
  if (!on_device) MG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_particles_init(mg_graph g, int64_t n, const int32_t* edge0,
                                       const double* x0, int inputs_on_device, uint32_t pid_base,
                                       uint64_t seed, uint32_t instance_id,
                                       mg_precision precision, void* stream, mg_particles* out) {
  if (!g || !out) return fail(MG_ERR_INVALID_ARG, "mg_particles_init: NULL argument");
  *out = nullptr;
  if (n < 1 || n > 2147483647LL) return fail(MG_ERR_INVALID_ARG, "need 1 <= n <= 2^31 - 1");
  if ((uint64_t)pid_base + (uint64_t)n > 4294967296ull)
    return fail(MG_ERR_INVALID_ARG, "pid_base + n exceeds 2^32");
  if (precision != MG_FP64 && precision != MG_FP32_MIXED && precision != MG_FP32)
    return fail(MG_ERR_INVALID_ARG, "unknown precision %d", (int)precision);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mg_particles p = new mg_particles_s();
  p->g = g;
  p->n = n;
  {
    mg_status c = check_positions(p, edge0, x0, inputs_on_device);
    if (c != MG_OK) {
      delete p;
      return c;
    }
  }
  p->pid_base = pid_base;
  p->seed = seed;
  p->instance = instance_id;
  p->prec = precision;
  mg_status s = dev_alloc(p->state, state_bytes(n, xbytes(p)), st);
  if (s == MG_OK) s = dev_alloc(p->counters, counter_bytes(g), st);
  if (s != MG_OK) {
    dev_free(p->state, st);
    delete p;
    return s;
  }
  state_layout(p);
  counter_layout(p);
  cudaError_t ce = cudaMemsetAsync(p->counters.p, 0, counter_bytes(g), st);
  if (ce != cudaSuccess) s = cuda_fail(ce, "mg_particles_init: memset");
  if (s == MG_OK) s = load_positions(p, edge0, x0, inputs_on_device, st);
  if (s != MG_OK) {
    dev_free(p->state, st);
    dev_free(p->counters, st);
    delete p;
    return s;
  }
  p->last_stream = st;
  g->refs++;
  *out = p;
  return MG_OK;
}

extern "C" mg_status mg_particles_reset(mg_particles p, const int32_t* edge0, const double* x0,
                                        int inputs_on_device, void* stream) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_particles_reset: NULL particles");
  mg_status s = check_positions(p, edge0, x0, inputs_on_device);  // before changing anything
  if (s != MG_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MG_CUDA(cudaMemsetAsync(p->counters.p, 0, counter_bytes(p->g), st));
  s = load_positions(p, edge0, x0, inputs_on_device, st);
  if (s != MG_OK) return s;
  p->step = 0;
  p->last_stream = st;
  return MG_OK;
}

extern "C" mg_status mg_particles_destroy(mg_particles p) {
  if (!p) return MG_OK;
  cudaStreamSynchronize(p->last_stream);
  dev_free(p->state, p->last_stream);
  dev_free(p->counters, p->last_stream);
  dev_free(p->hist_tmp, p->last_stream);
  dev_free(p->bins_tmp, p->last_stream);
  p->g->refs--;
  delete p;
  return MG_OK;
}

extern "C" mg_status mg_particles_info(mg_particles p, int64_t* n, int32_t* precision,
                                       uint64_t* step) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_particles_info: NULL particles");
  if (n) *n = p->n;
  if (precision) *precision = (int32_t)p->prec;
  if (step) *step = p->step;
  return MG_OK;
}

namespace {

// Dynamic shared memory the fused kernel may take per block beside its ring
// of normals (32 KB): the jump words (8 KB), then staged tables, counters and
// histogram (16 KB), so that four blocks of 256 threads -- the most the
// registers allow -- stay resident on an SM (4 x 56 KB of its 228 KB).
constexpr size_t kSmemBudget = 24 * 1024;

}  // namespace

extern "C" mg_status mg_particles_set_tuning(mg_particles p, int32_t split_batch,
                                             int64_t steps_per_launch, int32_t max_blocks) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_particles_set_tuning: NULL particles");
  if (split_batch < 0 || split_batch > 32)
    return fail(MG_ERR_INVALID_ARG, "split_batch must be in [0, 32]");
  if (steps_per_launch < 0) return fail(MG_ERR_INVALID_ARG, "steps_per_launch must be >= 0");
  if (max_blocks < 0) return fail(MG_ERR_INVALID_ARG, "max_blocks must be >= 0");
  p->split_batch = split_batch;
  p->steps_per_launch = steps_per_launch;
  p->max_blocks = max_blocks;
  return MG_OK;
}

namespace {

// Default number of pending lanes that triggers a batched split pass (a
// warp also resolves its pending lanes whenever no other lane can move).  A
// pass costs about the same whatever number of lanes it resolves, while a
// pending lane idles until it runs, so the best batch grows with the cost of
// a split.  Measured on the 16-edge Langevin star (2^24 particles, one GB300,
// particle-steps/s): FP32-mixed, whose binary64 root makes splits dear,
// 3.48e11 at 1, 3.72 at 4, 3.74 at 5, 3.70 at 6, 3.47 at 8; FP32 4.42e11 at
// 1, 4.49 at 3, 4.40 at 5; FP64 8.62e9 at 1, 8.74 at 2, 8.07 at 4.
int32_t default_split_batch(mg_precision prec) {
  switch (prec) {
    case MG_FP32: return 3;
    case MG_FP32_MIXED: return 5;
    default: return 2;
  }
}

}  // namespace

namespace {

mg::Keys keys_of(uint64_t seed) {
  mg::Keys k{};
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {
    k.rk[2 * r] = k0 + r * 0x9E3779B9u;
    k.rk[2 * r + 1] = k1 + r * 0xBB67AE85u;
  }
  return k;
}

// Per-set launch arguments and shared-memory plan: the normal ring always;
// then the tables (when their size is at most stage_limit), the counters and
// the histogram, as long as the total stays within the budget.
struct Plan {
  mg::SimArgs a{};
  bool f64 = false, stage = true, counters = true, shist = false;
  bool var = false;           // a kVarSigma kernel (stages the diffusion slopes too)
  int32_t hist_len = 0;
  int32_t counter_bytes = 4;  // 8 for the range kernel
  size_t smem(bool with_hist, const mg_graph g) const {
    return mg::smem_layout(g->V, g->E, g->S, g->view.G, f64, stage, counters,
                           (with_hist && shist) ? hist_len : 0, mg::kBlock, counter_bytes, var)
        .total;
  }
};

// The kernel mode of a set: its precision, plus kVarSigma when its graph has
// position-dependent diffusion.
int kernel_mode(mg_particles p) {
  return (int)p->prec | (p->g->var_sigma ? mg::kVarSigma : 0);
}

Plan plan_launch(mg_particles p, double dt, int32_t M, int32_t hist_bins, uint32_t* hist_out,
                 size_t stage_limit, int32_t split_batch, bool var) {
  const mg_graph g = p->g;
  Plan pl;
  pl.f64 = p->prec == MG_FP64;
  pl.var = var;
  mg::SimArgs& a = pl.a;
  a.g = g->view;
  a.s = p->sv;
  a.c = p->cv;
  a.n = p->n;
  a.range = mg::kBlock;
  a.pid_base = p->pid_base;
  a.instance = p->instance;
  a.dt = dt;
  a.sqrt_dt = std::sqrt(dt);
  a.dt_f = (float)a.dt;
  a.sqrt_dt_f = (float)a.sqrt_dt;
  a.M = M;
  a.split_batch = split_batch > 0 ? split_batch : default_split_batch(p->prec);
  a.hist_bins = hist_bins;
  a.hist = hist_out;
  pl.hist_len = hist_bins > 0 ? g->E * hist_bins : 0;
  pl.shist = hist_bins > 0;
  const size_t budget = kSmemBudget + 128u * mg::kBlock;  // + the normal ring
  const int32_t G = g->view.G;
  const size_t tables =
      mg::smem_layout(g->V, g->E, g->S, G, pl.f64, true, false, 0, mg::kBlock, 4, var).total -
      mg::smem_layout(g->V, g->E, g->S, G, pl.f64, false, false, 0, mg::kBlock, 4, var).total;
  if (tables > stage_limit) pl.stage = false;
  if (pl.smem(true, g) > budget) pl.shist = false;
  if (pl.smem(true, g) > budget) pl.counters = false;
  if (pl.smem(true, g) > budget) pl.stage = false;
  a.stage_smem = pl.stage;
  a.smem_counters = pl.counters;
  a.smem_hist = pl.shist;
  return pl;
}

// Most EM-Steps one launch may take: the kernel's loop guard, 32 steps
// (2M + 2) + 64, must fit 32 bits (and so does the per-lane step counter);
// with 32-bit shared counters in blocks of 256 particles, 2^32 / (256 (2M + 1))
// so that they cannot wrap.
int64_t max_steps_per_launch(int32_t M, bool smem_counters) {
  int64_t chunk = (int64_t)((4294967295ull - 64ull) / (32ull * (2ull * (uint64_t)M + 2ull)));
  if (smem_counters) {
    const int64_t cap = (int64_t)(4294967295ull / (256ull * (2ull * (uint64_t)M + 1ull)));
    if (chunk > cap) chunk = cap;
  }
  return chunk < 1 ? 1 : chunk;
}

// Particles per block of mg_simulate: 256 (one per thread, em_step_kernel),
// fewer for a set that cannot fill the GPU's resident blocks (see below),
// unless particles can die and the set is larger than the blocks resident at
// once (or max_blocks): then the set is spread evenly over those blocks and
// em_range_kernel's lanes claim the next particle when theirs dies or
// finishes, so no lane idles beside its warp's slowest particle.  On such
// graphs the particles' work is uneven even before many die (tracers near
// short edges split far more often), and with one split per lane per pass
// the range kernel is the faster at every launch length measured on the
// synthetic vascular network (2^24 tracers, binary32): range / tile
// throughput 1.30 at 16 EM-Steps per launch (4% absorbed), 1.21 at 128
// (19%), 1.21 at 250, 1.26 at 500, 1.57 at 1000, 2.06 at 2000 (81%);
// FP32-mixed 1.30 to 1.37 at 32 to 128.  An explicit max_blocks bounds its
// block count.
int64_t block_range(mg_particles p, size_t smem) {
  const int64_t tiles = (p->n + mg::kBlock - 1) / mg::kBlock;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  if (p->max_blocks == 0) {
    // one particle per thread; a set smaller than the resident blocks x 256
    // is spread over more blocks of fewer particles (a multiple of 32, at
    // least 32; the other threads idle), so that every SM gets work: the
    // warps are latency-bound, and one SM running eight of them is slower
    // than four SMs running two each
    const int per_sm = mg::em_step_blocks_per_sm(kernel_mode(p), smem);
    const int64_t slots = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
    if (tiles < slots) {
      const int64_t want = (p->n + slots - 1) / slots;
      return std::min<int64_t>(mg::kBlock, std::max<int64_t>(32, (want + 31) / 32 * 32));
    }
  }
  if (!p->g->has_absorbing) return mg::kBlock;
  const int per_sm = mg::em_range_blocks_per_sm(kernel_mode(p), smem);
  int64_t blocks = (int64_t)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  if (p->max_blocks > 0 && p->max_blocks < blocks) blocks = p->max_blocks;
  if (tiles <= blocks) return mg::kBlock;
  return (p->n + blocks - 1) / blocks;
}

mg_status check_step_args(double dt, int64_t steps, int32_t M, int32_t hist_bins,
                          const uint32_t* hist_out) {
  // the binary32 modes carry dt and the time left as normal binary32 numbers
  if (!(dt >= 1e-30 && dt <= 1e30)) return fail(MG_ERR_INVALID_ARG, "dt must be in [1e-30, 1e30]");
  if (steps < 0) return fail(MG_ERR_INVALID_ARG, "steps must be >= 0");
  if (M < 1 || M > 1024) return fail(MG_ERR_INVALID_ARG, "max_splits_M must be in [1, 1024]");
  if (hist_bins < 0) return fail(MG_ERR_INVALID_ARG, "hist_bins must be >= 0");
  if (hist_bins > 0 && !hist_out) return fail(MG_ERR_INVALID_ARG, "hist_bins > 0 needs hist_out");
  if (hist_bins > 0) return check_memory(hist_out, Mem::kDevice, "hist_out");
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_simulate(mg_particles p, double dt, int64_t steps, int32_t M,
                                 int32_t hist_bins, uint32_t* hist_out, void* stream) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_simulate: NULL particles");
  mg_status s = check_step_args(dt, steps, M, hist_bins, hist_out);
  if (s != MG_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mg_graph g = p->g;
  Plan pl = plan_launch(p, dt, M, hist_bins, hist_out, (size_t)-1, p->split_batch,
                        p->g->var_sigma);
  const mg::Keys keys = keys_of(p->seed);
  int64_t first = std::min(steps, max_steps_per_launch(M, false));
  if (p->steps_per_launch > 0) first = std::min(first, p->steps_per_launch);
  pl.a.range = block_range(p, pl.smem(true, g));
  if (pl.a.range > mg::kBlock) {  // blocks run many particles: 64-bit counters
    pl.counter_bytes = 8;
    if (pl.counters && pl.smem(true, g) > kSmemBudget + 128u * mg::kBlock) {
      pl.counters = false;
      pl.a.smem_counters = 0;
    }
  }
  int64_t chunk = max_steps_per_launch(M, pl.counters);
  if (p->steps_per_launch > 0 && p->steps_per_launch < chunk) chunk = p->steps_per_launch;
  int64_t done = 0;
  do {
    const int64_t now = (steps - done < chunk) ? steps - done : chunk;
    pl.a.steps = now;
    const bool last = done + now >= steps;
    pl.a.hist_bins = (last && hist_bins > 0) ? hist_bins : 0;
    pl.a.smem_hist = (last && pl.shist) ? 1 : 0;
    cudaError_t ce = mg::launch_em_step(kernel_mode(p), pl.a, keys, pl.smem(last, g), st);
    if (ce != cudaSuccess) return cuda_fail(ce, "mg_simulate: launch");
    done += now;
  } while (done < steps);
  p->step += (uint64_t)steps;
  p->last_stream = st;
  return MG_OK;
}

extern "C" mg_status mg_simulate_sampled(mg_particles p, double dt, int64_t steps, int32_t M,
                                         int64_t every, int32_t hist_bins, uint32_t* hist_out,
                                         void* stream) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_simulate_sampled: NULL particles");
  if (every < 1) return fail(MG_ERR_INVALID_ARG, "every must be >= 1");
  if (hist_bins < 1 || !hist_out)
    return fail(MG_ERR_INVALID_ARG, "mg_simulate_sampled needs hist_bins >= 1 and hist_out");
  mg_status s = check_step_args(dt, steps, M, hist_bins, hist_out);
  if (s != MG_OK) return s;
  const int64_t snaps = steps / every;
  for (int64_t k = 0; k < snaps; ++k) {
    s = mg_simulate(p, dt, every, M, hist_bins, hist_out, stream);
    if (s != MG_OK) return s;
  }
  const int64_t rest = steps - snaps * every;
  return rest > 0 ? mg_simulate(p, dt, rest, M, 0, nullptr, stream) : MG_OK;
}

// ------------------------------------------------------------------ batches

struct mg_batch_s {
  struct Member {
    mg_particles p;
    double dt;
    int64_t steps;
    int32_t M, hist_bins;
    uint32_t* hist;
  };
  std::vector<Member> members;
  bool have_seed = false;
  uint64_t seed = 0;
  mg_precision prec = MG_FP64;
  bool var = false;             // members need the position-dependent diffusion kernel
  int32_t split_batch = 0;      // 0: the precision's default
  int64_t stage_limit = -1;     // < 0: stage whatever fits the budget
  int32_t blocks_per_sm = 0;    // 0: occupancy maximum
  bool dirty = true;
  // device side (rebuilt when dirty)
  DevBuf buf;                   // SimArgs[n_inst] | BatchItem[n_items] | head
  mg::SimArgs* d_insts = nullptr;
  mg::BatchItem* d_items = nullptr;
  uint32_t* d_head = nullptr;
  int32_t n_items = 0;
  size_t smem = 0;
  int blocks = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
  cudaStream_t last_stream = nullptr;
};

namespace {

void batch_drop_graph(mg_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Builds the instance table and the work queue: one item per 256 particles,
// instances with more steps first (longest-processing-time order).
mg_status batch_build(mg_batch b, cudaStream_t st) {
  const size_t n_inst = b->members.size();
  std::vector<mg::SimArgs> insts(n_inst);
  std::vector<size_t> order(n_inst);
  size_t smem = 0;
  const size_t stage_limit = b->stage_limit < 0 ? (size_t)-1 : (size_t)b->stage_limit;
  // one kernel for all members: the position-dependent one if any member's
  // graph needs it (it gives bit-identical results for constant diffusion,
  // sigma_e + 0 x being sigma_e)
  b->var = false;
  for (const auto& mb : b->members) b->var = b->var || mb.p->g->var_sigma;
  for (size_t m = 0; m < n_inst; ++m) {
    const auto& mb = b->members[m];
    Plan pl = plan_launch(mb.p, mb.dt, mb.M, mb.hist_bins, mb.hist, stage_limit, b->split_batch,
                          b->var);
    pl.a.steps = mb.steps;
    insts[m] = pl.a;
    smem = std::max(smem, pl.smem(true, mb.p->g));
    if (mb.steps > max_steps_per_launch(mb.M, pl.counters))
      return fail(MG_ERR_INVALID_ARG, "mg_batch: member %zu takes more steps than one launch allows",
                  m);
    order[m] = m;
  }
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    return b->members[x].steps > b->members[y].steps;
  });
  std::vector<mg::BatchItem> items;
  for (size_t m : order) {
    if (b->members[m].steps == 0) continue;
    const int64_t tiles = (b->members[m].p->n + mg::kBlock - 1) / mg::kBlock;
    for (int64_t t = 0; t < tiles; ++t) items.push_back({(int32_t)m, (int32_t)t});
  }
  if (items.size() > 2147483647u) return fail(MG_ERR_INVALID_ARG, "mg_batch: too many work items");
  const size_t o_inst = 0, o_items = a256(n_inst * sizeof(mg::SimArgs));
  const size_t o_head = a256(o_items + items.size() * sizeof(mg::BatchItem));
  const size_t total = o_head + 256;
  if (b->buf.bytes < total) {
    dev_free(b->buf, st);
    mg_status s = dev_alloc(b->buf, total, st);
    if (s != MG_OK) return s;
  }
  unsigned char* base = static_cast<unsigned char*>(b->buf.p);
  b->d_insts = reinterpret_cast<mg::SimArgs*>(base + o_inst);
  b->d_items = reinterpret_cast<mg::BatchItem*>(base + o_items);
  b->d_head = reinterpret_cast<uint32_t*>(base + o_head);
  MG_CUDA(cudaMemcpyAsync(b->d_insts, insts.data(), n_inst * sizeof(mg::SimArgs),
                          cudaMemcpyHostToDevice, st));
  if (!items.empty())
    MG_CUDA(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(mg::BatchItem),
                            cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaStreamSynchronize(st));  // the host vectors go out of scope
  b->n_items = (int32_t)items.size();
  b->smem = smem;
  int per_sm = mg::em_batch_blocks_per_sm((int)b->prec | (b->var ? mg::kVarSigma : 0), smem);
  if (per_sm < 1) return fail(MG_ERR_INVALID_ARG, "mg_batch: the kernel does not fit an SM");
  if (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) per_sm = b->blocks_per_sm;
  int dev = 0, sms = 0;
  MG_CUDA(cudaGetDevice(&dev));
  MG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  b->blocks = std::max(1, std::min(per_sm * sms, b->n_items));
  b->dirty = false;
  return MG_OK;
}

mg_status batch_enqueue(mg_batch b, cudaStream_t st) {
  MG_CUDA(cudaMemsetAsync(b->d_head, 0, 4, st));
  if (b->n_items > 0) {
    cudaError_t ce = mg::launch_em_batch((int)b->prec | (b->var ? mg::kVarSigma : 0), b->d_insts,
                                         b->d_items, b->n_items, b->d_head,
                                         keys_of(b->seed), b->smem, b->blocks, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "mg_batch_run: launch");
  }
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_batch_create(mg_batch* out) {
  if (!out) return fail(MG_ERR_INVALID_ARG, "mg_batch_create: NULL argument");
  *out = new mg_batch_s();
  return MG_OK;
}

extern "C" mg_status mg_batch_add(mg_batch b, mg_particles p, double dt, int64_t steps, int32_t M,
                                  int32_t hist_bins, uint32_t* hist_out) {
  if (!b || !p) return fail(MG_ERR_INVALID_ARG, "mg_batch_add: NULL argument");
  mg_status s = check_step_args(dt, steps, M, hist_bins, hist_out);
  if (s != MG_OK) return s;
  if (b->members.empty()) {
    b->seed = p->seed;
    b->prec = p->prec;
  } else {
    if (p->seed != b->seed) return fail(MG_ERR_INVALID_ARG, "mg_batch_add: members share one seed");
    if (p->prec != b->prec) return fail(MG_ERR_INVALID_ARG, "mg_batch_add: members share one precision");
  }
  for (const auto& m : b->members)
    if (m.p == p) return fail(MG_ERR_INVALID_ARG, "mg_batch_add: a particle set is already a member");
  b->members.push_back({p, dt, steps, M, hist_bins, hist_out});
  b->dirty = true;
  return MG_OK;
}

extern "C" mg_status mg_batch_clear(mg_batch b) {
  if (!b) return fail(MG_ERR_INVALID_ARG, "mg_batch_clear: NULL batch");
  b->members.clear();
  b->dirty = true;
  return MG_OK;
}

extern "C" mg_status mg_batch_set_tuning(mg_batch b, int32_t split_batch, int64_t stage_limit_bytes,
                                         int32_t blocks_per_sm) {
  if (!b) return fail(MG_ERR_INVALID_ARG, "mg_batch_set_tuning: NULL batch");
  if (split_batch < 0 || split_batch > 32 || blocks_per_sm < 0)
    return fail(MG_ERR_INVALID_ARG, "mg_batch_set_tuning: split_batch in [0, 32], blocks_per_sm >= 0");
  b->split_batch = split_batch;
  b->stage_limit = stage_limit_bytes;
  b->blocks_per_sm = blocks_per_sm;
  b->dirty = true;
  return MG_OK;
}

extern "C" mg_status mg_batch_run(mg_batch b, int use_graph, void* stream) {
  if (!b) return fail(MG_ERR_INVALID_ARG, "mg_batch_run: NULL batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (use_graph && st == nullptr)
    return fail(MG_ERR_INVALID_ARG, "mg_batch_run: graph replay needs a non-default stream");
  if (b->dirty) {
    batch_drop_graph(b);
    mg_status s = batch_build(b, st);
    if (s != MG_OK) return s;
  }
  if (use_graph) {
    if (!b->exec || b->graph_stream != st) {
      batch_drop_graph(b);
      MG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      mg_status s = batch_enqueue(b, st);
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (s != MG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "mg_batch_run: capture");
      b->graph = graph;
      MG_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
      b->graph_stream = st;
    }
    MG_CUDA(cudaGraphLaunch(b->exec, st));
  } else {
    mg_status s = batch_enqueue(b, st);
    if (s != MG_OK) return s;
  }
  for (auto& m : b->members) {
    m.p->step += (uint64_t)m.steps;
    m.p->last_stream = st;
  }
  b->last_stream = st;
  return MG_OK;
}

extern "C" mg_status mg_batch_info(mg_batch b, int32_t* n_members, int32_t* n_items,
                                   int32_t* blocks) {
  if (!b) return fail(MG_ERR_INVALID_ARG, "mg_batch_info: NULL batch");
  if (n_members) *n_members = (int32_t)b->members.size();
  if (n_items) *n_items = b->n_items;
  if (blocks) *blocks = b->blocks;
  return MG_OK;
}

extern "C" mg_status mg_batch_destroy(mg_batch b) {
  if (!b) return MG_OK;
  cudaStreamSynchronize(b->last_stream);
  batch_drop_graph(b);
  dev_free(b->buf, b->last_stream);
  delete b;
  return MG_OK;
}

extern "C" mg_status mg_synchronize(mg_particles p) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_synchronize: NULL particles");
  MG_CUDA(cudaStreamSynchronize(p->last_stream));
  uint32_t err = 0;
  MG_CUDA(cudaMemcpy(&err, p->cv.err, 4, cudaMemcpyDeviceToHost));
  if (err) {
    MG_CUDA(cudaMemset(p->cv.err, 0, 4));
    return fail(MG_ERR_DEVICE_FAULT, "device error bits 0x%x (1: edge out of range, 2: position "
                "outside [0, l_e] or NaN, 4: random stream exhausted, 8: loop guard)", err);
  }
  return MG_OK;
}

extern "C" mg_status mg_histogram(mg_particles p, int32_t bins, uint32_t* out, int out_on_device,
                                  void* stream) {
  if (!p || !out) return fail(MG_ERR_INVALID_ARG, "mg_histogram: NULL argument");
  if (bins < 1) return fail(MG_ERR_INVALID_ARG, "bins must be >= 1");
  {
    mg_status s = check_memory(out, out_on_device ? Mem::kDevice : Mem::kHost, "out");
    if (s != MG_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mg_graph g = p->g;
  const size_t bytes = (size_t)g->E * bins * 4;
  uint32_t* dst = out;
  if (!out_on_device) {
    if (p->hist_tmp.bytes < bytes) {
      dev_free(p->hist_tmp, st);
      mg_status s = dev_alloc(p->hist_tmp, bytes, st);
      if (s != MG_OK) return s;
    }
    dst = static_cast<uint32_t*>(p->hist_tmp.p);
  }
  MG_CUDA(cudaMemsetAsync(dst, 0, bytes, st));
  const bool sm = bytes <= 96 * 1024;
  cudaError_t ce = (p->prec == MG_FP64)
                       ? mg::launch_histogram_f64(g->view, p->sv.edge, p->sv.x, p->n, bins, dst, sm, st)
                       : mg::launch_histogram_f32(g->view, p->sv.edge, p->sv.x, p->n, bins, dst, sm, st);
  if (ce != cudaSuccess) return cuda_fail(ce, "mg_histogram: launch");
  p->last_stream = st;
  if (!out_on_device) MG_CUDA(copy_to_host(out, dst, bytes, st));
  return MG_OK;
}

extern "C" mg_status mg_histogram_binned(mg_particles p, const int32_t* bin_offsets,
                                         const double* bin_upper, uint32_t* out,
                                         int out_on_device, void* stream) {
  if (!p || !bin_offsets || !out)
    return fail(MG_ERR_INVALID_ARG, "mg_histogram_binned: NULL argument");
  {
    mg_status s = check_host({{bin_offsets, "bin_offsets"}, {bin_upper, "bin_upper"}});
    if (s == MG_OK) s = check_memory(out, out_on_device ? Mem::kDevice : Mem::kHost, "out");
    if (s != MG_OK) return s;
  }
  const mg_graph g = p->g;
  if (bin_offsets[0] != 0) return fail(MG_ERR_INVALID_ARG, "bin_offsets[0] must be 0");
  for (int32_t e = 0; e < g->E; ++e)
    if (bin_offsets[e + 1] < bin_offsets[e])
      return fail(MG_ERR_INVALID_ARG, "bin_offsets must be non-decreasing (edge %d)", e);
  const int32_t nb = bin_offsets[g->E];
  if (nb > 0 && !bin_upper) return fail(MG_ERR_INVALID_ARG, "mg_histogram_binned: NULL bin_upper");
  for (int32_t e = 0; e < g->E; ++e)
    for (int32_t j = bin_offsets[e]; j < bin_offsets[e + 1]; ++j) {
      const double u = bin_upper[j];
      const double prev = (j == bin_offsets[e]) ? 0.0 : bin_upper[j - 1];
      if (!(std::isfinite(u) && u > prev))
        return fail(MG_ERR_INVALID_ARG,
                    "edge %d: bin boundaries must be finite, > 0 and increasing (bin %d)", e, j);
    }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool f64 = p->prec == MG_FP64;
  // device tables: offsets, then boundaries in the state's precision
  // (binary32: the smallest binary32 >= the boundary)
  std::vector<unsigned char> host;
  const size_t o_up = a256((size_t)(g->E + 1) * 4);
  const size_t tbytes = o_up + (size_t)nb * (f64 ? 8 : 4) + 16;
  host.assign(tbytes, 0);
  memcpy(host.data(), bin_offsets, (size_t)(g->E + 1) * 4);
  for (int32_t j = 0; j < nb; ++j) {
    if (f64) {
      memcpy(host.data() + o_up + 8 * (size_t)j, &bin_upper[j], 8);
    } else {
      float f = (float)bin_upper[j];
      if ((double)f < bin_upper[j]) f = std::nextafter(f, INFINITY);
      memcpy(host.data() + o_up + 4 * (size_t)j, &f, 4);
    }
  }
  const size_t obytes = (size_t)(nb > 0 ? nb : 1) * 4;
  const size_t need = a256(tbytes) + (out_on_device ? 0 : a256(obytes));
  if (p->bins_tmp.bytes < need) {
    dev_free(p->bins_tmp, st);
    mg_status s = dev_alloc(p->bins_tmp, need, st);
    if (s != MG_OK) return s;
  }
  unsigned char* base = static_cast<unsigned char*>(p->bins_tmp.p);
  uint32_t* dst = out_on_device ? out : reinterpret_cast<uint32_t*>(base + a256(tbytes));
  MG_CUDA(cudaMemcpyAsync(base, host.data(), tbytes, cudaMemcpyHostToDevice, st));
  if (nb > 0) {
    MG_CUDA(cudaMemsetAsync(dst, 0, (size_t)nb * 4, st));
    cudaError_t ce = mg::launch_histogram_binned(f64, p->sv.edge, p->sv.x, p->n,
                                                 reinterpret_cast<const int32_t*>(base),
                                                 base + o_up, nb, dst, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "mg_histogram_binned: launch");
  }
  p->last_stream = st;
  if (!out_on_device) {
    if (nb > 0) MG_CUDA(cudaMemcpyAsync(out, dst, (size_t)nb * 4, cudaMemcpyDeviceToHost, st));
  }
  // the host table must outlive the upload
  MG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

extern "C" mg_status mg_exit_counts(mg_particles p, uint64_t* slot_exits, uint64_t* absorbed,
                                    uint64_t* truncations, uint64_t* particle_steps, void* stream) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_exit_counts: NULL particles");
  {
    mg_status s = check_host({{slot_exits, "slot_exits"}, {absorbed, "absorbed"},
                              {truncations, "truncations"}, {particle_steps, "particle_steps"}});
    if (s != MG_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mg_graph g = p->g;
  const size_t nw = (size_t)g->S + g->V + 2;
  std::vector<uint64_t> fallback;
  uint64_t* h = static_cast<uint64_t*>(g_stage.get(8 * nw));  // pinned, else ordinary
  if (!h) {
    fallback.resize(nw);
    h = fallback.data();
  }
  MG_CUDA(cudaMemcpyAsync(h, p->counters.p, 8 * nw, cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  if (slot_exits) memcpy(slot_exits, h, 8 * (size_t)g->S);
  if (absorbed) memcpy(absorbed, h + g->S, 8 * (size_t)g->V);
  if (truncations) *truncations = h[g->S + g->V];
  if (particle_steps) *particle_steps = h[g->S + g->V + 1];
  return MG_OK;
}

extern "C" mg_status mg_counters_reset(mg_particles p, void* stream) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_counters_reset: NULL particles");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MG_CUDA(cudaMemsetAsync(p->counters.p, 0, 8 * ((size_t)p->g->S + p->g->V + 2), st));
  p->last_stream = st;
  return MG_OK;
}

extern "C" mg_status mg_state_get(mg_particles p, int32_t* edge, double* x, uint32_t* n_draw,
                                  uint32_t* hits, uint32_t* first_hits, uint32_t* flags,
                                  uint64_t* step, void* stream) {
  if (!p) return fail(MG_ERR_INVALID_ARG, "mg_state_get: NULL particles");
  {
    mg_status s = check_host({{edge, "edge"}, {x, "x"}, {n_draw, "n_draw"}, {hits, "hits"},
                              {first_hits, "first_hits"}, {flags, "flags"}, {step, "step"}});
    if (s != MG_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)p->n;
  if (edge) MG_CUDA(cudaMemcpyAsync(edge, p->sv.edge, 4 * n, cudaMemcpyDeviceToHost, st));
  std::vector<float> xf;
  if (x) {
    if (p->prec == MG_FP64) {
      MG_CUDA(cudaMemcpyAsync(x, p->sv.x, 8 * n, cudaMemcpyDeviceToHost, st));
    } else {
      xf.resize(n);
      MG_CUDA(cudaMemcpyAsync(xf.data(), p->sv.x, 4 * n, cudaMemcpyDeviceToHost, st));
    }
  }
  if (n_draw) MG_CUDA(cudaMemcpyAsync(n_draw, p->sv.n_draw, 4 * n, cudaMemcpyDeviceToHost, st));
  if (hits) MG_CUDA(cudaMemcpyAsync(hits, p->sv.hits, 4 * n, cudaMemcpyDeviceToHost, st));
  if (first_hits)
    MG_CUDA(cudaMemcpyAsync(first_hits, p->sv.first_hits, 4 * n, cudaMemcpyDeviceToHost, st));
  if (flags) MG_CUDA(cudaMemcpyAsync(flags, p->sv.flags, 4 * n, cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  if (x && p->prec != MG_FP64)
    for (size_t i = 0; i < n; ++i) x[i] = (double)xf[i];
  if (step) *step = p->step;
  return MG_OK;
}

extern "C" mg_status mg_state_set(mg_particles p, const int32_t* edge, const double* x,
                                  const uint32_t* n_draw, const uint32_t* hits,
                                  const uint32_t* first_hits, const uint32_t* flags,
                                  uint64_t step, void* stream) {
  if (!p || !edge || !x || !n_draw || !hits || !first_hits || !flags)
    return fail(MG_ERR_INVALID_ARG, "mg_state_set: NULL argument");
  {
    mg_status s = check_host({{edge, "edge"}, {x, "x"}, {n_draw, "n_draw"}, {hits, "hits"},
                              {first_hits, "first_hits"}, {flags, "flags"}});
    if (s != MG_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)p->n;
  const mg_graph g = p->g;
  {
    const double* len = g->length.data();
    const int32_t E = g->E;
    const int64_t i = first_bad((int64_t)n, [&](int64_t k) {
      const int32_t e = edge[k];
      if (e < -1 || e >= E) return true;
      return e >= 0 && !(x[k] >= 0.0 && x[k] <= len[e] && std::isfinite(x[k]));
    });
    if (i < (int64_t)n) {
      if (edge[i] < -1 || edge[i] >= E)
        return fail(MG_ERR_INVALID_ARG, "particle %lld: edge out of range", (long long)i);
      return fail(MG_ERR_INVALID_ARG, "particle %lld: x outside [0, l_e]", (long long)i);
    }
  }
  std::vector<float> xf;
  MG_CUDA(cudaMemcpyAsync(p->sv.edge, edge, 4 * n, cudaMemcpyHostToDevice, st));
  if (p->prec == MG_FP64) {
    MG_CUDA(cudaMemcpyAsync(p->sv.x, x, 8 * n, cudaMemcpyHostToDevice, st));
  } else {
    xf.resize(n);
    for (size_t i = 0; i < n; ++i) xf[i] = (float)x[i];
    MG_CUDA(cudaMemcpyAsync(p->sv.x, xf.data(), 4 * n, cudaMemcpyHostToDevice, st));
  }
  MG_CUDA(cudaMemcpyAsync(p->sv.n_draw, n_draw, 4 * n, cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaMemcpyAsync(p->sv.hits, hits, 4 * n, cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaMemcpyAsync(p->sv.first_hits, first_hits, 4 * n, cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaMemcpyAsync(p->sv.flags, flags, 4 * n, cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaStreamSynchronize(st));
  p->step = step;
  p->last_stream = st;
  return MG_OK;
}

extern "C" mg_status mg_hit_root(int32_t mode, int64_t n, const float* A, const float* B,
                                 const float* C, double* s, void* stream) {
  if (mode != MG_FP64 && mode != MG_FP32_MIXED && mode != MG_FP32)
    return fail(MG_ERR_INVALID_ARG, "mg_hit_root: unknown precision mode %d", (int)mode);
  if (n < 0) return fail(MG_ERR_INVALID_ARG, "mg_hit_root: n < 0");
  if (n == 0) return MG_OK;
  if (!A || !B || !C || !s) return fail(MG_ERR_INVALID_ARG, "mg_hit_root: NULL argument");
  for (const auto& q : {std::pair<const void*, const char*>{A, "A"}, {B, "B"}, {C, "C"}, {s, "s"}}) {
    mg_status st = check_memory(q.first, Mem::kDevice, q.second);
    if (st != MG_OK) return st;
  }
  cudaError_t ce =
      mg::launch_hit_root(mode, n, A, B, C, s, static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess) return cuda_fail(ce, "mg_hit_root: launch");
  return MG_OK;
}

extern "C" const char* mg_last_error(void) { return g_err.c_str(); }

extern "C" const char* mg_version(void) { return "libmetricgraph 0.1 (sm_103a)"; }

// Read-only view of a particle set for other translation units of the
// library (the positions, edges and graph tables a kernel reads).
bool mg_particles_view(mg_particles p, mg::GraphView* g, const int32_t** edge, const void** x,
                       int64_t* n, int* precision) {
  if (!p) return false;
  *g = p->g->view;
  *edge = p->sv.edge;
  *x = p->sv.x;
  *n = p->n;
  *precision = (int)p->prec;
  return true;
}

// Records an error message from another translation unit of the library.
mg_status mg_fail_message(mg_status st, const char* msg) { return fail(st, "%s", msg); }
