// mg_types.h -- device-side table layouts shared by the host builder and the
// kernels of libmetricgraph (not part of the public C ABI).
#pragma once
#include <cstddef>
#include <cstdint>

#if defined(__CUDACC__)
#define MG_HD __host__ __device__
#else
#define MG_HD
#endif

namespace mg {

enum : int32_t { kEndInit = 0, kEndTerm = 1, kDead = -1 };
enum : int32_t { kVertexStandard = 0, kVertexAbsorbing = 1 };
// device-error bits (same values as MG_DEVERR_* in the public header)
enum : uint32_t { kErrBadEdge = 1u, kErrNan = 2u, kErrStream = 4u, kErrStuck = 8u };
// threads per block of the fused kernel
constexpr int kThreads = 256;
// precision modes (same values as mg_precision)
enum : int { kModeF64 = 0, kModeMixed = 1, kModeF32 = 2 };
// A kernel's mode argument is a precision mode, plus kVarSigma for graphs
// with position-dependent diffusion sigma_e(x) = sigma_e + sigma1_e x.
constexpr int kVarSigma = 4;
MG_HD constexpr int prec_of(int mode) { return mode & 3; }
MG_HD constexpr bool var_sigma(int mode) { return (mode & kVarSigma) != 0; }

// One edge (Definition 1) with its drift mu_e(x) = c0 + c1 x and diffusion
// sigma_e; 32 bytes so a warp loads it with one 16-byte pair per lane.
struct alignas(16) EdgeRec32 {
  float L, c0, c1, sigma;               // L = +inf for a semi-infinite edge
  int32_t src, dst, slot_init, slot_term; // dst = -1: vertex at infinity
};

struct alignas(16) EdgeRec64 {
  double L, c0, c1, sigma;
  int32_t src, dst, slot_init, slot_term;
};

// One (vertex, incident edge end) with its integer jump threshold T in
// [0, 2^32]: slot j of v is drawn when u < T_j and u >= T_{j-1}.  Stored as
// tm1 = T - 1 (so u < T is u <= tm1 in 32 bits); slots with T = 0 (zero
// weight ahead of every positive one) hold 0 and are never compared, since
// the guide table below never points at them.
struct alignas(16) SlotRec {
  uint32_t tm1;
  int32_t edge, end, pad;
};

// Slots of vertex v are [begin, end); kind is mg_vertex_kind.  guide: offset
// of v's guide table (Chen and Asau, 1974) of 2^gb entries, gb the smallest
// with 2^gb >= end - begin: entry k is the first slot j with T_j > k 2^(32-gb),
// so the slot drawn by u is found by a forward scan from entry u >> (32 - gb).
struct alignas(16) VtxRec {
  int32_t begin, end, kind, guide;
};

// Read-only view of a graph on the device (global memory, or shared memory
// after staging).
struct GraphView {
  int32_t V, E, S, G;  // G: guide table entries of all vertices
  const EdgeRec32* e32;
  const EdgeRec64* e64;
  const SlotRec* slot;
  const VtxRec* vtx;
  const int32_t* guide;
  const double* range;  // histogram range per edge
  const float* s1_32;   // diffusion slope sigma1_e per edge (zeros for constant sigma)
  const double* s1_64;
};

// Particle state, structure of arrays.
struct StateView {
  int32_t* edge;
  void* x;  // float* (binary32 modes) or double* (binary64)
  uint32_t* n_draw;  // normals used so far
  uint32_t* hits;
  uint32_t* first_hits;
  uint32_t* flags;
};

struct CounterView {
  unsigned long long* exits;     // [S]
  unsigned long long* absorbed;  // [V]
  unsigned long long* trunc;     // [1]
  unsigned long long* psteps;    // [1] particle-steps taken while alive
  uint32_t* err;                 // [1] device-error bits
};

// Philox round keys of a seed: (seed lo + r W0, seed hi + r W1), r = 0..9.
struct Keys {
  uint32_t rk[20];
};

// One particle set's share of a launch of the fused EM-Step kernel (the
// whole launch for mg_simulate, one instance of a batch otherwise).
struct SimArgs {
  GraphView g;
  StateView s;
  CounterView c;
  int64_t n;
  uint32_t pid_base;
  uint32_t instance;
  int64_t steps;
  double dt, sqrt_dt;
  float dt_f, sqrt_dt_f;  // the same rounded to binary32 (binary32 coefficients)
  int32_t M;
  int32_t hist_bins;    // 0: no fused histogram
  uint32_t* hist;       // [E * hist_bins]
  int32_t split_batch;  // pending lanes that trigger a batched split pass
  int32_t stage_smem;   // graph tables staged in shared memory
  int32_t smem_counters;// exit/absorbed counters privatised in shared memory
  int32_t smem_hist;    // histogram privatised in shared memory
  int64_t range;        // particles per block: <= 256 em_step_kernel, > 256 the range kernel
};

// Dynamic shared memory of the fused kernel: the ring of buffered normals
// and the jump words of each thread, then staged tables (with the diffusion
// slopes for kVarSigma kernels), privatised counters and the privatised
// histogram (each of these three optional).
struct SmemLayout {
  size_t ring, jump, edges, slots, vtx, guide, sig1, exits, absorbed, hist, total;
};

MG_HD inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

MG_HD inline SmemLayout smem_layout(int32_t V, int32_t E, int32_t S, int32_t G, bool f64,
                                    bool stage, bool counters, int32_t hist_len, int32_t block,
                                    int32_t counter_bytes = 4, bool var = false) {
  SmemLayout l{};
  size_t off = 0;
  l.ring = off;  // buffered normals, each stored twice: 32 KB at 256 threads
  off += align16((size_t)(f64 ? 16 : 32) * block * (f64 ? 8 : 4));
  l.jump = off;  // the jump draws of two Philox blocks, 8 words per thread (right after the ring)
  off += align16((size_t)8 * block * 4);
  if (stage) {
    l.edges = off; off += align16((size_t)E * (f64 ? sizeof(EdgeRec64) : sizeof(EdgeRec32)));
    l.slots = off; off += align16((size_t)S * sizeof(SlotRec));
    l.vtx = off; off += align16((size_t)V * sizeof(VtxRec));
    l.guide = off; off += align16((size_t)G * sizeof(int32_t));
    if (var) { l.sig1 = off; off += align16((size_t)E * (f64 ? 8 : 4)); }
  }
  if (counters) {  // 4-byte (tiles) or 8-byte (range kernel) counters
    l.exits = off; off += align16((size_t)S * counter_bytes);
    l.absorbed = off; off += align16((size_t)V * counter_bytes);
  }
  l.hist = off;
  off += align16((size_t)hist_len * 4);
  l.total = off;
  return l;
}

// A work item of the batched kernel: 256 particles (one block) of an
// instance, from particle tile * kThreads on.
struct BatchItem {
  int32_t inst;
  int32_t tile;
};

}  // namespace mg
