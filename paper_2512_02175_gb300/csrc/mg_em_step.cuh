// mg_em_step.cuh -- the fused EM-Step kernel of libmetricgraph.
//
// One thread advances one particle (edge e, position x) through many
// EM-Steps of the timestep-splitting Euler-Maruyama scheme ("Sampling on
// Metric Graphs", Algorithms 1 and 2), keeping the particle in registers for
// the whole launch (Section 3.1: state in registers, global memory only for
// the ensemble statistics).  Per step:
//
//   fast path  one Euler-Maruyama sub-step x + mu_e(x) dt + sigma_e sqrt(dt) W
//              that stays inside (0, l_e): two FMAs and two compares, with W
//              from a Philox-4x32-10 block shared by four consecutive steps.
//   slow path  the sub-step leaves the edge (or starts at a vertex): solve for
//              the hitting fraction alpha, keep (1 - alpha) h, draw the next
//              edge from b_v with an integer threshold table, restart from the
//              vertex with |W| into the new edge, repeat up to M times.
//
// Counters (exits per slot, absorptions, truncations) and the optional
// snapshot histogram are privatised in shared memory when they fit and
// flushed with one atomic per nonzero entry per block.
//
// Precision: kF64 = true computes everything in binary64 in the same order as
// the plain CPU reference (the translation unit is built without FMA
// contraction); kF64 = false keeps positions, increments and normals in
// binary32 and only the hitting fraction and remaining time in binary64.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "mg_types.h"

namespace mg {

// ------------------------------------------------------------------ Philox

struct U4 {
  uint32_t x, y, z, w;
};

// Philox-4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As
// Easy as 1, 2, 3" (SC'11).  Ten rounds; round keys rk[2r], rk[2r+1] are the
// key plus r times the Weyl increments, precomputed on the host.
__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            const uint32_t* __restrict__ rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
    const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// ------------------------------------------------------------- Box-Muller

// binary64: u = (2w + 1) 2^-33, r = sqrt(-2 ln u_a), theta = 2 pi u_b.
__device__ __forceinline__ double u01_f64(uint32_t w) {
  return ((double)w * 2.0 + 1.0) * 0x1p-33;
}
__device__ __forceinline__ void box_muller_f64(uint32_t wa, uint32_t wb, double& zc, double& zs) {
  const double ua = u01_f64(wa), ub = u01_f64(wb);
  const double r = sqrt(-2.0 * log(ua));
  const double th = 6.283185307179586 * ub;
  double s, c;
  sincos(th, &s, &c);
  zc = r * c;
  zs = r * s;
}

// binary32: u = (2 (w >> 9) + 1) 2^-24, formed exactly from the top 23 bits
// (1 + m 2^-23 minus 1 - 2^-24), so the FP32 and FP64 modes see the same
// words.  cos(2 pi u) = -cos(2 pi u - pi) keeps the hardware sine/cosine on
// (-pi, pi).  lg2/sqrt/sin/cos are the approximate hardware instructions.
__device__ __forceinline__ float u01_f32(uint32_t w) {
  return __uint_as_float((w >> 9) | 0x3f800000u) - 0.99999994f;
}
__device__ __forceinline__ void box_muller_f32(uint32_t wa, uint32_t wb, float& zc, float& zs) {
  const float ua = u01_f32(wa), ub = u01_f32(wb);
  const float r2 = -1.38629436112f * __log2f(ua);  // -2 ln u
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
  const float th = fmaf(ub, 6.28318530718f, -3.14159265359f);
  float s, c;
  __sincosf(th, &s, &c);
  zc = -r * c;
  zs = -r * s;
}

template <bool kF64>
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb,
                                           std::conditional_t<kF64, double, float>& zc,
                                           std::conditional_t<kF64, double, float>& zs) {
  if constexpr (kF64) box_muller_f64(wa, wb, zc, zs);
  else box_muller_f32(wa, wb, zc, zs);
}

// ---------------------------------------------------- hitting-fraction root

// First root s in [0, 1] of A s^2 + B s + C = 0 with C >= 0 (s = sqrt(alpha)
// of the partial step): A = 0 gives -C/B; otherwise (-B - d)/(2A) for B > 0
// and the equal 2C/(-B + d) for B <= 0, each free of cancellation on its
// side; d = sqrt(max(B^2 - 4AC, 0)); the result is clamped to [0, 1].
__device__ __forceinline__ double hit_root(double A, double B, double C) {
  double s;
  if (A == 0.0) {
    s = (B == 0.0) ? 0.0 : -C / B;
  } else {
    const double disc = B * B - 4.0 * A * C;
    const double d = sqrt(disc > 0.0 ? disc : 0.0);
    if (B > 0.0) {
      s = (-B - d) / (2.0 * A);
    } else {
      const double den = -B + d;
      s = (den == 0.0) ? 0.0 : (2.0 * C) / den;
    }
  }
  if (!(s > 0.0)) s = 0.0;
  if (s > 1.0) s = 1.0;
  return s;
}

// --------------------------------------------------------------- the edge

template <bool kF64>
struct EdgeRegs {
  using R = std::conditional_t<kF64, double, float>;
  R L, c0, c1, sigma;
  int32_t src, dst, slot_init, slot_term;
  // fast-path coefficients for a full step of length dt (FP32 mode):
  // x + (c0 + c1 x) dt + sigma sqrt(dt) W = x Q + P + S W
  float P, Q, S;
};

template <bool kF64>
__device__ __forceinline__ void load_edge(const GraphView& g, int32_t e, double dt,
                                          double sqrt_dt, EdgeRegs<kF64>& r) {
  if constexpr (kF64) {
    const EdgeRec64 q = g.e64[e];
    r.L = q.L; r.c0 = q.c0; r.c1 = q.c1; r.sigma = q.sigma;
    r.src = q.src; r.dst = q.dst; r.slot_init = q.slot_init; r.slot_term = q.slot_term;
  } else {
    const EdgeRec32 q = g.e32[e];
    r.L = q.L; r.c0 = q.c0; r.c1 = q.c1; r.sigma = q.sigma;
    r.src = q.src; r.dst = q.dst; r.slot_init = q.slot_init; r.slot_term = q.slot_term;
    r.P = q.c0 * (float)dt;
    r.Q = fmaf(q.c1, (float)dt, 1.0f);
    r.S = q.sigma * (float)sqrt_dt;
  }
}

// Slot of vertex v drawn by u: the first j in [begin, end) with u < T_j.
__device__ __forceinline__ int32_t choose_slot(const GraphView& g, const VtxRec& vr, uint32_t u) {
  int32_t lo = vr.begin, hi = vr.end - 1;  // the last threshold is 2^32 > u
  while (lo < hi) {  // thresholds are non-decreasing: binary search
    const int32_t mid = (lo + hi) >> 1;
    if ((uint64_t)u < g.slot[mid].T) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Per-thread accumulators that are reduced once per block.
struct ThreadCounters {
  uint32_t trunc;
};

struct BlockCounters {
  uint32_t* exits;     // shared [S] or nullptr (then global atomics)
  uint32_t* absorbed;  // shared [V] or nullptr
};

__device__ __forceinline__ void count_exit(const CounterView& c, const BlockCounters& b,
                                           int32_t slot) {
  if (b.exits) atomicAdd(&b.exits[slot], 1u);
  else atomicAdd(&c.exits[slot], 1ull);
}
__device__ __forceinline__ void count_absorbed(const CounterView& c, const BlockCounters& b,
                                               int32_t v) {
  if (b.absorbed) atomicAdd(&b.absorbed[v], 1u);
  else atomicAdd(&c.absorbed[v], 1ull);
}

// ------------------------------------------------------------ the EM-Step

template <bool kF64>
struct Particle {
  using R = std::conditional_t<kF64, double, float>;
  int32_t e;
  R x;
  bool at_v;  // x is an endpoint of e: the particle sits at that vertex
  uint32_t hits, first_hits, flags;
  EdgeRegs<kF64> ed;
};

// The whole EM-Step from its first sub-step on, once that sub-step is known
// to leave the edge or to start at a vertex (Algorithm 2, with the |W| rule of
// Algorithm 1 for sub-steps from a vertex).  W: the step's first normal.
__device__ __forceinline__ float absr(float v) { return fabsf(v); }
__device__ __forceinline__ double absr(double v) { return fabs(v); }

template <bool kF64>
__device__ __forceinline__ void em_step_split(Particle<kF64>& p, std::conditional_t<kF64, double, float> W,
                                           const SimArgs& a, const GraphView& g,
                                           const BlockCounters& bc, ThreadCounters& tc,
                                           uint32_t pid) {
  using R = std::conditional_t<kF64, double, float>;
  double h = a.dt;  // time left in this step (binary64 in both modes)
  int32_t k = 0;    // splits taken in this step
  for (;;) {
    int32_t at_end = -1;
    if (p.at_v) at_end = (p.x == (R)0) ? kEndInit : kEndTerm;
    if (at_end == kEndInit) W = absr(W);
    else if (at_end == kEndTerm) W = -absr(W);

    // Euler-Maruyama sub-step over the time left
    const R xs = p.x;
    R a_, b_, xt;
    if constexpr (kF64) {
      const double mu = p.ed.c0 + p.ed.c1 * xs;
      a_ = mu * h;
      b_ = p.ed.sigma * sqrt(h) * W;
      xt = xs + a_ + b_;
      const double L = p.ed.L;
      const double tol = 1e-9 * ((isfinite(L) && L > 1.0) ? L : 1.0);
      if (fabs(xt) < tol || (isfinite(L) && fabs(L - xt) < tol)) p.flags |= 1u;
    } else {
      const float hf = (float)h;
      const float mu = fmaf(p.ed.c1, xs, p.ed.c0);
      a_ = mu * hf;
      b_ = p.ed.sigma * sqrtf(hf) * W;
      xt = xs + a_ + b_;
    }
    if (xt > (R)0 && xt < p.ed.L) {  // stays inside the open edge
      if (at_end >= 0) {
        const int32_t slot = (at_end == kEndInit) ? p.ed.slot_init : p.ed.slot_term;
        count_exit(a.c, bc, slot);
      }
      p.x = xt;
      p.at_v = false;
      return;
    }

    // vertex hit: partial step to the vertex (binary64)
    const bool hit_init = !(xt > (R)0);
    const int32_t v = hit_init ? p.ed.src : p.ed.dst;
    const double A = hit_init ? (double)a_ : -(double)a_;
    const double B = hit_init ? (double)b_ : -(double)b_;
    const double C = hit_init ? (double)xs : (double)p.ed.L - (double)xs;
    const double s = hit_root(A, B, C);
    const double alpha = s * s;
    h = (1.0 - alpha) * h;
    if constexpr (kF64) {
      if (h < 1e-9 * a.dt) p.flags |= 1u;
    }
    const uint32_t j = p.hits;
    p.hits = j + 1u;
    if (at_end < 0) p.first_hits++;
    ++k;

    const VtxRec vr = g.vtx[v];
    if (vr.kind == kVertexAbsorbing) {
      count_absorbed(a.c, bc, v);
      p.e = kDead;
      return;
    }
    // draws of the j-th hit: u = w0 picks the slot, (w2, w3) the next normal
    const U4 w = philox4x32_10(j, pid, 1u, a.instance, a.rk);
    const int32_t slot = choose_slot(g, vr, w.x);
    const SlotRec sr = g.slot[slot];
    p.e = sr.edge;
    load_edge<kF64>(g, p.e, a.dt, a.sqrt_dt, p.ed);
    p.x = (sr.end == kEndInit) ? (R)0 : p.ed.L;
    p.at_v = true;
    if (k == a.M) {  // split cap: stay at the vertex (Theorem 1)
      tc.trunc++;
      return;
    }
    if (h <= 0.0) return;
    R zc, zs;
    box_muller<kF64>(w.z, w.w, zc, zs);
    W = zc;
  }
}

// One EM-Step with its first normal W: the fast interior sub-step, else the
// split path.  Returns false once the particle is absorbed.
template <bool kF64>
__device__ __forceinline__ bool em_step(Particle<kF64>& p, std::conditional_t<kF64, double, float> W,
                                        const SimArgs& a, const GraphView& g,
                                        const BlockCounters& bc, ThreadCounters& tc, uint32_t pid) {
  using R = std::conditional_t<kF64, double, float>;
  R xt;
  if constexpr (kF64) {
    const double mu = p.ed.c0 + p.ed.c1 * p.x;
    const double a_ = mu * a.dt;
    const double b_ = p.ed.sigma * a.sqrt_dt * W;
    xt = p.x + a_ + b_;
  } else {
    xt = fmaf(p.ed.S, W, fmaf(p.x, p.ed.Q, p.ed.P));
  }
  if (!p.at_v && xt > (R)0 && xt < p.ed.L) {
    if constexpr (kF64) {
      const double L = p.ed.L;
      const double tol = 1e-9 * ((isfinite(L) && L > 1.0) ? L : 1.0);
      if (fabs(xt) < tol || (isfinite(L) && fabs(L - xt) < tol)) p.flags |= 1u;
    }
    p.x = xt;
    return true;
  }
  em_step_split<kF64>(p, W, a, g, bc, tc, pid);
  return p.e >= 0;
}

// ---------------------------------------------------------- shared staging

template <typename T>
__device__ __forceinline__ void block_copy(T* dst, const T* src, int32_t n) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  const int32_t n16 = (int32_t)(((size_t)n * sizeof(T)) / 16);
  for (int32_t k = threadIdx.x; k < n16; k += blockDim.x) d[k] = s[k];
}

template <typename T>
__device__ __forceinline__ void block_zero(T* dst, int32_t n) {
  for (int32_t k = threadIdx.x; k < n; k += blockDim.x) dst[k] = 0;
}

// Histogram bin of position x on edge e (the set's precision):
// min(floor(x * (bins / range_e)), bins - 1), floored at 0.
template <bool kF64>
__device__ __forceinline__ int32_t hist_bin(std::conditional_t<kF64, double, float> x, double range,
                                            int32_t bins) {
  const double scale = (double)bins / range;
  int32_t b;
  if constexpr (kF64) {
    const double f = floor(x * scale);
    b = (f < 0.0) ? 0 : (f > (double)(bins - 1)) ? bins - 1 : (int32_t)f;
  } else {
    const float f = floorf(x * (float)scale);
    b = (f < 0.0f) ? 0 : (f > (float)(bins - 1)) ? bins - 1 : (int32_t)f;
  }
  return b;
}

// ------------------------------------------------------------- the kernel

template <bool kF64>
__global__ void __launch_bounds__(256) em_step_kernel(const __grid_constant__ SimArgs a) {
  using R = std::conditional_t<kF64, double, float>;
  extern __shared__ __align__(16) unsigned char smem[];
  GraphView g = a.g;
  const int32_t hist_len = a.smem_hist ? g.E * a.hist_bins : 0;
  const SmemLayout lay = smem_layout(g.V, g.E, g.S, kF64, a.stage_smem, a.smem_counters, hist_len);
  if (a.stage_smem) {
    if constexpr (kF64) {
      block_copy(reinterpret_cast<EdgeRec64*>(smem + lay.edges), g.e64, g.E);
      g.e64 = reinterpret_cast<const EdgeRec64*>(smem + lay.edges);
    } else {
      block_copy(reinterpret_cast<EdgeRec32*>(smem + lay.edges), g.e32, g.E);
      g.e32 = reinterpret_cast<const EdgeRec32*>(smem + lay.edges);
    }
    block_copy(reinterpret_cast<SlotRec*>(smem + lay.slots), g.slot, g.S);
    block_copy(reinterpret_cast<VtxRec*>(smem + lay.vtx), g.vtx, g.V);
    g.slot = reinterpret_cast<const SlotRec*>(smem + lay.slots);
    g.vtx = reinterpret_cast<const VtxRec*>(smem + lay.vtx);
  }
  BlockCounters bc{nullptr, nullptr};
  if (a.smem_counters) {
    bc.exits = reinterpret_cast<uint32_t*>(smem + lay.exits);
    bc.absorbed = reinterpret_cast<uint32_t*>(smem + lay.absorbed);
    block_zero(bc.exits, g.S);
    block_zero(bc.absorbed, g.V);
  }
  uint32_t* shist = a.smem_hist ? reinterpret_cast<uint32_t*>(smem + lay.hist) : nullptr;
  if (shist) block_zero(shist, hist_len);
  __syncthreads();

  ThreadCounters tc{0};
  uint64_t psteps = 0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    Particle<kF64> p;
    p.e = a.s.edge[i];
    p.x = reinterpret_cast<const R*>(a.s.x)[i];
    p.hits = a.s.hits[i];
    p.first_hits = a.s.first_hits[i];
    p.flags = a.s.flags[i];
    const uint32_t pid = a.pid_base + (uint32_t)i;
    bool ok = p.e >= kDead && p.e < g.E;
    if (!ok) atomicOr(a.c.err, kErrBadEdge);
    if (ok && p.e >= 0) {
      load_edge<kF64>(g, p.e, a.dt, a.sqrt_dt, p.ed);
      if (!(p.x >= (R)0 && p.x <= p.ed.L)) {
        atomicOr(a.c.err, kErrNan);
        ok = false;
      }
      p.at_v = (p.x == (R)0) || (p.x == p.ed.L);
    }
    if (ok && p.e >= 0 && a.steps > 0) {
      const uint64_t t0 = a.t_begin, t1 = a.t_begin + (uint64_t)a.steps;
      uint64_t t = t0;
      bool alive = true;
      // head: steps up to the next multiple of four
      if (t & 3u) {
        const U4 w = philox4x32_10((uint32_t)(t >> 2), pid, 0u, a.instance, a.rk);
        R z[4];
        box_muller<kF64>(w.x, w.y, z[0], z[1]);
        box_muller<kF64>(w.z, w.w, z[2], z[3]);
#pragma unroll
        for (int l = 1; l < 4; ++l) {
          if (alive && (int)(t & 3u) == l && t < t1) {
            alive = em_step<kF64>(p, z[l], a, g, bc, tc, pid);
            if (alive) ++t;
          }
        }
      }
      // body: whole groups of four steps share one Philox block
      const uint64_t g_end = t1 >> 2;
      for (uint64_t grp = t >> 2; alive && grp < g_end; ++grp) {
        const U4 w = philox4x32_10((uint32_t)grp, pid, 0u, a.instance, a.rk);
        R z0, z1, z2, z3;
        box_muller<kF64>(w.x, w.y, z0, z1);
        box_muller<kF64>(w.z, w.w, z2, z3);
        t = grp << 2;
        if (!(alive = em_step<kF64>(p, z0, a, g, bc, tc, pid))) break;
        ++t;
        if (!(alive = em_step<kF64>(p, z1, a, g, bc, tc, pid))) break;
        ++t;
        if (!(alive = em_step<kF64>(p, z2, a, g, bc, tc, pid))) break;
        ++t;
        if (!(alive = em_step<kF64>(p, z3, a, g, bc, tc, pid))) break;
        t = (grp + 1) << 2;
      }
      // tail: the last t1 mod 4 steps
      if (alive && t < t1) {
        const U4 w = philox4x32_10((uint32_t)(t >> 2), pid, 0u, a.instance, a.rk);
        R z[4];
        box_muller<kF64>(w.x, w.y, z[0], z[1]);
        box_muller<kF64>(w.z, w.w, z[2], z[3]);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          if (alive && (int)(t & 3u) == l && t < t1) {
            alive = em_step<kF64>(p, z[l], a, g, bc, tc, pid);
            if (alive) ++t;
          }
        }
      }
      // a particle absorbed during step t took steps t0 .. t
      psteps = alive ? (uint64_t)a.steps : (t - t0 + 1);
    }
    if (ok) {
      a.s.edge[i] = p.e;
      reinterpret_cast<R*>(a.s.x)[i] = p.x;
      a.s.hits[i] = p.hits;
      a.s.first_hits[i] = p.first_hits;
      a.s.flags[i] = p.flags;
      // fused snapshot histogram of the final position
      if (a.hist_bins > 0 && p.e >= 0) {
        const int32_t bin = hist_bin<kF64>(p.x, g.range[p.e], a.hist_bins);
        const int32_t key = p.e * a.hist_bins + bin;
        if (shist) atomicAdd(&shist[key], 1u);
        else atomicAdd(&a.hist[key], 1u);
      }
    }
  }

  // per-warp reduction of the scalar counters
  uint32_t tr = tc.trunc;
  unsigned long long ps = psteps;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tr += __shfl_down_sync(0xffffffffu, tr, off);
    ps += __shfl_down_sync(0xffffffffu, ps, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (tr) atomicAdd(a.c.trunc, (unsigned long long)tr);
    if (ps) atomicAdd(a.c.psteps, ps);
  }
  __syncthreads();
  if (a.smem_counters) {
    for (int32_t k = threadIdx.x; k < g.S; k += blockDim.x)
      if (bc.exits[k]) atomicAdd(&a.c.exits[k], (unsigned long long)bc.exits[k]);
    for (int32_t k = threadIdx.x; k < g.V; k += blockDim.x)
      if (bc.absorbed[k]) atomicAdd(&a.c.absorbed[k], (unsigned long long)bc.absorbed[k]);
  }
  if (shist)
    for (int32_t k = threadIdx.x; k < hist_len; k += blockDim.x)
      if (shist[k]) atomicAdd(&a.hist[k], shist[k]);
}

// Snapshot histogram of the living particles (no stepping).
template <bool kF64>
__global__ void __launch_bounds__(256) histogram_kernel(GraphView g, const int32_t* __restrict__ edge,
                                                        const void* __restrict__ xv, int64_t n,
                                                        int32_t bins, uint32_t* __restrict__ out,
                                                        int32_t use_smem) {
  using R = std::conditional_t<kF64, double, float>;
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
    const int32_t key = e * bins + hist_bin<kF64>(x[i], g.range[e], bins);
    if (use_smem) atomicAdd(&sh[key], 1u);
    else atomicAdd(&out[key], 1u);
  }
  if (use_smem) {
    __syncthreads();
    for (int32_t k = threadIdx.x; k < len; k += blockDim.x)
      if (sh[k]) atomicAdd(&out[k], sh[k]);
  }
}

}  // namespace mg
