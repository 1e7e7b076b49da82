// mg_em_step.cuh -- the fused EM-Step kernel of libmetricgraph.
//
// One thread advances one particle (edge e, position x) through many
// EM-Steps of the timestep-splitting Euler-Maruyama scheme ("Sampling on
// Metric Graphs", Algorithms 1 and 2), keeping the particle in registers for
// the whole launch (Section 3.1: state in registers, global memory only for
// the ensemble statistics).
//
// Every Euler-Maruyama sub-step -- the first of a step, and each one that
// continues a step from a vertex after a split -- takes the next normal of
// the particle's own counter-based stream (Philox-4x32-10 + Box-Muller, four
// normals per block), buffered per thread in a ring of 16 in shared memory.
// A warp loops in iterations; per lane and iteration:
//
//   split     a lane whose last sub-step ended outside (0, l_e) is pending;
//             the warp resolves its pending lanes together in one pass --
//             hitting fraction, time left, jump draw, next edge, and the
//             sub-step from the vertex, repeated while it hits again -- so
//             the long split path runs with many lanes active instead of one.
//             A particle's draws depend only on its own counters, so batching
//             does not change results;
//   refill    the ring is topped up to at least kSub + 1 normals;
//   vertex    a lane sitting at a vertex at the start of a step takes its
//             sub-step from the vertex: W = +-|z| into the edge;
//   interior  then kSub sub-steps (8 in the binary32 modes, 4 in binary64)
//             x~ = x + mu_e(x) dt + sigma_e sqrt(dt) z, two FMAs and a range
//             test each, branch-free; the first that leaves (0, l_e) makes
//             the lane pending.
//
// Counters (exits per slot, absorptions, truncations) and the optional
// snapshot histogram are privatised in shared memory when they fit and
// flushed with one atomic per nonzero entry per block.  em_step_kernel runs
// one particle per thread; em_range_kernel (graphs whose particles can die)
// lets a lane claim the next particle of its block's range when its own
// dies or finishes; em_batch_kernel runs 256-particle tiles of many sets.
//
// Precision modes (template kMode):
//   kModeF64    everything in binary64, in the same operation order as the
//               plain CPU reference (the translation unit is built without
//               FMA contraction);
//   kModeMixed  positions, increments and normals in binary32; the split's
//               hitting fraction -- the root s to binary64 accuracy,
//               alpha = s^2 -- and the time left h in binary64;
//   kModeF32    everything in binary32.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "mg_log_table.h"
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
    // each product as one 32 x 32 -> 64-bit multiply (both halves at once)
    const uint64_t m0 = (uint64_t)0xD2511F53u * c0, m1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t lo0 = (uint32_t)m0, hi0 = (uint32_t)(m0 >> 32);
    const uint32_t lo1 = (uint32_t)m1, hi1 = (uint32_t)(m1 >> 32);
    const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
    const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// Two Philox-4x32-10 blocks with counters (c0a, c1, c2, c3) and (c0b, c1, c2,
// c3), their rounds interleaved so that the two independent multiply chains
// overlap.
__device__ __forceinline__ void philox4x32_10_x2(uint32_t c0a, uint32_t c0b, uint32_t c1,
                                                 uint32_t c2, uint32_t c3,
                                                 const uint32_t* __restrict__ rk, U4& wa,
                                                 U4& wb) {
  uint32_t a0 = c0a, a1 = c1, a2 = c2, a3 = c3;
  uint32_t b0 = c0b, b1 = c1, b2 = c2, b3 = c3;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t am0 = (uint64_t)0xD2511F53u * a0, am1 = (uint64_t)0xCD9E8D57u * a2;
    const uint64_t bm0 = (uint64_t)0xD2511F53u * b0, bm1 = (uint64_t)0xCD9E8D57u * b2;
    const uint32_t alo0 = (uint32_t)am0, ahi0 = (uint32_t)(am0 >> 32);
    const uint32_t alo1 = (uint32_t)am1, ahi1 = (uint32_t)(am1 >> 32);
    const uint32_t blo0 = (uint32_t)bm0, bhi0 = (uint32_t)(bm0 >> 32);
    const uint32_t blo1 = (uint32_t)bm1, bhi1 = (uint32_t)(bm1 >> 32);
    const uint32_t an0 = ahi1 ^ a1 ^ rk[2 * r], an2 = ahi0 ^ a3 ^ rk[2 * r + 1];
    const uint32_t bn0 = bhi1 ^ b1 ^ rk[2 * r], bn2 = bhi0 ^ b3 ^ rk[2 * r + 1];
    a0 = an0; a1 = alo1; a2 = an2; a3 = alo0;
    b0 = bn0; b1 = blo1; b2 = bn2; b3 = blo0;
  }
  wa = {a0, a1, a2, a3};
  wb = {b0, b1, b2, b3};
}

// ------------------------------------------------------------- Box-Muller

// binary64: u = (2w + 1) 2^-33, r = sqrt(-2 ln u_a), theta = 2 pi u_b.
// u is assembled from its bits with integer instructions (the value is exact:
// 2w + 1 has at most 33 significant bits), which keeps three operations per
// uniform off GB300's slow binary64 pipe: with m = 2w + 1 = 2^t (1 + f),
// u = 2^(t - 33) (1 + f).
__device__ __forceinline__ double u01_f64(uint32_t w) {
  const uint64_t m = 2ull * w + 1ull;                 // 1 .. 2^33 - 1
  const int t = 63 - __clzll((long long)m);           // 0 .. 32
  const uint64_t frac = (m << (52 - t)) & 0x000FFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(((uint64_t)(1023 + t - 33) << 52) | frac));
}
// ln u for u = (2w + 1) 2^-33 in binary64, correctly rounded (checked
// against a 40-digit logarithm on 63 000 inputs by a CPU emulation of these
// steps), with fewer binary64 operations than a general logarithm -- the
// binary64 pipe bounds the binary64 mode:
//   u = 2^-k f with f in [1 - 2^-8, 2 - 2^-7) (exact, from the bits of 2w + 1);
//   c = the table's binary64 value nearest 64 / (64 + j), j = round(64 (f - 1))
//   (c = 1 for f < 1), so that ln u = -k ln 2 - ln c + log1p(f c - 1);
//   f c = ph + pl exactly (a product and its fused-multiply-add remainder),
//   r = ph - 1 exact, |r| <= 2^-7;
//   log1p(r + pl) = r + r^2 q(r) + pl (1 - r), q by the series of log1p to
//   r^8 (the next term is below 2^-56 of r);
//   -k ln 2 - ln c as one pair of binary64 numbers per (k, j) (a table
//   written by gen_log_table.py, one 16-byte load), its sum with r kept
//   exactly (Dekker's fast two-sum: |k ln 2 + ln c| >= |r| wherever the
//   former is nonzero, since |r| <= 1 / (2 (64 + j)) while k ln 2 + ln c =
//   ln(2^k 64 / (64 + j)) is zero or at least ln(128 / 127) in magnitude).
// Near u = 1 (k = 0, c = 1) the result is r + r^2 q alone: full relative
// accuracy.
__device__ __forceinline__ double ln_u01(uint32_t w) {
  const uint64_t m = 2ull * w + 1ull;        // 1 .. 2^33 - 1
  const int t = 63 - __clzll((long long)m);  // 0 .. 32
  const uint64_t frac = (m << (52 - t)) & 0x000FFFFFFFFFFFFFull;
  int k = 33 - t;  // u = 2^-k f, f = 1 + frac 2^-52
  int j = 0;
  double f;
  if (frac >= 0x000FE00000000000ull) {  // f >= 2 - 2^-7: use f / 2 in [1 - 2^-8, 1)
    f = __longlong_as_double((long long)((1022ull << 52) | frac));
    k -= 1;
  } else {
    f = __longlong_as_double((long long)((1023ull << 52) | frac));
    j = (int)((frac + (1ull << 45)) >> 46);  // 0 .. 63
  }
  const double c = __ldg(&kLogC[j]);
  const double ph = f * c;
  const double pl = fma(f, c, -ph);
  const double r = ph - 1.0;
  double q = fma(r, -0.125, 1.0 / 7.0);
  q = fma(q, r, -1.0 / 6.0);
  q = fma(q, r, 0.2);
  q = fma(q, r, -0.25);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double2 v = __ldg(&kLogKJ[64 * k + j]);  // -k ln 2 - ln c = v.x + v.y
  const double t1 = v.x + r, e1 = r - (t1 - v.x);
  const double small = (v.y + e1) + fma(-pl, r, pl);
  return t1 + fma(r * r, q, small);
}

__device__ __forceinline__ void box_muller_f64(uint32_t wa, uint32_t wb, double& zc, double& zs) {
  const double ub = u01_f64(wb);
  const double r = sqrt(-2.0 * ln_u01(wa));
  const double th = 6.283185307179586 * ub;
  double s, c;
  sincos(th, &s, &c);
  zc = r * c;
  zs = r * s;
}

// binary32: u = (2 (w >> 9) + 1) 2^-24, formed exactly from the top 23 bits
// (1 + m 2^-23 minus 1 - 2^-24; m < 2^23, so adding the exponent bits is an
// OR), so the binary32 and binary64 modes see the same words.  cos(2 pi u) =
// -cos(2 pi u - pi) keeps the hardware sine/cosine on (-pi, pi).
// lg2/sqrt/sin/cos are the approximate hardware instructions in their
// flush-to-zero forms: their arguments here are normal numbers (u >= 2^-24,
// |2 pi u - pi| >= 2^-23), for which the results are the same, and the
// forms without it spend instructions on subnormal arguments (on the
// 16-edge star the flush-to-zero forms run 2% faster).
__device__ __forceinline__ float u01_f32(uint32_t w) {
  return __uint_as_float((w >> 9) + 0x3f800000u) - 0.99999994f;
}
__device__ __forceinline__ void box_muller_f32(uint32_t wa, uint32_t wb, float& zc, float& zs) {
  const float ua = u01_f32(wa), ub = u01_f32(wb);
  float lg;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(ua));
  const float r2 = -1.38629436112f * lg;  // -2 ln u
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(r2));
  const float th = fmaf(ub, 6.28318530718f, -3.14159265359f);
  float s, c;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(th));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(th));
  zc = -r * c;
  zs = -r * s;
}

// ------------------------------------------- binary32 <-> binary64 by bits

// binary64 h in [0, 2^128) to binary32, truncated (rounded toward zero),
// with integer operations; values below 2^-126 give 0.  The binary32 time of
// the FP32-mixed mode's sub-step coefficients: the binary64 h stays the time
// left, and truncating rather than rounding to nearest saves the rounding
// step's operations in every split (1% on the 16-edge star) at an error of
// at most one binary32 ulp in those coefficients.
__device__ __forceinline__ float narrow_f64_rz(double h) {
  const uint32_t hi = (uint32_t)__double2hiint(h), lo = (uint32_t)__double2loint(h);
  return (hi < 0x38100000u) ? 0.0f : __uint_as_float(((hi - (896u << 20)) << 3) | (lo >> 29));
}

// ---------------------------------------------------- hitting-fraction root

// First root s in [0, 1] of A s^2 + B s + C = 0 with C >= 0 (s = sqrt(alpha)
// of the partial step): A = 0 gives -C/B; otherwise (-B - d)/(2A) for B > 0
// and the equal 2C/(-B + d) for B <= 0, each free of cancellation on its
// side; d = sqrt(max(B^2 - 4AC, 0)); the result is clamped to [0, 1].
template <typename T>
__device__ __forceinline__ T hit_root(T A, T B, T C) {
  T s;
  if (A == T(0)) {
    s = (B == T(0)) ? T(0) : -C / B;
  } else {
    const T disc = B * B - T(4) * A * C;
    const T d = sqrt(disc > T(0) ? disc : T(0));
    if (B > T(0)) {
      s = (-B - d) / (T(2) * A);
    } else {
      const T den = -B + d;
      s = (den == T(0)) ? T(0) : (T(2) * C) / den;
    }
  }
  if (!(s > T(0))) s = T(0);
  if (s > T(1)) s = T(1);
  return s;
}

// The same root in binary32 with the hardware's approximate reciprocal and
// square root (a few ulp; the result is clamped to [0, 1] all the same),
// branch-free: one quotient num / den picks the side's cancellation-free
// form.  For A = 0, d = |B| and the B <= 0 form is 2C / (2|B|) = -C/B, while
// B > 0 gives a zero denominator (no root in [0, 1]); den = 0 gives 0.
__device__ __forceinline__ float hit_root_fast(float A, float B, float C) {
  const float disc = fmaf(B, B, -4.0f * A * C);
  float d;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(d) : "f"(fmaxf(disc, 0.0f)));
  const bool pos = B > 0.0f;
  const float num = pos ? -B - d : 2.0f * C;
  const float den = pos ? 2.0f * A : d - B;
  float rden;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rden) : "f"(den));
  float s = num * rden;
  if (!(s > 0.0f) || den == 0.0f) s = 0.0f;  // negative, NaN, or no root
  return fminf(s, 1.0f);
}

// Sum a + b = s + e exactly (Knuth's two-sum, no ordering assumption); the
// _rn intrinsics keep the compiler from fusing any of it into an FMA.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Exact widening of a binary32 v to binary64 with integer operations (sign
// kept, exponent rebiased, mantissa shifted up 29 bits).  Subnormal inputs,
// below 2^-126 -- far under any coefficient of a sub-step -- become a zero of
// the same sign.
__device__ __forceinline__ double widen_f32(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t mag = b & 0x7fffffffu;
  const bool normal = mag >= 0x00800000u;
  const uint32_t hi = (b & 0x80000000u) | (normal ? (mag >> 3) + (896u << 20) : 0u);
  const uint32_t lo = normal ? (mag << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// s in [0, 1] from a binary64 s: NaN and negative values give 0, values
// above 1 give 1 (comparisons of the bit patterns).
__device__ __forceinline__ double clamp_unit(double s) {
  const long long b = __double_as_longlong(s);
  if (!(b > 0ll) || (b & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) return 0.0;  // <= 0, NaN
  return (b > 0x3FF0000000000000ll) ? 1.0 : s;
}

// The first root in [0, 1] of A s^2 + B s + C = 0 for binary32 coefficients,
// solved in binary64 by the closed form of hit_root<double> on the widened
// coefficients, with the same binary64 result: B^2 and 4AC are exact in
// binary64, so the discriminant is rounded once (one fused multiply-add);
// square root and quotient are CUDA's correctly rounded binary64 operations.
// Tests of the coefficients run on the binary32 inputs (the same outcomes).
__device__ __forceinline__ double hit_root_f64_closed(float A, float B, float C) {
  double s;
  if (A == 0.0f) {
    s = (B == 0.0f) ? 0.0 : -widen_f32(C) / widen_f32(B);
  } else {
    const double B64 = widen_f32(B);
    const double t = widen_f32(4.0f * A) * widen_f32(C);  // exact
    const double disc = fma(B64, B64, -t);
    const double d = (__double_as_longlong(disc) > 0ll) ? sqrt(disc) : 0.0;
    if (B > 0.0f) {
      s = (-B64 - d) / widen_f32(2.0f * A);
    } else {
      const double den = d - B64;
      s = ((__double_as_longlong(den) & 0x7FFFFFFFFFFFFFFFll) == 0ll)
              ? 0.0
              : widen_f32(2.0f * C) / den;
    }
  }
  return clamp_unit(s);
}

// Exact product a b = p + e (the FMA gives the rounding error exactly).
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
  return p;
}

// The same root to binary64 accuracy, refined in binary32 error-free
// arithmetic (GB300's binary64 pipe runs at about 1/70 of the binary32 rate,
// so the refinement keeps off it).  From the binary32 root s0:
//   f(s0) = (A s0 + B) s0 + C is split exactly into binary32 terms (exact
//   products by FMA, Knuth's two-sums): f0 + f0l to ~2^-70 of the terms;
//   f'(s0) = 2 A s0 + B as d + dl;
//   Newton step 1: t = -f0 / d (a binary32 correction of ~2^-22 s0);
//   f(s0 + t) = f(s0) + t f'(s0) + A t^2, again to ~2^-68 of the terms
//   (t d exactly, the rest small), so that
//   Newton step 2: t2 = -f(s0 + t) / d leaves s = s0 + t + t2 good to
//   ~2^-66 s0.
// ok = false for a second correction beyond 2^-40 s0 (a nearly double root,
// where Newton's method converges slowly): the caller falls back to the
// closed form in binary64.  s0 = 0: no root in (0, 1], or C = 0.
struct RootParts {
  float s0, t, t2;
  bool ok;
};

__device__ __forceinline__ RootParts hit_root_parts(float A, float B, float C) {
  RootParts r{hit_root_fast(A, B, C), 0.0f, 0.0f, true};
  const float s0 = r.s0;
  if (!(s0 > 0.0f)) return r;
  float pae, ge, qe, we, re, rse, a1e, a2e, f0e, de, ue, ve;
  const float pa = two_prod(A, s0, pae);   // A s0
  const float g = two_sum(pa, B, ge);      // A s0 + B = g + ge + pae
  const float q = two_prod(g, s0, qe);     // g s0
  const float w = two_sum(q, C, we);       // g s0 + C = w + we + qe
  const float rr = two_sum(ge, pae, re);   // (ge + pae) s0 = rr s0 + re s0
  const float rs = two_prod(rr, s0, rse);
  const float a1 = two_sum(we, qe, a1e);
  const float a2 = two_sum(a1, rs, a2e);
  const float lo = ((a1e + a2e) + rse) + re * s0;
  const float f0 = two_sum(w, a2, f0e);
  const float f0l = f0e + lo;              // f(s0) = f0 + f0l
  const float d = two_sum(2.0f * pa, B, de);
  const float dl = de + 2.0f * pae;        // f'(s0) = d + dl
  float rd;  // 1 / f'(s0), shared by both corrections
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(d));
  const float t = -f0 * rd;
  const float u = two_prod(t, d, ue);
  const float v = two_sum(f0, u, ve);
  const float f1 = v + ((((ve + f0l) + ue) + t * dl) + A * (t * t));
  const float t2 = -f1 * rd;
  r.t = t;
  r.t2 = t2;
  r.ok = fabsf(t2) <= 0x1p-40f * s0;
  return r;
}

// The root s in binary64: (s0 + t) exactly, then + t2 (one rounding).
__device__ __forceinline__ double hit_root_f64_eft(float A, float B, float C) {
  const RootParts r = hit_root_parts(A, B, C);
  if (!(r.s0 > 0.0f)) return 0.0;
  if (!r.ok) return hit_root_f64_closed(A, B, C);
  return clamp_unit((widen_f32(r.s0) + widen_f32(r.t)) + widen_f32(r.t2));
}

// The hitting fraction alpha = s^2 of that root in binary64, with one
// binary64 addition and one FMA: sa = s0 + t exactly, alpha = sa^2 + 2 sa t2
// (t2^2 < 2^-80 s^2 is dropped, and 2 sa t2 is taken as 2 s0 t2 in binary32,
// within 2^-20 of itself: ~2^-63 of alpha), clamped to [0, 1].
__device__ __forceinline__ double hit_alpha_f64(float A, float B, float C) {
  const RootParts r = hit_root_parts(A, B, C);
  if (!(r.s0 > 0.0f)) return 0.0;
  if (!r.ok) {
    const double s = hit_root_f64_closed(A, B, C);
    return s * s;
  }
  const double sa = widen_f32(r.s0) + widen_f32(r.t);
  const double alpha = fma(sa, sa, widen_f32(2.0f * r.s0 * r.t2));
  return (__double_as_longlong(alpha) > 0x3FF0000000000000ll) ? 1.0 : alpha;
}

// Slot of vertex v drawn by u: the first j in [begin, end) with u < T_j
// (thresholds are non-decreasing and the last is 2^32 > u).  The guide entry
// of u's bucket is that j or an earlier slot of v (every slot before it has
// T_j <= the bucket's lower end <= u), so a forward scan from it finds j; it
// stops at the last slot at the latest (tm1 = 2^32 - 1 >= u).
__device__ __forceinline__ int32_t choose_slot(const GraphView& g, const VtxRec& vr, uint32_t u) {
  const int32_t d = vr.end - vr.begin;
  const uint32_t gb = (d > 1) ? 32u - (uint32_t)__clz(d - 1) : 0u;  // 2^gb >= d
  int32_t j = g.guide[vr.guide + (int32_t)__funnelshift_l(u, 0u, gb)];  // u >> (32 - gb)
  while (u > g.slot[j].tm1) ++j;
  return j;
}

// Exit and absorption counters of a block, privatised in shared memory when
// they fit: 32-bit for a tile of 256 particles (one launch cannot overflow
// them), 64-bit for the range kernel, whose blocks run many particles.
template <typename C>
struct BlockCountersT {
  C* exits;     // shared [S] or nullptr (then global atomics)
  C* absorbed;  // shared [V] or nullptr
};
using BlockCounters = BlockCountersT<uint32_t>;
using BlockCounters64 = BlockCountersT<unsigned long long>;

template <typename C>
__device__ __forceinline__ void count_exit(const CounterView& c, const BlockCountersT<C>& b,
                                           int32_t slot) {
  if (b.exits) atomicAdd(&b.exits[slot], (C)1);
  else atomicAdd(&c.exits[slot], 1ull);
}
template <typename C>
__device__ __forceinline__ void count_absorbed(const CounterView& c, const BlockCountersT<C>& b,
                                               int32_t v) {
  if (b.absorbed) atomicAdd(&b.absorbed[v], (C)1);
  else atomicAdd(&c.absorbed[v], 1ull);
}

// ---------------------------------------------------------------- the lane

template <int kMode>
struct Types {
  using R = std::conditional_t<prec_of(kMode) == kModeF64, double, float>;  // positions, normals
  using H = std::conditional_t<prec_of(kMode) == kModeF32, float, double>;  // alpha, time left
  // interior sub-steps per loop iteration, and the ring of buffered normals:
  // kRing per thread, each stored twice (rows n % kRing and n % kRing + kRing)
  static constexpr int kSub = (prec_of(kMode) == kModeF64) ? 4 : 8;
  static constexpr bool kVar = var_sigma(kMode);  // sigma_e(x) = sigma_e + sigma1_e x
  static constexpr uint32_t kRing = 2 * kSub;
};

// Jump draws: the u32 of a particle's hit j is word j & 3 of Philox block
// (j >> 2, pid, 1, instance).  A thread keeps two blocks of its particle's
// words in shared memory, [8][kThreads] right after the ring of normals
// (block b in rows 4 (b & 1) .. 4 (b & 1) + 3, so hit j reads row j & 7);
// jtop is the first hit whose word is not there yet.  Blocks are computed
// ahead of the hits, warp-wide, in the refill phase -- whenever a lane of the
// warp has used up its words, every lane with room for a block computes its
// next one, so one Philox evaluation serves many lanes.  A split pass takes
// one hit per lane and a refill phase follows every pass, so a lane always
// holds its next word when it splits (the split only reads it: computing a
// missing block there as well cost 3% on the vascular network, for code that
// never ran).
template <int kMode>
__device__ __forceinline__ uint32_t* jump_words(const typename Types<kMode>::R* ring) {
  return reinterpret_cast<uint32_t*>(const_cast<typename Types<kMode>::R*>(ring) +
                                     2 * Types<kMode>::kRing * kThreads) +
         threadIdx.x;
}

// Stores the words of block b (its slot b & 1).
__device__ __forceinline__ void store_jump_block(uint32_t* jw, uint32_t b, const U4& w) {
  uint32_t* r = jw + (b & 1u) * 4u * kThreads;
  r[0 * kThreads] = w.x;
  r[1 * kThreads] = w.y;
  r[2 * kThreads] = w.z;
  r[3 * kThreads] = w.w;
}

// A particle just loaded: the block holding its next hit.
template <int kMode>
__device__ __forceinline__ uint32_t prime_jump_words(uint32_t hits,
                                                     const typename Types<kMode>::R* ring,
                                                     const SimArgs& a, const Keys& keys,
                                                     uint32_t pid) {
  store_jump_block(jump_words<kMode>(ring), hits >> 2,
                   philox4x32_10(hits >> 2, pid, 1u, a.instance, keys.rk));
  return (hits & ~3u) + 4u;
}

// Sign handling of the normal of a sub-step: W = (z & wand) | wor on the sign
// bit (z itself inside an edge, +|z| at an init end, -|z| at a term end).
__device__ __forceinline__ float apply_sign(float z, uint32_t wand, uint32_t wor) {
  return __uint_as_float((__float_as_uint(z) & wand) | wor);
}
__device__ __forceinline__ double apply_sign(double z, uint32_t wand, uint32_t wor) {
  const int lo = __double2loint(z);
  const int hi = (int)(((uint32_t)__double2hiint(z) & wand) | wor);
  return __hiloint2double(hi, lo);
}

template <int kMode>
struct Lane {
  using R = typename Types<kMode>::R;
  using H = typename Types<kMode>::H;
  // particle
  int32_t e;
  R x;
  uint32_t n_draw, n_gen, hits, first_hits, flags;
  uint32_t jtop;  // first hit whose jump word is not in shared memory yet
  // current edge
  R L;
  R tol;  // binary64 mode: branch margin 1e-9 max(1, l_e)
  // binary64 mode: bit patterns bounding the band (l_e - tol, l_e + tol)
  long long near_lo, near_hi;
  // sub-step coefficients for the time h of the current sub-step:
  //   binary32: x~ = x Q + P + S W, P = c0 h, Q = 1 + c1 h, S = sigma sqrt(h)
  //   binary64: x~ = (x + (c0 + c1 x) h) + S W, S = sigma sqrt(h)
  R P, Q, S;
  R Pm, Qm, Sm;  // the same for a whole step (h = dt)
  R c0, c1;      // binary64 mode
  // position-dependent diffusion (kVar): binary32 modes S1 = sigma1 sqrt(h),
  // so that the noise of a sub-step from x is (S + S1 x) W; binary64 mode
  // sigma_e(x) = sg0 + sg1 x and rh = sqrt(h)
  R S1, S1m;
  R sg0, sg1, rh;
  H h;           // time left in the current step
  float hf;      // binary32-mixed mode: h truncated to binary32 (narrow_f64_rz)
  uint32_t wand, wor;
  int32_t cur_slot;  // slot of the vertex end the particle sits at
  int32_t k;         // splits in the current step
  uint32_t left;     // steps left in this launch
  bool at_v;         // at a vertex: the next sub-step leaves it (W = +-|z|)
  bool in_cont;      // ... and continues a step after a split (time left h)
  bool pending;      // the last sub-step ended outside (0, l_e): split next
  bool active;
};

template <int kMode>
__device__ __forceinline__ void set_vertex_sign(Lane<kMode>& p, int32_t end) {
  p.wand = 0x7fffffffu;
  p.wor = (end == kEndInit) ? 0u : 0x80000000u;
}

// Load edge e into the lane and set its whole-step coefficients (h = dt).
template <int kMode>
__device__ __forceinline__ void enter_edge(Lane<kMode>& p, const GraphView& g, int32_t e,
                                           const SimArgs& a) {
  p.e = e;
  if constexpr (prec_of(kMode) == kModeF64) {
    const EdgeRec64& q = g.e64[e];
    p.L = q.L;
    p.c0 = q.c0;
    p.c1 = q.c1;
    p.Sm = q.sigma * a.sqrt_dt;
    if constexpr (Types<kMode>::kVar) {
      p.sg0 = q.sigma;
      p.sg1 = g.s1_64[e];
    }
    p.tol = 1e-9 * ((isfinite(q.L) && q.L > 1.0) ? q.L : 1.0);
    // the band around the terminal end as bit patterns of non-negative
    // binary64 numbers (empty for l_e = +inf), so that the near-branch test
    // of every sub-step is integer comparisons (the subtraction l_e - x~ it
    // replaces ran on the binary64 pipe once per sub-step)
    const double lo = q.L - p.tol;
    p.near_lo = lo > 0.0 ? __double_as_longlong(lo) : 0ll;
    p.near_hi = __double_as_longlong(q.L + p.tol);
  } else {
    const EdgeRec32& q = g.e32[e];
    p.L = q.L;
    p.Pm = q.c0 * a.dt_f;
    p.Qm = fmaf(q.c1, a.dt_f, 1.0f);
    p.Sm = q.sigma * a.sqrt_dt_f;
    if constexpr (Types<kMode>::kVar) p.S1m = g.s1_32[e] * a.sqrt_dt_f;
  }
}

template <int kMode>
__device__ __forceinline__ void use_step_coefficients(Lane<kMode>& p, const SimArgs& a) {
  if constexpr (prec_of(kMode) == kModeF32) p.h = a.dt_f;
  else p.h = a.dt;
  if constexpr (prec_of(kMode) == kModeMixed) p.hf = a.dt_f;
  if constexpr (prec_of(kMode) != kModeF64) {
    p.P = p.Pm;
    p.Q = p.Qm;
    if constexpr (Types<kMode>::kVar) p.S1 = p.S1m;
  } else if constexpr (Types<kMode>::kVar) {
    p.rh = a.sqrt_dt;
  }
  p.S = p.Sm;
}

// Coefficients of a sub-step over the time left h on the current edge (its
// record q, already loaded, in the binary32 modes).
template <int kMode>
__device__ __forceinline__ void use_rest_coefficients(Lane<kMode>& p, const GraphView& g,
                                                      const EdgeRec32& q) {
  if constexpr (prec_of(kMode) == kModeF64) {
    if constexpr (Types<kMode>::kVar) p.rh = sqrt(p.h);
    else p.S = g.e64[p.e].sigma * sqrt(p.h);
  } else {
    float hf;
    if constexpr (prec_of(kMode) == kModeMixed) {
      p.hf = narrow_f64_rz(p.h);
      hf = p.hf;
    } else {
      hf = p.h;
    }
    float rh;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rh) : "f"(hf));
    p.P = q.c0 * hf;
    p.Q = fmaf(q.c1, hf, 1.0f);
    p.S = q.sigma * rh;
    if constexpr (Types<kMode>::kVar) p.S1 = g.s1_32[p.e] * rh;
  }
}

// Ring of buffered normals, kRing per thread, each stored twice: normal n of
// the thread sits at rows n % kRing and n % kRing + kRing of
// ring[2 kRing][kThreads], so kSub + 1 consecutive normals from row n % kRing
// are read at fixed offsets.  A lane refills (four at a time) only while it
// holds at most kSub and is not pending, so the normal of a pending sub-step
// stays readable until its split has used it.  A stream never wraps: a lane
// that would pass 2^32 - 16 normals stops with kErrStream.
template <int kMode>
__device__ __forceinline__ void refill(Lane<kMode>& p, typename Types<kMode>::R* ring,
                                       const SimArgs& a, const Keys& keys, uint32_t pid) {
  using R = typename Types<kMode>::R;
  if (p.n_gen >= 0xFFFFFFF0u) {
    atomicOr(a.c.err, kErrStream);
    p.active = false;
    p.pending = false;
    return;
  }
  const U4 w = philox4x32_10(p.n_gen >> 2, pid, 0u, a.instance, keys.rk);
  R z0, z1, z2, z3;
  if constexpr (prec_of(kMode) == kModeF64) {
    box_muller_f64(w.x, w.y, z0, z1);
    box_muller_f64(w.z, w.w, z2, z3);
  } else {
    box_muller_f32(w.x, w.y, z0, z1);
    box_muller_f32(w.z, w.w, z2, z3);
  }
  constexpr uint32_t K = Types<kMode>::kRing;
  R* r = ring + (p.n_gen & (K - 1u)) * kThreads + threadIdx.x;  // a multiple of 4
  r[0 * kThreads] = z0;
  r[1 * kThreads] = z1;
  r[2 * kThreads] = z2;
  r[3 * kThreads] = z3;
  r[(K + 0) * kThreads] = z0;
  r[(K + 1) * kThreads] = z1;
  r[(K + 2) * kThreads] = z2;
  r[(K + 3) * kThreads] = z3;
  p.n_gen += 4;
}

// Eight normals at once (binary32 modes): the next two Philox blocks of the
// lane's stream, computed interleaved.  Only for a lane that holds at most
// kSub = 8 normals, so that the ring's 16 cannot overflow.
template <int kMode>
__device__ __forceinline__ void refill8(Lane<kMode>& p, typename Types<kMode>::R* ring,
                                        const SimArgs& a, const Keys& keys, uint32_t pid) {
  static_assert(prec_of(kMode) != kModeF64, "binary32 modes only");
  if (p.n_gen >= 0xFFFFFFF0u - 4u) {
    atomicOr(a.c.err, kErrStream);
    p.active = false;
    p.pending = false;
    return;
  }
  U4 wa, wb;
  philox4x32_10_x2(p.n_gen >> 2, (p.n_gen >> 2) + 1u, pid, 0u, a.instance, keys.rk, wa, wb);
  float z[8];
  box_muller_f32(wa.x, wa.y, z[0], z[1]);
  box_muller_f32(wa.z, wa.w, z[2], z[3]);
  box_muller_f32(wb.x, wb.y, z[4], z[5]);
  box_muller_f32(wb.z, wb.w, z[6], z[7]);
  constexpr uint32_t K = Types<kMode>::kRing;
  float* ra = ring + (p.n_gen & (K - 1u)) * kThreads + threadIdx.x;
  float* rb = ring + ((p.n_gen + 4u) & (K - 1u)) * kThreads + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ra[k * kThreads] = z[k];
    ra[(K + k) * kThreads] = z[k];
    rb[k * kThreads] = z[4 + k];
    rb[(K + k) * kThreads] = z[4 + k];
  }
  p.n_gen += 8;
}

// The refills of an iteration: top the buffer up to at least kSub + 1
// normals (an iteration uses up to kSub + 1; a lane that went pending with an
// empty buffer needs up to three blocks of four).  Binary32 modes take two
// blocks at once whenever any are needed (the lane holds at most 8, so 16
// fit), and a third for an empty buffer.
template <int kMode>
__device__ __forceinline__ void refill_iteration(Lane<kMode>& p, typename Types<kMode>::R* ring,
                                                 const SimArgs& a, const Keys& keys,
                                                 uint32_t pid) {
  // jump words: when a lane of the warp has none left, every lane with a
  // used-up slot computes its next block (the warp evaluates Philox once)
  if (__any_sync(0xffffffffu, p.active && p.hits >= p.jtop) && p.active &&
      p.jtop - p.hits <= 4u) {
    store_jump_block(jump_words<kMode>(ring), p.jtop >> 2,
                     philox4x32_10(p.jtop >> 2, pid, 1u, a.instance, keys.rk));
    p.jtop += 4u;
  }
  constexpr uint32_t kSub = (uint32_t)Types<kMode>::kSub;
  const uint32_t held = p.n_gen - p.n_draw;
  const uint32_t n_ref = (p.active && !p.pending && held <= kSub) ? (kSub + 4u - held) >> 2 : 0u;
  if constexpr (prec_of(kMode) != kModeF64) {
    if (n_ref > 0u) refill8<kMode>(p, ring, a, keys, pid);
    if (n_ref > 2u) refill<kMode>(p, ring, a, keys, pid);
  } else {
    if (n_ref > 0u) refill<kMode>(p, ring, a, keys, pid);
    if (n_ref > 1u) refill<kMode>(p, ring, a, keys, pid);
  }
}

// Binary64 noise sigma_e(x) sqrt(h) W of a sub-step from x, in the oracle's
// order of operations: (sigma_e(x) sqrt(h)) W.
template <int kMode>
__device__ __forceinline__ double noise_f64(const Lane<kMode>& p, double x, double W) {
  if constexpr (Types<kMode>::kVar) return ((p.sg0 + p.sg1 * x) * p.rh) * W;
  else return p.S * W;
}

// End point of a sub-step with normal W over the lane's current time h.
template <int kMode>
__device__ __forceinline__ typename Types<kMode>::R sub_step_end(const Lane<kMode>& p,
                                                                 typename Types<kMode>::R W) {
  if constexpr (prec_of(kMode) == kModeF64) {
    const double mu = p.c0 + p.c1 * p.x;
    const double a_ = mu * p.h;
    const double b_ = noise_f64(p, p.x, W);
    return p.x + a_ + b_;
  } else if constexpr (Types<kMode>::kVar) {
    // x (Q + S1 W) + (S W + P), as the interior sub-steps compute it
    return fmaf(p.x, fmaf(p.S1, W, p.Q), fmaf(p.S, W, p.P));
  } else {
    // x Q + (S W + P): the same expression (and rounding) as the interior
    // sub-steps, so a recomputed end point falls on the same side
    return fmaf(p.x, p.Q, fmaf(p.S, W, p.P));
  }
}

// Comparisons of binary64 numbers on their bit patterns, for numbers that
// are not NaN: a non-negative binary64 number orders as its bits read as a
// signed 64-bit integer, a negative one reads negative.  Exactly the
// floating-point comparisons, on the integer pipes instead of GB300's slow
// binary64 pipe.  abs_below(v, b): |v| < b for b >= 0.
__device__ __forceinline__ bool abs_below(double v, double b) {
  return (__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll) < __double_as_longlong(b);
}

// x~ in (0, l_e) for binary64, l_e > 0 (+inf on a semi-infinite edge)
__device__ __forceinline__ bool inside(double xt, double L) {
  const long long b = __double_as_longlong(xt);
  return (b > 0) & (b < __double_as_longlong(L));
}

template <int kMode>
__device__ __forceinline__ void mark_near_branch(Lane<kMode>& p, typename Types<kMode>::R xt) {
  if constexpr (prec_of(kMode) == kModeF64) {
    // |x~| < tol, or x~ in (l_e - tol, l_e + tol); a negative x~ within tol
    // of l_e is within tol of 0 as well
    const long long b = __double_as_longlong(xt);
    if (abs_below(xt, p.tol) || (b > p.near_lo && b < p.near_hi)) p.flags |= 1u;
  }
}

// The sub-step of a lane at a vertex: into the edge with |z|; ending inside
// it is an exit through the vertex slot and closes the step.
template <int kMode, typename BC>
__device__ __forceinline__ void vertex_sub_step(Lane<kMode>& p,
                                                const typename Types<kMode>::R* ring,
                                                const SimArgs& a, const BC& bc) {
  using R = typename Types<kMode>::R;
  const R z = ring[(p.n_draw & (Types<kMode>::kRing - 1u)) * kThreads + threadIdx.x];
  p.n_draw++;
  const R xt = sub_step_end(p, apply_sign(z, p.wand, p.wor));
  mark_near_branch(p, xt);
  bool in;
  if constexpr (prec_of(kMode) == kModeF64) in = inside(xt, p.L);
  else in = xt > R(0) && xt < p.L;
  if (in) {
    count_exit(a.c, bc, p.cur_slot);
    if (p.in_cont) use_step_coefficients(p, a);
    p.k = 0;
    p.at_v = false;
    p.in_cont = false;
    p.wand = 0xffffffffu;
    p.wor = 0u;
    p.x = xt;
    if (--p.left == 0u) p.active = false;
  } else {
    p.pending = true;
  }
}

// Up to kSub interior sub-steps over whole steps (h = dt, W = z), stopping
// at the first that ends outside (0, l_e) -- the lane is then pending -- or,
// with kCheckLeft, when the launch's steps are done.  Branch-free: every
// unrolled sub-step is evaluated and a running "all inside so far" predicate
// decides which ones count.  Ring rows past the lane's generated normals may
// be read (in bounds: at most kRing - 1 + kSub - 1 < 2 kRing) but never count.
template <int kMode, bool kCheckLeft>
__device__ __forceinline__ void interior_sub_steps(Lane<kMode>& p, const typename Types<kMode>::R* ring,
                                              bool run) {
  using R = typename Types<kMode>::R;
  constexpr uint32_t kSub = (uint32_t)Types<kMode>::kSub;
  const R* r = ring + (p.n_draw & (Types<kMode>::kRing - 1u)) * kThreads + threadIdx.x;
  const uint32_t lim = kCheckLeft ? (p.left < kSub ? p.left : kSub) : kSub;
  uint32_t n_in = 0;
  bool go = run;
  // binary32: the end points are chained unselected (xc), so each sub-step
  // adds one FMA on x to the dependency chain; xc equals x for every
  // sub-step that counts
  R xc = p.x;
#pragma unroll
  for (int q = 0; q < (int)kSub; ++q) {
    const bool att = go && (!kCheckLeft || (uint32_t)q < lim);
    const R z = r[q * kThreads];
    R xt;
    if constexpr (prec_of(kMode) == kModeF64) {
      const double mu = p.c0 + p.c1 * p.x;
      const double a_ = mu * p.h;
      const double b_ = noise_f64(p, p.x, z);
      xt = p.x + a_ + b_;
      if (att) mark_near_branch(p, xt);
    } else if constexpr (Types<kMode>::kVar) {
      xt = fmaf(xc, fmaf(p.S1m, z, p.Qm), fmaf(p.Sm, z, p.Pm));
      xc = xt;
    } else {
      xt = fmaf(xc, p.Qm, fmaf(p.Sm, z, p.Pm));
      xc = xt;
    }
    bool in;
    if constexpr (prec_of(kMode) == kModeF64) in = att & inside(xt, p.L);
    else in = att & (xt > R(0)) & (xt < p.L);
    p.x = in ? xt : p.x;
    n_in += in ? 1u : 0u;
    go = in;
  }
  const bool out = run && n_in < lim;
  p.n_draw += n_in + (out ? 1u : 0u);
  p.left -= n_in;
  p.pending = p.pending | out;
  if (p.left == 0u) p.active = false;
}

// Resolve the pending vertex hit: partial step to the vertex, time left,
// jump draw, next edge, and the coefficients of the rest of the step.
template <int kMode, typename BC>
__device__ __forceinline__ void split(Lane<kMode>& p, const GraphView& g, const SimArgs& a,
                                      const BC& bc, const typename Types<kMode>::R* ring,
                                      uint32_t& trunc) {
  using R = typename Types<kMode>::R;
  p.pending = false;
  // the jump draw of this hit (j = hits so far), stored ahead by the refill
  // phase; a lane without it would be a library bug, reported as such
  if (p.hits >= p.jtop) atomicOr(a.c.err, kErrStuck);
  const uint32_t u = jump_words<kMode>(ring)[(p.hits & 7u) * kThreads];
  const R xs = p.x;
  // the pending sub-step again: its normal is still in the ring
  const R Wp = apply_sign(
      ring[((p.n_draw - 1u) & (Types<kMode>::kRing - 1u)) * kThreads + threadIdx.x], p.wand,
      p.wor);
  const bool hit_init = !(sub_step_end(p, Wp) > R(0));
  // the hit vertex and its record first: the load's latency (a round trip to
  // L2 for graphs whose tables stay out of shared memory) overlaps the
  // hitting-fraction arithmetic below; v < 0 (the far end of a semi-infinite
  // edge, reached only by an overflow) reads vertex 0 and is reported below
  int32_t v;
  if constexpr (prec_of(kMode) == kModeF64) v = hit_init ? g.e64[p.e].src : g.e64[p.e].dst;
  else v = hit_init ? g.e32[p.e].src : g.e32[p.e].dst;
  const VtxRec vr = g.vtx[v < 0 ? 0 : v];
  bool rest;  // time is left in the step after this hit
  if constexpr (prec_of(kMode) == kModeF64) {
    const double mu = p.c0 + p.c1 * xs;
    const double a_ = mu * p.h;
    const double b_ = noise_f64(p, xs, Wp);
    const double A = hit_init ? a_ : -a_;
    const double B = hit_init ? b_ : -b_;
    const double C = hit_init ? xs : p.L - xs;
    const double s = hit_root<double>(A, B, C);
    const double alpha = s * s;
    p.h = (1.0 - alpha) * p.h;
    if (p.h < 1e-9 * a.dt) p.flags |= 1u;
    rest = p.h > 0.0;
  } else {
    // increments of the pending sub-step in binary32: a = mu(x) h, b = S W
    const EdgeRec32& q = g.e32[p.e];
    float hf;
    if constexpr (prec_of(kMode) == kModeMixed) hf = p.hf;
    else hf = p.h;
    const float a_ = fmaf(q.c1, xs, q.c0) * hf;
    float b_;
    if constexpr (Types<kMode>::kVar) b_ = fmaf(p.S1, xs, p.S) * Wp;
    else b_ = p.S * Wp;
    const float A = hit_init ? a_ : -a_;
    const float B = hit_init ? b_ : -b_;
    const float C = hit_init ? xs : p.L - xs;
    if constexpr (prec_of(kMode) == kModeMixed) {
      // the hitting fraction and the time left in binary64: the root to
      // binary64 accuracy, alpha = s^2, h <- h - alpha h
      const double alpha = hit_alpha_f64(A, B, C);
      p.h = fma(-alpha, p.h, p.h);
      // h (1 - alpha) > 0 exactly when alpha < 1, and stays positive when rounded
      rest = __double_as_longlong(alpha) < 0x3FF0000000000000ll;
    } else {
      const float s = hit_root_fast(A, B, C);
      p.h = fmaf(-s * s, p.h, p.h);
      rest = p.h > 0.0f;
    }
  }
  const uint32_t j = p.hits;
  p.hits = j + 1u;
  if (!p.at_v) p.first_hits++;
  p.k++;
  if (v < 0) {
    // the far end of a semi-infinite edge: only an end point that overflowed
    // to +inf gets here (a drift pushing the particle off to infinity)
    atomicOr(a.c.err, kErrNan);
    p.active = false;
    return;
  }
  if (vr.kind == kVertexAbsorbing) {
    count_absorbed(a.c, bc, v);
    p.e = kDead;
    p.active = false;
    return;
  }
  const int32_t slot = choose_slot(g, vr, u);
  const SlotRec sr = g.slot[slot];
  EdgeRec32 qn{};  // the new edge (binary32 modes)
  if constexpr (prec_of(kMode) == kModeF64) {
    enter_edge<kMode>(p, g, sr.edge, a);
  } else {
    p.e = sr.edge;
    qn = g.e32[sr.edge];
    p.L = qn.L;
    p.Pm = qn.c0 * a.dt_f;
    p.Qm = fmaf(qn.c1, a.dt_f, 1.0f);
    p.Sm = qn.sigma * a.sqrt_dt_f;
    if constexpr (Types<kMode>::kVar) p.S1m = g.s1_32[sr.edge] * a.sqrt_dt_f;
  }
  p.x = (sr.end == kEndInit) ? R(0) : p.L;
  p.at_v = true;
  p.cur_slot = slot;
  set_vertex_sign(p, sr.end);
  if (p.k == a.M || !rest) {  // the step ends at the vertex
    if (p.k == a.M) trunc++;
    p.k = 0;
    p.in_cont = false;
    use_step_coefficients(p, a);
    if (--p.left == 0) p.active = false;
    return;
  }
  p.in_cont = true;
  use_rest_coefficients(p, g, qn);
}

// A pending lane's part of a split pass: one split, then -- when time is left
// in the step -- the sub-step from the vertex into the new edge, which may
// reach a vertex again and leave the lane pending for a later pass.  One
// split per lane per pass: a lane whose sub-steps keep hitting vertices (a
// chain of up to M splits in a step, common on short edges against a strong
// drift) no longer holds its whole warp in the pass; its warp's other lanes
// move on meanwhile.  Measured on one GB300 against resolving whole chains in
// a pass: the synthetic vascular network 1.06e11 -> 2.01e11 particle-steps/s
// in FP32 (2.52e9 -> 3.15e9 in FP64), the 3-edge Brownian star +6%, the
// 16-edge Langevin star (no chains) and the 512-instance batch unchanged.
template <int kMode, typename BC>
__device__ __forceinline__ void split_and_continue(Lane<kMode>& p, const GraphView& g,
                                                   const SimArgs& a, const Keys& keys,
                                                   const BC& bc,
                                                   typename Types<kMode>::R* ring, uint32_t pid,
                                                   uint32_t& trunc) {
  if (!p.pending) return;
  split<kMode>(p, g, a, bc, ring, trunc);
  if (!p.active || !p.in_cont) return;
  if (p.n_gen == p.n_draw) {  // the split used up the buffer
    refill<kMode>(p, ring, a, keys, pid);
    if (!p.active) return;
  }
  vertex_sub_step<kMode>(p, ring, a, bc);
}

// Histogram bin of position x on edge e (the set's precision):
// min(floor(x * (bins / range_e)), bins - 1), floored at 0.
template <typename R>
__device__ __forceinline__ int32_t hist_bin(R x, double range, int32_t bins) {
  const double scale = (double)bins / range;
  int32_t b;
  if constexpr (std::is_same<R, double>::value) {
    const double f = floor(x * scale);
    b = (f < 0.0) ? 0 : (f > (double)(bins - 1)) ? bins - 1 : (int32_t)f;
  } else {
    const float f = floorf(x * (float)scale);
    b = (f < 0.0f) ? 0 : (f > (float)(bins - 1)) ? bins - 1 : (int32_t)f;
  }
  return b;
}

// Copies n elements in 16-byte pieces, rounding the byte count up to a
// multiple of 16: both sides are padded to 16 bytes (the device tables to 256).
template <typename T>
__device__ __forceinline__ void block_copy(T* dst, const T* src, int32_t n) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  const int32_t n16 = (int32_t)(((size_t)n * sizeof(T) + 15) / 16);
  for (int32_t k = threadIdx.x; k < n16; k += blockDim.x) d[k] = s[k];
}

template <typename T>
__device__ __forceinline__ void block_zero(T* dst, int32_t n) {
  for (int32_t k = threadIdx.x; k < n; k += blockDim.x) dst[k] = 0;
}

// ------------------------------------------------------------- the kernel

// A block's view of its working set: graph tables (staged in shared memory
// when they fit), privatised counters and histogram, the normal ring.
template <int kMode>
struct BlockSetup {
  GraphView g;
  BlockCounters64 bc;
  uint32_t* shist;
  int32_t hist_len;
  typename Types<kMode>::R* ring;
};

// Stages the tables and zeroes the privatised counters (the caller
// synchronises the block before use).
template <int kMode>
__device__ __forceinline__ BlockSetup<kMode> setup_block(const SimArgs& a, unsigned char* smem) {
  using R = typename Types<kMode>::R;
  constexpr bool kF64 = prec_of(kMode) == kModeF64;
  BlockSetup<kMode> b;
  b.g = a.g;
  GraphView& g = b.g;
  b.hist_len = a.smem_hist ? g.E * a.hist_bins : 0;
  const SmemLayout lay = smem_layout(g.V, g.E, g.S, g.G, kF64, a.stage_smem, a.smem_counters,
                                     b.hist_len, kThreads, 8, Types<kMode>::kVar);
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
    block_copy(reinterpret_cast<int32_t*>(smem + lay.guide), g.guide, g.G);
    g.slot = reinterpret_cast<const SlotRec*>(smem + lay.slots);
    g.vtx = reinterpret_cast<const VtxRec*>(smem + lay.vtx);
    g.guide = reinterpret_cast<const int32_t*>(smem + lay.guide);
    if constexpr (Types<kMode>::kVar) {
      if constexpr (kF64) {
        block_copy(reinterpret_cast<double*>(smem + lay.sig1), g.s1_64, g.E);
        g.s1_64 = reinterpret_cast<const double*>(smem + lay.sig1);
      } else {
        block_copy(reinterpret_cast<float*>(smem + lay.sig1), g.s1_32, g.E);
        g.s1_32 = reinterpret_cast<const float*>(smem + lay.sig1);
      }
    }
  }
  b.bc = BlockCounters64{nullptr, nullptr};
  if (a.smem_counters) {
    b.bc.exits = reinterpret_cast<unsigned long long*>(smem + lay.exits);
    b.bc.absorbed = reinterpret_cast<unsigned long long*>(smem + lay.absorbed);
    block_zero(b.bc.exits, g.S);
    block_zero(b.bc.absorbed, g.V);
  }
  b.shist = a.smem_hist ? reinterpret_cast<uint32_t*>(smem + lay.hist) : nullptr;
  if (b.shist) block_zero(b.shist, b.hist_len);
  b.ring = reinterpret_cast<R*>(smem + lay.ring);
  return b;
}

// Adds the block's privatised counters and histogram to the global ones
// (after the block's last use of them).
template <int kMode>
__device__ __forceinline__ void flush_block(const SimArgs& a, const BlockSetup<kMode>& b) {
  __syncthreads();
  if (a.smem_counters) {
    for (int32_t k = threadIdx.x; k < b.g.S; k += blockDim.x)
      if (b.bc.exits[k]) atomicAdd(&a.c.exits[k], b.bc.exits[k]);
    for (int32_t k = threadIdx.x; k < b.g.V; k += blockDim.x)
      if (b.bc.absorbed[k]) atomicAdd(&a.c.absorbed[k], b.bc.absorbed[k]);
  }
  if (b.shist)
    for (int32_t k = threadIdx.x; k < b.hist_len; k += blockDim.x)
      if (b.shist[k]) atomicAdd(&a.hist[k], b.shist[k]);
}

// One iteration of a warp after its liveness check: the split pass (one
// vertex hit of each pending lane and its sub-step from the vertex), the
// refills, the sub-step from a vertex, and kSub interior sub-steps.
template <int kMode, typename BC>
__device__ __forceinline__ void iteration(Lane<kMode>& p, const GraphView& g, const SimArgs& a,
                                          const Keys& keys, const BC& bc,
                                          typename Types<kMode>::R* ring, uint32_t pid,
                                          uint32_t& trunc, uint32_t am) {
  const uint32_t full = 0xffffffffu;
  const uint32_t pm = __ballot_sync(full, p.pending);
  if (pm != 0u && (__popc(pm) >= a.split_batch || pm == am)) {
    split_and_continue<kMode>(p, g, a, keys, bc, ring, pid, trunc);
  }
  refill_iteration<kMode>(p, ring, a, keys, pid);
  constexpr uint32_t kSub = (uint32_t)Types<kMode>::kSub;
  if (p.active && !p.pending && p.at_v) vertex_sub_step<kMode>(p, ring, a, bc);
  const bool run = p.active && !p.pending && !p.at_v;
  if (__all_sync(full, !run || p.left >= kSub)) interior_sub_steps<kMode, false>(p, ring, run);
  else interior_sub_steps<kMode, true>(p, ring, run);
}

// One block's tile of a particle set: particle i of the calling thread
// (i >= a.n: an idle lane that still takes part in the block's barriers).
template <int kMode>
__device__ __forceinline__ void run_tile(const SimArgs& a, const Keys& keys, int64_t i,
                                         unsigned char* smem) {
  using R = typename Types<kMode>::R;
  constexpr bool kF64 = prec_of(kMode) == kModeF64;
  GraphView g = a.g;
  const int32_t hist_len = a.smem_hist ? g.E * a.hist_bins : 0;
  const SmemLayout lay = smem_layout(g.V, g.E, g.S, g.G, kF64, a.stage_smem, a.smem_counters,
                                     hist_len, kThreads, 4, Types<kMode>::kVar);
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
    block_copy(reinterpret_cast<int32_t*>(smem + lay.guide), g.guide, g.G);
    g.slot = reinterpret_cast<const SlotRec*>(smem + lay.slots);
    g.vtx = reinterpret_cast<const VtxRec*>(smem + lay.vtx);
    g.guide = reinterpret_cast<const int32_t*>(smem + lay.guide);
    if constexpr (Types<kMode>::kVar) {
      if constexpr (kF64) {
        block_copy(reinterpret_cast<double*>(smem + lay.sig1), g.s1_64, g.E);
        g.s1_64 = reinterpret_cast<const double*>(smem + lay.sig1);
      } else {
        block_copy(reinterpret_cast<float*>(smem + lay.sig1), g.s1_32, g.E);
        g.s1_32 = reinterpret_cast<const float*>(smem + lay.sig1);
      }
    }
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
  R* ring = reinterpret_cast<R*>(smem + lay.ring);
  __syncthreads();

  uint32_t trunc = 0;
  uint64_t psteps = 0;
  const uint32_t pid = a.pid_base + (uint32_t)i;
  Lane<kMode> p;
  p.active = false;
  p.pending = false;
  bool ok = false, alive0 = false;
  if (i < a.n) {
    p.e = a.s.edge[i];
    p.x = reinterpret_cast<const R*>(a.s.x)[i];
    p.n_draw = a.s.n_draw[i];
    p.hits = a.s.hits[i];
    p.first_hits = a.s.first_hits[i];
    p.flags = a.s.flags[i];
    ok = p.e >= kDead && p.e < g.E;
    if (!ok) atomicOr(a.c.err, kErrBadEdge);
    if (ok && p.e >= 0) {
      const R x0 = p.x;
      enter_edge<kMode>(p, g, p.e, a);
      p.x = x0;
      if (!(p.x >= R(0) && p.x <= p.L && isfinite(p.x))) {  // finite: L may be +inf
        atomicOr(a.c.err, kErrNan);
        ok = false;
      }
    }
    alive0 = ok && p.e >= 0;
    if (alive0 && a.steps > 0) {
      p.active = true;
      p.left = (uint32_t)a.steps;
      p.k = 0;
      p.in_cont = false;
      use_step_coefficients(p, a);
      p.at_v = (p.x == R(0)) || (p.x == p.L);
      p.wand = 0xffffffffu;
      p.wor = 0u;
      p.cur_slot = -1;
      if (p.at_v) {
        const int32_t end = (p.x == R(0)) ? kEndInit : kEndTerm;
        if constexpr (kF64) p.cur_slot = (end == kEndInit) ? g.e64[p.e].slot_init : g.e64[p.e].slot_term;
        else p.cur_slot = (end == kEndInit) ? g.e32[p.e].slot_init : g.e32[p.e].slot_term;
        set_vertex_sign(p, end);
      }
      p.n_gen = p.n_draw & ~3u;
      refill<kMode>(p, ring, a, keys, pid);
      p.jtop = prime_jump_words<kMode>(p.hits, ring, a, keys, pid);
    }
  }

  // Iterations of at most kSub + 1 sub-steps per lane (one from a vertex,
  // kSub interior); pending vertex hits resolved in warp-wide batches (split_batch
  // lanes, or whenever nothing else moves).  Every iteration moves some lane
  // forward by a sub-step or a split, and a lane has at most 2M + 1 of those
  // per step, so the loop ends within 32 steps (2M + 2) iterations; the cap turns a
  // logic error into a reported fault instead of a hang (the host keeps it
  // within 32 bits).
  const uint32_t full = 0xffffffffu;
  const uint32_t cap = 32u * (uint32_t)a.steps * (uint32_t)(2 * a.M + 2) + 64u;
  uint32_t iters = 0;
  for (;;) {
    const uint32_t am = __ballot_sync(full, p.active);
    if (am == 0u) break;
    if (++iters > cap) {
      if (p.active) atomicOr(a.c.err, kErrStuck);
      break;
    }
    const uint32_t pm = __ballot_sync(full, p.pending);
    if (pm != 0u && (__popc(pm) >= a.split_batch || pm == am)) {
      split_and_continue<kMode>(p, g, a, keys, bc, ring, pid, trunc);
    }
    refill_iteration<kMode>(p, ring, a, keys, pid);
    constexpr uint32_t kSub = (uint32_t)Types<kMode>::kSub;
    if (p.active && !p.pending && p.at_v) vertex_sub_step<kMode>(p, ring, a, bc);
    const bool run = p.active && !p.pending && !p.at_v;
    if (__all_sync(full, !run || p.left >= kSub)) interior_sub_steps<kMode, false>(p, ring, run);
    else interior_sub_steps<kMode, true>(p, ring, run);
  }

  if (ok && i < a.n) {
    // steps taken while alive: an absorbed particle took the step it died in
    if (alive0 && a.steps > 0)
      psteps = (uint64_t)a.steps - p.left + ((p.e < 0) ? 1u : 0u);
    a.s.edge[i] = p.e;
    reinterpret_cast<R*>(a.s.x)[i] = p.x;
    a.s.n_draw[i] = p.n_draw;
    a.s.hits[i] = p.hits;
    a.s.first_hits[i] = p.first_hits;
    a.s.flags[i] = p.flags;
    if (a.hist_bins > 0 && p.e >= 0) {
      const int32_t bin = hist_bin<R>(p.x, g.range[p.e], a.hist_bins);
      const int32_t key = p.e * a.hist_bins + bin;
      if (shist) atomicAdd(&shist[key], 1u);
      else atomicAdd(&a.hist[key], 1u);
    }
  }

  // per-warp reduction of the scalar counters
  uint32_t tr = trunc;
  unsigned long long ps = psteps;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tr += __shfl_down_sync(full, tr, off);
    ps += __shfl_down_sync(full, ps, off);
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

// A block's claim on its range of particles (range kernel), in shared
// memory: the next unclaimed index, the end of the range, and the block's
// totals of steps taken while alive and of truncated steps.
struct RangeCtl {
  unsigned long long next;
  long long hi;
  unsigned long long psteps, trunc;
};

// Loads particle i into the lane (state, edge, whole-step coefficients and
// the first four normals of its stream) and returns whether it moves: alive,
// valid and with steps to take.  A particle that does not move is written
// back at once (if valid: unchanged, plus its histogram bin); an invalid edge
// or position sets the device-error bit and leaves it untouched.
template <int kMode>
__device__ __forceinline__ bool load_particle(Lane<kMode>& p, uint32_t& pid, const SimArgs& a,
                                              const Keys& keys, const GraphView& g,
                                              typename Types<kMode>::R* ring, uint32_t* shist,
                                              int64_t i) {
  using R = typename Types<kMode>::R;
  pid = a.pid_base + (uint32_t)i;
  p.active = false;
  p.pending = false;
  p.e = a.s.edge[i];
  p.x = reinterpret_cast<const R*>(a.s.x)[i];
  p.n_draw = a.s.n_draw[i];
  p.hits = a.s.hits[i];
  p.first_hits = a.s.first_hits[i];
  p.flags = a.s.flags[i];
  bool ok = p.e >= kDead && p.e < g.E;
  if (!ok) atomicOr(a.c.err, kErrBadEdge);
  if (ok && p.e >= 0) {
    const R x0 = p.x;
    enter_edge<kMode>(p, g, p.e, a);
    p.x = x0;
    if (!(p.x >= R(0) && p.x <= p.L && isfinite(p.x))) {  // finite: L may be +inf
      atomicOr(a.c.err, kErrNan);
      ok = false;
    }
  }
  if (!ok) return false;
  if (p.e < 0 || a.steps <= 0) {  // dead, or nothing to do: only the histogram
    if (a.hist_bins > 0 && p.e >= 0) {
      const int32_t key = p.e * a.hist_bins + hist_bin<R>(p.x, g.range[p.e], a.hist_bins);
      if (shist) atomicAdd(&shist[key], 1u);
      else atomicAdd(&a.hist[key], 1u);
    }
    return false;
  }
  p.active = true;
  p.left = (uint32_t)a.steps;
  p.k = 0;
  p.in_cont = false;
  use_step_coefficients(p, a);
  p.at_v = (p.x == R(0)) || (p.x == p.L);
  p.wand = 0xffffffffu;
  p.wor = 0u;
  p.cur_slot = -1;
  if (p.at_v) {
    const int32_t end = (p.x == R(0)) ? kEndInit : kEndTerm;
    if constexpr (prec_of(kMode) == kModeF64)
      p.cur_slot = (end == kEndInit) ? g.e64[p.e].slot_init : g.e64[p.e].slot_term;
    else
      p.cur_slot = (end == kEndInit) ? g.e32[p.e].slot_init : g.e32[p.e].slot_term;
    set_vertex_sign(p, end);
  }
  p.n_gen = p.n_draw & ~3u;
  refill<kMode>(p, ring, a, keys, pid);
  p.jtop = prime_jump_words<kMode>(p.hits, ring, a, keys, pid);
  return true;
}

// Writes back a particle that moved in this launch: state, steps taken while
// alive (an absorbed particle took the step it died in), its truncations and
// its bin of the fused snapshot histogram.
template <int kMode>
__device__ __forceinline__ void finish_particle(const Lane<kMode>& p, uint32_t pid,
                                                uint32_t& trunc, const SimArgs& a,
                                                const GraphView& g, uint32_t* shist,
                                                RangeCtl* ctl) {
  using R = typename Types<kMode>::R;
  const int64_t i = (int64_t)(uint32_t)(pid - a.pid_base);
  atomicAdd(&ctl->psteps,
            (unsigned long long)((uint64_t)a.steps - p.left + ((p.e < 0) ? 1u : 0u)));
  if (trunc) atomicAdd(&ctl->trunc, (unsigned long long)trunc);
  trunc = 0;
  a.s.edge[i] = p.e;
  reinterpret_cast<R*>(a.s.x)[i] = p.x;
  a.s.n_draw[i] = p.n_draw;
  a.s.hits[i] = p.hits;
  a.s.first_hits[i] = p.first_hits;
  a.s.flags[i] = p.flags;
  if (a.hist_bins > 0 && p.e >= 0) {
    const int32_t key = p.e * a.hist_bins + hist_bin<R>(p.x, g.range[p.e], a.hist_bins);
    if (shist) atomicAdd(&shist[key], 1u);
    else atomicAdd(&a.hist[key], 1u);
  }
}

// One block's range [lo, hi) of a particle set, for sets whose particles can
// die (absorbing vertices): thread t starts with particle lo + t, and a lane
// whose particle has taken all its steps or died writes it back and claims
// the next particle of the range, so lanes stay busy until the range runs out
// instead of idling beside their warp's last survivor.  A particle's result
// does not depend on the lane, block or order that runs it.
template <int kMode>
__device__ __forceinline__ void run_range(const SimArgs& a, const Keys& keys, int64_t lo,
                                          int64_t hi, unsigned char* smem, RangeCtl* ctl) {
  const BlockSetup<kMode> blk = setup_block<kMode>(a, smem);
  const GraphView& g = blk.g;
  if (threadIdx.x == 0) {
    ctl->next = (unsigned long long)(lo + blockDim.x);
    ctl->hi = hi;
    ctl->psteps = 0;
    ctl->trunc = 0;
  }
  __syncthreads();

  uint32_t trunc = 0;  // truncated steps of the lane's current particle
  uint32_t pid = 0;    // global id of the lane's particle
  Lane<kMode> p;
  p.active = false;
  p.pending = false;
  bool held = false;   // the lane holds a moving particle (to be written back)
  bool claim = true;   // the block's range may still have particles for it
  if (lo + (int64_t)threadIdx.x < hi)
    held = load_particle<kMode>(p, pid, a, keys, g, blk.ring, blk.shist,
                                lo + (int64_t)threadIdx.x);

  // As in run_tile, plus: between two iterations in which a lane of the warp
  // takes a new particle, every iteration moves one of the at most 32
  // particles held by a sub-step or a split, so `iters`, restarted whenever a
  // lane takes a particle, stays within 32 steps (2M + 2) + 64.
  const uint32_t full = 0xffffffffu;
  const uint32_t cap = 32u * (uint32_t)a.steps * (uint32_t)(2 * a.M + 2) + 64u;
  uint32_t iters = 0;
  for (;;) {
    bool took = false;
    if (!p.active && claim) {
      // write back the finished particle, then claim the next one that moves
      if (held) finish_particle<kMode>(p, pid, trunc, a, g, blk.shist, ctl);
      held = false;
      do {
        const int64_t nx = (int64_t)atomicAdd(&ctl->next, 1ull);
        if (nx >= ctl->hi) {
          claim = false;
          break;
        }
        took = true;
        held = load_particle<kMode>(p, pid, a, keys, g, blk.ring, blk.shist, nx);
      } while (!held);
    }
    if (__any_sync(full, took)) iters = 0;
    const uint32_t am = __ballot_sync(full, p.active);
    if (am == 0u) break;
    if (++iters > cap) {
      if (p.active) atomicOr(a.c.err, kErrStuck);
      break;
    }
    iteration<kMode>(p, g, a, keys, blk.bc, blk.ring, pid, trunc, am);
  }
  // after the last particle, or a loop left through the cap: write back what
  // the lane holds
  if (held) finish_particle<kMode>(p, pid, trunc, a, g, blk.shist, ctl);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ctl->trunc) atomicAdd(a.c.trunc, ctl->trunc);
    if (ctl->psteps) atomicAdd(a.c.psteps, ctl->psteps);
  }
  flush_block<kMode>(a, blk);
}

// The range form of the fused EM-Step kernel: block b runs particles
// [b range, (b + 1) range) of one set with lanes that claim particles.
// (binary32 modes: at most 64 registers, four blocks per SM, like the tile
// kernel; binary64 unconstrained.)
template <int kMode>
__global__ void __launch_bounds__(256, (prec_of(kMode) == kModeF64) ? 0 : 4)
    em_range_kernel(const __grid_constant__ SimArgs a, const __grid_constant__ Keys keys) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RangeCtl ctl;
  const int64_t lo = (int64_t)blockIdx.x * a.range;
  const int64_t hi = (lo + a.range < a.n) ? lo + a.range : a.n;
  run_range<kMode>(a, keys, lo, hi, smem, &ctl);
}

// The fused EM-Step kernel over one particle set: block b takes particles
// b * r .. b * r + r - 1, r = a.range (256, or fewer for a set too small to
// fill the GPU's resident blocks).
template <int kMode>
__global__ void __launch_bounds__(256, (prec_of(kMode) == kModeF64) ? 2 : 4) em_step_kernel(const __grid_constant__ SimArgs a,
                                                      const __grid_constant__ Keys keys) {
  extern __shared__ __align__(16) unsigned char smem[];
  // a.range <= 256 particles per block; the block's other threads are idle
  const int64_t i =
      (threadIdx.x < a.range) ? (int64_t)blockIdx.x * a.range + threadIdx.x : a.n;
  run_tile<kMode>(a, keys, i, smem);
}

// The batched, persistent form: each block pops work items -- 256 particles
// of one instance -- from a queue (ordered longest first by the host) until
// it is empty, copying the instance's arguments to shared memory and running
// the same tile body, so a particle's result does not depend on the batch.
// (binary32 modes: at most 64 registers, four blocks per SM.)
template <int kMode>
__global__ void __launch_bounds__(256, (prec_of(kMode) == kModeF64) ? 0 : 4)
    em_batch_kernel(const SimArgs* __restrict__ insts,
                                                       const BatchItem* __restrict__ items,
                                                       int32_t n_items, uint32_t* head,
                                                       const __grid_constant__ Keys keys) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) SimArgs sa;
  __shared__ int32_t s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int32_t)atomicAdd(head, 1u);
    __syncthreads();
    const int32_t it = s_item;
    if (it >= n_items) break;
    const BatchItem bi = items[it];
    const uint32_t* src = reinterpret_cast<const uint32_t*>(insts + bi.inst);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
    for (int k = threadIdx.x; k < (int)(sizeof(SimArgs) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    run_tile<kMode>(sa, keys, (int64_t)bi.tile * kThreads + threadIdx.x, smem);
    __syncthreads();
  }
}

}  // namespace mg
