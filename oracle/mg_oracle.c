/*
 * mg_oracle.c -- plain FP64 CPU oracle for the timestep-splitting
 * Euler-Maruyama scheme on metric graphs (arXiv 2512.02175).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, by the smoke check and
 * by the CPU-baseline leg of the benchmark; never by the library.  It shares
 * no code with the CUDA path.
 *
 * Written for a reader who checks it against the paper by eye: one particle,
 * one step, one sub-step at a time, in the order of Algorithm 2 (general
 * graph), with the star-graph reading of Algorithm 1 for sub-steps that start
 * at a vertex.  Readings of the paper that it implements (where the text is
 * garbled, ambiguous or inconsistent):
 *
 *  R1  A sub-step that starts at a vertex moves into its edge: the normal is
 *      used as |W| (Algorithm 1, while loop), pointed into the edge at either
 *      end.  Algorithm 2 keeps the sign of W; Algorithm 1 and the proofs of
 *      Theorems 1-2 use |W|.
 *  R2  At the terminal end the distance is l_e - x and the increment enters
 *      with the opposite sign, so the quadratic solved is
 *      (-a) s^2 + (-b) s + (l_e - x) = 0 with a = mu h, b = sigma sqrt(h) W.
 *  R3  The interior is the open interval (0, l_e); the side hit is the side of
 *      the endpoint of the sub-step (Algorithm 2, hit test).
 *  R4  The jump law b_v is sampled with integer thresholds: slot j of vertex
 *      v is the first with u < T_j, T_j = floor(C_j 2^32) from the FP64
 *      running sums C_j of the normalised weights, the last forced to 2^32.
 *  R5  The hitting fraction alpha uses the drift and diffusion of the edge
 *      the sub-step was taken on (the h_k recursion in the proof of
 *      Theorem 1).
 *  R6  At most M splits per step (Theorem 1 bounds their number): on the
 *      M-th split the particle stays at the vertex on the chosen edge, the
 *      rest of the step is dropped and a truncation is counted.
 *  R7  An absorbing vertex removes the particle (edge = -1).
 *  R8  Exit counts: a sub-step that starts at a vertex and ends inside the
 *      edge counts one exit through that (vertex, edge, end) slot; this is
 *      the event whose law Corollary 1 states.
 *  R15 Position-dependent diffusion (the edge generator allows any C^1
 *      sigma_e; here the affine sigma_e(x) = sigma_e + sigma1_e x): like the
 *      drift, it is evaluated at the sub-step's starting point x_s (Algorithm
 *      1 evaluates mu_e and sigma_e there), so the increment is
 *      sigma_e(x_s) sqrt(h) W and the split's quadratic keeps B =
 *      sigma_e(x_s) sqrt(h) W.
 */
#include "mg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox */

/* Philox-4x32 round constants and Weyl key increments as published by
 * Salmon et al. (2011). */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: add the Weyl constants before each later round */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double or_u01(uint32_t w) {
  /* (2w + 1) 2^-33: every step exact in FP64, never 0 or 1 */
  return ((double)w * 2.0 + 1.0) * 0x1p-33;
}

void or_box_muller(uint32_t wa, uint32_t wb, double* z_cos, double* z_sin) {
  double ua = or_u01(wa);
  double ub = or_u01(wb);
  double r = sqrt(-2.0 * log(ua));
  double theta = 6.283185307179586 * ub; /* 2 pi rounded to FP64 */
  *z_cos = r * cos(theta);
  *z_sin = r * sin(theta);
}

static void key_of_seed(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
}

double or_normal(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t n) {
  uint32_t key[2], ctr[4], w[4];
  key_of_seed(seed, key);
  ctr[0] = n >> 2;
  ctr[1] = pid;
  ctr[2] = 0u; /* tag 0: normals of the sub-steps */
  ctr[3] = instance;
  or_philox4x32_10(ctr, key, w);
  double zc, zs;
  switch ((int)(n & 3u)) {
    case 0: or_box_muller(w[0], w[1], &zc, &zs); return zc;
    case 1: or_box_muller(w[0], w[1], &zc, &zs); return zs;
    case 2: or_box_muller(w[2], w[3], &zc, &zs); return zc;
    default: or_box_muller(w[2], w[3], &zc, &zs); return zs;
  }
}

uint32_t or_split_draw(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t j) {
  uint32_t key[2], ctr[4], w[4];
  key_of_seed(seed, key);
  ctr[0] = j >> 2; /* four draws per block */
  ctr[1] = pid;
  ctr[2] = 1u; /* tag 1: draws of vertex hits */
  ctr[3] = instance;
  or_philox4x32_10(ctr, key, w);
  return w[j & 3u];
}

/* ------------------------------------------------------------------- graph */

static void* xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

void or_graph_free(or_graph* g) {
  if (!g) return;
  free(g->src); free(g->dst); free(g->length); free(g->c0); free(g->c1);
  free(g->sigma); free(g->sigma1); free(g->w_init); free(g->w_term); free(g->hist_range);
  free(g->kind); free(g->vtx_off); free(g->slot_edge); free(g->slot_end);
  free(g->slot_T); free(g->slot_of_end);
  free(g);
}

int or_graph_build(int32_t V, int32_t E, const int32_t* src, const int32_t* dst,
                   const double* length, const double* c0, const double* c1,
                   const double* sigma, const double* w_init, const double* w_term,
                   const double* hist_range, const uint8_t* kind, or_graph** out) {
  *out = NULL;
  if (V < 1 || E < 1) return -1;
  for (int32_t e = 0; e < E; ++e) {
    if (src[e] < 0 || src[e] >= V) return -1;
    if (dst[e] < -1 || dst[e] >= V) return -1;
    if (dst[e] == -1) {
      if (!(isinf(length[e]) && length[e] > 0)) return -1;
    } else if (!(isfinite(length[e]) && length[e] > 0)) {
      return -1;
    }
    if (!(isfinite(sigma[e]) && sigma[e] > 0)) return -1;
    if (!isfinite(c0[e]) || !isfinite(c1[e])) return -1;
    if (!(isfinite(w_init[e]) && w_init[e] >= 0)) return -1;
    if (dst[e] >= 0 && !(isfinite(w_term[e]) && w_term[e] >= 0)) return -1;
    if (hist_range && !(isfinite(hist_range[e]) && hist_range[e] > 0)) return -1;
  }
  if (kind)
    for (int32_t v = 0; v < V; ++v)
      if (kind[v] > OR_VERTEX_ABSORBING) return -1;

  or_graph* g = (or_graph*)xcalloc(1, sizeof(or_graph));
  g->n_vertices = V;
  g->n_edges = E;
  g->src = (int32_t*)xcalloc(E, 4); g->dst = (int32_t*)xcalloc(E, 4);
  g->length = (double*)xcalloc(E, 8); g->c0 = (double*)xcalloc(E, 8);
  g->c1 = (double*)xcalloc(E, 8); g->sigma = (double*)xcalloc(E, 8);
  g->sigma1 = (double*)xcalloc(E, 8); /* constant diffusion unless set */
  g->w_init = (double*)xcalloc(E, 8); g->w_term = (double*)xcalloc(E, 8);
  g->hist_range = (double*)xcalloc(E, 8);
  g->kind = (uint8_t*)xcalloc(V, 1);
  memcpy(g->src, src, 4 * (size_t)E); memcpy(g->dst, dst, 4 * (size_t)E);
  memcpy(g->length, length, 8 * (size_t)E); memcpy(g->c0, c0, 8 * (size_t)E);
  memcpy(g->c1, c1, 8 * (size_t)E); memcpy(g->sigma, sigma, 8 * (size_t)E);
  memcpy(g->w_init, w_init, 8 * (size_t)E);
  for (int32_t e = 0; e < E; ++e) {
    g->w_term[e] = (dst[e] >= 0) ? w_term[e] : 0.0;
    /* histogram range: given, else the length, else 1 for a semi-infinite edge */
    if (hist_range) g->hist_range[e] = hist_range[e];
    else g->hist_range[e] = (dst[e] >= 0) ? length[e] : 1.0;
  }
  if (kind) memcpy(g->kind, kind, (size_t)V);

  /* slots: one per (vertex, incident edge end), ordered by vertex, then edge
   * id, then init end before term end (a self-loop has two) -- the incident
   * edge sets E(v) of the paper, with orientations */
  g->vtx_off = (int32_t*)xcalloc((size_t)V + 1, 4);
  int32_t S = 0;
  for (int32_t e = 0; e < E; ++e) S += (dst[e] >= 0) ? 2 : 1;
  g->n_slots = S;
  g->slot_edge = (int32_t*)xcalloc(S, 4);
  g->slot_end = (uint8_t*)xcalloc(S, 1);
  g->slot_T = (uint64_t*)xcalloc(S, 8);
  g->slot_of_end = (int32_t*)xcalloc(2 * (size_t)E, 4);
  for (int32_t i = 0; i < 2 * E; ++i) g->slot_of_end[i] = -1;
  double* wslot = (double*)xcalloc(S, 8);
  int32_t s = 0;
  for (int32_t v = 0; v < V; ++v) { /* plain O(V E) scan: obviously ordered */
    g->vtx_off[v] = s;
    for (int32_t e = 0; e < E; ++e) {
      if (src[e] == v) {
        g->slot_edge[s] = e; g->slot_end[s] = OR_END_INIT; wslot[s] = g->w_init[e];
        g->slot_of_end[2 * e + OR_END_INIT] = s; ++s;
      }
      if (dst[e] == v) {
        g->slot_edge[s] = e; g->slot_end[s] = OR_END_TERM; wslot[s] = g->w_term[e];
        g->slot_of_end[2 * e + OR_END_TERM] = s; ++s;
      }
    }
  }
  g->vtx_off[V] = s;

  /* jump thresholds (reading R4) */
  for (int32_t v = 0; v < V; ++v) {
    int32_t lo = g->vtx_off[v], hi = g->vtx_off[v + 1];
    if (lo == hi) continue;
    double wtot = 0.0;
    for (int32_t j = lo; j < hi; ++j) wtot = wtot + wslot[j];
    if (g->kind[v] == OR_VERTEX_STANDARD && !(wtot > 0.0)) {
      free(wslot);
      or_graph_free(g);
      return -1; /* b_v must be a distribution (Definition 4) */
    }
    double cum = 0.0;
    for (int32_t j = lo; j < hi; ++j) {
      cum = cum + wslot[j];
      double c = (wtot > 0.0) ? cum / wtot : 1.0;
      double t = floor(c * 4294967296.0);
      g->slot_T[j] = (t >= 4294967296.0) ? 4294967296ull : (uint64_t)t;
    }
    g->slot_T[hi - 1] = 4294967296ull;
  }
  free(wslot);
  *out = g;
  return 0;
}

int or_graph_set_sigma1(or_graph* g, const double* sigma1) {
  for (int32_t e = 0; e < g->n_edges; ++e) {
    if (!isfinite(sigma1[e])) return -1;
    if (g->dst[e] < 0) {
      if (sigma1[e] < 0.0) return -1;
    } else if (!(g->sigma[e] + sigma1[e] * g->length[e] > 0.0)) {
      return -1;
    }
  }
  memcpy(g->sigma1, sigma1, 8 * (size_t)g->n_edges);
  return 0;
}

int32_t or_graph_n_slots(const or_graph* g) { return g->n_slots; }

void or_graph_slots(const or_graph* g, int32_t* vtx_off, int32_t* slot_edge,
                    uint8_t* slot_end, uint64_t* slot_T) {
  memcpy(vtx_off, g->vtx_off, 4 * ((size_t)g->n_vertices + 1));
  memcpy(slot_edge, g->slot_edge, 4 * (size_t)g->n_slots);
  memcpy(slot_end, g->slot_end, (size_t)g->n_slots);
  memcpy(slot_T, g->slot_T, 8 * (size_t)g->n_slots);
}

int32_t or_choose_slot(const or_graph* g, int32_t v, uint32_t u) {
  for (int32_t j = g->vtx_off[v]; j < g->vtx_off[v + 1]; ++j)
    if ((uint64_t)u < g->slot_T[j]) return j;
  return g->vtx_off[v + 1] - 1; /* unreachable: the last threshold is 2^32 */
}

/* --------------------------------------------------------- hitting fraction */

/* The partial sub-step of Algorithms 1-2: the particle reaches the vertex at
 * the fraction alpha of the remaining time h where
 *   d + alpha mu h + sigma sqrt(alpha h) W = 0   (init end, d = x),
 * i.e. with s = sqrt(alpha):  A s^2 + B s + C = 0,  A = mu h, B = sigma
 * sqrt(h) W, C = d >= 0.  Since the sub-step ends beyond the vertex,
 * A + B + C <= 0, so a root lies in [0,1]; we want the first one.
 *   A = 0:  s = -C/B (B = 0 means the sub-step did not move: s = 0).
 *   A != 0: roots (-B -+ sqrt(B^2 - 4AC)) / (2A).  The first crossing is
 *           (-B - d)/(2A), which equals 2C/(-B + d); each form is used on the
 *           side where it has no cancellation (B > 0 resp. B <= 0).
 * Rounding can leave the discriminant slightly negative or s slightly outside
 * [0,1]; both are clamped. */
double or_root(double A, double B, double C) {
  double s;
  if (A == 0.0) {
    s = (B == 0.0) ? 0.0 : -C / B;
  } else {
    double disc = B * B - 4.0 * A * C;
    double d = sqrt(disc > 0.0 ? disc : 0.0);
    if (B > 0.0) {
      s = (-B - d) / (2.0 * A);
    } else {
      double den = -B + d;
      s = (den == 0.0) ? 0.0 : (2.0 * C) / den;
    }
  }
  if (!(s > 0.0)) s = 0.0; /* also maps NaN to 0 */
  if (s > 1.0) s = 1.0;
  return s;
}

/* ------------------------------------------------------------------ EM-Step */

static double philox_normal(or_draws* self, or_particle* p) {
  double z = or_normal(self->seed, self->instance, self->pid, p->n_draw);
  p->n_draw++;
  return z;
}

static uint32_t philox_split(or_draws* self, const or_particle* p, uint32_t j) {
  (void)p;
  return or_split_draw(self->seed, self->instance, self->pid, j);
}

static double injected_normal(or_draws* self, or_particle* p) {
  p->n_draw++;
  return (self->pos_z < self->n_z) ? self->zs[self->pos_z++] : 0.0;
}

static uint32_t injected_split(or_draws* self, const or_particle* p, uint32_t j) {
  (void)p; (void)j;
  return (self->pos_u < self->n_u) ? self->us[self->pos_u++] : 0u;
}

int or_em_step(const or_graph* g, or_particle* p, double dt, int32_t M, or_draws* rnd,
               or_counters* cnt) {
  if (p->edge == OR_DEAD) return 0;
  double h = dt; /* time left in this step */
  int32_t k = 0; /* splits taken in this step */
  for (;;) {
    int32_t e = p->edge;
    double l = g->length[e];
    /* a particle sits at a vertex exactly when x is an endpoint (the
     * interior is open, R3, so only a split puts it there) */
    int at_end = -1;
    if (p->x == 0.0) at_end = OR_END_INIT;
    else if (p->x == l) at_end = OR_END_TERM;
    double W = rnd->normal(rnd, p);               /* Sample W ~ N(0,1) */
    if (at_end == OR_END_INIT) W = fabs(W);       /* R1 */
    else if (at_end == OR_END_TERM) W = -fabs(W); /* R1 */

    /* Euler-Maruyama sub-step (Eq. of the scheme on the real line) */
    double xs = p->x;
    double mu = g->c0[e] + g->c1[e] * xs;
    double sig = g->sigma[e] + g->sigma1[e] * xs; /* R15 */
    double a = mu * h;
    double b = sig * sqrt(h) * W;
    double xt = xs + a + b;

    double tol = 1e-9 * ((isfinite(l) && l > 1.0) ? l : 1.0);
    if (fabs(xt) < tol || (isfinite(l) && fabs(l - xt) < tol)) p->flags |= OR_FLAG_NEAR;

    if (xt > 0.0 && xt < l) { /* no vertex hit (R3) */
      if (at_end >= 0) cnt->exits[g->slot_of_end[2 * e + at_end]]++; /* R8 */
      p->x = xt;
      return k;
    }

    /* vertex hit: partial step to the vertex (R2, R3, R5) */
    int hit_init = (xt <= 0.0);
    int32_t v = hit_init ? g->src[e] : g->dst[e];
    double A = hit_init ? a : -a;
    double B = hit_init ? b : -b;
    double C = hit_init ? xs : l - xs;
    double s = or_root(A, B, C);
    double alpha = s * s;
    h = (1.0 - alpha) * h; /* remaining time */
    if (h < 1e-9 * dt) p->flags |= OR_FLAG_NEAR;
    uint32_t j = p->hits;
    p->hits = j + 1u;
    if (at_end < 0) p->first_hits++;
    k++;

    if (g->kind[v] == OR_VERTEX_ABSORBING) { /* R7 */
      cnt->absorbed[v]++;
      p->edge = OR_DEAD;
      return k;
    }

    /* sample the next edge from b_v (R4) and restart at its end */
    uint32_t u = rnd->split(rnd, p, j);
    int32_t slot = or_choose_slot(g, v, u);
    int32_t e2 = g->slot_edge[slot];
    p->edge = e2;
    p->x = (g->slot_end[slot] == OR_END_INIT) ? 0.0 : g->length[e2];

    if (k == M) { /* R6 */
      cnt->truncations++;
      return k;
    }
    if (h <= 0.0) return k;
    /* the rest of the step continues from the vertex with the next normal */
  }
}

void or_simulate(const or_graph* g, int64_t n, const uint32_t* pid, int32_t* edge,
                 double* x, uint32_t* n_draw, uint32_t* hits, uint32_t* first_hits,
                 uint32_t* flags, uint64_t seed, uint32_t instance, double dt,
                 int64_t steps, int32_t M, uint64_t* exits, uint64_t* absorbed,
                 uint64_t* truncations, int64_t* particle_steps) {
  or_counters cnt;
  cnt.exits = exits;
  cnt.absorbed = absorbed;
  cnt.truncations = 0;
  int64_t ps = 0;
  for (int64_t i = 0; i < n; ++i) {
    or_particle p;
    p.edge = edge[i]; p.x = x[i]; p.n_draw = n_draw[i]; p.hits = hits[i];
    p.first_hits = first_hits[i]; p.flags = flags[i];
    or_draws rnd;
    memset(&rnd, 0, sizeof rnd);
    rnd.normal = philox_normal;
    rnd.split = philox_split;
    rnd.seed = seed; rnd.instance = instance; rnd.pid = pid[i];
    for (int64_t st = 0; st < steps; ++st) {
      if (p.edge == OR_DEAD) break;
      or_em_step(g, &p, dt, M, &rnd, &cnt);
      ps++;
    }
    edge[i] = p.edge; x[i] = p.x; n_draw[i] = p.n_draw; hits[i] = p.hits;
    first_hits[i] = p.first_hits; flags[i] = p.flags;
  }
  *truncations += cnt.truncations;
  if (particle_steps) *particle_steps += ps;
}

void or_histogram(const or_graph* g, int64_t n, const int32_t* edge, const double* x,
                  int32_t B, uint64_t* hist) {
  for (int64_t i = 0; i < n; ++i) {
    int32_t e = edge[i];
    if (e == OR_DEAD) continue;
    double scale = (double)B / g->hist_range[e];
    double f = floor(x[i] * scale);
    int64_t bin = (f < 0.0) ? 0 : (f > (double)(B - 1)) ? (int64_t)(B - 1) : (int64_t)f;
    hist[(int64_t)e * B + bin]++;
  }
}

void or_histogram_binned(const or_graph* g, int64_t n, const int32_t* edge, const double* x,
                         const int32_t* off, const double* up, uint64_t* hist) {
  (void)g;
  for (int64_t i = 0; i < n; ++i) {
    int32_t e = edge[i];
    if (e == OR_DEAD || off[e] == off[e + 1]) continue;
    int32_t j = off[e];
    while (j < off[e + 1] - 1 && !(x[i] < up[j])) j++;
    hist[j]++;
  }
}

int or_em_step_injected(const or_graph* g, int32_t* edge, double* x, uint32_t* n_draw,
                        uint32_t* hits, uint32_t* first_hits, uint32_t* flags, double dt,
                        int32_t M, const double* zs, int32_t n_z, const uint32_t* us,
                        int32_t n_u, uint64_t* exits, uint64_t* absorbed,
                        uint64_t* truncations) {
  or_particle p;
  p.edge = *edge; p.x = *x; p.n_draw = *n_draw; p.hits = *hits; p.first_hits = *first_hits;
  p.flags = *flags;
  or_draws rnd;
  memset(&rnd, 0, sizeof rnd);
  rnd.normal = injected_normal;
  rnd.split = injected_split;
  rnd.zs = zs; rnd.n_z = n_z; rnd.us = us; rnd.n_u = n_u;
  or_counters cnt;
  cnt.exits = exits; cnt.absorbed = absorbed; cnt.truncations = 0;
  int k = or_em_step(g, &p, dt, M, &rnd, &cnt);
  *edge = p.edge; *x = p.x; *n_draw = p.n_draw; *hits = p.hits; *first_hits = p.first_hits;
  *flags = p.flags;
  *truncations += cnt.truncations;
  return k;
}
