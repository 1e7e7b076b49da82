/*
 * mg_oracle.h -- plain, slow FP64 CPU oracle for the timestep-splitting
 * Euler-Maruyama scheme on metric graphs ("Sampling on Metric Graphs",
 * arXiv 2512.02175).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check in
 * __graft_entry__ and the CPU-baseline leg of bench.py may load this code.
 * It shares no source, header, table or constant with the CUDA library; the
 * two agree only because both follow the same written rules (the paper's
 * Algorithms 1 and 2 plus the readings listed with each function).
 *
 * Everything is FP64, written without fused multiply-adds (compile with
 * -ffp-contract=off), one particle at a time, one step at a time.
 */
#ifndef MG_ORACLE_H
#define MG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- random */

/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As
 * Easy as 1, 2, 3", SC'11): ten rounds of the 4x32 S-box with the Weyl key
 * schedule.  ctr[4], key[2] in; out[4] out. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* u = (2w+1) 2^-33, an exact double in (0,1). */
double or_u01(uint32_t w);

/* Box & Muller (1958): r = sqrt(-2 ln u_a), theta = 2 pi u_b,
 * z_cos = r cos(theta), z_sin = r sin(theta). */
void or_box_muller(uint32_t wa, uint32_t wb, double* z_cos, double* z_sin);

/* The n-th normal of particle pid (one per Euler-Maruyama sub-step, in
 * order): block (n>>2, pid, 0, instance) under key (seed lo, seed hi); lane
 * n&3 picks z_cos(w0,w1), z_sin(w0,w1), z_cos(w2,w3), z_sin(w2,w3). */
double or_normal(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t n);

/* The uniform 32-bit draw of the j-th vertex hit of particle pid (it picks
 * the next edge): word w[j&3] of block (j>>2, pid, 1, instance), four draws
 * per block. */
uint32_t or_split_draw(uint64_t seed, uint32_t instance, uint32_t pid, uint32_t j);

/* ----------------------------------------------------------------- graph */

#define OR_END_INIT 0
#define OR_END_TERM 1
#define OR_VERTEX_STANDARD 0
#define OR_VERTEX_ABSORBING 1
#define OR_DEAD (-1)

typedef struct {
  int32_t n_vertices, n_edges;
  /* per edge (Definition 1): init vertex, term vertex (-1: vertex at
   * infinity, length = +inf), length l_e, drift mu_e(x) = c0 + c1 x,
   * diffusion sigma_e, unnormalised jump weights b at each end, histogram
   * range (l_e unless the edge is semi-infinite). */
  int32_t *src, *dst;
  double *length, *c0, *c1, *sigma, *w_init, *w_term, *hist_range;
  /* diffusion slope: sigma_e(x) = sigma + sigma1 x (zero unless set by
   * or_graph_set_sigma1) */
  double* sigma1;
  uint8_t* kind; /* per vertex */
  /* CSR of vertex-edge incidences ("slots"), ordered by (vertex, edge id,
   * init end before term end). */
  int32_t n_slots;
  int32_t* vtx_off;     /* [V+1] */
  int32_t* slot_edge;   /* [S] */
  uint8_t* slot_end;    /* [S] */
  uint64_t* slot_T;     /* [S] integer jump thresholds in [0, 2^32] */
  int32_t* slot_of_end; /* [2E] slot of (edge, end); -1 if absent */
} or_graph;

/* Copies the description and builds the slots and thresholds.  Returns 0,
 * or a negative code for an invalid description. */
int or_graph_build(int32_t n_vertices, int32_t n_edges, const int32_t* src,
                   const int32_t* dst, const double* length, const double* c0,
                   const double* c1, const double* sigma, const double* w_init,
                   const double* w_term, const double* hist_range,
                   const uint8_t* kind, or_graph** out);
void or_graph_free(or_graph* g);
/* Position-dependent diffusion sigma_e(x) = sigma_e + sigma1_e x (x from
 * e_init), positive on the whole edge: sigma_e + sigma1_e l_e > 0 on a
 * finite edge, sigma1_e >= 0 on a semi-infinite one.  Returns 0, or a
 * negative code (nothing changed) for an invalid slope. */
int or_graph_set_sigma1(or_graph* g, const double* sigma1);
int32_t or_graph_n_slots(const or_graph* g);
void or_graph_slots(const or_graph* g, int32_t* vtx_off, int32_t* slot_edge,
                    uint8_t* slot_end, uint64_t* slot_T);

/* Slot chosen at vertex v for the draw u: the first slot j of v with
 * u < T_j. */
int32_t or_choose_slot(const or_graph* g, int32_t v, uint32_t u);

/* Smallest root s in [0,1] of A s^2 + B s + C = 0 (C >= 0), s = sqrt(alpha);
 * see or_em_step for where it comes from. */
double or_root(double A, double B, double C);

/* ------------------------------------------------------------- particles */

typedef struct {
  int32_t edge;        /* OR_DEAD once absorbed */
  double x;            /* position on the edge, measured from e_init */
  uint32_t n_draw;     /* normals used so far (= index of the next one) */
  uint32_t hits;       /* vertex hits so far (= index of the next split draw) */
  uint32_t first_hits; /* hits that started from the interior of an edge */
  uint32_t flags;      /* bit 0: trajectory passed within 1e-9 of a branch */
} or_particle;

#define OR_FLAG_NEAR 1u

typedef struct {
  uint64_t* exits;      /* [S] sub-steps leaving a vertex into the slot's edge */
  uint64_t* absorbed;   /* [V] */
  uint64_t truncations; /* steps that hit the split cap M */
} or_counters;

/* Source of the random draws (Philox normally; tests inject hand-chosen
 * sequences): normal() returns the particle's next normal and advances
 * p->n_draw; split() returns the u32 of the particle's j-th vertex hit. */
typedef struct or_draws {
  double (*normal)(struct or_draws* self, or_particle* p);
  uint32_t (*split)(struct or_draws* self, const or_particle* p, uint32_t j);
  uint64_t seed;
  uint32_t instance, pid;
  /* injection */
  const double* zs;
  const uint32_t* us;
  int32_t n_z, n_u, pos_z, pos_u;
} or_draws;

/* One EM-Step of length dt (Algorithm 2 with the readings of Algorithm 1).
 * Returns the number of splits. */
int or_em_step(const or_graph* g, or_particle* p, double dt, int32_t M, or_draws* rnd,
               or_counters* cnt);

/* Advance particles i = 0..n-1 (global ids pid[i]) by `steps` EM-Steps.
 * State arrays are updated in place; counters accumulate. */
void or_simulate(const or_graph* g, int64_t n, const uint32_t* pid, int32_t* edge,
                 double* x, uint32_t* n_draw, uint32_t* hits, uint32_t* first_hits,
                 uint32_t* flags, uint64_t seed, uint32_t instance, double dt,
                 int64_t steps, int32_t M, uint64_t* exits, uint64_t* absorbed,
                 uint64_t* truncations, int64_t* particle_steps);

/* Snapshot histogram of living particles: B bins of width range_e/B per
 * edge, bin = clamp(floor(x * (B / range_e)), 0, B-1); hist[E*B] accumulates. */
void or_histogram(const or_graph* g, int64_t n, const int32_t* edge, const double* x,
                  int32_t B, uint64_t* hist);

/* Snapshot histogram with bins of any width per edge (Section 4.1 estimates
 * densities by histograms; the bins of edge e are off[e] .. off[e+1]-1 with
 * upper boundaries up[j], increasing within the edge).  A living particle at
 * x on e counts in the first bin j of e with x < up[j], else in e's last bin;
 * an edge without bins counts nothing.  hist[off[E]] accumulates. */
void or_histogram_binned(const or_graph* g, int64_t n, const int32_t* edge, const double* x,
                         const int32_t* off, const double* up, uint64_t* hist);

/* Test hook: one EM-Step of one particle with injected draws: the normals
 * zs[0..n_z) of its sub-steps in order, the u32s us[0..n_u) of its hits. */
int or_em_step_injected(const or_graph* g, int32_t* edge, double* x, uint32_t* n_draw,
                        uint32_t* hits, uint32_t* first_hits, uint32_t* flags, double dt,
                        int32_t M, const double* zs, int32_t n_z, const uint32_t* us,
                        int32_t n_u, uint64_t* exits, uint64_t* absorbed,
                        uint64_t* truncations);

#ifdef __cplusplus
}
#endif
#endif
