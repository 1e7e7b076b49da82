/*
 * mg.h -- C ABI of libmetricgraph: the timestep-splitting Euler-Maruyama
 * scheme for diffusions on metric graphs ("Sampling on Metric Graphs",
 * arXiv 2512.02175), run on one NVIDIA GB300 (sm_103a).
 *
 * Conventions (every entry point):
 *  - Returns an mg_status; no C++ exception crosses this boundary.  On an
 *    error, mg_last_error() returns a message for the calling thread.
 *  - Pointers marked "host" are caller-owned host memory, read (or written)
 *    only during the call.  Pointers marked "device" are caller-owned device
 *    memory on the current CUDA device (managed memory and mapped pinned host
 *    memory qualify).  A device pointer to ordinary host memory or to another
 *    device's memory, and a host pointer to device memory, are rejected
 *    (MG_ERR_INVALID_ARG) before anything runs; array lengths are the
 *    caller's.  Handles (mg_graph, mg_particles) are library-owned and freed
 *    by their _destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL: the legacy default
 *    stream).  Calls that take a stream are stream-ordered and may return
 *    before the GPU work finishes; errors found on the GPU are reported by the
 *    next mg_synchronize or by any call that reads results back.  The library
 *    orders work on one handle only within one stream: a caller that moves a
 *    handle to another stream orders the two (an event, or a synchronize).
 *  - Device memory is obtained through the allocator set by
 *    mg_set_allocator (default: cudaMalloc/cudaFree).
 *  - Floating-point inputs are IEEE binary64.  Integers are fixed width.
 *
 * Notation follows the paper: a metric graph (V, E, l) has edges e identified
 * with intervals (0, l_e); e_init and e_term are the vertices at x = 0 and
 * x = l_e (Definition 1).  A particle is a pair (e, x).  b_v is the
 * vertex-edge jump distribution of the standard gluing conditions
 * (Definition 4); E(v) is the set of edges incident to v.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_graph_s* mg_graph;
typedef struct mg_particles_s* mg_particles;

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,   /* an argument violates the stated contract */
  MG_ERR_OUT_OF_MEMORY = 2, /* the allocator returned NULL */
  MG_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in mg_last_error) */
  MG_ERR_TIMEOUT = 4,       /* a bounded wait ran out */
  MG_ERR_CANCELLED = 5,     /* work was cancelled by the caller */
  MG_ERR_BUSY = 6,          /* the handle is still referenced */
  MG_ERR_DEVICE_FAULT = 7   /* a kernel flagged an invariant violation */
} mg_status;

typedef enum {
  MG_FP64 = 0,       /* every step in binary64 */
  MG_FP32_MIXED = 1, /* positions, increments and normals in binary32; the
                        hitting fraction alpha and the time left of a split
                        in binary64; counts in integers */
  MG_FP32 = 2        /* everything in binary32; counts in integers */
} mg_precision;

typedef enum { MG_VERTEX_STANDARD = 0, MG_VERTEX_ABSORBING = 1 } mg_vertex_kind;

/* Device-error bits reported with MG_ERR_DEVICE_FAULT. */
#define MG_DEVERR_BAD_EDGE 1u  /* a particle's edge index out of range */
#define MG_DEVERR_NAN 2u       /* a position was NaN, infinite or outside [0, l_e], or
                                  overflowed to infinity (the particle stops) */
#define MG_DEVERR_STREAM 4u    /* a particle used up its 2^32 - 16 normals */
#define MG_DEVERR_STUCK 8u     /* the kernel's loop guard fired (a library bug) */

/* Description of a metric graph (Definition 1; drift and diffusion of the
 * edge generator, Eq. (generator_edge); jump weights of the standard
 * gluing conditions, Definition 4).  All arrays host, length n_edges unless
 * noted; copied by mg_graph_create. */
typedef struct {
  int32_t n_vertices;          /* >= 1 */
  int32_t n_edges;             /* >= 1 */
  const int32_t* edge_src;     /* e_init in [0, n_vertices) */
  const int32_t* edge_dst;     /* e_term in [0, n_vertices), or -1: the edge is
                                  semi-infinite (a vertex at infinity) */
  const double* length;        /* l_e > 0 finite; +INFINITY iff edge_dst == -1 */
  const double* drift_c0;      /* mu_e(x) = c0 + c1 x, x measured from e_init */
  const double* drift_c1;
  const double* sigma;         /* diffusion sigma_e > 0, constant on the edge */
  const double* weight_init;   /* >= 0: unnormalised b_{v e} at v = e_init */
  const double* weight_term;   /* >= 0: unnormalised b_{v e} at v = e_term
                                  (ignored for semi-infinite edges) */
  const double* hist_range;    /* NULL, or > 0 finite: the histogram covers
                                  [0, hist_range_e); NULL means l_e (1 for a
                                  semi-infinite edge) */
  const uint8_t* vertex_kind;  /* [n_vertices] mg_vertex_kind, or NULL (all
                                  standard) */
  const double* sigma_slope;   /* NULL (constant diffusion), or the slope k_e of a
                                  position-dependent diffusion sigma_e(x) = sigma_e
                                  + k_e x (x from e_init; the edge generator allows
                                  any C^1 sigma_e, Section 2.2), evaluated at each
                                  sub-step's starting point as Algorithm 1 evaluates
                                  the coefficients; finite, with sigma_e(x) > 0 on
                                  the whole edge (k_e >= 0 on a semi-infinite one) */
} mg_graph_desc;

/* ---------------------------------------------------------------- memory */

/* Allocation hooks (e.g. a framework's caching allocator).  alloc returns
 * device memory of at least `bytes` bytes usable on `stream`, or NULL;
 * free releases it.  Passing NULL for both restores cudaMalloc/cudaFree.
 * Set before creating handles; memory is freed with the hooks that
 * allocated it. */
typedef void* (*mg_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*mg_free_fn)(void* ptr, void* stream, void* ctx);
mg_status mg_set_allocator(mg_alloc_fn alloc, mg_free_fn free_fn, void* ctx);

/* ----------------------------------------------------------------- graph */

/* Validates `desc`, builds the incident-edge table ("slots": one per
 * (vertex, incident edge end), ordered by vertex, then edge id, then init end
 * before term end; a self-loop has two) and the integer jump thresholds that
 * sample b_v (T_j = floor(2^32 C_j) from the binary64 running sums C_j of the
 * normalised weights of v's slots, the last forced to 2^32; slot j is the
 * first with u < T_j for a uniform 32-bit u), and uploads them to the current
 * device.  MG_ERR_INVALID_ARG for: a vertex id out of range; a length <= 0 or
 * NaN, infinite on a finite edge or finite on a semi-infinite one; sigma <= 0;
 * a non-finite drift; a negative weight; a standard vertex with incident
 * slots whose weights sum to 0; a bad hist_range or vertex kind; a slope that
 * is not finite or lets sigma_e(x) reach 0 on the edge. */
mg_status mg_graph_create(const mg_graph_desc* desc, mg_graph* out);

/* MG_ERR_BUSY while particle sets created on the graph are alive. */
mg_status mg_graph_destroy(mg_graph g);

/* Sizes of the graph: any output pointer may be NULL. */
mg_status mg_graph_info(mg_graph g, int32_t* n_vertices, int32_t* n_edges, int32_t* n_slots);

/* Copies the slot table to host arrays: vtx_off[n_vertices + 1] (slots of v
 * are vtx_off[v] .. vtx_off[v+1]-1), slot_edge[n_slots], slot_end[n_slots]
 * (0 init, 1 term), slot_threshold[n_slots] (T_j in [0, 2^32]).  Any pointer
 * may be NULL. */
mg_status mg_graph_slots(mg_graph g, int32_t* vtx_off, int32_t* slot_edge, uint8_t* slot_end,
                         uint64_t* slot_threshold);

/* ------------------------------------------------------------- particles */

/* Creates a set of n particles on g (1 <= n <= 2^31 - 1).  edge0[n], x0[n]:
 * starting edges and positions, host arrays, or device arrays when
 * inputs_on_device != 0; 0 <= x0 <= l_e and finite (x0 = 0 or l_e starts the
 * particle at that vertex; a semi-infinite edge has no far vertex).  Host
 * arrays have been copied when the call returns (pinned memory included).  Particle i has the global id pid = pid_base + i (must not
 * wrap 2^32).  Its random numbers are Philox-4x32-10 (Salmon et al., SC'11)
 * blocks under the key (seed mod 2^32, seed >> 32):
 *   the n-th normal (one per Euler-Maruyama sub-step -- the first of a step
 *   and each one after a split, in order) is Box-Muller of block
 *   (n >> 2, pid, 0, instance_id): lanes n & 3 = 0..3 take r cos and r sin of
 *   words (w0, w1), then of (w2, w3), with u = (2w + 1) 2^-33 (binary64) or
 *   (2 (w >> 9) + 1) 2^-24 (binary32 modes);
 *   the j-th vertex hit draws its next edge with word w0 of block
 *   (j, pid, 1, instance_id),
 * so results do not depend on how particles are sharded or batched.  The
 * state holds, per particle: edge (-1 once absorbed), position x, n_draw
 * (normals used), hits, first_hits (hits that started inside the edge), flags
 * (bit 0: the binary64 trajectory passed within 1e-9 max(1, l_e) of a
 * branch).  Step counter and all counters start at 0.  Host inputs are
 * validated (MG_ERR_INVALID_ARG); device inputs are validated by the kernel
 * (reported by mg_synchronize). */
mg_status mg_particles_init(mg_graph g, int64_t n, const int32_t* edge0, const double* x0,
                            int inputs_on_device, uint32_t pid_base, uint64_t seed,
                            uint32_t instance_id, mg_precision precision, void* stream,
                            mg_particles* out);

/* Re-initialises the positions of an existing set (same n, graph, seed,
 * precision) from edge0/x0 as in mg_particles_init, and zeroes its per-particle
 * counters, step counter and global counters.  Host inputs are checked before
 * anything changes (MG_ERR_INVALID_ARG leaves the set as it was) and have been
 * copied when the call returns; device inputs are read stream-ordered. */
mg_status mg_particles_reset(mg_particles p, const int32_t* edge0, const double* x0,
                             int inputs_on_device, void* stream);

mg_status mg_particles_destroy(mg_particles p);

/* Launch tuning of a set (the results do not depend on it): split_batch =
 * pending vertex hits in a warp that trigger a batched split pass (1..32; 0:
 * the library's default for the precision), steps_per_launch = largest number
 * of EM-Steps per kernel launch (0: no limit beyond the library's own),
 * max_blocks = for graphs with absorbing vertices, the most blocks of 256
 * threads a launch uses: a set larger than that is spread evenly over the
 * blocks, whose lanes take the next particle when theirs dies or finishes
 * (0: the library's choice -- the blocks resident on the GPU at once). */
mg_status mg_particles_set_tuning(mg_particles p, int32_t split_batch, int64_t steps_per_launch,
                                  int32_t max_blocks);

/* Advances every particle by `steps` EM-Steps of length dt (Algorithm 2 of
 * the paper, with sub-steps from a vertex taken into the edge with |W| as in
 * Algorithm 1): an Euler-Maruyama sub-step x + mu_e(x) h + sigma_e sqrt(h) W;
 * if it leaves the open interval (0, l_e), the partial step to the vertex
 * (first root s = sqrt(alpha) in [0,1] of the sub-step's quadratic path),
 * h <- (1 - alpha) h, the next edge drawn from b_v, and a new sub-step from
 * that vertex; at most max_splits_M splits per step (a step that reaches M
 * stays at the vertex and counts a truncation; Theorem 1); an absorbing
 * vertex removes the particle.  Exits (a sub-step from a vertex that ends
 * inside its edge), absorptions and truncations accumulate into the set's
 * counters.  1e-30 <= dt <= 1e30, steps >= 0, max_splits_M >= 1.
 * If hist_bins > 0 and hist_out != NULL, the snapshot occupancy histogram of
 * the final positions (as mg_histogram) is ADDED to the device array
 * hist_out[n_edges * hist_bins] (uint32, caller-zeroed) in the same kernel.
 * Stream-ordered. */
mg_status mg_simulate(mg_particles p, double dt, int64_t steps, int32_t max_splits_M,
                      int32_t hist_bins, uint32_t* hist_out, void* stream);

/* Time-averaged occupancy.  Section 4.1 estimates a steady-state density by a
 * histogram of the particles after a long run; averaging snapshots over time
 * lowers its noise.  Advances every particle by `steps` EM-Steps exactly as
 * mg_simulate does (bit-identical results) and ADDS the snapshot histogram of
 * the positions after every `every` EM-Steps -- steps / every snapshots, the
 * last after step (steps / every) * every; a remainder runs without one -- to
 * the device array hist_out[n_edges * hist_bins] (uint32, caller-zeroed;
 * bins as mg_histogram).  Divided by (snapshots x living particles) it is the
 * occupancy averaged over those times.  A bin must stay below 2^32 counts
 * (snapshots x n < 2^32 suffices).  every >= 1, hist_bins >= 1, hist_out
 * non-NULL; otherwise as mg_simulate.  Stream-ordered. */
mg_status mg_simulate_sampled(mg_particles p, double dt, int64_t steps, int32_t max_splits_M,
                              int64_t every, int32_t hist_bins, uint32_t* hist_out, void* stream);

/* ---------------------------------------------------------------- batches
 *
 * A batch advances many particle sets (instances: different graphs, sizes,
 * dt, step counts, M) in one launch of a persistent kernel: its blocks pop
 * work items -- 256 particles of one instance -- from a queue ordered by
 * decreasing step count, and run on each the same per-particle code as
 * mg_simulate, so every particle's result is bit-identical alone and in any
 * batch.  Members share one seed and one precision (instances differ by
 * instance_id and pid); a member must stay alive while the batch uses it. */
typedef struct mg_batch_s* mg_batch;

mg_status mg_batch_create(mg_batch* out);

/* Adds particle set p, to be advanced by `steps` EM-Steps of length dt with at
 * most max_splits_M splits per step, optionally adding its final-position
 * histogram to hist_out (device, [n_edges * hist_bins]), as mg_simulate does.
 * MG_ERR_INVALID_ARG for a different seed or precision than the first
 * member's, a set added twice, or the step arguments mg_simulate rejects. */
mg_status mg_batch_add(mg_batch b, mg_particles p, double dt, int64_t steps, int32_t max_splits_M,
                       int32_t hist_bins, uint32_t* hist_out);

mg_status mg_batch_clear(mg_batch b);

/* Launch tuning (the results do not depend on it): split_batch as in
 * mg_particles_set_tuning (0: default), stage_limit_bytes: a member's graph
 * tables are staged in shared memory only when they take at most this many
 * bytes (< 0: whenever they fit), blocks_per_sm: resident blocks of the
 * persistent kernel per SM (0: the occupancy maximum). */
mg_status mg_batch_set_tuning(mg_batch b, int32_t split_batch, int64_t stage_limit_bytes,
                              int32_t blocks_per_sm);

/* Advances every member once (stream-ordered).  The first run after a
 * change builds the instance table and work queue in device memory; with
 * use_graph != 0 it also captures the launch into a CUDA graph on `stream`
 * (which must not be the legacy default stream) and later runs replay it. */
mg_status mg_batch_run(mg_batch b, int use_graph, void* stream);

/* Members, work items and persistent blocks of the last build. */
mg_status mg_batch_info(mg_batch b, int32_t* n_members, int32_t* n_items, int32_t* blocks);

mg_status mg_batch_destroy(mg_batch b);

/* Waits for the set's stream work and reports any device-error bits as
 * MG_ERR_DEVICE_FAULT (the bits are in mg_last_error's message and are
 * cleared). */
mg_status mg_synchronize(mg_particles p);

/* Snapshot occupancy histogram of the living particles: `bins` equal bins
 * per edge over [0, hist_range_e); bin = min(floor(x * (bins / range_e)),
 * bins - 1), computed in the set's precision.  out[n_edges * bins] uint32 is
 * overwritten; it is device memory when out_on_device != 0 (stream-ordered),
 * else host memory (the call synchronises). */
mg_status mg_histogram(mg_particles p, int32_t bins, uint32_t* out, int out_on_device,
                       void* stream);

/* The same histogram as mg_histogram with a host output, for callers that
 * cannot let the library allocate device memory -- a fixed, pre-reserved
 * memory budget, code that must not synchronise the device the way
 * cudaMalloc/cudaFree can, or an allocator hook that is not safe to call at
 * this point.  The paper has no counterpart: it is a property of this
 * library.  The counts are staged in a static device array of at most
 * 2^20 counts (n_edges * bins; 4 MiB, held on every GPU that loads the
 * library until the process exits); larger requests return
 * MG_ERR_INVALID_ARG.  Nothing is allocated: no cudaMalloc, cudaFree or
 * allocator hook is called.  out[n_edges * bins] is host memory, overwritten;
 * the call synchronises `stream`.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it; if the
 * library's device code is not loaded on that device yet (CUDA's lazy module
 * loading), that lookup loads it, reserving the array, and may synchronise
 * the device -- so make the first call during set-up, before any stream
 * capture.  cudaDeviceReset frees the array: do not call this entry point on
 * a device after resetting it.  All calls share the one array, which keeps
 * the previous call's counts (each call clears what it uses): calls that
 * overlap on the GPU, from different streams or threads, race. */
mg_status mg_histogram_static(mg_particles p, int32_t bins, uint32_t* out, void* stream);

/* Snapshot histogram with bins of any width per edge (the paper's densities
 * are histograms of the particles' positions, Section 4.1; here each edge
 * takes its own bin boundaries).  bin_offsets[n_edges + 1] (host, int32):
 * the bins of edge e are bin_offsets[e] .. bin_offsets[e+1]-1, bin_offsets[0]
 * = 0, non-decreasing (an edge may have none); bin_upper[bin_offsets[n_edges]]
 * (host, binary64): the bins' upper boundaries, finite, > 0 and strictly
 * increasing within an edge.  A living particle at x on e counts in the first
 * bin j of e with x < bin_upper[j] -- half-open bins, as the uniform bins of
 * mg_histogram -- or in e's last bin when x is at or beyond every boundary;
 * edges without bins and dead particles count nothing.  For binary32 states
 * the boundaries are rounded up to binary32, which decides every comparison
 * exactly as in binary64.  out[bin_offsets[n_edges]] (uint32) is overwritten:
 * host memory (synchronises) or device memory (out_on_device != 0,
 * stream-ordered).  MG_ERR_INVALID_ARG for malformed offsets or boundaries. */
mg_status mg_histogram_binned(mg_particles p, const int32_t* bin_offsets, const double* bin_upper,
                              uint32_t* out, int out_on_device, void* stream);

/* Copies the set's counters to host arrays (synchronises): slot_exits[n_slots]
 * (in the slot order of mg_graph_slots), absorbed[n_vertices], truncations[1],
 * particle_steps[1] (steps taken by living particles).  Any pointer may be
 * NULL. */
mg_status mg_exit_counts(mg_particles p, uint64_t* slot_exits, uint64_t* absorbed,
                         uint64_t* truncations, uint64_t* particle_steps, void* stream);

/* Zeroes the set's counters (stream-ordered). */
mg_status mg_counters_reset(mg_particles p, void* stream);

/* Checkpoint: copies the full particle state to host arrays (synchronises);
 * positions are returned in binary64.  step: EM-Steps taken so far.  Any
 * pointer may be NULL. */
mg_status mg_state_get(mg_particles p, int32_t* edge, double* x, uint32_t* n_draw, uint32_t* hits,
                       uint32_t* first_hits, uint32_t* flags, uint64_t* step, void* stream);

/* Resume: overwrites the particle state from host arrays (all required) and
 * the step counter; with the counter-based random numbers the continuation is
 * bit-identical to an uninterrupted run. */
mg_status mg_state_set(mg_particles p, const int32_t* edge, const double* x,
                       const uint32_t* n_draw, const uint32_t* hits, const uint32_t* first_hits,
                       const uint32_t* flags, uint64_t step, void* stream);

/* The hitting fraction of a split (Section 3, the partial sub-step of
 * Algorithms 1 and 2): a sub-step x + a + b (a = mu_e h, b = sigma_e sqrt(h) W)
 * that ends beyond a vertex at distance C >= 0 reaches it after the fraction
 * alpha = s^2 of its time h, s the first root in [0, 1] of A s^2 + B s + C = 0
 * (A = a, B = b at e_init; A = -a, B = -b at e_term).  Computes s for n
 * coefficient triples with the device function that precision mode `mode`
 * uses in its kernels:
 *   MG_FP64        the closed form in binary64: d = sqrt(max(B^2 - 4AC, 0)),
 *                  s = (-B - d) / (2A) for B > 0, 2C / (-B + d) otherwise,
 *                  -C / B for A = 0, clamped to [0, 1] (correctly rounded
 *                  binary64 square root and quotient);
 *   MG_FP32_MIXED  the binary64 root of the FP32-mixed mode (the binary32
 *                  coefficients widened exactly; see mg_precision);
 *   MG_FP32        the binary32 root with the hardware's approximate square
 *                  root and reciprocal.
 * A, B, C: device, binary32 [n] (coefficients as the binary32 modes form
 * them); s: device, binary64 [n], overwritten.  n >= 0.  Stream-ordered. */
mg_status mg_hit_root(int32_t mode, int64_t n, const float* A, const float* B, const float* C,
                      double* s, void* stream);

/* n, precision and step counter of a set; any pointer may be NULL. */
mg_status mg_particles_info(mg_particles p, int64_t* n, int32_t* precision, uint64_t* step);

/* Message of the last error on the calling thread ("" if none). */
const char* mg_last_error(void);

/* Library version string. */
const char* mg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
