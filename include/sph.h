/*
 * sph.h -- C ABI of libsph, the GB300 (sm_103a) SPH neighbour-interaction
 * hot path after Schaller, Gonnet, Chalk, Draper, "SWIFT: Using task-based
 * parallelism, fully asynchronous communication, and graph partition-based
 * domain decomposition for strong scaling on more than 100,000 cores",
 * PASC '16.
 *
 * Problem statement (Section 2): particles with position x, velocity v,
 * internal energy u, mass m and smoothing length h in a periodic box. The
 * density stage solves each h_i so that the weighted neighbour number
 * N_i(h) = (4 pi / 3) h^3 sum_j W(r_ij, h) equals n_ngb, and evaluates
 * rho_i (Eq. rho), Omega_i and P_i; the force stage evaluates Eqs. (dvdt) and
 * (dudt); the integrator task (Section 3.1) updates positions and velocities.
 * W is the cubic spline with support radius h (W(r,h) = (8/pi) w(r/h) / h^3,
 * w(q) = 1 - 6q^2 + 6q^3 below q = 1/2, 2(1-q)^3 up to q = 1).
 *
 * Conventions shared by every call:
 *   - Return value: 0 (SPH_OK) on success, else a negative SPH_E* code;
 *     sph_last_error() then holds a one-line message.
 *   - Device pointers are CUDA global-memory addresses on the device that was
 *     current when sph_create() ran; host pointers are ordinary host memory.
 *   - All work is enqueued on the stream given to sph_create(). Calls that
 *     must decide on device results (the smoothing-length iteration, status
 *     reads, sph_stats) synchronise that stream; the others return as soon as
 *     the work is enqueued.
 *   - Ownership: the caller owns every buffer it passes and keeps it alive
 *     for the duration of the call; the library copies inputs into its own
 *     particle store (sorted by cell) and never frees caller memory. Results
 *     come back in the caller's original particle order.
 *   - Particle arrays are in "caller order": particle k of box b is entry
 *     box_offsets[b] + k. Vectors are row-major [N][3].
 */
#ifndef SPH_ABI_H_INCLUDED
#define SPH_ABI_H_INCLUDED

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SPH_OK 0
#define SPH_EINVAL (-1)        /* bad argument (null pointer, N < 1, h <= 0, m <= 0, u < 0, box <= 0) */
#define SPH_ENOMEM (-2)        /* device allocation failed or workspace too small */
#define SPH_ECUDA (-3)         /* a CUDA runtime call failed */
#define SPH_ENOTCONVERGED (-4) /* smoothing-length iteration hit max_iter */
#define SPH_EBOXTOOSMALL (-5)  /* some h would exceed L/3 of its box */
#define SPH_ENONPHYSICAL (-6)  /* rho <= 0, Omega <= 0 or u <= 0 */
#define SPH_ETIMEOUT (-7)      /* a bounded device-side wait gave up */
#define SPH_ESTATE (-8)        /* call out of order (e.g. sph_force before sph_density) */

/* ---- fields for sph_get ---- */
#define SPH_X 0      /* double [N][3] positions (wrapped into [0, L)) */
#define SPH_V 1      /* float  [N][3] velocities */
#define SPH_U 2      /* float  [N]    internal energy per unit mass */
#define SPH_H 3      /* double [N]    smoothing lengths */
#define SPH_RHO 4    /* float  [N]    density, Eq. (rho) */
#define SPH_OMEGA 5  /* float  [N]    Omega = 1 + h/(3 rho) drho/dh */
#define SPH_P 6      /* float  [N]    pressure P = (gamma - 1) rho u */
#define SPH_A 7      /* float  [N][3] dv/dt, Eq. (dvdt) */
#define SPH_DUDT 8   /* float  [N]    du/dt, Eq. (dudt) */
#define SPH_NNGB 9   /* int32  [N]    #{j != i : r_ij < h_i} at the converged h */
#define SPH_NITER 10 /* int32  [N]    density passes the particle's h needed */
#define SPH_NFORCE 11 /* int32 [N]    #{j != i : r_ij < max(h_i, h_j)} */
#define SPH_M 12     /* float  [N]    masses */
#define SPH_CELL 13  /* int32  [N][4] the grid cell the particle was binned into at the last
                        regrid (Section 3.1 cells): integer coordinates (ix, iy, iz) of its
                        top cell in its box, ix = floor(x / w_x) exactly for the FP64 x
                        (wrapped into [0, L)) and the FP64 width w_x of sph_grid, and, 4th,
                        the level of its octree leaf inside that top cell (0: the top cell) */
#define SPH_LEAF_CELL 14 /* int32 [N][3] integer coordinates of the particle's octree leaf
                        cell (edge w / 2^level) inside its top cell at the last regrid: the
                        leading `level` bits of floor((x - ix w) x (1 / w) x 1024) per axis */
#define SPH_NFIELDS 15

/* ---- interaction-kernel forms ---- */
#define SPH_MODE_PLAIN 0   /* one launch per density pass, host-driven h iteration */
#define SPH_MODE_BATCHED 1 /* one block per group of <= 32 particles, h iteration inside the
                              kernel; particles it cannot finish go to the per-pass form */
#define SPH_MODE_SYMMETRIC 2 /* density as SPH_MODE_PLAIN; force from pair tasks between
                                octree leaves that evaluate each pair once and update both
                                particles (Section 3.1, pair symmetry), the top cells
                                coloured so that the cells one launch runs share no
                                neighbour: no atomics, fixed summation order. FP32 sums
                                only (precision is not used by this force) */

/* ---- precision ---- */
#define SPH_PREC_FP32 0  /* FP32 pair arithmetic and accumulation */
#define SPH_PREC_KAHAN 1 /* FP32 pair arithmetic, compensated (Kahan) accumulation */

typedef struct sph_ctx sph_ctx; /* opaque, owned by the library */

typedef struct {
  double gamma;    /* adiabatic index (P = (gamma - 1) rho u) */
  double n_ngb;    /* target weighted neighbour number (> 32/3) */
  double h_tol;    /* converged when |N_i - n_ngb| <= h_tol * n_ngb and, to first order, h_i
                      lies within 5e-7 h_i of the root (|N_i - n_ngb| <= 5e-7 N_i d ln N/d ln h),
                      or the next step would move h_i by <= 5e-7 h_i */
  int max_iter;    /* density passes before SPH_ENOTCONVERGED */
  int n_split;     /* split octree cells holding more particles than this (8..256) */
  int precision;   /* SPH_PREC_* */
  int mode;        /* SPH_MODE_* */
  int profile;     /* 1: time each stage with CUDA events on the context stream */
  int pair_sort;   /* 1: sort each leaf's particles along the 13 pair axes (Section 3.1)
                      before the first per-pass kernel after a regrid, and let the
                      per-pass kernels visit only the source particles whose key along a
                      pair's axis is within reach; 0: visit whole source leaves (same
                      results, more pairs tested). The batched kernels do not use them. */
  int reuse_grid;  /* 1: sph_step keeps the grid of the last regrid while every particle
                      stays within reach of its top cell (h_max + 2 x the largest distance
                      outside its cell <= the cell width), refreshing positions and boxes
                      only, and runs those steps as one CUDA graph in the batched FP32
                      form; 0: regrid every step (same results up to summation order) */
  int tile;        /* batched first-tier stage: 0 small (more blocks per SM), 1 large
                      (fewer groups to the second tier on clumped inputs), 2 the density
                      as 1 and the force's first tier per group: the small stage for the
                      groups whose stage in the last force call held <= 640 entries, the
                      large one for the rest (an occupancy bin per group) */
  double cell_factor; /* top-cell edge >= cell_factor x the largest h where the box allows
                         (1 <= cell_factor <= 4; >= 1 x always) */
  int reuse_lists;  /* batched form, neighbour cache: keep each group's staged neighbours
                       and per-lane neighbour lists in device memory after the density; the
                       force of the same call takes its pairs from them (plus the pairs
                       reached by a neighbour's larger h), and later density calls reuse
                       them while a bound on the distance moved since they were built (the
                       summed |v dt| of the drifts) shows them complete for the current h.
                       0: off, search anew in every call; 1: on for sets of >= 16384 target
                       groups (smaller sets are latency-bound, where the cache's extra
                       kernels cost more than they save); 2: on always. Results are the
                       same up to summation order. */
  int work_queue;   /* batched form (Section 3.2, task queue and costs): how the
                       first-tier kernels share the target groups out among their
                       blocks. 0: a fixed grid stride. 1 (default): as 2 for sets of
                       >= 2^20 groups, else as 0. 2: every block claims 32 groups at a
                       time from a queue in group order until it is empty (neighbouring
                       groups stay together in time). 3: the same queue in measured
                       cost order: chunks of 32 groups, costliest first, a group's cost
                       being its duration in the last call (first: target count x task
                       count). Results are identical in every mode. */
} sph_params;

typedef struct {
  int64_t n_particles;
  int64_t n_boxes;
  int64_t n_top_cells;        /* cells of the top grids (edge >= largest h) */
  int64_t n_leaves;           /* octree leaves after recursive splitting */
  int64_t n_pairs_density;    /* leaf-pair tasks in the density lists */
  int64_t n_pairs_force;      /* leaf-pair tasks in the force lists */
  int64_t density_interactions; /* sum_i #{j != i: r_ij < h_i}, converged pass */
  int64_t force_interactions;   /* sum_i #{j != i: r_ij < max(h_i, h_j)} */
  int64_t density_pair_candidates; /* (i, j) pairs tested in all density passes */
  int64_t force_pair_candidates;   /* (i, j) pairs tested in the force pass */
  int32_t density_passes;     /* density passes of the last sph_density */
  int32_t rebuilds;           /* grid / list rebuilds in the last sph_density */
  int32_t max_iter_used;      /* most passes any particle needed */
  int32_t batched_fallbacks;  /* particles the batched kernels left to the per-pass form */
  double h_min, h_max;        /* extremes of the converged h */
  int32_t stage_max_density;  /* largest candidate stage of a batched density group */
  int32_t stage_max_force;    /* largest candidate stage of a batched force group */
  /* Cumulative since sph_create (never reset): */
  int64_t total_density_interactions; /* converged-pass density interactions */
  int64_t total_force_interactions;
  int64_t kernel_launches;    /* CUDA kernels this context enqueued */
  int64_t density_launches;   /* launches of the density interaction kernel */
  int64_t force_launches;     /* launches of the force interaction kernel */
  /* Stage times in ms (CUDA events on the context stream; profile = 1 only).
   * Each brackets the stage's launches; stages that read device counters
   * back include the host round trip. */
  double t_grid_ms;           /* cell keys, counting sort, octree split, gather */
  double t_lists_ms;          /* leaf-pair task lists */
  double t_density_ms;        /* density interaction kernel only */
  double t_ghost_ms;          /* h update / finalisation kernel */
  double t_force_ms;          /* force interaction kernel only */
  double t_integrate_ms;      /* kick / drift kernels */
  double t_sort_ms;           /* pair-axis sorts of every leaf (pair_sort = 1) */
  /* Last sph_density + sph_force, batched form (same results either way):
   * direct_list_warps = density warps whose per-lane neighbour lists
   * overflowed and that read their pre-filtered candidates directly, plus
   * force warps that built their lists in more than one round;
   * direct_stage_warps = density warps whose candidates overflowed and that
   * read the group's whole stage, plus force warps that filtered the stage in
   * more than one chunk. */
  int32_t direct_list_warps;
  int32_t direct_stage_warps;
  /* Particles of the last sph_density + sph_force that the batched kernels
   * left to the per-pass form, by cause: [0] density, third-tier walk
   * frontier overflowed or h outgrew the top-cell width, [1] density, h not
   * converged in max_iter passes, [2] force, third-tier walk frontier
   * overflowed, [3] zero. */
  int32_t fallback_causes[4];
  /* Batched form, last sph_density + sph_force ([0] density, [1] force):
   * groups whose stage overflowed and that the second tier staged again by
   * each target's own radius (first at the first tier's stage size, then,
   * if that still overflowed, in a larger stage), and (group, warp) entries
   * whose targets the third tier computed one warp per target (stage or
   * task-slot overflow, or an h beyond the staged radius). */
  int32_t tier2_groups[2];
  int32_t tier3_entries[2];
  int64_t sort_launches;      /* pair-axis sort launches (cumulative since sph_create) */
  int64_t reused_steps;       /* steps run on the previous step's grid (cumulative) */
  int64_t redone_steps;       /* of those, steps redone on a new grid because a particle had
                                 moved too far from its top cell (cumulative) */
  int64_t graph_steps;        /* of those, steps launched as one CUDA graph (cumulative) */
  /* Neighbour cache (reuse_lists = 1), batched form, last density / force: */
  int64_t n_groups;           /* target groups (<= 32 consecutive particles of a top cell) */
  int64_t cache_density_groups; /* groups whose density ran on their stored neighbours */
  int64_t cache_force_groups;   /* groups whose force ran on the density's neighbours */
  int64_t cache_built_groups;   /* groups whose density searched anew and stored them */
  int64_t cache_relist_warps;   /* warps on stored neighbours whose h or motion made them
                                   rebuild their per-lane lists from the stored stage */
} sph_stats_t;

/* Default parameters: gamma = 5/3, n_ngb = 48, h_tol = 1e-6, max_iter = 30,
 * n_split = 64, FP32, batched mode, pair sorts on, grid reuse on, profiling
 * off, tile 0, cell_factor 2, list reuse on. */
void sph_default_params(sph_params *p);

/* Create a context on the current CUDA device. `cuda_stream` is a
 * cudaStream_t (NULL: the legacy default stream). Errors: SPH_EINVAL for a
 * null `out` or out-of-range parameters, SPH_ECUDA if no device is usable. */
int sph_create(sph_ctx **out, const sph_params *p, void *cuda_stream);

/* Device bytes of the fixed-size per-particle and per-cell store for
 * `n_total` particles in `n_boxes` boxes. The variable-size leaf-pair task
 * lists are not included: the library allocates and grows those itself. */
int sph_workspace_size(const sph_ctx *ctx, int64_t n_total, int n_boxes, size_t *bytes);

/* Hand the library a caller-allocated device block for the fixed-size store
 * (at least sph_workspace_size bytes, 256-byte aligned). The caller keeps it
 * alive until sph_destroy or the next sph_set_workspace. Without it the
 * library allocates the store itself. Errors: SPH_EINVAL (null / unaligned). */
int sph_set_workspace(sph_ctx *ctx, void *dev_ptr, size_t bytes);

/* Load particles (Section 2 problem statement). Host arrays: box_offsets
 * (n_boxes + 1, int64, box_offsets[0] = 0, non-decreasing), box_len
 * (n_boxes x 3, edge lengths). Device arrays, caller order: x double[N][3]
 * (wrapped into the box on load), v float[N][3], m float[N] (> 0),
 * u float[N] (>= 0), h double[N] initial smoothing-length guesses (> 0; the
 * density stage iterates from them). Builds the cell grid and the leaf-pair
 * task lists. Errors: SPH_EINVAL, SPH_ENOMEM, SPH_EBOXTOOSMALL, SPH_ECUDA. */
int sph_init(sph_ctx *ctx, int n_boxes, const int64_t *box_offsets, const double *box_len,
             const double *x, const float *v, const float *m, const float *u, const double *h);

/* Density stage: iterate every h_i to N_i(h_i) = n_ngb (within h_tol), with
 * rho_i (Eq. rho), Omega_i, P_i at the converged h (Section 2; the ghost task
 * of Section 3.1 is the per-particle finalisation). Rebuilds the grid and
 * lists when an h outgrows them. Synchronises the stream. Errors:
 * SPH_ENOTCONVERGED, SPH_EBOXTOOSMALL, SPH_ENONPHYSICAL, SPH_ECUDA. */
int sph_density(sph_ctx *ctx);

/* Force stage, Eqs. (dvdt) and (dudt), over j with r_ij < max(h_i, h_j).
 * Requires a completed sph_density on the current positions (SPH_ESTATE
 * otherwise). Asynchronous. */
int sph_force(sph_ctx *ctx);

/* n_steps kick-drift-kick steps with global time step dt (> 0): half kick,
 * drift (FP64 positions, periodic wrap; h carried along as the starting
 * guess of the next iteration, h exp(-dt (du/dt) / (3 (gamma - 1) u))), grid
 * rebuild or reuse (reuse_grid), density, force with velocities and
 * energies predicted to the end of the step, half kick.
 * Requires sph_force on the current state first (SPH_ESTATE). Errors as
 * sph_density, plus SPH_ENONPHYSICAL when some u becomes <= 0. */
int sph_step(sph_ctx *ctx, double dt, int n_steps);

/* Copy one SPH_* field into `dev_out` (device, caller order, layout as listed
 * at the field). Asynchronous. Errors: SPH_EINVAL (unknown field / null),
 * SPH_ESTATE (field not computed yet). */
int sph_get(sph_ctx *ctx, int field, void *dev_out);

/* Autotuner (no counterpart in the paper; the paper tunes its cell split
 * threshold by hand, Section 3.1). On the loaded state, times one
 * sph_density + sph_force for every combination of tile (0, 1, 2; batched form
 * only), n_split (16, 32, 64, 128) and cell_factor (1.5, 2, 2.5, 3), each on its own
 * grid, best of 2, and keeps the fastest in the context's parameters; then
 * rebuilds the grid and leaves density and force computed on the current
 * state. Results do not depend on these parameters beyond summation order.
 * Outputs (host pointers, each may be NULL): the chosen tile, n_split,
 * cell_factor, and the best time in ms. Synchronises. Errors: SPH_ESTATE
 * before sph_init, or those of sph_density / sph_force. */
int sph_autotune(sph_ctx *ctx, int *tile_out, int *n_split_out, double *cell_factor_out,
                 double *ms_out);

/* Pair-axis sort of the current grid along direction `axis` (0..12; the
 * integer offsets (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1)
 * (0,1,1) (0,1,-1) (1,1,1) (1,1,-1) (1,-1,1) (1,-1,-1), normalised), Section
 * 3.1: the particles of every octree leaf ranked by x . e_axis (ties by
 * position in the leaf). Writes two int32 device arrays of N entries, one per
 * slot of the library's leaf-ordered store: `leaf_out[s]` = the leaf holding
 * slot s (leaves occupy consecutive slots), `order_out[s]` = the caller
 * index of the particle of rank s - (first slot of that leaf). Asynchronous.
 * Errors: SPH_EINVAL (axis out of range, null output), SPH_ESTATE (no
 * particles loaded, or pair_sort = 0). */
int sph_get_pair_order(sph_ctx *ctx, int axis, int32_t *order_out, int32_t *leaf_out);

/* FP32 fused multiply-add rate of `device`, measured (no counterpart in the
 * paper; the second denominator of the interaction kernels' FP32 roofline,
 * beside SM count x 128 lanes x 2 flops x the maximum SM clock). Runs
 * independent FFMA chains at full occupancy on a private stream, best of 5
 * timed launches (~1 ms each) after a warm-up; an FFMA counts as 2 flops.
 * Writes TFLOP/s to *tflops_out and the best launch time (ms) to *ms_out
 * (host pointers; ms_out may be NULL). The calling thread's current device is
 * restored. Synchronises that device's work on its own stream only.
 * Errors: SPH_EINVAL (null tflops_out, bad device), SPH_ENOMEM, SPH_ECUDA. */
int sph_fp32_peak(int device, double *tflops_out, double *ms_out);

/* Top grid of box `box` (0 <= box < n_boxes) as of the last regrid (Section
 * 3.1: cells no smaller than the largest smoothing length): cells per axis
 * (n_out, host int32[3]) and the FP64 cell widths w = L / n (w_out, host
 * double[3]; either may be NULL). Errors: SPH_EINVAL (box out of range),
 * SPH_ESTATE (no particles loaded). */
int sph_grid(const sph_ctx *ctx, int box, int32_t *n_out, double *w_out);

/* Counters of the last density/force calls (synchronises the stream). */
int sph_stats(sph_ctx *ctx, sph_stats_t *out);

/* Message of the last failed call on this context ("" if none). */
const char *sph_last_error(const sph_ctx *ctx);

/* Release the context and every buffer the library allocated. NULL is a no-op. */
void sph_destroy(sph_ctx *ctx);

/* ---- allocation-free density stage (no counterpart in the paper) ----
 *
 * For callers that may not allocate device memory on their calls: a host
 * framework that owns the whole GPU through its own memory pool, or code
 * where a cudaMalloc/cudaFree (which can also synchronise the device) is not
 * allowed. The regular entry points allocate a particle store and task lists;
 * this one allocates nothing itself. It runs the same density sums and the
 * same smoothing-length update rule as the per-pass density form for ONE
 * periodic box of at most SPH_NOALLOC_MAX_PARTICLES particles, finding
 * neighbours by scanning all particles (minimum image), and keeps its
 * per-particle scratch (~0.9 MB) in a fixed device array of this library's
 * CUDA module.
 *
 *   n          particles, 1 <= n <= SPH_NOALLOC_MAX_PARTICLES (else SPH_EINVAL)
 *   box_len    host, 3 edge lengths of the periodic box (> 0)
 *   x          device, double [n][3] positions (inside or outside the box)
 *   m          device, float [n] masses (> 0)
 *   h0         device, double [n] initial smoothing-length guesses (> 0)
 *   n_ngb, h_tol, max_iter   as in sph_params
 *   h_out      device, double [n]: converged h
 *   rho_out    device, float [n]: density, the same sum as sph_density's
 *   omega_out  device, float [n]: Omega = 1 + h/(3 rho) drho/dh
 *   cuda_stream  cudaStream_t of the work (NULL: legacy default stream)
 * Returns SPH_OK, SPH_EINVAL (bad arguments, or some m <= 0, h0 <= 0 or a
 * non-finite x, m, h0), SPH_ECUDA, SPH_EBOXTOOSMALL, SPH_ENONPHYSICAL or
 * SPH_ENOTCONVERGED.
 *
 * Memory: the scratch array is loaded with the module, on each device that
 * uses the library: at context creation under CUDA_MODULE_LOADING=EAGER,
 * otherwise (lazy loading, the CUDA default) when the module is first used
 * on that device, which can be this call's first call. Make one warm-up call
 * per device (or run with CUDA_MODULE_LOADING=EAGER) before relying on "no
 * allocation"; the array then stays until the process exits. The first call
 * on a device also looks up the array's device address
 * (cudaGetSymbolAddress).
 *
 * Synchronisation: the call copies a status word to the host and
 * synchronises the stream after every iteration pass, so it cannot be
 * captured into a CUDA graph. All calls share the one scratch array: calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it. */
#define SPH_NOALLOC_MAX_PARTICLES 16384
int sph_density_noalloc(int n, const double *box_len, const double *x, const float *m,
                        const double *h0, double n_ngb, double h_tol, int max_iter,
                        double *h_out, float *rho_out, float *omega_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SPH_ABI_H_INCLUDED */
