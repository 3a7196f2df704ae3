// sph_internal.cuh -- device data layout and launch wrappers shared by the
// translation units of libsph (CUDA, sm_103a). Not part of the public ABI.
//
// Particle store: every per-particle array is in "sorted order": particles of
// one octree leaf are contiguous, leaves follow the depth-first (Morton) order
// of the octree of their top cell, top cells follow box then cell index
// (Section 3.1: cells of edge >= the largest h, split recursively).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace sph {

// Kernel-launch counter of the context whose API call is running on this
// thread (set at API entry); every launch wrapper adds its launches.
extern thread_local long long *g_launch_count;
inline void note_launch(int k = 1) {
  if (g_launch_count) *g_launch_count += k;
}

constexpr int kMaxDepth = 10;   // octree levels below a top cell (1024 sub-cells per edge)
constexpr int kWarp = 32;
constexpr float kInvPi = 0.318309886183790671538f;

// Error bits a kernel may raise in the device status word.
enum : int {
  kErrHCap = 1,        // an h outgrew its leaf's density-list cap -> rebuild lists
  kErrHGrid = 2,       // an h outgrew the top-cell width -> rebuild the grid
  kErrBoxTooSmall = 4, // an h would exceed L/3 of its box
  kErrNonPhysical = 8, // rho <= 0, Omega <= 0, or u <= 0
  kErrNotConverged = 16,
  kErrListOverflow = 32,
  kErrInvalidInput = 64, // m <= 0, u < 0, h <= 0 or a non-finite input
};

struct BoxDev {
  double L[3];     // edge lengths
  double w[3];     // top-cell widths L / n
  int n[3];        // top cells per axis (>= 3)
  int cell_base;   // first global top-cell id of this box
  int first, count;  // particle range (the same in caller and sorted order)
  float eps;       // pruning margin in top-cell-relative units
  float pad;
  double iw[3];    // 1 / w
  double hcap;     // largest allowed h: min(L) / (3 (1 + 1e-6))
  float wf[3];     // w rounded to FP32 (neighbour-cell shifts in the walks)
  float pad2;
};

struct Node {
  int start, count;  // particle range in sorted order
  int child;         // first of 8 consecutive children, -1 for a leaf
  int parent;        // -1 for a top cell
  int cell;          // global top-cell id
  int leaf;          // leaf index (leaves only)
  int level;         // 0 = top cell
  int ix, iy, iz;    // integer coordinates at `level` inside the top cell
  float lo[3], hi[3];  // particle bounding box, relative to the top-cell origin
  float hmax;        // largest h of the node's particles
  int box;
};

struct Leaf {
  int start, count;
  int node, box;
  double o[3];       // leaf-cell origin relative to its top-cell origin
  float of[3];       // o rounded to FP32 (box arithmetic with a pruning margin only)
  int pad;
};

// One entry of a leaf's task list: the source leaf and the shift that maps
// the source leaf's particle coordinates into the target leaf's frame
// (origin_S + image offset - origin_T, rounded once to FP32).
struct Task {
  float sx, sy, sz;
  int src;
};

// Per-context counters written by kernels (device side).
struct DevCounters {
  unsigned long long dens_inter;      // converged-pass density interactions
  unsigned long long force_inter;
  unsigned long long dens_cand;       // (i, j) pairs tested, all density passes
  unsigned long long force_cand;
  int unconverged;
  int status;                         // kErr* bits
  int max_iter_used;
  int n_active;
  int n_frontier;
  int fallback;                       // particles the batched kernels left to the per-pass form
  int stage_max[2];                   // largest group stage (density, force) of the batched form
  int direct[2];                      // batched warp-groups that read their candidates
                                      // directly (a list overflowed) / the whole stage
  int queued[2];                      // groups queued for the second (larger-stage) tier
  int walk_queued;                    // groups queued for the tight walk
  int queued2[2];                     // (group, warp) entries queued for the third tier
  int why[4];                         // batched fallbacks: density third-tier walk (frontier
                                      // or h beyond the top cell), density passes, force
                                      // third-tier walk, (zero)
  int cache_used[2];                  // groups whose density / force ran on the stored
                                      // neighbour cache (no walk, no staging tests)
  int cache_built;                    // groups whose density built (and stored) a new cache
  int cache_relist;                   // warps on a stored stage that rebuilt their lists
  int queued_big[2];                  // groups the tight tier at the first-tier stage size
                                      // passed on to the large-stage tier
  int step_status;                    // kErr* bits of the kicks and the grid check (last
                                      // field: the density's counter reset keeps it)
};

// ---- cubic spline, support q < 1 (Section 2: h is the radius of the
// sphere of particles considered; W(r,h) = (8/pi) w(r/h) / h^3) ----
__device__ __forceinline__ void w_and_dw(float q, float &w, float &dw) {
  // inner piece 1 - 6q^2 + 6q^3, outer piece 2(1-q)^3, written in the power
  // basis so one Horner chain serves both: coefficients are selected, not
  // branched on.
  const bool in = q < 0.5f;
  const float c0 = in ? 1.f : 2.f, c1 = in ? 0.f : -6.f, c2 = in ? -6.f : 6.f,
              c3 = in ? 6.f : -2.f;
  const float d0 = in ? 0.f : -6.f, d1 = in ? -12.f : 12.f, d2 = in ? 18.f : -6.f;
  w = fmaf(fmaf(fmaf(c3, q, c2), q, c1), q, c0);
  dw = fmaf(fmaf(d2, q, d1), q, d0);
}

__device__ __forceinline__ float dw_only(float q) {
  const bool in = q < 0.5f;
  const float d0 = in ? 0.f : -6.f, d1 = in ? -12.f : 12.f, d2 = in ? 18.f : -6.f;
  float dw = fmaf(fmaf(d2, q, d1), q, d0);
  return q < 1.f ? dw : 0.f;
}

// ---- one smoothing-length update (the ghost step, Section 2: the number of
// neighbours is kept constant) shared by every density form ----
struct HIter {
  double h;      // current smoothing length
  double lo, hi; // bracket: N(lo) < n_ngb <= N(hi); hi = 1e308 while open
  float hf;      // h rounded to FP32 (the kernels' working copy)
  float fprev;   // |N - n_ngb| of the previous pass
  __device__ __forceinline__ void start(double h0, double lo0, double hi0, float fprev0) {
    h = h0;
    lo = lo0;
    hi = hi0;
    hf = (float)h0;
    fprev = fprev0;
  }
};

// Largest relative distance of an accepted h from the root, to first order:
// |N - n_ngb| / (N s) with s = d ln N / d ln h. It keeps h well inside the
// 1e-6 h band within which integer neighbour counts may differ from exact
// arithmetic, also for particles whose N is flat in h (small s).
constexpr float kHAcc = 5e-7f;

// Weighted neighbour number N = (32/3) sum w and dN/dh = -(32/(3h)) sum q w'
// from the FP32 sums at h. Returns true when h is accepted: |N - n_ngb| <=
// tol_n (= h_tol n_ngb; this test is FP64) and |N - n_ngb| <= kHAcc N s, or
// the next step would move h by at most 5e-7 h (the resolution of FP32
// sums). Otherwise moves h by Newton
// on ln N(ln h) (exponent s = h N'/N = -(sum q w') / (sum w) measured, so
// steep N near clusters does not overshoot), clamped to [h/8, 2h] and to
// hcap (L/3), bisecting the bracket when the step leaves it or |f| failed to
// halve well above the FP32 noise. *st receives kErrBoxTooSmall when the
// root lies beyond hcap. The bracket and h are FP64; the step factor, the
// halving test and the Newton step-size test are FP32 (FP64 runs at 1/64 of
// the FP32 rate on this part, so the pass does as few FP64 operations as
// the FP64 test and bracket need).
__device__ __forceinline__ bool h_newton_step(HIter &it, float sw, float sqdw, double n_ngb,
                                              double tol_n, double hcap, int *st) {
  const double f = fma(32.0 / 3.0, (double)sw, -n_ngb);
  const float ff = (float)f;
  if (fabs(f) <= tol_n && sw > 0.f &&
      fabsf(ff) <= kHAcc * (32.f / 3.f) * sw * (-sqdw / sw))  // N s = (32/3) sum(-q w')
    return true;
  const double h = it.h;
  double lo = it.lo, hi = it.hi;
  if (f < 0.0)
    lo = h;
  else
    hi = h;
  const bool open = hi >= 1e300;
  const float s_ln = sw > 0.f ? -sqdw / sw : 0.f;  // d ln N / d ln h
  float fac = 2.f;
  if (s_ln > 0.f) fac = __expf(__logf((float)n_ngb / ((32.f / 3.f) * sw)) / s_ln);
  fac = fminf(fmaxf(fac, 0.125f), 2.f);
  double hn = h * (double)fac;
  bool newton = true;
  if (!open && (!(hn > lo && hn < hi) ||
                (fabsf(ff) > 0.5f * it.fprev && fabsf(ff) > 1e-4f * (float)n_ngb))) {
    hn = 0.5 * (lo + hi);
    newton = false;
  }
  it.fprev = fabsf(ff);
  if (hn > hcap) {
    if (h >= hcap * (1.0 - 1e-12) && f < 0.0) *st |= kErrBoxTooSmall;
    hn = hcap;
    newton = false;
  }
  const bool tiny = newton ? fabsf(fac - 1.f) <= 5e-7f : fabs(hn - h) <= 5e-7 * h;
  if (tiny && !(*st & kErrBoxTooSmall)) return true;
  it.h = hn;
  it.hf = (float)hn;
  it.lo = lo;
  it.hi = hi;
  return false;
}

// The same step with h and its bracket held in FP32 (the batched kernels:
// h needs ~3e-6 relative accuracy for rho to 1e-5, FP32 gives 6e-8); the
// acceptance test |N - n_ngb| <= tol_n stays FP64. hi = +inf while open.
struct HIterF {
  float h, lo, hi, fprev;
  __device__ __forceinline__ void start(float h0) {
    h = h0;
    lo = 0.f;
    hi = __int_as_float(0x7f800000);
    fprev = __int_as_float(0x7f800000);
  }
};

__device__ __forceinline__ bool h_newton_step_f(HIterF &it, float sw, float sqdw, double n_ngb,
                                                double tol_n, float hcap, int *st) {
  const double f = fma(32.0 / 3.0, (double)sw, -n_ngb);
  const float ff = (float)f;
  if (fabs(f) <= tol_n && fabsf(ff) <= kHAcc * (32.f / 3.f) * -sqdw) return true;  // N s
  const float h = it.h;
  float lo = it.lo, hi = it.hi;
  if (ff < 0.f)
    lo = h;
  else
    hi = h;
  const bool open = !(hi < 3e38f);
  const float nn = (float)n_ngb;
  const float s_ln = sw > 0.f ? -sqdw / sw : 0.f;  // d ln N / d ln h
  float fac = 2.f;
  if (s_ln > 0.f) fac = __expf(__logf(nn / ((32.f / 3.f) * sw)) / s_ln);
  fac = fminf(fmaxf(fac, 0.125f), 2.f);
  float hn = h * fac;
  bool newton = true;
  if (!open && (!(hn > lo && hn < hi) ||
                (fabsf(ff) > 0.5f * it.fprev && fabsf(ff) > 1e-4f * nn))) {
    hn = 0.5f * (lo + hi);
    newton = false;
  }
  it.fprev = fabsf(ff);
  if (hn > hcap) {
    if (h >= hcap && ff < 0.f) *st |= kErrBoxTooSmall;
    hn = hcap;
    newton = false;
  }
  const bool tiny = newton ? fabsf(fac - 1.f) <= 5e-7f : fabsf(hn - h) <= 5e-7f * h;
  if (tiny && !(*st & kErrBoxTooSmall)) return true;
  it.h = hn;
  it.lo = lo;
  it.hi = hi;
  return false;
}

// Per-particle quantities at a converged h from the density sums `s`
// (sum w, sum q w', sum m w, sum m (3w + q w')) and the internal energy u:
// rho (Eq. rho), Omega = 1 + h/(3 rho) drho/dh, P = (gamma - 1) rho u, and the
// force-stage record (h, 1/h, A (8/pi) h^-4, h^2) with A = P / (Omega rho^2).
// FP32 arithmetic (relative error ~1e-7).
__device__ __forceinline__ bool finalise_density(float hf, float4 s, float u, float gm1,
                                                 float *rho_o, float *omega_o, float *P_o,
                                                 float4 *fi_o) {
  const float c8pi = 2.546479089470325f;  // 8 / pi
  const float hinv = 1.f / hf;
  const float hinv3 = hinv * hinv * hinv;
  const float rho = c8pi * s.z * hinv3;
  const float drho = -c8pi * s.w * hinv3 * hinv;
  const float omega = 1.f + hf / (3.f * rho) * drho;
  const float P = gm1 * rho * u;
  const float A = P / (omega * rho * rho);
  *rho_o = rho;
  *omega_o = omega;
  *P_o = P;
  *fi_o = make_float4(hf, hinv, A * c8pi * hinv3 * hinv, hf * hf);
  return rho > 0.f && omega > 0.f && u >= 0.f;
}

// ---- pair-axis sorts (Section 3.1: particles are sorted along the axis of
// each pair of neighbouring cells before the density tasks run) ----
constexpr int kAxes = 13;
// Integer offsets to 13 of the 26 neighbouring cells; the other 13 are their
// negatives. Each has its first non-zero component positive.
static __constant__ signed char kAxisDir[kAxes][3] = {
    {1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0},   {1, -1, 0},  {1, 0, 1},  {1, 0, -1},
    {0, 1, 1},  {0, 1, -1}, {1, 1, 1},  {1, 1, -1},  {1, -1, 1},  {1, -1, -1}};

// Unit vector of direction k.
__device__ __forceinline__ float3 axis_vec(int k) {
  const float a = kAxisDir[k][0], b = kAxisDir[k][1], c = kAxisDir[k][2];
  const int nz = (a != 0.f) + (b != 0.f) + (c != 0.f);
  const float s = nz == 1 ? 1.f : (nz == 2 ? 0.70710678118654752f : 0.57735026918962576f);
  return make_float3(a * s, b * s, c * s);
}

__device__ __forceinline__ float axis_key(float4 p, float3 e) {
  return fmaf(p.x, e.x, fmaf(p.y, e.y, p.z * e.z));
}

// Direction (of the 13) most nearly parallel to the offset d, with |d . e|.
// Computed by a whole warp (lanes 0..12 score one direction each); every lane
// receives the winner. Ties go to the lowest index.
__device__ __forceinline__ int warp_best_axis(float dx, float dy, float dz) {
  const int lane = threadIdx.x & 31;
  float v = -1.f;
  if (lane < kAxes) {
    const float3 e = axis_vec(lane);
    v = fabsf(fmaf(dx, e.x, fmaf(dy, e.y, dz * e.z)));
  }
  float m = v;
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const unsigned hit = __ballot_sync(0xffffffffu, v == m);
  return __ffs(hit) - 1;
}

// Window [lo, hi] of keys (along direction k, in the source leaf's frame,
// where keys are sorted) that can reach any of the warp's targets: lanes pass
// their key d_i (target frame) and reach R_i (<= 0 or an inactive lane: no
// contribution). `sd` = shift . e_k maps source keys into the target frame.
// Returns false when no lane is active. The pad covers FP32 rounding of the
// keys and the shift (relative 1e-5 of the magnitudes involved).
__device__ __forceinline__ bool warp_key_window(bool act, float d, float R, float sd, float &lo,
                                                float &hi) {
  float l = act ? d - R : 3e38f, h = act ? d + R : -3e38f;
  float mag = act ? fabsf(d) + R : 0.f;
  for (int o = 16; o; o >>= 1) {
    l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
    h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
    mag = fmaxf(mag, __shfl_xor_sync(0xffffffffu, mag, o));
  }
  if (!(l <= h)) return false;
  const float pad = 1e-5f * (mag + fabsf(sd)) + 1e-30f;
  lo = l - sd - pad;
  hi = h - sd + pad;
  return true;
}

// Sorted-rank range [r0, r1) of a source leaf's keys (count entries from
// `key`) inside [lo, hi]: counted by warp ballots over coalesced loads (keys
// ascend, so the counts are the bounds).
__device__ __forceinline__ void warp_key_range(const float *key, int count, float lo, float hi,
                                               int &r0, int &r1) {
  const int lane = threadIdx.x & 31;
  int below = 0, upto = 0;
  for (int b = 0; b < count; b += 32) {
    const int k = b + lane;
    const float v = k < count ? key[k] : 3e38f;
    below += __popc(__ballot_sync(0xffffffffu, k < count && v < lo));
    upto += __popc(__ballot_sync(0xffffffffu, k < count && v <= hi));
  }
  r0 = below;
  r1 = upto;
}

// Target group of the batched kernels: up to 32 consecutive particles (sorted
// order) of one top cell, one warp lane each.
struct Group {
  int start, count;
  int cell, box;
  double o[3];          // frame origin: leaf-cell origin of the first particle
                        // (relative to the top-cell origin)
  float tlo[3], thi[3]; // bounding box, relative to the top-cell origin
  float flo[3], fhi[3]; // bounding box in the group frame
  float hmax;           // largest h of the group
  int pad;
};

// ---- host-side launch wrappers (grid.cu) ----
struct GridArgs {
  int n;                 // particles
  int n_boxes;
  const BoxDev *boxes;   // device
  int n_cells;           // total top cells
  int n_split;
  const double *x0, *x1, *x2;  // positions (current order)
  int *cell_of;          // [n] scratch
  unsigned *morton;      // [n] Morton code per current slot
  unsigned *morton_tmp;  // [n] Morton code in new order
  unsigned *morton_scr;  // [n] scratch for the octant scatter
  int *cell_count;       // [n_cells + 1]
  int *cell_start;       // [n_cells + 1]
  int *cursor;           // [n_cells]
  int *order;            // [n] new slot -> old slot
  int *order_tmp;        // [n]
  const int *orig;       // [n] original index of old slot (tie-break)
};

void launch_cell_keys(const GridArgs &g, cudaStream_t s);
void launch_cell_scatter(const GridArgs &g, cudaStream_t s);
void exclusive_scan_int(const int *in, int *out, int n, void *tmp, size_t tmp_bytes,
                        cudaStream_t s);
size_t scan_tmp_bytes(int n);
void launch_init_top_nodes(Node *nodes, const GridArgs &g, cudaStream_t s);
void launch_frontier_top(const Node *nodes, int n_cells, int n_split, int *frontier,
                         DevCounters *ctr, cudaStream_t s);
void launch_split_level(Node *nodes, const int *frontier, int n_frontier, int child_base,
                        int level, int n_split, int *next_frontier, DevCounters *ctr,
                        const GridArgs &g, cudaStream_t s);
void launch_mark_leaves(const Node *nodes, int n_nodes, int *flag, cudaStream_t s);
void launch_fill_leaves(Node *nodes, int n_nodes, const int *leaf_idx_excl, Leaf *leaves,
                        const BoxDev *boxes, int n_boxes, cudaStream_t s);
void launch_sort_leaves(const Leaf *leaves, int n_leaves, int *order, const int *orig,
                        const unsigned *morton, cudaStream_t s);

struct GeomArgs {
  int n_leaves;
  const Leaf *leaves;
  Node *nodes;
  const BoxDev *boxes;
  int n_boxes;
  const double *x0, *x1, *x2;
  const float *m;
  const float *hf;     // h as float, sorted order
  float4 *pm;          // out: leaf-relative position, mass
  unsigned *maxout;    // optional out, per box: largest distance outside the top cell (float bits)
};
void launch_leaf_geometry(const GeomArgs &a, int n_nodes, cudaStream_t s);
// After a drift on an unchanged grid: empty every node box, then refill them
// and the leaf-relative positions (k_leaf_geometry).
void launch_refresh_geometry(const GeomArgs &a, int n_nodes, cudaStream_t s);
// kErrHGrid into *status when some box's h_max (1 + 1e-6) + 2 out > its top-cell
// width (boxout[b]: box b's largest out-of-cell distance, float bits).
void launch_grid_check(const double *h, int n, const BoxDev *boxes, int nb,
                       unsigned long long *hext, const unsigned *boxout, int *status,
                       cudaStream_t s);
void launch_leaf_hmax(const GeomArgs &a, int n_nodes, cudaStream_t s);
void launch_h_guess(const GeomArgs &a, double n_ngb, double *h, float *hf, cudaStream_t s);
// Top-cell coordinates + leaf level ([N][4]) and leaf-cell coordinates
// ([N][3]) per particle in caller order (either output may be null).
void launch_get_cells(const int *orig, const int *leaf_of, const Leaf *leaves, const Node *nodes,
                      const BoxDev *boxes, int n, int *out4, int *out3, cudaStream_t s);

// ---- axis_sort.cu ----
struct AxisSortArgs {
  int n_leaves;
  const Leaf *leaves;
  const float4 *pm;     // leaf-relative positions (sorted order)
  int n;                // particles (stride of one direction's arrays)
  float *skey;          // out: [kAxes][n] keys in rank order within each leaf
  int *sidx;            // out: [kAxes][n] leaf-local index of each rank
};
void launch_axis_sort(const AxisSortArgs &a, cudaStream_t s);
void launch_get_pair_order(const Leaf *leaves, const int *leaf_of, const int *sidx,
                           const int *orig, int n, int axis, int *order_out, int *leaf_out,
                           cudaStream_t s);

// per-box largest h (dmax[nb]) and global min / max (dminmax[2]), as ordered
// int64 bit patterns of non-negative doubles (dminmax[0] holds the minimum)
void launch_h_extremes(const double *h, int n, const BoxDev *boxes, int n_boxes,
                       unsigned long long *dmax, unsigned long long *dminmax, cudaStream_t s);
void launch_validate(const double *x, const float *v, const float *m, const float *u,
                     const double *h, int n, int *status, cudaStream_t s);
void launch_reset_iteration(unsigned char *done, int *niter, double *hlo, double *hhi,
                            float *fprev, int n, cudaStream_t s);

struct ListArgs {
  int n_leaves;
  const Leaf *leaves;
  const Node *nodes;
  const BoxDev *boxes;
  int n_boxes;
  int force;           // 0: density (gather, d < cap_T), 1: force (d < max(hT, hS))
  float cap_factor;    // density cap = cap_factor * hmax_T
  int *count;          // [n_leaves + 1]
  const int *offset;   // [n_leaves + 1] (fill pass)
  Task *tasks;         // fill pass
  const int *active;   // optional subset of target leaves (NULL = all)
  int n_targets;
  int *status;         // kErrListOverflow if a walk ran out of stack
  int *flag;           // [n_targets] 1: the warp walk's frontier overflowed for this target
};
// Count pass (a.tasks null) or fill pass: one warp per target leaf, breadth
// first; the few targets whose frontier overflows are walked by one thread
// each, depth first (same tasks, another order, the same in both passes).
void launch_build_lists(const ListArgs &a, cudaStream_t s);

// ---- interact.cu ----
struct DensArgs {
  int n_active;
  const int *active;     // active target leaves
  const Leaf *leaves;
  const int *list_off;   // [n_leaves + 1]
  const Task *tasks;
  const float4 *pm;
  const float *hf;
  const unsigned char *done;  // per particle converged flag
  float4 *sums;          // sum w, sum q w', sum m w, sum m (3w + q w')
  int *cnt;
  DevCounters *ctr;
  int kahan;
  const float *skey;     // pair-axis sorts ([kAxes][n]); null: visit whole source leaves
  const int *sidx;
  int n;
};
void launch_density(const DensArgs &a, cudaStream_t s);

struct GhostArgs {
  int n;
  double n_ngb, tol, gamma;
  int max_iter;
  const Leaf *leaves;
  const int *leaf_of;     // per particle leaf index
  const Node *nodes;
  const BoxDev *boxes;
  int n_boxes;
  float cap_factor;
  double *h;
  double *hlo, *hhi;
  float *fprev;           // |N - n_ngb| of the previous pass (step safeguard)
  float *hf;
  const float4 *sums;
  const int *cnt;
  const float4 *vu;       // u in .w (predicted u during a step)
  unsigned char *done;
  int *niter;
  int *nngb;
  float *rho, *omega, *P;
  float4 *force_i;        // (h, 1/h, A (8/pi) h^-4, m) for the force stage
  DevCounters *ctr;
};
void launch_ghost(const GhostArgs &a, cudaStream_t s);
void launch_active_leaves(const Leaf *leaves, int n_leaves, const unsigned char *done,
                          int *active, DevCounters *ctr, cudaStream_t s);

struct ForceArgs {
  int n_leaves;                // targets: n_targets leaves, active[t] (or t when null)
  const int *active;
  int n_targets;
  const unsigned char *skip;   // optional: particles already finished (not written)
  const Leaf *leaves;
  const int *list_off;
  const Task *tasks;
  const float4 *pm;
  const float4 *fi;       // (h, 1/h, A', m)
  const float4 *vu;       // predicted v, u
  float4 *acc;            // out: a, du/dt
  int *nforce;
  DevCounters *ctr;
  int kahan;
  const Node *nodes;      // source-leaf largest h (reach of a pair along a sort axis)
  const float *skey;      // pair-axis sorts ([kAxes][n]); null: visit whole source leaves
  const int *sidx;
  int n;
};
void launch_force(const ForceArgs &a, cudaStream_t s);

// ---- symmetric.cu (SPH_MODE_SYMMETRIC force) ----
struct SymArgs {
  const int *cells;       // the top cells of one colour class (global ids)
  int n_cells;
  const int *cell_leaf;   // [n_cells total + 1] first leaf of each top cell
  const Leaf *leaves;
  const int *list_off;    // the per-pass force task lists of every leaf (leaf index order)
  const Task *tasks;
  const float4 *pm, *fi, *vu;
  float4 *acc;            // in/out: a, du/dt (zeroed before the first colour)
  int *nforce;            // in/out (zeroed before the first colour)
  DevCounters *ctr;
};
void launch_force_sym(const SymArgs &a, cudaStream_t s);
void launch_leaf_cells(const Leaf *leaves, const Node *nodes, int n_leaves, int *out,
                       cudaStream_t s);
// Host: cell_leaf (n_cells + 1), and the cells that hold leaves grouped by
// colour class (colour_cells, with offsets colour_off).
void sym_colours(const std::vector<BoxDev> &boxes, int n_cells, const std::vector<int> &leaf_cell,
                 std::vector<int> &cell_leaf, std::vector<int> &colour_cells,
                 std::vector<int> &colour_off);

// ---- batched.cu ----
struct GroupBuildArgs {
  int n_nodes;
  const Node *nodes;
  int n_cells;
  const int *cell_start, *cell_count;
  const BoxDev *boxes;
  int n_boxes;
  int *gcount;           // [n_nodes + 1] groups per node (scanned in place to offsets)
  Group *groups;
  int n_groups;
  const Leaf *leaves;
  const int *leaf_of;
  const float4 *pm;
  const float *hf;
  float4 *gpos;          // out (geometry): position in the group frame, mass
};
void launch_group_count(const GroupBuildArgs &a, cudaStream_t s);
void launch_group_fill(const GroupBuildArgs &a, cudaStream_t s);
void launch_group_geometry(const GroupBuildArgs &a, cudaStream_t s);
void launch_group_hmax(const GroupBuildArgs &a, cudaStream_t s);

// ---- neighbour cache of the batched form (density stage and per-lane
// lists kept in HBM) ----
//
// The first tier of the density stores, per group, the particles of its
// stage (index and task slot, in the stage's segment layout) and each warp's
// per-lane neighbour lists (16-bit stage indices, padded to a multiple of 4
// with the stage sentinel). The force of the same call reuses them: its
// pairs r < max(h_i, h_j) are the listed ones, plus stage particles whose own
// h reaches a target from beyond its list (found by a warp filter and
// checked against the lists), plus particles outside the stage whose h
// reaches the group (a walk that only follows nodes of large h: such a group
// takes the full force path). Later density calls reuse a group's cache
// while it is provably complete: dpath[i] bounds how far particle i has moved
// since the cache epoch began (sum of |v dt| over the drifts), delta = the
// largest dpath of the particles held by the 27 top cells around the group's
// cell (on a reused grid every pair in range lies within them), D = the
// stage's largest dpath. A stage built with
// radius Rg around the group box then still holds every j with r_ij < Rg -
// dpath_i - delta, and a list built with radius rl every staged j with r_ij <
// rl - dpath_i - D: the kernel checks h_i against both and rebuilds the lists
// (or sends the warp to the third tier) when h_i outgrows them.
struct GroupCache {
  int wc[4];       // staged entries per warp
  int tpad[4];     // stored list rows per warp (-1: none stored)
  int wok[4];      // the warp finished in the first tier on per-lane lists (last call)
  float Rg;        // stage radius at the build (distance from the group box)
  int stage_ok;    // the stored stage is complete (built in the first tier, no overflow)
  int pad[2];
};
static_assert(sizeof(GroupCache) == 64, "GroupCache layout");

struct CacheCtl {
  int build_all;   // 1: the next density builds every group's cache (new epoch)
  int fail;        // groups whose stored stage motion made incomplete (this call)
  int n_groups;
  int lfail;       // warps whose stored lists motion made incomplete (this call)
  int force_off;   // 1: this force call skips the cache (far-reacher walk not run)
  int fused;       // groups whose force ran on the cache in the last call that tried
  int probe;       // calls left before a skipped force cache is tried again
  int pad;
};

struct CacheArgs {
  GroupCache *meta;        // [n_groups]
  int *sj;                 // [n_groups * ns] particle index per stage slot
  unsigned short *slot;    // [n_groups * ns] task slot per stage slot
  unsigned short *list;    // [n_groups * 4 * lane_cap * 32] rows of 32 lanes
  float *rl;               // [n] radius the particle's stored list was built with
  float *dpath;            // [n] path length since the epoch began (upper bound)
  const unsigned *dmax_cell; // [n_cells] largest dpath per top cell (float bits)
  unsigned char *gmode;    // [n_groups] 1: this density call reuses the stored cache
  unsigned char *fuse;     // [n_groups] 1: this force call reuses it
  CacheCtl *ctl;
  const Task *tasks;       // the density's task slots (the stored stage's shifts)
  const int *tcount;       // the density's task count per group
  int ns;                  // stage slots per group (layout stride)
  int lane_cap;            // list entries per lane (layout stride)
};

struct GroupListArgs {
  int n_groups;
  const Group *groups;
  const Leaf *leaves;
  const Node *nodes;
  const BoxDev *boxes;
  int force;             // 0: density stage radius, 1: max(hmax_G, hmax_S)
  float skin;            // density stage radius = min(skin * hmax_G, top-cell width)
  int tcap;              // task slots per group
  int *count;            // [n_groups] tasks found (> tcap: overflow)
  Task *tasks;           // [n_groups * tcap]
  int *status;
  const int *leaf_of;    // targets of the tight walk
  const float4 *pm;
  const float *hf;
  int *walk_queue;       // [n_groups] groups whose walk overflowed (null: no tight walk)
  int *walk_queued;      // device count of walk_queue, zero on entry
  unsigned char *wmode;  // (density, optional) per group: 0 the group-box walk found its
                         // tasks, 1 the tight walk did (each target's own sphere only)
  int cache_on;          // the neighbour cache is in use (density: skip the walk of groups
                         // whose stored stage is valid; force: far-reacher walk first, and
                         // no walk for groups whose force reuses the cache)
  CacheArgs cache;
  DevCounters *ctr;
};
// The walk packs (node, neighbour code) into one int: node indices below 2^26.
constexpr int kWalkMaxNodes = 1 << 26;
void launch_group_lists(const GroupListArgs &a, cudaStream_t s);

// Work queue of a first-tier launch (task cost ordering, Section 3.2): the
// blocks claim the groups kClaim queue positions at a time through *head,
// in the order `order` gives (null: group order; -1 entries: no group).
// The block that ran group g writes its duration to cost[g] (SM clock
// cycles, from the group's fetch to the block's next fetch), which orders
// the next call. head == nullptr: a static grid stride over the groups.
struct WorkQueue {
  const int *order;
  int *head;
  float *cost;
};
constexpr int kCostBins = 2048;   // cost buckets: 8 per octave
// The queue order: chunks of 32 consecutive groups, costliest first (a
// group's cost: cost[g] where measured, > 0, else the estimate count x
// tasks from its walk), each chunk's groups in group order. order:
// ceil(n_groups / 32) * 32 ints; bins: kCostBins ints; cbin:
// ceil(n_groups / 32) ints. The n_heads queue heads are zeroed.
void launch_cost_order(const Group *groups, int n_groups, const int *tcount, const float *cost,
                       int *order, int *bins, int *cbin, int *heads, int n_heads,
                       cudaStream_t s);

struct BatchDensArgs {
  int n_groups;
  const Group *groups;
  const int *tcount;     // tasks of group g: tasks[g * tcap + k], k < tcount[g]
  int tcap;
  const Task *tasks;
  const Leaf *leaves;
  const int *leaf_of;
  const float4 *pm;
  const float4 *gpos;    // targets: position in their group's frame, mass
  const BoxDev *boxes;
  double *h;
  float *hf;
  const float4 *vu;      // u in .w for P
  double n_ngb, tol, gamma;
  int max_iter;
  float skin_stage;      // stage radius factor (matches the list build)
  float skin_list;       // per-lane list and sub-cluster candidate radius factor
  int kahan;             // compensated sums
  unsigned char *done;
  int *niter, *nngb;
  float *rho, *omega, *P;
  float4 *fi;
  DevCounters *ctr;
  int *queue;            // [n_groups] groups handed to the second tier (tight stage)
  int *queue2;           // [n_groups * 4] (group, warp) handed to the third tier
  int *queue_big;        // [n_groups] groups the second tier hands to its large stage
  const Node *nodes;     // the third tier walks the octrees itself
  int tile;              // first-tier stage size: 0 small (high occupancy), 1 large
  // per group, 1: its tasks came from the tight walk, so its stage is complete
  // only within each target's own starting radius min(skin_stage h_i, w), not
  // within Rg of the group box
  const unsigned char *wmode;
  int cache_on;
  CacheArgs cache;
  // first tier: the work queue (heads: [0] the launch on stored stages,
  // [1] the launch that stages anew)
  WorkQueue wq;
};
void launch_density_batched(const BatchDensArgs &a, cudaStream_t s);
// The next call's epoch decision (one thread): a new epoch when motion made
// more than an eighth of the groups restage, or of the warps rebuild their
// lists, in this call.
void launch_cache_decide(CacheCtl *ctl, cudaStream_t s);
// A new epoch: every group builds (and stores) its cache in the next density.
void launch_cache_init(CacheCtl *ctl, int n_groups, cudaStream_t s);
// Before a force call (one thread): when fewer than an eighth of the groups
// could take their force from the cache in the last call that tried, skip
// the far-reacher walk and the cached force for the next 15 calls, then try
// again.
void launch_force_gate(CacheCtl *ctl, cudaStream_t s);
// Stage capacity and list entries per lane of the first tier of `tile`.
int cache_stage_slots(int tile);
int cache_lane_cap(int tile);

struct BatchForceArgs {
  int n_groups;
  const Group *groups;
  const int *tcount;
  int tcap;
  const Task *tasks;
  const Leaf *leaves;
  const int *leaf_of;
  const float4 *pm;
  const float4 *gpos;    // targets: position in their group's frame, mass
  const float4 *fi;
  const float4 *vu;
  float4 *acc;
  int *nforce;
  unsigned char *fdone;  // per particle: force written by the batched kernel
  DevCounters *ctr;
  int *queue;            // [n_groups] groups handed to the second tier (tight stage)
  int *queue2;           // [n_groups * 4] (group, warp) handed to the third tier
  int *queue_big;        // [n_groups] groups the second tier hands to its large stage
  const Node *nodes;     // the third tier walks the octrees itself
  const BoxDev *boxes;
  int kahan;             // compensated sums
  int tile;              // first-tier stage size: 0 small (high occupancy), 1 large,
                         // 2 per group by its last stage (gstage): small where it fitted
  int cache_on;
  CacheArgs cache;
  WorkQueue wq;          // first tier: the work queue
  int *gstage;           // [n_groups] out, first tier: the stage each group needed, kNW x its
                         // largest warp share (-1 unknown)
  const int *border;     // tile 2: the groups, those for the small stage first
  const int *bsplit;     // tile 2: how many are for the small stage (device)
  int bin;               // first-tier launch of tile 2: 1 small, 2 large; 0 otherwise
};
void launch_force_batched(const BatchForceArgs &a, cudaStream_t s);
// Tile 2: the groups whose last first-tier force stage held at most `fit`
// entries (and was measured) first, the rest after, each part in group
// order; *split = the size of the first part. flag, excl: n_groups + 1 ints.
void launch_force_bins(const int *gstage, int n_groups, int fit, int *flag, int *excl,
                       void *scan_tmp, size_t scan_tmp_bytes, int *order, int *split,
                       cudaStream_t s);

// ---- integrate.cu ----
struct StoreArrays {
  double *x0, *x1, *x2, *h, *hlo, *hhi;
  float4 *vu, *vu_pred, *acc;
  float *m;
  int *orig;
};
// wx: wrapped caller-order positions, SoA (x0 = wx, x1 = wx + n, x2 = wx + 2n)
void launch_load_caller(const StoreArrays &dst, const int *order, int n, const double *wx,
                        const float *v, const float *m, const float *u, const double *h,
                        cudaStream_t s);
void launch_permute(const StoreArrays &dst, const StoreArrays &src, const int *order, int n,
                    cudaStream_t s);
void launch_wrap_cell_keys_from_caller(const double *x, const BoxDev *boxes, int n_boxes, int n,
                                       double *x0, double *x1, double *x2, cudaStream_t s);
// save: when not null, the step's starting x, h, (v, u) and (a, du/dt) are
// copied there as they are read (the state a redone step restarts from);
// done / fdone: when not null, the per-particle finished flags of the density
// and force are cleared on the way
// The neighbour cache's motion bound, updated by the drift (optional):
// dpath[s] += |v dt| (or = 0 when ctl->build_all: the coming density starts
// a new epoch), and dmax_cell[c] = max(dmax_cell[c], dpath) over the
// particles of top cell c (zeroed by the caller).
struct DriftCache {
  float *dpath;
  unsigned *dmax_cell;
  const CacheCtl *ctl;
  const int *leaf_of;
  const Leaf *leaves;
  const Node *nodes;
};
void launch_kick_drift(StoreArrays st, int n, double dt, const BoxDev *boxes, int n_boxes,
                       double gamma, float *hf, const StoreArrays *save, unsigned char *done,
                       unsigned char *fdone, DevCounters *ctr, cudaStream_t s,
                       const DriftCache *dc = nullptr);
void launch_kick(StoreArrays st, int n, double dt, DevCounters *ctr, cudaStream_t s);
void launch_h_to_float(const double *h, float *hf, int n, cudaStream_t s);
void launch_leaf_of(const Leaf *leaves, int n_leaves, int *leaf_of, cudaStream_t s);
void launch_get(int field, void *out, const int *orig, int n, const StoreArrays &st,
                const float *rho, const float *omega, const float *P, const int *nngb,
                const int *niter, const int *nforce, cudaStream_t s);

}  // namespace sph
