// sph_api.cu -- C ABI entry points and host orchestration of libsph.
//
// Order of work per call (Section 3.1 task hierarchy, sort -> density ->
// ghost -> force -> integrator, mapped to stream-ordered kernel launches):
//   sph_init     wrap positions, build grid (A1), split cells (A2), gather
//                the particle store into leaf order, leaf geometry.
//   sph_density  batched form (default): group frames and h maxima, group
//                walk, the three density tiers with the h iteration inside
//                (A4, A5), no host round trip between them; per-pass form,
//                and any target the batched tiers leave: repeat { leaf h
//                maxima, active leaves, density task lists, density gather
//                (A4), ghost h update (A5) } until every h has converged.
//                The grid is rebuilt when an h outgrows it.
//   sph_force    batched: group h maxima, group walk, the three force tiers
//                (A6); per-pass: force task lists, force gather.
//   sph_step     kick + drift, position refresh on the reused grid (or a
//                regrid), density, force (predicted v, u), kick, grid check;
//                steady batched steps replay one captured CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/sph.h"
#include "sph_internal.cuh"

using namespace sph;

namespace {

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct sph_ctx {
  sph_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;

  // fixed store: caller workspace (bump allocated) or library allocations
  char *ws = nullptr;
  size_t ws_bytes = 0, ws_used = 0;
  std::vector<void *> owned;
  int64_t alloc_n = -1;  // store currently laid out for (alloc_n, alloc_nb, alloc_ws)
  int alloc_nb = -1;
  char *alloc_ws = nullptr;

  int n = 0, nb = 0;
  std::vector<BoxDev> boxes_h;
  BoxDev *boxes_d = nullptr;
  StoreArrays st{}, st2{};
  float *hf = nullptr;
  float4 *pm = nullptr, *sums = nullptr, *fi = nullptr;
  float4 *gpos = nullptr;  // position in the particle's batched group frame, mass
  float *skey = nullptr;  // pair-axis sorts: [kAxes][n] keys, rank order per leaf
  int *sidx = nullptr;    // [kAxes][n] leaf-local index of each rank
  int *cnt = nullptr, *niter = nullptr, *nngb = nullptr, *nforce = nullptr, *leaf_of = nullptr;
  unsigned char *done = nullptr, *fdone = nullptr;
  float *rho = nullptr, *omega = nullptr, *P = nullptr, *fprev = nullptr;
  int *cell_of = nullptr, *order = nullptr, *order_tmp = nullptr, *flag = nullptr,
      *excl = nullptr, *ident = nullptr;
  unsigned *mkey = nullptr, *msrt = nullptr, *mscr = nullptr;
  double *wx = nullptr;
  unsigned long long *hext = nullptr;  // per-box max h, then global min, max

  // growable, library-owned
  // batched form: target groups and their task lists
  DevBuf gcount, groups, gd_off, gd_tasks, gf_off, gf_tasks, gqueue, lflag, gwmode;
  // task cost ordering: measured cost per group (density, force), the order
  // of the next first-tier launch, its bins and queue heads
  DevBuf gcost_d, gcost_f, gorder, gbins, gcbin;
  // tile 2: each group's last first-tier force stage size, and the partition
  DevBuf gstage, gbflag, gbexcl, gborder, gbsplit;
  int n_groups = 0;
  bool groups_valid = false;
  int64_t n_gd_tasks = 0, n_gf_tasks = 0;
  DevBuf cell_count, cell_start, cursor, nodes, frontier, frontier2, leaves, scan_tmp, active,
      dens_off, dens_tasks, force_off, force_tasks;
  int n_cells = 0, n_nodes = 0, n_leaves = 0;
  int64_t n_dens_tasks = 0, n_force_tasks = 0;

  // neighbour cache of the batched form: the density's stage and per-lane
  // lists kept in HBM for the force and for later calls
  DevBuf vc_meta, vc_sj, vc_slot, vc_list, vc_rl, vc_dpath, vc_dmax, vc_gmode, vc_fuse, vc_ctl;
  bool vc_valid = false;  // laid out for the current groups and tile, epoch started
  int vc_tile = -1;

  DevCounters *ctr = nullptr;    // device
  DevCounters *ctr_h = nullptr;  // pinned host mirror

  bool loaded = false, grid_valid = false, density_valid = false, force_valid = false;
  bool sorts_valid = false;  // pair-axis sorts match the current grid
  bool groups_geom_valid = false;  // group frames and boxes match the current positions
  bool grid_reusable = false;      // the last step's grid passed the reach check
  int reuse_streak = 0;            // steps run in a row on the current grid
  int regrids_in_step = 0;
  long long grid_stamp = 0;        // bumped by every regrid (sizes, buffers, store swap)
  // symmetric force: the coloured cells of the current grid
  DevBuf sym_cells, sym_cell_leaf, sym_leafcell;
  std::vector<int> sym_off;
  long long sym_stamp = -1;
  // steady steps as one CUDA graph (batched form on a reused grid)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  long long graph_stamp = -1;
  long long graph_kernels = 0, graph_dens = 0, graph_force = 0;
  unsigned graph_stage_mask = 0;   // stages whose events the graph records
  bool capturing = false;
  long long graph_steps = 0;
  unsigned *boxout = nullptr;      // per box: largest distance outside the top cell
  int last_passes = 0, last_rebuilds = 0;
  // cumulative counters and stage timers
  long long launches = 0, dens_launches = 0, force_launches = 0, sort_launches = 0;
  long long reused_steps = 0, redone_steps = 0;
  unsigned long long total_dens_inter = 0, total_force_inter = 0;
  bool force_pending = false;  // force counters on the device not yet added to the totals
  cudaEvent_t ev[9][2] = {};
  bool ev_pending[9] = {};
  double t_ms[9] = {};
};

namespace sph {
thread_local long long *g_launch_count = nullptr;
}

namespace {

// Timed stages. The walks before the density and before the force, and the
// two kicks, have separate slots so one captured step records each once.
enum Stage { kGrid = 0, kLists, kDens, kGhost, kForce, kInteg, kSort, kLists2, kInteg2, kNStages };
static_assert(kNStages == 9, "event arrays of sph_ctx");

// Points the launch counter at this context for the duration of an API call.
struct LaunchScope {
  long long *prev;
  explicit LaunchScope(sph_ctx *c) : prev(g_launch_count) { g_launch_count = &c->launches; }
  ~LaunchScope() { g_launch_count = prev; }
};

// Inside a stream capture an event record must be an external event node to
// take a timestamp when the graph runs (a plain record only orders streams).
void record(sph_ctx *c, cudaEvent_t e) {
  if (c->capturing)
    cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(e, c->stream);
}
void tic(sph_ctx *c, Stage s) {
  if (c->p.profile) record(c, c->ev[s][0]);
}
void toc(sph_ctx *c, Stage s) {
  if (!c->p.profile) return;
  record(c, c->ev[s][1]);
  c->ev_pending[s] = true;
  if (c->capturing) c->graph_stage_mask |= 1u << s;
}
// Add the elapsed time of every bracket whose closing event was recorded.
void collect_timers(sph_ctx *c) {
  if (!c->p.profile) return;
  for (int s = 0; s < kNStages; ++s) {
    if (!c->ev_pending[s]) continue;
    if (cudaEventSynchronize(c->ev[s][1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[s][0], c->ev[s][1]) == cudaSuccess)
      c->t_ms[s] += ms;
    else
      cudaGetLastError();  // a timer is diagnostics: never fail the call over it
    c->ev_pending[s] = false;
  }
}

}  // namespace

namespace {

int fail(sph_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

#define CUDA_TRY(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(c, SPH_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

#define TRY(call)            \
  do {                       \
    int rc_ = (call);        \
    if (rc_) return rc_;     \
  } while (0)

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int ensure(sph_ctx *c, DevBuf &b, size_t bytes, bool keep = false) {
  if (bytes == 0) bytes = 256;
  if (b.bytes >= bytes) return SPH_OK;
  size_t nb = std::max(bytes, b.bytes + b.bytes / 2);
  void *np = nullptr;
  if (cudaMalloc(&np, nb) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SPH_ENOMEM, "device allocation of %zu bytes failed", nb);
  }
  if (keep && b.p && b.bytes) {
    CUDA_TRY(cudaMemcpyAsync(np, b.p, b.bytes, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  if (b.p) cudaFree(b.p);
  b.p = np;
  b.bytes = nb;
  return SPH_OK;
}

void release(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

template <class T>
T *as(DevBuf &b) {
  return reinterpret_cast<T *>(b.p);
}

// Bytes of every fixed-size per-particle array, in allocation order.
struct FixedLayout {
  std::vector<size_t> sizes;
  size_t total = 0;
};

FixedLayout fixed_layout(int64_t n, int nb) {
  FixedLayout L;
  const size_t N = (size_t)n;
  auto add = [&](size_t b) {
    L.sizes.push_back(b);
    L.total += align256(b);
  };
  for (int copy = 0; copy < 2; ++copy) {
    for (int k = 0; k < 6; ++k) add(N * sizeof(double));  // x0 x1 x2 h hlo hhi
    for (int k = 0; k < 3; ++k) add(N * sizeof(float4));  // vu vu_pred acc
    add(N * sizeof(float));                               // m
    add(N * sizeof(int));                                 // orig
  }
  add(N * sizeof(float));          // hf
  add(N * sizeof(float4));         // pm
  add(N * sizeof(float4));         // gpos
  add((size_t)kAxes * N * sizeof(float));  // skey
  add((size_t)kAxes * N * sizeof(int));    // sidx
  add(N * sizeof(float4));         // sums
  add(N * sizeof(float4));         // fi
  for (int k = 0; k < 5; ++k) add(N * sizeof(int));  // cnt niter nngb nforce leaf_of
  add(N);                          // done
  add(N);                          // fdone
  for (int k = 0; k < 4; ++k) add(N * sizeof(float));  // rho omega P fprev
  add(N * sizeof(int));            // cell_of
  add(N * sizeof(int));            // order
  add(N * sizeof(int));            // order_tmp
  add((N + 1) * sizeof(int));      // flag
  add((N + 1) * sizeof(int));      // excl
  add(N * sizeof(int));            // ident
  for (int k = 0; k < 3; ++k) add(N * sizeof(unsigned));  // mkey msrt mscr
  add(3 * N * sizeof(double));     // wx
  add((size_t)(nb + 2) * sizeof(unsigned long long));     // hext
  add((size_t)nb * sizeof(unsigned));                      // boxout
  add((size_t)nb * sizeof(BoxDev));                        // boxes
  return L;
}

int alloc_fixed(sph_ctx *c, int64_t n, int nb) {
  if (c->alloc_n == n && c->alloc_nb == nb && c->alloc_ws == c->ws) return SPH_OK;  // reuse
  c->alloc_n = -1;
  FixedLayout L = fixed_layout(n, nb);
  for (void *p : c->owned) cudaFree(p);
  c->owned.clear();
  char *base = nullptr;
  if (c->ws) {
    if (c->ws_bytes < L.total)
      return fail(c, SPH_ENOMEM, "workspace of %zu bytes is below the %zu needed", c->ws_bytes,
                  L.total);
    base = c->ws;
  } else {
    void *p = nullptr;
    if (cudaMalloc(&p, L.total) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, SPH_ENOMEM, "device allocation of %zu bytes failed", L.total);
    }
    c->owned.push_back(p);
    base = (char *)p;
  }
  size_t off = 0, k = 0;
  auto take = [&](auto *&ptr) {
    ptr = reinterpret_cast<std::remove_reference_t<decltype(ptr)>>(base + off);
    off += align256(L.sizes[k++]);
  };
  StoreArrays *S[2] = {&c->st, &c->st2};
  for (int copy = 0; copy < 2; ++copy) {
    take(S[copy]->x0);
    take(S[copy]->x1);
    take(S[copy]->x2);
    take(S[copy]->h);
    take(S[copy]->hlo);
    take(S[copy]->hhi);
    take(S[copy]->vu);
    take(S[copy]->vu_pred);
    take(S[copy]->acc);
    take(S[copy]->m);
    take(S[copy]->orig);
  }
  take(c->hf);
  take(c->pm);
  take(c->gpos);
  take(c->skey);
  take(c->sidx);
  take(c->sums);
  take(c->fi);
  take(c->cnt);
  take(c->niter);
  take(c->nngb);
  take(c->nforce);
  take(c->leaf_of);
  take(c->done);
  take(c->fdone);
  take(c->rho);
  take(c->omega);
  take(c->P);
  take(c->fprev);
  take(c->cell_of);
  take(c->order);
  take(c->order_tmp);
  take(c->flag);
  take(c->excl);
  take(c->ident);
  take(c->mkey);
  take(c->msrt);
  take(c->mscr);
  take(c->wx);
  take(c->hext);
  take(c->boxout);
  take(c->boxes_d);
  c->alloc_n = n;
  c->alloc_nb = nb;
  c->alloc_ws = c->ws;
  return SPH_OK;
}

__global__ void k_iota(int *a, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

int read_counters(sph_ctx *c) {
  CUDA_TRY(cudaMemcpyAsync(c->ctr_h, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->force_pending) {
    c->total_force_inter += c->ctr_h->force_inter;
    c->force_pending = false;
  }
  collect_timers(c);
  return SPH_OK;
}

int sync_check(sph_ctx *c) {
  CUDA_TRY(cudaGetLastError());
  return SPH_OK;
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
}

// Choose top-grid cells per box from the largest h: edge >= cell_factor h_max
// where the box allows (headroom for h growth and for drift on a reused
// grid), never below h_max, >= 3 per axis.
int choose_grid(sph_ctx *c, const std::vector<double> &hmax_box) {
  int base = 0;
  for (int b = 0; b < c->nb; ++b) {
    BoxDev &B = c->boxes_h[b];
    if (B.count == 0) {  // an empty box keeps a minimal 3x3x3 grid
      for (int d = 0; d < 3; ++d) {
        B.n[d] = 3;
        B.w[d] = B.L[d] / 3.0;
        B.iw[d] = 1.0 / B.w[d];
        B.wf[d] = (float)B.w[d];
      }
      B.eps = (float)(1e-5 * std::max(B.w[0], std::max(B.w[1], B.w[2])));
      B.hcap = std::min(B.L[0], std::min(B.L[1], B.L[2])) / (3.0 * (1.0 + 1e-6));
      B.cell_base = base;
      base += 27;
      continue;
    }
    const double hm = hmax_box[b] * (1.0 + 1e-6);
    const double lmin = std::min(B.L[0], std::min(B.L[1], B.L[2]));
    if (!(hm > 0.0)) return fail(c, SPH_EINVAL, "box %d has a non-positive smoothing length", b);
    if (hm > lmin / 3.0 * (1.0 + 1e-12))
      return fail(c, SPH_EBOXTOOSMALL, "box %d: h = %g exceeds L/3 = %g", b, hmax_box[b],
                  lmin / 3.0);
    const int64_t cap = std::max<int64_t>(27, 2 * (int64_t)B.count);
    for (int d = 0; d < 3; ++d) {
      int64_t nd = (int64_t)std::floor(B.L[d] / (c->p.cell_factor * hm));
      if (nd < 3) nd = (int64_t)std::floor(B.L[d] / hm);
      nd = std::max<int64_t>(3, std::min<int64_t>(nd, 1024));
      B.n[d] = (int)nd;
    }
    while ((int64_t)B.n[0] * B.n[1] * B.n[2] > cap) {
      int d = 0;
      for (int k = 1; k < 3; ++k)
        if (B.n[k] > B.n[d]) d = k;
      if (B.n[d] <= 3) break;
      B.n[d] = std::max(3, B.n[d] * 3 / 4);
    }
    double wmax = 0.0;
    for (int d = 0; d < 3; ++d) {
      B.w[d] = B.L[d] / B.n[d];
      B.iw[d] = 1.0 / B.w[d];
      B.wf[d] = (float)B.w[d];
      wmax = std::max(wmax, B.w[d]);
    }
    B.eps = (float)(1e-5 * wmax);
    B.hcap = lmin / (3.0 * (1.0 + 1e-6));
    B.cell_base = base;
    base += B.n[0] * B.n[1] * B.n[2];
  }
  c->n_cells = base;
  CUDA_TRY(cudaMemcpyAsync(c->boxes_d, c->boxes_h.data(), sizeof(BoxDev) * c->nb,
                           cudaMemcpyHostToDevice, c->stream));
  return SPH_OK;
}

int h_extremes(sph_ctx *c, const double *h, std::vector<double> &hmax_box, double &hmin,
               double &hmax) {
  std::vector<unsigned long long> init(c->nb + 2, 0ull);
  init[c->nb] = ~0ull;
  CUDA_TRY(cudaMemcpyAsync(c->hext, init.data(), sizeof(unsigned long long) * init.size(),
                           cudaMemcpyHostToDevice, c->stream));
  launch_h_extremes(h, c->n, c->boxes_d, c->nb, c->hext, c->hext + c->nb, c->stream);
  CUDA_TRY(cudaMemcpyAsync(init.data(), c->hext, sizeof(unsigned long long) * init.size(),
                           cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  hmax_box.resize(c->nb);
  for (int b = 0; b < c->nb; ++b) hmax_box[b] = bits_to_double(init[b]);
  hmin = bits_to_double(init[c->nb]);
  hmax = bits_to_double(init[c->nb + 1]);
  return SPH_OK;
}

// A1 + A2: grid, recursive split, leaves, store gather, leaf geometry.
// from_caller: positions come from the wrapped caller copy (c->wx) and the
// store is loaded from the caller arrays passed in.
int build_grid_inner(sph_ctx *c, bool from_caller, const float *cv, const float *cm, const float *cu,
               const double *ch) {
  std::vector<double> hmax_box;
  double hmin, hmax;
  TRY(h_extremes(c, from_caller ? ch : c->st.h, hmax_box, hmin, hmax));
  TRY(choose_grid(c, hmax_box));

  const int n = c->n, C = c->n_cells;
  TRY(ensure(c, c->cell_count, sizeof(int) * (C + 1)));
  TRY(ensure(c, c->cell_start, sizeof(int) * (C + 1)));
  TRY(ensure(c, c->cursor, sizeof(int) * (C + 1)));
  TRY(ensure(c, c->scan_tmp, scan_tmp_bytes(std::max(C + 1, n + 1))));
  CUDA_TRY(cudaMemsetAsync(c->cell_count.p, 0, sizeof(int) * (C + 1), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->cursor.p, 0, sizeof(int) * (C + 1), c->stream));

  GridArgs g{};
  g.n = n;
  g.n_boxes = c->nb;
  g.boxes = c->boxes_d;
  g.n_cells = C;
  g.n_split = c->p.n_split;
  if (from_caller) {
    g.x0 = c->wx;
    g.x1 = c->wx + n;
    g.x2 = c->wx + 2 * (size_t)n;
    g.orig = c->ident;
  } else {
    g.x0 = c->st.x0;
    g.x1 = c->st.x1;
    g.x2 = c->st.x2;
    g.orig = c->st.orig;
  }
  g.cell_of = c->cell_of;
  g.morton = c->mkey;
  g.morton_tmp = c->msrt;
  g.morton_scr = c->mscr;
  g.cell_count = as<int>(c->cell_count);
  g.cell_start = as<int>(c->cell_start);
  g.cursor = as<int>(c->cursor);
  g.order = c->order;
  g.order_tmp = c->order_tmp;

  launch_cell_keys(g, c->stream);
  exclusive_scan_int(g.cell_count, g.cell_start, C + 1, c->scan_tmp.p, c->scan_tmp.bytes,
                     c->stream);
  launch_cell_scatter(g, c->stream);

  // A2: recursive octant split
  size_t want_nodes = (size_t)C + (size_t)n / 4 + 1024;
  TRY(ensure(c, c->nodes, sizeof(Node) * want_nodes));
  TRY(ensure(c, c->frontier, sizeof(int) * want_nodes));
  TRY(ensure(c, c->frontier2, sizeof(int) * want_nodes));
  launch_init_top_nodes(as<Node>(c->nodes), g, c->stream);
  CUDA_TRY(cudaMemsetAsync(&c->ctr->n_frontier, 0, sizeof(int), c->stream));
  launch_frontier_top(as<Node>(c->nodes), C, c->p.n_split, as<int>(c->frontier), c->ctr,
                      c->stream);
  TRY(read_counters(c));
  int nf = c->ctr_h->n_frontier;
  int n_nodes = C;
  for (int level = 0; level < kMaxDepth && nf > 0; ++level) {
    const size_t need = (size_t)n_nodes + 8 * (size_t)nf;
    if (sizeof(Node) * need > c->nodes.bytes) {
      TRY(ensure(c, c->nodes, sizeof(Node) * need * 3 / 2, true));
      TRY(ensure(c, c->frontier, sizeof(int) * need * 3 / 2, true));
      TRY(ensure(c, c->frontier2, sizeof(int) * need * 3 / 2, false));
    }
    CUDA_TRY(cudaMemsetAsync(&c->ctr->n_frontier, 0, sizeof(int), c->stream));
    launch_split_level(as<Node>(c->nodes), as<int>(c->frontier), nf, n_nodes, level,
                       c->p.n_split, as<int>(c->frontier2), c->ctr, g, c->stream);
    n_nodes += 8 * nf;
    TRY(read_counters(c));
    nf = c->ctr_h->n_frontier;
    std::swap(c->frontier, c->frontier2);
  }
  c->n_nodes = n_nodes;

  // leaves, in slot order
  CUDA_TRY(cudaMemsetAsync(c->flag, 0, sizeof(int) * (n + 1), c->stream));
  launch_mark_leaves(as<Node>(c->nodes), n_nodes, c->flag, c->stream);
  exclusive_scan_int(c->flag, c->excl, n + 1, c->scan_tmp.p, c->scan_tmp.bytes, c->stream);
  int nl = 0;
  CUDA_TRY(cudaMemcpyAsync(&nl, c->excl + n, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->n_leaves = nl;
  TRY(ensure(c, c->leaves, sizeof(Leaf) * (size_t)std::max(nl, 1)));
  TRY(ensure(c, c->active, sizeof(int) * (size_t)(nl + 1)));
  launch_fill_leaves(as<Node>(c->nodes), n_nodes, c->excl, as<Leaf>(c->leaves), c->boxes_d, c->nb,
                     c->stream);
  launch_sort_leaves(as<Leaf>(c->leaves), nl, c->order, g.orig, g.morton, c->stream);

  // gather the store into leaf order
  if (from_caller) {
    launch_load_caller(c->st, c->order, n, c->wx, cv, cm, cu, ch, c->stream);
  } else {
    launch_permute(c->st2, c->st, c->order, n, c->stream);
    std::swap(c->st, c->st2);
  }
  launch_leaf_of(as<Leaf>(c->leaves), nl, c->leaf_of, c->stream);
  launch_h_to_float(c->st.h, c->hf, n, c->stream);
  GeomArgs ga{nl, as<Leaf>(c->leaves), as<Node>(c->nodes), c->boxes_d, c->nb,
              c->st.x0, c->st.x1, c->st.x2, c->st.m, c->hf, c->pm};
  launch_leaf_geometry(ga, n_nodes, c->stream);
  TRY(sync_check(c));
  CUDA_TRY(cudaMemsetAsync(c->boxout, 0, sizeof(unsigned) * (size_t)c->nb, c->stream));
  ++c->grid_stamp;
  c->grid_valid = true;
  c->groups_valid = false;
  c->groups_geom_valid = false;
  c->density_valid = false;
  c->force_valid = false;
  ++c->regrids_in_step;
  return SPH_OK;
}

int build_grid(sph_ctx *c, bool from_caller, const float *cv, const float *cm, const float *cu,
               const double *ch) {
  tic(c, kGrid);
  int rc = build_grid_inner(c, from_caller, cv, cm, cu, ch);
  toc(c, kGrid);
  c->sorts_valid = false;
  return rc;
}

// A3: every leaf's particles sorted along the 13 pair axes, once per grid,
// before the first per-pass (leaf-pair task) kernel that prunes with them.
// The batched kernels do not read them, so a step they finish alone sorts
// nothing.
void ensure_sorts(sph_ctx *c) {
  if (!c->p.pair_sort || c->sorts_valid) return;
  tic(c, kSort);
  AxisSortArgs sa{c->n_leaves, as<Leaf>(c->leaves), c->pm, c->n, c->skey, c->sidx};
  launch_axis_sort(sa, c->stream);
  toc(c, kSort);
  ++c->sort_launches;
  c->sorts_valid = true;
}

GeomArgs geom_args(sph_ctx *c) {
  return GeomArgs{c->n_leaves, as<Leaf>(c->leaves), as<Node>(c->nodes), c->boxes_d, c->nb,
                  c->st.x0, c->st.x1, c->st.x2, c->st.m, c->hf, c->pm};
}

// Count pass, scan, fill pass of a task list over `n_targets` target leaves.
int build_lists_inner(sph_ctx *c, bool force, const int *active, int n_targets, DevBuf &off,
                      DevBuf &tasks, int64_t &n_tasks) {
  TRY(ensure(c, off, sizeof(int) * (size_t)(n_targets + 1)));
  TRY(ensure(c, c->lflag, sizeof(int) * (size_t)std::max(n_targets, 1)));
  ListArgs la{};
  la.n_leaves = c->n_leaves;
  la.leaves = as<Leaf>(c->leaves);
  la.nodes = as<Node>(c->nodes);
  la.boxes = c->boxes_d;
  la.n_boxes = c->nb;
  la.force = force ? 1 : 0;
  la.cap_factor = 1.0f;
  la.count = as<int>(off);
  la.offset = nullptr;
  la.tasks = nullptr;
  la.active = active;
  la.n_targets = n_targets;
  la.status = &c->ctr->status;
  la.flag = as<int>(c->lflag);
  CUDA_TRY(cudaMemsetAsync(as<int>(off) + n_targets, 0, sizeof(int), c->stream));
  launch_build_lists(la, c->stream);
  exclusive_scan_int(as<int>(off), as<int>(off), n_targets + 1, c->scan_tmp.p, c->scan_tmp.bytes,
                     c->stream);
  int total = 0;
  CUDA_TRY(cudaMemcpyAsync(&total, as<int>(off) + n_targets, sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (total < 0) return fail(c, SPH_ENOMEM, "task list exceeds 2^31 entries");
  TRY(ensure(c, tasks, sizeof(Task) * (size_t)std::max(total, 1)));
  la.offset = as<int>(off);
  la.tasks = as<Task>(tasks);
  launch_build_lists(la, c->stream);
  n_tasks = total;
  return sync_check(c);
}

int build_lists(sph_ctx *c, bool force, const int *active, int n_targets, DevBuf &off,
                DevBuf &tasks, int64_t &n_tasks) {
  tic(c, kLists);
  int rc = build_lists_inner(c, force, active, n_targets, off, tasks, n_tasks);
  toc(c, kLists);
  return rc;
}

int check_status(sph_ctx *c, int st) {
  if (st & kErrBoxTooSmall)
    return fail(c, SPH_EBOXTOOSMALL, "a smoothing length would exceed L/3 of its box");
  if (st & kErrNonPhysical)
    return fail(c, SPH_ENONPHYSICAL, "non-physical state (rho <= 0, Omega <= 0 or u <= 0)");
  if (st & kErrListOverflow) return fail(c, SPH_ECUDA, "tree walk stack overflow");
  return SPH_OK;
}

GroupBuildArgs group_args(sph_ctx *c) {
  GroupBuildArgs ga{};
  ga.n_nodes = c->n_nodes;
  ga.nodes = as<Node>(c->nodes);
  ga.n_cells = c->n_cells;
  ga.cell_start = as<int>(c->cell_start);
  ga.cell_count = as<int>(c->cell_count);
  ga.boxes = c->boxes_d;
  ga.n_boxes = c->nb;
  ga.gcount = as<int>(c->gcount);
  ga.groups = as<Group>(c->groups);
  ga.n_groups = c->n_groups;
  ga.leaves = as<Leaf>(c->leaves);
  ga.leaf_of = c->leaf_of;
  ga.pm = c->pm;
  ga.hf = c->hf;
  ga.gpos = c->gpos;
  return ga;
}

// Target groups of the batched form: <= 32 consecutive particles per top cell.
int build_groups(sph_ctx *c) {
  const int C = c->n_nodes;
  TRY(ensure(c, c->gcount, sizeof(int) * (size_t)(C + 1)));
  TRY(ensure(c, c->scan_tmp, scan_tmp_bytes(std::max(C + 1, c->n + 1))));
  CUDA_TRY(cudaMemsetAsync(as<int>(c->gcount) + C, 0, sizeof(int), c->stream));
  GroupBuildArgs ga = group_args(c);
  launch_group_count(ga, c->stream);
  exclusive_scan_int(ga.gcount, ga.gcount, C + 1, c->scan_tmp.p, c->scan_tmp.bytes, c->stream);
  int ng = 0;
  CUDA_TRY(cudaMemcpyAsync(&ng, ga.gcount + C, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->n_groups = ng;
  TRY(ensure(c, c->groups, sizeof(Group) * (size_t)std::max(ng, 1)));
  // queue, queue2 (4 per group), queue_big
  TRY(ensure(c, c->gqueue, sizeof(int) * (size_t)std::max(ng, 1) * 6));
  // new groups: no measured cost yet (the first order is the estimate)
  TRY(ensure(c, c->gcost_d, sizeof(float) * (size_t)std::max(ng, 1)));
  TRY(ensure(c, c->gcost_f, sizeof(float) * (size_t)std::max(ng, 1)));
  const size_t n_chunks = (size_t)std::max(ng, 1) / 32 + 1;
  TRY(ensure(c, c->gorder, sizeof(int) * n_chunks * 32));
  TRY(ensure(c, c->gbins, sizeof(int) * (kCostBins + 4)));
  TRY(ensure(c, c->gcbin, sizeof(int) * n_chunks));
  TRY(ensure(c, c->gstage, sizeof(int) * (size_t)std::max(ng, 1)));
  TRY(ensure(c, c->gbflag, sizeof(int) * (size_t)(ng + 1)));
  TRY(ensure(c, c->gbexcl, sizeof(int) * (size_t)(ng + 1)));
  TRY(ensure(c, c->gborder, sizeof(int) * (size_t)std::max(ng, 1)));
  TRY(ensure(c, c->gbsplit, sizeof(int)));
  // new groups: no stage measured yet (tile 2 puts them on the large stage)
  CUDA_TRY(cudaMemsetAsync(c->gstage.p, 0xff, sizeof(int) * (size_t)std::max(ng, 1), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->gcost_d.p, 0, sizeof(float) * (size_t)std::max(ng, 1), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->gcost_f.p, 0, sizeof(float) * (size_t)std::max(ng, 1), c->stream));
  ga = group_args(c);
  launch_group_fill(ga, c->stream);
  launch_group_geometry(ga, c->stream);
  c->groups_valid = true;
  c->groups_geom_valid = true;
  c->vc_valid = false;  // new groups and particle order: the cache starts a new epoch
  return sync_check(c);
}

// Groups below which the cache is not used: such sets are bound by launch
// and memory latency, where the cache's extra kernels cost more than the
// searches they save.
constexpr int kCacheMinGroups = 16384;

bool cache_on(const sph_ctx *c) {
  return c->p.mode == SPH_MODE_BATCHED &&
         (c->p.reuse_lists == 2 || (c->p.reuse_lists == 1 && c->n_groups >= kCacheMinGroups));
}

CacheArgs cache_args(sph_ctx *c) {
  CacheArgs a{};
  a.meta = as<GroupCache>(c->vc_meta);
  a.sj = as<int>(c->vc_sj);
  a.slot = as<unsigned short>(c->vc_slot);
  a.list = as<unsigned short>(c->vc_list);
  a.rl = as<float>(c->vc_rl);
  a.dpath = as<float>(c->vc_dpath);
  a.dmax_cell = as<unsigned>(c->vc_dmax);
  a.gmode = as<unsigned char>(c->vc_gmode);
  a.fuse = as<unsigned char>(c->vc_fuse);
  a.ctl = as<CacheCtl>(c->vc_ctl);
  a.tasks = as<Task>(c->gd_tasks);
  a.tcount = as<int>(c->gd_off);
  a.ns = cache_stage_slots(c->p.tile);
  a.lane_cap = cache_lane_cap(c->p.tile);
  return a;
}

DriftCache drift_cache(sph_ctx *c) {
  DriftCache d{};
  d.dpath = as<float>(c->vc_dpath);
  d.dmax_cell = as<unsigned>(c->vc_dmax);
  d.ctl = as<CacheCtl>(c->vc_ctl);
  d.leaf_of = c->leaf_of;
  d.leaves = as<Leaf>(c->leaves);
  d.nodes = as<Node>(c->nodes);
  return d;
}

// Lay the neighbour cache out for the current groups and tile and start a new
// epoch (every group builds; path lengths from zero). Not inside a capture:
// the steady step is captured only once a density has prepared it.
int cache_prepare(sph_ctx *c) {
  if (!cache_on(c) || (c->vc_valid && c->vc_tile == c->p.tile)) return SPH_OK;
  if (c->capturing) return fail(c, SPH_ESTATE, "neighbour cache laid out inside a capture");
  const size_t ng = (size_t)std::max(c->n_groups, 1), n = (size_t)std::max(c->n, 1);
  const size_t ns = (size_t)cache_stage_slots(c->p.tile), lc = (size_t)cache_lane_cap(c->p.tile);
  TRY(ensure(c, c->vc_meta, sizeof(GroupCache) * ng));
  TRY(ensure(c, c->vc_sj, sizeof(int) * ng * ns));
  TRY(ensure(c, c->vc_slot, sizeof(unsigned short) * ng * ns));
  TRY(ensure(c, c->vc_list, sizeof(unsigned short) * ng * 4 * lc * 32));
  TRY(ensure(c, c->vc_rl, sizeof(float) * n));
  TRY(ensure(c, c->vc_dpath, sizeof(float) * n));
  TRY(ensure(c, c->vc_dmax, sizeof(unsigned) * (size_t)std::max(c->n_cells, 1)));
  TRY(ensure(c, c->vc_gmode, ng));
  TRY(ensure(c, c->vc_fuse, ng));
  TRY(ensure(c, c->vc_ctl, sizeof(CacheCtl)));
  CUDA_TRY(cudaMemsetAsync(c->vc_meta.p, 0, sizeof(GroupCache) * ng, c->stream));
  CUDA_TRY(cudaMemsetAsync(c->vc_dpath.p, 0, sizeof(float) * n, c->stream));
  CUDA_TRY(cudaMemsetAsync(c->vc_dmax.p, 0, sizeof(unsigned) * (size_t)std::max(c->n_cells, 1),
                           c->stream));
  CUDA_TRY(cudaMemsetAsync(c->vc_fuse.p, 0, ng, c->stream));
  launch_cache_init(as<CacheCtl>(c->vc_ctl), c->n_groups, c->stream);
  c->vc_valid = true;
  c->vc_tile = c->p.tile;
  return sync_check(c);
}

constexpr int kTaskCap = 384;  // task slots per group

// Group task lists: one walk, written into fixed per-group slots (no host
// round trip).
int build_group_lists(sph_ctx *c, bool force, float skin, DevBuf &cnt, DevBuf &tasks) {
  const Stage stage = force ? kLists2 : kLists;
  if (c->n_nodes >= kWalkMaxNodes)
    return fail(c, SPH_ENOMEM, "octree of %d nodes exceeds the walk's node index (2^26)",
                c->n_nodes);
  tic(c, stage);
  const int ng = c->n_groups;
  TRY(ensure(c, cnt, sizeof(int) * (size_t)std::max(ng, 1)));
  TRY(ensure(c, tasks, sizeof(Task) * (size_t)std::max(ng, 1) * kTaskCap));
  TRY(ensure(c, c->gwmode, (size_t)std::max(ng, 1)));
  GroupListArgs la{};
  la.n_groups = ng;
  la.groups = as<Group>(c->groups);
  la.leaves = as<Leaf>(c->leaves);
  la.nodes = as<Node>(c->nodes);
  la.boxes = c->boxes_d;
  la.force = force ? 1 : 0;
  la.skin = skin;
  la.tcap = kTaskCap;
  la.count = as<int>(cnt);
  la.tasks = as<Task>(tasks);
  la.status = &c->ctr->status;
  la.leaf_of = c->leaf_of;
  la.pm = c->pm;
  la.hf = c->hf;
  la.walk_queue = as<int>(c->gqueue);  // free until the interaction kernels run
  la.walk_queued = &c->ctr->walk_queued;
  la.ctr = c->ctr;
  la.wmode = force ? nullptr : as<unsigned char>(c->gwmode);
  la.cache_on = cache_on(c) && c->vc_valid;
  if (la.cache_on) la.cache = cache_args(c);
  CUDA_TRY(cudaMemsetAsync(la.walk_queued, 0, sizeof(int), c->stream));
  launch_group_lists(la, c->stream);
  toc(c, stage);
  return sync_check(c);
}

// Radii of the batched density, as multiples of h from before the call: the
// stage (group walk and staging) covers 1.06 x the group's largest h, a
// warp's candidates 1.02 x its sub-cluster's largest h, a lane's list 1.02 x
// its target's h. Steady steps start from h carried by the drift, so the
// iteration rarely leaves these radii; when a target's h does, its warp
// refilters or rebuilds its lists, and beyond the stage the target goes to
// the third tier.
constexpr float kSkinStage = 1.06f;
constexpr float kSkinList = 1.02f;

// Batched density: every particle whose group fits the stage and converges
// inside the kernel is finished here; the rest keep done = 0 for the
// per-pass loop.
// The kernels of the batched density (group frames if stale, h maxima, the
// walk, the three tiers), no host reads.
// `hmax_current`: the node and group h maxima still hold for the current h
// (a steady step: h has not changed since the last force's walk).
// Which (v, u) the pressure and the force use: the current ones, or those
// predicted to the end of a step. Passed as a choice, not a pointer: a regrid
// inside a call permutes the store by swapping its two copies, so the array
// is looked up at each use.
enum VuSel { kVuCurrent = 0, kVuPredicted = 1 };
const float4 *vu_of(const sph_ctx *c, VuSel sel) {
  return sel == kVuPredicted ? c->st.vu_pred : c->st.vu;
}

// Groups from which the first tier claims its groups from a work queue
// (work_queue = 1): at least 32 claims of 32 groups for every block the
// GPU holds at once. Below that a claim is a large share of a block's work
// and the fixed grid stride balances as well.
constexpr int kQueueMinGroups = 1 << 20;

// Tile 2: a group takes the small first-tier force stage (704 entries) when
// its last stage held at most this many (a margin for the motion since).
constexpr int kForceSmallFit = 640;

// 0: grid stride; 1: work queue in group order; 2: work queue in measured
// cost order.
int queue_mode(const sph_ctx *c) {
  switch (c->p.work_queue) {
    case 1: return c->n_groups >= kQueueMinGroups ? 1 : 0;
    case 2: return 1;
    case 3: return 2;
    default: return 0;
  }
}

// The work queue of a first-tier launch: heads [head0, head0 + n_heads) of
// gbins; in cost order, ordered from the costs the last call measured.
void work_queue(sph_ctx *c, const int *tcount, float *cost, int head0, int n_heads,
                WorkQueue &wq) {
  int *heads = as<int>(c->gbins) + kCostBins + head0;
  const int mode = queue_mode(c);
  if (mode == 2)
    launch_cost_order(as<Group>(c->groups), c->n_groups, tcount, cost, as<int>(c->gorder),
                      as<int>(c->gbins), as<int>(c->gcbin), heads, n_heads, c->stream);
  else
    cudaMemsetAsync(heads, 0, sizeof(int) * n_heads, c->stream);
  wq = WorkQueue{mode == 2 ? as<int>(c->gorder) : nullptr, heads, cost};
}

int enqueue_density_batched(sph_ctx *c, VuSel vu_for_P, bool hmax_current = false) {
  if (!c->groups_valid) TRY(build_groups(c));
  TRY(cache_prepare(c));
  if (!c->groups_geom_valid) {  // positions moved on an unchanged grid
    launch_group_geometry(group_args(c), c->stream);
    c->groups_geom_valid = true;
  }
  if (!hmax_current) {
    launch_group_hmax(group_args(c), c->stream);
    launch_leaf_hmax(geom_args(c), c->n_nodes, c->stream);
  }
  TRY(build_group_lists(c, false, kSkinStage, c->gd_off, c->gd_tasks));
  BatchDensArgs da{};
  da.n_groups = c->n_groups;
  da.groups = as<Group>(c->groups);
  da.tcount = as<int>(c->gd_off);
  da.tcap = kTaskCap;
  da.tasks = as<Task>(c->gd_tasks);
  da.leaves = as<Leaf>(c->leaves);
  da.leaf_of = c->leaf_of;
  da.pm = c->pm;
  da.boxes = c->boxes_d;
  da.h = c->st.h;
  da.hf = c->hf;
  da.vu = vu_of(c, vu_for_P);
  da.n_ngb = c->p.n_ngb;
  da.tol = c->p.h_tol;
  da.gamma = c->p.gamma;
  da.max_iter = c->p.max_iter;
  da.skin_stage = kSkinStage;
  da.skin_list = kSkinList;
  da.kahan = c->p.precision == SPH_PREC_KAHAN;
  da.done = c->done;
  da.niter = c->niter;
  da.nngb = c->nngb;
  da.rho = c->rho;
  da.omega = c->omega;
  da.P = c->P;
  da.fi = c->fi;
  da.ctr = c->ctr;
  da.queue = as<int>(c->gqueue);  // ctr->queued, queued2 were zeroed with the counters
  da.queue2 = as<int>(c->gqueue) + c->n_groups;
  da.queue_big = as<int>(c->gqueue) + 5 * (size_t)c->n_groups;
  da.gpos = c->gpos;
  da.tile = c->p.tile;
  da.nodes = as<Node>(c->nodes);
  da.wmode = as<unsigned char>(c->gwmode);
  da.cache_on = cache_on(c) && c->vc_valid;
  if (da.cache_on) da.cache = cache_args(c);
  // heads [0], [1]: the first-tier launches on stored stages and anew
  if (queue_mode(c)) work_queue(c, as<int>(c->gd_off), as<float>(c->gcost_d), 0, 2, da.wq);
  tic(c, kDens);
  launch_density_batched(da, c->stream);
  toc(c, kDens);
  if (da.cache_on) launch_cache_decide(da.cache.ctl, c->stream);
  ++c->dens_launches;
  return sync_check(c);
}

int density_batched(sph_ctx *c, VuSel vu_for_P) {
  TRY(enqueue_density_batched(c, vu_for_P));
  TRY(read_counters(c));
  TRY(check_status(c, c->ctr_h->status));
  c->last_passes = c->ctr_h->max_iter_used;
  return SPH_OK;
}

int density_impl(sph_ctx *c, VuSel vu_for_P) {
  if (!c->grid_valid) TRY(build_grid(c, false, nullptr, nullptr, nullptr, nullptr));
  const int n = c->n;
  launch_h_guess(geom_args(c), c->p.n_ngb, c->st.h, c->hf, c->stream);
  launch_reset_iteration(c->done, c->niter, c->st.hlo, c->st.hhi, c->fprev, n, c->stream);
  CUDA_TRY(cudaMemsetAsync(c->ctr, 0, offsetof(DevCounters, step_status), c->stream));
  c->last_passes = 0;
  c->last_rebuilds = 0;
  if (c->p.mode == SPH_MODE_BATCHED) {
    TRY(density_batched(c, vu_for_P));
    for (int r = 0; r < 2 && (c->ctr_h->status & kErrHGrid); ++r) {
      // some h outgrew its top cell: regrid with the grown h and start again
      TRY(build_grid(c, false, nullptr, nullptr, nullptr, nullptr));
      launch_reset_iteration(c->done, c->niter, c->st.hlo, c->st.hhi, c->fprev, n, c->stream);
      CUDA_TRY(cudaMemsetAsync(c->ctr, 0, offsetof(DevCounters, step_status), c->stream));
      ++c->last_rebuilds;
      TRY(density_batched(c, vu_for_P));
    }
    if (c->ctr_h->fallback == 0 && !(c->ctr_h->status & kErrHGrid)) {
      // every particle finished in the batched kernels: no per-pass remainder
      c->total_dens_inter += c->ctr_h->dens_inter;
      c->density_valid = true;
      c->force_valid = false;
      return SPH_OK;
    }
  }
  const int max_passes = c->p.max_iter + 8;
  for (int pass = 0;; ++pass) {
    if (pass >= max_passes)
      return fail(c, SPH_ENOTCONVERGED, "smoothing lengths did not converge in %d passes",
                  c->p.max_iter);
    GeomArgs ga = geom_args(c);
    launch_leaf_hmax(ga, c->n_nodes, c->stream);
    CUDA_TRY(cudaMemsetAsync(&c->ctr->n_active, 0, sizeof(int), c->stream));
    launch_active_leaves(as<Leaf>(c->leaves), c->n_leaves, c->done, as<int>(c->active), c->ctr,
                         c->stream);
    TRY(read_counters(c));
    const int n_active = c->ctr_h->n_active;
    if (n_active == 0) break;
    ++c->last_passes;
    TRY(build_lists(c, false, as<int>(c->active), n_active, c->dens_off, c->dens_tasks,
                    c->n_dens_tasks));
    DensArgs da{};
    da.n_active = n_active;
    da.active = as<int>(c->active);
    da.leaves = as<Leaf>(c->leaves);
    da.list_off = as<int>(c->dens_off);
    da.tasks = as<Task>(c->dens_tasks);
    da.pm = c->pm;
    da.hf = c->hf;
    da.done = c->done;
    da.sums = c->sums;
    da.cnt = c->cnt;
    da.ctr = c->ctr;
    da.kahan = c->p.precision == SPH_PREC_KAHAN;
    da.skey = c->p.pair_sort ? c->skey : nullptr;
    da.sidx = c->sidx;
    da.n = c->n;
    ensure_sorts(c);
    tic(c, kDens);
    launch_density(da, c->stream);
    toc(c, kDens);
    ++c->dens_launches;
    CUDA_TRY(cudaMemsetAsync(&c->ctr->unconverged, 0, 2 * sizeof(int), c->stream));
    GhostArgs gh{};
    gh.n = n;
    gh.n_ngb = c->p.n_ngb;
    gh.tol = c->p.h_tol;
    gh.gamma = c->p.gamma;
    gh.max_iter = c->p.max_iter;
    gh.leaves = as<Leaf>(c->leaves);
    gh.leaf_of = c->leaf_of;
    gh.nodes = as<Node>(c->nodes);
    gh.boxes = c->boxes_d;
    gh.n_boxes = c->nb;
    gh.cap_factor = 1.0f;
    gh.h = c->st.h;
    gh.hlo = c->st.hlo;
    gh.hhi = c->st.hhi;
    gh.fprev = c->fprev;
    gh.hf = c->hf;
    gh.sums = c->sums;
    gh.cnt = c->cnt;
    gh.vu = vu_of(c, vu_for_P);
    gh.done = c->done;
    gh.niter = c->niter;
    gh.nngb = c->nngb;
    gh.rho = c->rho;
    gh.omega = c->omega;
    gh.P = c->P;
    gh.force_i = c->fi;
    gh.ctr = c->ctr;
    tic(c, kGhost);
    launch_ghost(gh, c->stream);
    toc(c, kGhost);
    TRY(sync_check(c));
    TRY(read_counters(c));
    const int st = c->ctr_h->status;
    TRY(check_status(c, st));
    if (st & kErrHGrid) {
      // an h outgrew its top cell: regrid with the current h and start the
      // converged bookkeeping again (the per-particle results are reordered)
      TRY(build_grid(c, false, nullptr, nullptr, nullptr, nullptr));
      launch_reset_iteration(c->done, c->niter, c->st.hlo, c->st.hhi, c->fprev, n, c->stream);
      CUDA_TRY(cudaMemsetAsync(&c->ctr->dens_inter, 0, sizeof(unsigned long long), c->stream));
      ++c->last_rebuilds;
      continue;
    }
    if (c->ctr_h->unconverged == 0) {
      c->last_passes += 0;
      continue;  // the next active-leaf scan finds none and ends the loop
    }
    if (st & kErrNotConverged)
      return fail(c, SPH_ENOTCONVERGED, "smoothing lengths did not converge in %d passes",
                  c->p.max_iter);
  }
  c->total_dens_inter += c->ctr_h->dens_inter;
  c->density_valid = true;
  c->force_valid = false;
  return SPH_OK;
}

// The kernels of the batched force, no host reads.
// `steady`: called from a steady step, whose start zeroed every counter and
// whose kick-drift cleared the force finished flags (the density writes none
// of the force's counters; any fallback there redoes the step).
int enqueue_force_batched(sph_ctx *c, VuSel vu_for_force, bool steady = false) {
  if (!c->groups_valid) TRY(build_groups(c));
  GroupBuildArgs gb = group_args(c);
  launch_group_hmax(gb, c->stream);
  GeomArgs ga = geom_args(c);
  launch_leaf_hmax(ga, c->n_nodes, c->stream);
  if (cache_on(c) && c->vc_valid) launch_force_gate(as<CacheCtl>(c->vc_ctl), c->stream);
  TRY(build_group_lists(c, true, 1.0f, c->gf_off, c->gf_tasks));
  if (!steady) {
    CUDA_TRY(cudaMemsetAsync(&c->ctr->force_inter, 0, sizeof(unsigned long long), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->ctr->force_cand, 0, sizeof(unsigned long long), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->ctr->unconverged, 0, sizeof(int), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->ctr->queued[1], 0, sizeof(int), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->ctr->queued2[1], 0, sizeof(int), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->ctr->queued_big[1], 0, sizeof(int), c->stream));
    CUDA_TRY(cudaMemsetAsync(c->fdone, 0, (size_t)c->n, c->stream));
  }
  BatchForceArgs fa{};
  fa.n_groups = c->n_groups;
  fa.groups = as<Group>(c->groups);
  fa.tcount = as<int>(c->gf_off);
  fa.tcap = kTaskCap;
  fa.tasks = as<Task>(c->gf_tasks);
  fa.leaves = as<Leaf>(c->leaves);
  fa.leaf_of = c->leaf_of;
  fa.pm = c->pm;
  fa.fi = c->fi;
  fa.vu = vu_of(c, vu_for_force);
  fa.acc = c->st.acc;
  fa.nforce = c->nforce;
  fa.fdone = c->fdone;
  fa.ctr = c->ctr;
  fa.queue = as<int>(c->gqueue);
  fa.queue2 = as<int>(c->gqueue) + c->n_groups;
  fa.queue_big = as<int>(c->gqueue) + 5 * (size_t)c->n_groups;
  fa.gpos = c->gpos;
  fa.tile = c->p.tile;
  fa.nodes = as<Node>(c->nodes);
  fa.boxes = c->boxes_d;
  fa.kahan = c->p.precision == SPH_PREC_KAHAN;
  fa.cache_on = cache_on(c) && c->vc_valid;
  if (fa.cache_on) fa.cache = cache_args(c);
  fa.gstage = as<int>(c->gstage);
  if (c->p.tile == 2) {  // the small stage for the groups whose last stage fitted it
    launch_force_bins(as<int>(c->gstage), c->n_groups, kForceSmallFit, as<int>(c->gbflag),
                      as<int>(c->gbexcl), c->scan_tmp.p, c->scan_tmp.bytes,
                      as<int>(c->gborder), as<int>(c->gbsplit), c->stream);
    fa.border = as<int>(c->gborder);
    fa.bsplit = as<int>(c->gbsplit);
  }
  // heads [2], [3]: the force's first-tier launch(es)
  if (queue_mode(c)) work_queue(c, as<int>(c->gf_off), as<float>(c->gcost_f), 2, 2, fa.wq);
  tic(c, kForce);
  launch_force_batched(fa, c->stream);
  toc(c, kForce);
  ++c->force_launches;
  return sync_check(c);
}

// Batched force; returns through *all_done whether every particle was
// finished (else the per-leaf form must run).
int force_batched(sph_ctx *c, VuSel vu_for_force, bool *all_done) {
  *all_done = false;
  TRY(enqueue_force_batched(c, vu_for_force));
  TRY(read_counters(c));
  c->force_pending = true;  // banked by the next read, with any per-leaf remainder
  *all_done = c->ctr_h->unconverged == 0;
  if (*all_done) c->force_valid = true;
  return SPH_OK;
}

// Symmetric force (SPH_MODE_SYMMETRIC): the per-pass force task lists of
// every leaf, the colour classes of the top cells (once per grid, through
// the host), then one launch per colour; results accumulate from zero.
int force_symmetric(sph_ctx *c, VuSel vu_for_force) {
  GeomArgs ga = geom_args(c);
  launch_leaf_hmax(ga, c->n_nodes, c->stream);
  TRY(build_lists(c, true, nullptr, c->n_leaves, c->force_off, c->force_tasks, c->n_force_tasks));
  const int nl = c->n_leaves;
  if (c->sym_stamp != c->grid_stamp) {
    TRY(ensure(c, c->sym_leafcell, sizeof(int) * (size_t)std::max(nl, 1)));
    launch_leaf_cells(as<Leaf>(c->leaves), as<Node>(c->nodes), nl, as<int>(c->sym_leafcell),
                      c->stream);
    std::vector<int> leaf_cell((size_t)nl), cell_leaf, cells;
    if (nl > 0)
      CUDA_TRY(cudaMemcpyAsync(leaf_cell.data(), c->sym_leafcell.p, sizeof(int) * (size_t)nl,
                               cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    sym_colours(c->boxes_h, c->n_cells, leaf_cell, cell_leaf, cells, c->sym_off);
    TRY(ensure(c, c->sym_cell_leaf, sizeof(int) * cell_leaf.size()));
    TRY(ensure(c, c->sym_cells, sizeof(int) * std::max(cells.size(), (size_t)1)));
    CUDA_TRY(cudaMemcpyAsync(c->sym_cell_leaf.p, cell_leaf.data(), sizeof(int) * cell_leaf.size(),
                             cudaMemcpyHostToDevice, c->stream));
    if (!cells.empty())
      CUDA_TRY(cudaMemcpyAsync(c->sym_cells.p, cells.data(), sizeof(int) * cells.size(),
                               cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
    c->sym_stamp = c->grid_stamp;
  }
  CUDA_TRY(cudaMemsetAsync(c->st.acc, 0, sizeof(float4) * (size_t)c->n, c->stream));
  CUDA_TRY(cudaMemsetAsync(c->nforce, 0, sizeof(int) * (size_t)c->n, c->stream));
  CUDA_TRY(cudaMemsetAsync(&c->ctr->force_inter, 0, sizeof(unsigned long long), c->stream));
  CUDA_TRY(cudaMemsetAsync(&c->ctr->force_cand, 0, sizeof(unsigned long long), c->stream));
  SymArgs sa{};
  sa.cell_leaf = as<int>(c->sym_cell_leaf);
  sa.leaves = as<Leaf>(c->leaves);
  sa.list_off = as<int>(c->force_off);
  sa.tasks = as<Task>(c->force_tasks);
  sa.pm = c->pm;
  sa.fi = c->fi;
  sa.vu = vu_of(c, vu_for_force);
  sa.acc = c->st.acc;
  sa.nforce = c->nforce;
  sa.ctr = c->ctr;
  tic(c, kForce);
  for (size_t k = 0; k + 1 < c->sym_off.size(); ++k) {
    sa.cells = as<int>(c->sym_cells) + c->sym_off[k];
    sa.n_cells = c->sym_off[k + 1] - c->sym_off[k];
    launch_force_sym(sa, c->stream);
  }
  toc(c, kForce);
  ++c->force_launches;
  c->force_pending = true;
  TRY(sync_check(c));
  c->force_valid = true;
  return SPH_OK;
}

int force_impl(sph_ctx *c, VuSel vu_for_force) {
  if (!c->density_valid) return fail(c, SPH_ESTATE, "sph_force needs sph_density first");
  if (c->p.mode == SPH_MODE_SYMMETRIC) {
    if (c->force_pending) TRY(read_counters(c));  // bank the previous force counters
    return force_symmetric(c, vu_for_force);
  }
  if (c->force_pending) TRY(read_counters(c));  // bank the previous force counters
  const int *active = nullptr;
  int n_targets = c->n_leaves;
  const unsigned char *skip = nullptr;
  if (c->p.mode == SPH_MODE_BATCHED) {
    bool all = false;
    TRY(force_batched(c, vu_for_force, &all));
    if (all) return SPH_OK;
    // groups that overflowed their stage: the per-leaf form finishes the
    // leaves holding their particles, skipping particles already done
    CUDA_TRY(cudaMemsetAsync(&c->ctr->n_active, 0, sizeof(int), c->stream));
    launch_active_leaves(as<Leaf>(c->leaves), c->n_leaves, c->fdone, as<int>(c->active), c->ctr,
                         c->stream);
    TRY(read_counters(c));
    // that read banked the batched counts; they are banked again, with the
    // remainder's, after the per-leaf pass
    c->total_force_inter -= c->ctr_h->force_inter;
    active = as<int>(c->active);
    n_targets = c->ctr_h->n_active;
    skip = c->fdone;
  }
  GeomArgs ga = geom_args(c);
  launch_leaf_hmax(ga, c->n_nodes, c->stream);
  TRY(build_lists(c, true, active, n_targets, c->force_off, c->force_tasks, c->n_force_tasks));
  if (!skip) {  // a remainder after the batched pass keeps adding to its counters
    CUDA_TRY(cudaMemsetAsync(&c->ctr->force_inter, 0, sizeof(unsigned long long), c->stream));
    CUDA_TRY(cudaMemsetAsync(&c->ctr->force_cand, 0, sizeof(unsigned long long), c->stream));
  }
  ForceArgs fa{};
  fa.n_leaves = c->n_leaves;
  fa.active = active;
  fa.n_targets = n_targets;
  fa.skip = skip;
  fa.leaves = as<Leaf>(c->leaves);
  fa.list_off = as<int>(c->force_off);
  fa.tasks = as<Task>(c->force_tasks);
  fa.pm = c->pm;
  fa.fi = c->fi;
  fa.vu = vu_of(c, vu_for_force);
  fa.acc = c->st.acc;
  fa.nforce = c->nforce;
  fa.ctr = c->ctr;
  fa.kahan = c->p.precision == SPH_PREC_KAHAN;
  fa.nodes = as<Node>(c->nodes);
  fa.skey = c->p.pair_sort ? c->skey : nullptr;
  fa.sidx = c->sidx;
  fa.n = c->n;
  ensure_sorts(c);
  tic(c, kForce);
  launch_force(fa, c->stream);
  toc(c, kForce);
  ++c->force_launches;
  c->force_pending = true;
  TRY(sync_check(c));
  c->force_valid = true;
  return SPH_OK;
}

// After a drift on an unchanged grid: leaf-relative positions, node boxes
// and the per-box out-of-cell distance from the new x (A1 and A2 skipped).
int refresh_grid(sph_ctx *c) {
  tic(c, kGrid);
  CUDA_TRY(cudaMemsetAsync(c->boxout, 0, sizeof(unsigned) * (size_t)c->nb, c->stream));
  GeomArgs ga = geom_args(c);
  ga.maxout = c->boxout;
  launch_refresh_geometry(ga, c->n_nodes, c->stream);
  toc(c, kGrid);
  c->groups_geom_valid = false;
  c->sorts_valid = false;
  c->density_valid = false;
  c->force_valid = false;
  return sync_check(c);
}

// Copies the state a step starts from (positions, h, v and u, accelerations)
// between the store and its second copy: kick-drift saves it into the second
// copy as it reads it, and a step on a reused grid that has to be redone is
// restored from there.
void copy_step_state(sph_ctx *c, const StoreArrays &from, const StoreArrays &to) {
  const size_t n = (size_t)c->n;
  cudaMemcpyAsync(to.x0, from.x0, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(to.x1, from.x1, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(to.x2, from.x2, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(to.h, from.h, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(to.vu, from.vu, n * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(to.acc, from.acc, n * sizeof(float4), cudaMemcpyDeviceToDevice, c->stream);
}

// One kick-drift-kick step (Section 3.1 integrator task around the density,
// ghost and force tasks), on the grid of the last regrid when `reuse`.
// Leaves the status words in ctr_h (read once at the end).
int step_once(sph_ctx *c, double dt, bool reuse) {
  c->regrids_in_step = 0;
  CUDA_TRY(cudaMemsetAsync(&c->ctr->step_status, 0, sizeof(int), c->stream));
  const bool vc = cache_on(c) && c->vc_valid;
  if (vc) CUDA_TRY(cudaMemsetAsync(c->vc_dmax.p, 0, sizeof(unsigned) * c->n_cells, c->stream));
  const DriftCache dc = drift_cache(c);
  tic(c, kInteg);
  launch_kick_drift(c->st, c->n, dt, c->boxes_d, c->nb, c->p.gamma, c->hf,
                    reuse ? &c->st2 : nullptr, nullptr, nullptr, c->ctr, c->stream,
                    vc ? &dc : nullptr);
  toc(c, kInteg);
  c->density_valid = false;
  c->force_valid = false;
  if (reuse) {
    TRY(refresh_grid(c));
  } else {
    c->grid_valid = false;
    TRY(build_grid(c, false, nullptr, nullptr, nullptr, nullptr));
  }
  TRY(density_impl(c, kVuPredicted));
  TRY(force_impl(c, kVuPredicted));
  tic(c, kInteg2);
  launch_kick(c->st, c->n, dt, c->ctr, c->stream);
  toc(c, kInteg2);
  launch_grid_check(c->st.h, c->n, c->boxes_d, c->nb, c->hext, c->boxout, &c->ctr->step_status,
                    c->stream);
  return read_counters(c);
}

// Everything a step on the reused grid issues in the batched form, with
// no host reads: the body of the captured graph. Mirrors step_once(reuse).
int enqueue_steady_step(sph_ctx *c, double dt) {
  CUDA_TRY(cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), c->stream));
  tic(c, kInteg);
  // also clears the density and force finished flags (the batched tiers keep
  // their h brackets in registers, so nothing else of the iteration state
  // needs resetting)
  const bool vc = cache_on(c) && c->vc_valid;
  if (vc) CUDA_TRY(cudaMemsetAsync(c->vc_dmax.p, 0, sizeof(unsigned) * c->n_cells, c->stream));
  const DriftCache dc = drift_cache(c);
  launch_kick_drift(c->st, c->n, dt, c->boxes_d, c->nb, c->p.gamma, c->hf, &c->st2, c->done,
                    c->fdone, c->ctr, c->stream, vc ? &dc : nullptr);
  toc(c, kInteg);
  tic(c, kGrid);
  CUDA_TRY(cudaMemsetAsync(c->boxout, 0, sizeof(unsigned) * (size_t)c->nb, c->stream));
  GeomArgs ga = geom_args(c);
  ga.maxout = c->boxout;
  launch_refresh_geometry(ga, c->n_nodes, c->stream);
  toc(c, kGrid);
  // no starting-guess pass: h is the last step's converged h carried by the
  // drift (the guess only replaces an h more than 2x away from the
  // leaf-density estimate); the h maxima of the last force still bound it to
  // within the stage skin, and a target whose h leaves its staged radius is
  // finished by the third tier
  launch_group_geometry(group_args(c), c->stream);
  c->groups_geom_valid = true;
  TRY(enqueue_density_batched(c, kVuPredicted, true));
  TRY(enqueue_force_batched(c, kVuPredicted, true));
  tic(c, kInteg2);
  launch_kick(c->st, c->n, dt, c->ctr, c->stream);
  toc(c, kInteg2);
  launch_grid_check(c->st.h, c->n, c->boxes_d, c->nb, c->hext, c->boxout, &c->ctr->step_status,
                    c->stream);
  return sync_check(c);
}

// Capture the steady step on a private stream (the caller's may be the legacy
// default stream, which cannot be captured); host-side counters that the
// capture advanced are taken back and replayed per launch.
int capture_steady_step(sph_ctx *c, double dt) {
  TRY(cache_prepare(c));
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (!c->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = c->stream;
  const long long l0 = c->launches, d0 = c->dens_launches, f0 = c->force_launches;
  c->stream = c->cap_stream;
  c->capturing = true;
  c->graph_stage_mask = 0;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? enqueue_steady_step(c, dt) : SPH_OK;
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c->stream, &g) : e;
  c->capturing = false;
  c->stream = user;
  c->graph_kernels = c->launches - l0;
  c->graph_dens = c->dens_launches - d0;
  c->graph_force = c->force_launches - f0;
  c->launches = l0;
  c->dens_launches = d0;
  c->force_launches = f0;
  for (int s = 0; s < kNStages; ++s)  // nothing was recorded yet
    if (c->graph_stage_mask & (1u << s)) c->ev_pending[s] = false;
  if (rc || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc ? rc : fail(c, SPH_ECUDA, "step capture failed: %s", cudaGetErrorString(e2));
  }
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    cudaGetLastError();
    return fail(c, SPH_ECUDA, "step graph instantiation failed: %s", cudaGetErrorString(e));
  }
  c->graph_dt = dt;
  c->graph_stamp = c->grid_stamp;
  return SPH_OK;
}

// One steady step as a graph launch, then one read of the counters.
int graph_step(sph_ctx *c, double dt) {
  if (!c->graph || c->graph_dt != dt || c->graph_stamp != c->grid_stamp)
    TRY(capture_steady_step(c, dt));
  CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
  c->launches += c->graph_kernels;
  c->dens_launches += c->graph_dens;
  c->force_launches += c->graph_force;
  for (int s = 0; s < kNStages; ++s)
    if (c->graph_stage_mask & (1u << s)) c->ev_pending[s] = true;
  c->force_pending = true;  // banked by the read below
  c->regrids_in_step = 0;
  ++c->graph_steps;
  TRY(read_counters(c));
  c->total_dens_inter += c->ctr_h->dens_inter;
  c->last_passes = c->ctr_h->max_iter_used;
  c->density_valid = true;
  c->force_valid = true;
  return SPH_OK;
}

}  // namespace

extern "C" {

void sph_default_params(sph_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->gamma = 5.0 / 3.0;
  p->n_ngb = 48.0;
  p->h_tol = 1e-6;
  p->max_iter = 30;
  p->n_split = 64;
  p->precision = SPH_PREC_FP32;
  p->mode = SPH_MODE_BATCHED;
  p->pair_sort = 1;
  p->reuse_grid = 1;
  p->tile = 0;
  p->cell_factor = 2.0;
  p->reuse_lists = 1;
  p->work_queue = 1;
}

int sph_create(sph_ctx **out, const sph_params *p, void *cuda_stream) {
  if (!out) return SPH_EINVAL;
  *out = nullptr;
  sph_params q;
  sph_default_params(&q);
  if (p) q = *p;
  if (!(q.gamma > 1.0) || !(q.n_ngb > 32.0 / 3.0) || !(q.h_tol > 0.0) || q.max_iter < 1 ||
      q.n_split < 8 || q.n_split > 256 ||
      (q.precision != SPH_PREC_FP32 && q.precision != SPH_PREC_KAHAN) ||
      (q.mode != SPH_MODE_PLAIN && q.mode != SPH_MODE_BATCHED && q.mode != SPH_MODE_SYMMETRIC) ||
      (q.pair_sort != 0 && q.pair_sort != 1) || (q.reuse_grid != 0 && q.reuse_grid != 1) ||
      q.tile < 0 || q.tile > 2 || !(q.cell_factor >= 1.0 && q.cell_factor <= 4.0) ||
      q.reuse_lists < 0 || q.reuse_lists > 2 || q.work_queue < 0 || q.work_queue > 3)
    return SPH_EINVAL;
  sph_ctx *c = new (std::nothrow) sph_ctx();
  if (!c) return SPH_ENOMEM;
  c->p = q;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaMalloc(&c->ctr, sizeof(DevCounters)) != cudaSuccess ||
      cudaMallocHost(&c->ctr_h, sizeof(DevCounters)) != cudaSuccess) {
    cudaGetLastError();
    if (c->ctr) cudaFree(c->ctr);
    delete c;
    return SPH_ECUDA;
  }
  std::memset(c->ctr_h, 0, sizeof(DevCounters));
  if (c->p.profile) {
    for (auto &pair : c->ev)
      for (auto &e : pair)
        if (cudaEventCreate(&e) != cudaSuccess) {
          cudaGetLastError();
          c->p.profile = 0;
        }
  }
  *out = c;
  return SPH_OK;
}

int sph_workspace_size(const sph_ctx *ctx, int64_t n_total, int n_boxes, size_t *bytes) {
  if (!ctx || !bytes || n_total < 1 || n_total > (int64_t)1 << 30 || n_boxes < 1)
    return SPH_EINVAL;
  *bytes = fixed_layout(n_total, n_boxes).total;
  return SPH_OK;
}

int sph_set_workspace(sph_ctx *c, void *dev_ptr, size_t bytes) {
  if (!c || !dev_ptr || ((uintptr_t)dev_ptr & 255)) return fail(c, SPH_EINVAL, "bad workspace");
  c->ws = (char *)dev_ptr;
  c->ws_bytes = bytes;
  c->loaded = false;
  return SPH_OK;
}

int sph_init(sph_ctx *c, int n_boxes, const int64_t *box_offsets, const double *box_len,
             const double *x, const float *v, const float *m, const float *u, const double *h) {
  if (!c) return SPH_EINVAL;
  LaunchScope ls(c);
  c->err.clear();
  if (n_boxes < 1 || !box_offsets || !box_len || !x || !v || !m || !u || !h)
    return fail(c, SPH_EINVAL, "null argument or n_boxes < 1");
  if (box_offsets[0] != 0) return fail(c, SPH_EINVAL, "box_offsets[0] must be 0");
  for (int b = 0; b < n_boxes; ++b) {
    if (box_offsets[b + 1] < box_offsets[b])
      return fail(c, SPH_EINVAL, "box_offsets must be non-decreasing");
    for (int d = 0; d < 3; ++d)
      if (!(box_len[3 * b + d] > 0.0) || !std::isfinite(box_len[3 * b + d]))
        return fail(c, SPH_EINVAL, "box %d has a non-positive edge", b);
  }
  const int64_t n = box_offsets[n_boxes];
  if (n < 1 || n > ((int64_t)1 << 30)) return fail(c, SPH_EINVAL, "N = %lld out of range", (long long)n);
  c->n = (int)n;
  c->nb = n_boxes;
  c->boxes_h.assign(n_boxes, BoxDev{});
  for (int b = 0; b < n_boxes; ++b) {
    BoxDev &B = c->boxes_h[b];
    for (int d = 0; d < 3; ++d) B.L[d] = box_len[3 * b + d];
    B.first = (int)box_offsets[b];
    B.count = (int)(box_offsets[b + 1] - box_offsets[b]);
  }
  c->loaded = false;
  c->grid_reusable = false;
  TRY(alloc_fixed(c, n, n_boxes));
  CUDA_TRY(cudaMemcpyAsync(c->boxes_d, c->boxes_h.data(), sizeof(BoxDev) * n_boxes,
                           cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), c->stream));
  launch_validate(x, v, m, u, h, c->n, &c->ctr->status, c->stream);
  TRY(read_counters(c));
  if (c->ctr_h->status & kErrInvalidInput)
    return fail(c, SPH_EINVAL, "inputs must be finite with m > 0, u >= 0 and h > 0");
  k_iota<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->ident, c->n);
  note_launch();
  launch_wrap_cell_keys_from_caller(x, c->boxes_d, c->nb, c->n, c->wx, c->wx + n,
                                    c->wx + 2 * (size_t)n, c->stream);
  TRY(build_grid(c, true, v, m, u, h));
  c->loaded = true;
  return SPH_OK;
}

int sph_density(sph_ctx *c) {
  if (!c) return SPH_EINVAL;
  LaunchScope ls(c);
  c->err.clear();
  if (!c->loaded) return fail(c, SPH_ESTATE, "sph_density before sph_init");
  return density_impl(c, kVuCurrent);
}

int sph_force(sph_ctx *c) {
  if (!c) return SPH_EINVAL;
  LaunchScope ls(c);
  c->err.clear();
  if (!c->loaded) return fail(c, SPH_ESTATE, "sph_force before sph_init");
  return force_impl(c, kVuCurrent);
}

int sph_step(sph_ctx *c, double dt, int n_steps) {
  if (!c) return SPH_EINVAL;
  LaunchScope ls(c);
  c->err.clear();
  if (!c->loaded || !c->force_valid)
    return fail(c, SPH_ESTATE, "sph_step needs sph_density and sph_force on the current state");
  if (!(dt > 0.0) || !std::isfinite(dt) || n_steps < 0)
    return fail(c, SPH_EINVAL, "dt must be positive and n_steps >= 0");
  for (int s = 0; s < n_steps; ++s) {
    const bool reuse = c->p.reuse_grid && c->grid_reusable && c->grid_valid;
    // a grid's first reused step runs host-driven; capturing pays from the second on
    const bool graph =
        reuse && c->reuse_streak >= 1 && c->p.mode == SPH_MODE_BATCHED && c->groups_valid;
    if (graph)
      TRY(graph_step(c, dt));
    else
      TRY(step_once(c, dt, reuse));
    if (reuse) ++c->reused_steps;
    int st = c->ctr_h->step_status;
    if (graph) {  // the graph has no per-pass form and no regrid: redo such a step
      st |= c->ctr_h->status & kErrHGrid;
      if (c->ctr_h->fallback > 0) st |= kErrHGrid;
    }
    if ((st & kErrHGrid) && reuse && c->regrids_in_step == 0) {
      ++c->redone_steps;
      // a particle moved too far from its top cell for the h it now has:
      // back to the step's starting state and redo the step on a new grid
      copy_step_state(c, c->st2, c->st);
      launch_h_to_float(c->st.h, c->hf, c->n, c->stream);
      TRY(step_once(c, dt, false));
      st = c->ctr_h->step_status;
    }
    TRY(check_status(c, (c->ctr_h->status | st) & ~kErrHGrid));
    c->grid_reusable = !(st & kErrHGrid);
    c->reuse_streak = c->regrids_in_step == 0 && reuse ? c->reuse_streak + 1 : 0;
  }
  return sync_check(c);
}

int sph_get(sph_ctx *c, int field, void *dev_out) {
  if (!c) return SPH_EINVAL;
  LaunchScope ls(c);
  c->err.clear();
  if (!dev_out || field < 0 || field >= SPH_NFIELDS)
    return fail(c, SPH_EINVAL, "unknown field %d or null output", field);
  if (!c->loaded) return fail(c, SPH_ESTATE, "no particles loaded");
  const bool needs_density = field == SPH_RHO || field == SPH_OMEGA || field == SPH_P ||
                             field == SPH_NNGB || field == SPH_NITER;
  const bool needs_force = field == SPH_A || field == SPH_DUDT || field == SPH_NFORCE;
  if (needs_density && !c->density_valid)
    return fail(c, SPH_ESTATE, "field %d needs sph_density on the current positions", field);
  if (needs_force && !c->force_valid)
    return fail(c, SPH_ESTATE, "field %d needs sph_force on the current state", field);
  if (field == SPH_CELL || field == SPH_LEAF_CELL) {
    if (!c->grid_valid)
      return fail(c, SPH_ESTATE, "field %d needs a grid of the current particles", field);
    launch_get_cells(c->st.orig, c->leaf_of, as<Leaf>(c->leaves), as<Node>(c->nodes),
                     c->boxes_d, c->n, field == SPH_CELL ? (int *)dev_out : nullptr,
                     field == SPH_LEAF_CELL ? (int *)dev_out : nullptr, c->stream);
    return sync_check(c);
  }
  launch_get(field, dev_out, c->st.orig, c->n, c->st, c->rho, c->omega, c->P, c->nngb, c->niter,
             c->nforce, c->stream);
  return sync_check(c);
}

int sph_grid(const sph_ctx *c, int box, int32_t *n_out, double *w_out) {
  if (!c) return SPH_EINVAL;
  if (!c->loaded) return SPH_ESTATE;
  if (box < 0 || box >= c->nb) return SPH_EINVAL;
  const BoxDev &B = c->boxes_h[box];
  for (int d = 0; d < 3; ++d) {
    if (n_out) n_out[d] = B.n[d];
    if (w_out) w_out[d] = B.w[d];
  }
  return SPH_OK;
}

int sph_autotune(sph_ctx *c, int *tile_out, int *n_split_out, double *cell_factor_out,
                 double *ms_out) {
  if (!c) return SPH_EINVAL;
  LaunchScope ls(c);
  c->err.clear();
  if (!c->loaded) return fail(c, SPH_ESTATE, "sph_autotune before sph_init");
  const sph_params keep = c->p;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, SPH_ECUDA, "event creation failed");
  }
  const int tiles = c->p.mode == SPH_MODE_BATCHED ? 3 : 1;
  const int splits[] = {16, 32, 64, 128};
  const double factors[] = {1.5, 2.0, 2.5, 3.0};
  double best = 1e300;
  sph_params best_p = keep;
  int rc = density_impl(c, kVuCurrent);  // converged h to start from
  for (int t = 0; t < tiles && rc == SPH_OK; ++t)
    for (int ns : splits)
      for (double cf : factors) {
        if (rc != SPH_OK) break;
        c->p.tile = t;
        c->p.n_split = ns;
        c->p.cell_factor = cf;
        c->grid_valid = false;
        rc = build_grid(c, false, nullptr, nullptr, nullptr, nullptr);
        double ms_min = 1e300;
        for (int rep = 0; rep < 2 && rc == SPH_OK; ++rep) {
          cudaEventRecord(e0, c->stream);
          rc = density_impl(c, kVuCurrent);
          if (rc == SPH_OK) rc = force_impl(c, kVuCurrent);
          cudaEventRecord(e1, c->stream);
          if (rc == SPH_OK && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms_min = std::min(ms_min, (double)ms);
          }
        }
        if (rc == SPH_OK && ms_min < best) {
          best = ms_min;
          best_p = c->p;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->p = rc == SPH_OK ? best_p : keep;
  c->grid_valid = false;  // rebuild the grid with the chosen parameters
  c->grid_reusable = false;
  if (rc != SPH_OK) return rc;
  TRY(build_grid(c, false, nullptr, nullptr, nullptr, nullptr));
  TRY(density_impl(c, kVuCurrent));
  TRY(force_impl(c, kVuCurrent));
  if (tile_out) *tile_out = c->p.tile;
  if (n_split_out) *n_split_out = c->p.n_split;
  if (cell_factor_out) *cell_factor_out = c->p.cell_factor;
  if (ms_out) *ms_out = best;
  return sync_check(c);
}

int sph_get_pair_order(sph_ctx *c, int axis, int32_t *order_out, int32_t *leaf_out) {
  if (!c) return SPH_EINVAL;
  LaunchScope ls(c);
  c->err.clear();
  if (axis < 0 || axis >= kAxes || !order_out || !leaf_out)
    return fail(c, SPH_EINVAL, "axis %d out of range or null output", axis);
  if (!c->loaded || !c->grid_valid) return fail(c, SPH_ESTATE, "no particles loaded");
  if (!c->p.pair_sort) return fail(c, SPH_ESTATE, "pair sorts are off (pair_sort = 0)");
  ensure_sorts(c);
  launch_get_pair_order(as<Leaf>(c->leaves), c->leaf_of, c->sidx, c->st.orig, c->n, axis,
                        order_out, leaf_out, c->stream);
  return sync_check(c);
}

int sph_stats(sph_ctx *c, sph_stats_t *out) {
  if (!c || !out) return SPH_EINVAL;
  LaunchScope ls(c);
  std::memset(out, 0, sizeof *out);
  out->n_particles = c->n;
  out->n_boxes = c->nb;
  if (!c->loaded) return SPH_OK;
  TRY(read_counters(c));
  out->n_top_cells = c->n_cells;
  out->n_leaves = c->n_leaves;
  out->n_pairs_density = c->n_dens_tasks;
  out->n_pairs_force = c->n_force_tasks;
  out->density_interactions = (int64_t)c->ctr_h->dens_inter;
  out->force_interactions = (int64_t)c->ctr_h->force_inter;
  out->density_pair_candidates = (int64_t)c->ctr_h->dens_cand;
  out->force_pair_candidates = (int64_t)c->ctr_h->force_cand;
  out->density_passes = c->last_passes;
  out->rebuilds = c->last_rebuilds;
  out->max_iter_used = c->ctr_h->max_iter_used;
  out->batched_fallbacks = c->ctr_h->fallback;
  out->stage_max_density = c->ctr_h->stage_max[0];
  out->stage_max_force = c->ctr_h->stage_max[1];
  out->total_density_interactions = (int64_t)c->total_dens_inter;
  out->total_force_interactions = (int64_t)c->total_force_inter;
  out->density_launches = c->dens_launches;
  out->force_launches = c->force_launches;
  out->t_grid_ms = c->t_ms[kGrid];
  out->t_lists_ms = c->t_ms[kLists] + c->t_ms[kLists2];
  out->t_density_ms = c->t_ms[kDens];
  out->t_ghost_ms = c->t_ms[kGhost];
  out->t_force_ms = c->t_ms[kForce];
  out->t_integrate_ms = c->t_ms[kInteg] + c->t_ms[kInteg2];
  out->t_sort_ms = c->t_ms[kSort];
  out->direct_list_warps = c->ctr_h->direct[0];
  out->direct_stage_warps = c->ctr_h->direct[1];
  for (int k = 0; k < 4; ++k) out->fallback_causes[k] = c->ctr_h->why[k];
  for (int k = 0; k < 2; ++k) {
    out->tier2_groups[k] = c->ctr_h->queued[k];
    out->tier3_entries[k] = c->ctr_h->queued2[k];
  }
  out->sort_launches = c->sort_launches;
  out->reused_steps = c->reused_steps;
  out->graph_steps = c->graph_steps;
  out->redone_steps = c->redone_steps;
  out->n_groups = c->n_groups;
  out->cache_density_groups = c->ctr_h->cache_used[0];
  out->cache_force_groups = c->ctr_h->cache_used[1];
  out->cache_built_groups = c->ctr_h->cache_built;
  out->cache_relist_warps = c->ctr_h->cache_relist;
  out->kernel_launches = c->launches;  // before the extremes kernel below
  std::vector<double> hb;
  double hmin = 0, hmax = 0;
  TRY(h_extremes(c, c->st.h, hb, hmin, hmax));
  out->h_min = hmin;
  out->h_max = hmax;
  return SPH_OK;
}

const char *sph_last_error(const sph_ctx *c) { return c ? c->err.c_str() : "null context"; }

void sph_destroy(sph_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  DevBuf *bufs[] = {&c->cell_count, &c->cell_start, &c->cursor,   &c->nodes,      &c->frontier,
                    &c->frontier2,  &c->leaves,     &c->scan_tmp, &c->active,     &c->dens_off,
                    &c->dens_tasks, &c->force_off,  &c->force_tasks, &c->gcount,
                    &c->groups,     &c->gd_off,     &c->gd_tasks, &c->gf_off,     &c->gf_tasks,
                    &c->gqueue,     &c->lflag,      &c->gwmode,   &c->gcost_d,    &c->gcost_f,
                    &c->gorder,     &c->gbins,      &c->gcbin,      &c->gstage,
                    &c->gbflag,     &c->gbexcl,     &c->gborder,    &c->gbsplit,    &c->sym_cells,
                    &c->sym_cell_leaf, &c->sym_leafcell, &c->vc_meta,
                    &c->vc_sj,
                    &c->vc_slot,    &c->vc_list,    &c->vc_rl,    &c->vc_dpath,   &c->vc_dmax,
                    &c->vc_gmode,   &c->vc_fuse,    &c->vc_ctl};
  for (DevBuf *b : bufs) release(*b);
  for (void *p : c->owned) cudaFree(p);
  if (c->ctr) cudaFree(c->ctr);
  if (c->ctr_h) cudaFreeHost(c->ctr_h);
  for (auto &pair : c->ev)
    for (auto &e : pair)
      if (e) cudaEventDestroy(e);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"
