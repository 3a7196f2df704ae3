// grid.cu -- cell grid, recursive cell splitting and leaf-pair task lists.
//
// Section 3.1 of the paper: the domain is cut into a grid of cells whose
// edge is at least the largest particle radius h, so two particles close
// enough to interact share a cell or lie in neighbouring cells; cells with
// too many particles are split recursively, and the tasks between split
// cells are replaced by tasks between their neighbouring sub-cells.
//
// GPU form:
//   A1  cell key per particle (integer, from FP64 positions), histogram,
//       exclusive scan, scatter (a counting sort by top cell).
//   A2  split every top cell holding more than n_split particles into 8
//       octants, level by level (a counting sort on octant keys per split
//       node), down to leaves of at most n_split particles.
//   Task lists: for every target leaf, the source leaves whose bounding box
//       lies within the interaction radius, found by walking the octrees of
//       the 27 neighbouring top cells (the refined self/pair task set), one
//       warp per target leaf, breadth first.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// exclusive scan of one value per thread across the block; *total = block sum
__device__ int block_excl_scan(int v, int *total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = warp_incl_scan(v, lane);
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = lane < nw ? ws[lane] : 0;
    t = warp_incl_scan(t, lane);
    ws[lane] = t;
  }
  __syncthreads();
  int pre = warp ? ws[warp - 1] : 0;
  *total = ws[nw - 1];
  __syncthreads();
  return pre + x - v;
}

__global__ void k_scan_reduce(const int *in, int n, int *bsum) {
  const int base = blockIdx.x * kScanTile;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = base + threadIdx.x * kScanItems + k;
    if (idx < n) s += in[idx];
  }
  int tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int *in, int *out, int n, const int *boff) {
  const int base = blockIdx.x * kScanTile;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = base + threadIdx.x * kScanItems + k;
    v[k] = idx < n ? in[idx] : 0;
    s += v[k];
  }
  int tot;
  int run = block_excl_scan(s, &tot) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = base + threadIdx.x * kScanItems + k;
    if (idx < n) out[idx] = run;
    run += v[k];
  }
}

size_t scan_tmp_bytes(int n) {
  size_t b = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    b += 2 * sizeof(int) * (size_t)(n + 1);
  }
  return b + 256;
}

// out[k] = sum_{j<k} in[k]; in and out may alias only if identical.
void exclusive_scan_int(const int *in, int *out, int n, void *tmp, size_t tmp_bytes,
                        cudaStream_t s) {
  if (n <= 0) return;
  if (n <= kScanTile) {
    k_scan_apply<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr); note_launch();
    return;
  }
  const int nb = (n + kScanTile - 1) / kScanTile;
  int *bsum = reinterpret_cast<int *>(tmp);
  int *boff = bsum + nb + 1;
  void *rest = boff + nb + 1;
  k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, bsum); note_launch();
  exclusive_scan_int(bsum, boff, nb, rest, tmp_bytes, s);
  k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, out, n, boff); note_launch();
}

// ------------------------------------------------------------- helpers

__device__ __forceinline__ int box_of_particle(const BoxDev *b, int nb, int k) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b[mid].first <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int box_of_cell(const BoxDev *b, int nb, int c) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b[mid].cell_base <= c)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ unsigned part1by2(unsigned x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

__device__ __forceinline__ void cell_coords(const BoxDev &B, int local, int c[3]) {
  c[2] = local % B.n[2];
  c[1] = (local / B.n[2]) % B.n[1];
  c[0] = local / (B.n[1] * B.n[2]);
}

// ------------------------------------------------------------------ A1

// Lanes of the warp whose `key` equals this lane's, and this lane's rank
// among them (inactive lanes pass a key no active lane uses).
__device__ __forceinline__ unsigned warp_peers(int key, int &rank) {
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  rank = __popc(peers & ((1u << (threadIdx.x & 31)) - 1u));
  return peers;
}

// Integer top-cell key and 30-bit Morton code (10 bits per axis inside the
// top cell) of every particle, plus the cell histogram. The cell index is
// c = floor(x / w) exactly, for the FP64 values x and w: a product with 1/w,
// corrected by one step either way where the sign of c w - x, taken from an
// fma (the exact product and difference, rounded once, so its sign is the
// exact sign), says the product was off. rel = x - c w (one fma, rounded
// once) lies in [0, w), and each Morton coordinate is floor(rel (1024 / w))
// with 1024 / w formed as (1 / w) x 1024 (exact power-of-two scaling).
// Histogram increments are aggregated over the lanes of a warp that share a
// cell.
__global__ void k_cell_keys(GridArgs g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = k < g.n;
  int cell = -1;
  if (valid) {
    const BoxDev &B = g.boxes[box_of_particle(g.boxes, g.n_boxes, k)];
    const double x[3] = {g.x0[k], g.x1[k], g.x2[k]};
    int ic[3];
    unsigned q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int c = (int)floor(__dmul_rn(x[d], B.iw[d]));
      if (fma((double)c, B.w[d], -x[d]) > 0.0)
        --c;  // c w > x
      else if (fma((double)(c + 1), B.w[d], -x[d]) <= 0.0)
        ++c;  // (c + 1) w <= x
      c = c < 0 ? 0 : (c >= B.n[d] ? B.n[d] - 1 : c);
      ic[d] = c;
      const double rel = fma(-(double)c, B.w[d], x[d]);
      int qi = (int)floor(__dmul_rn(rel, __dmul_rn(B.iw[d], (double)(1 << kMaxDepth))));
      qi = qi < 0 ? 0 : (qi > (1 << kMaxDepth) - 1 ? (1 << kMaxDepth) - 1 : qi);
      q[d] = (unsigned)qi;
    }
    cell = B.cell_base + (ic[0] * B.n[1] + ic[1]) * B.n[2] + ic[2];
    g.cell_of[k] = cell;
    g.morton[k] = (part1by2(q[0]) << 2) | (part1by2(q[1]) << 1) | part1by2(q[2]);
  }
  int rank;
  const unsigned peers = warp_peers(cell, rank);
  if (valid && rank == 0) atomicAdd(&g.cell_count[cell], __popc(peers));
}

void launch_cell_keys(const GridArgs &g, cudaStream_t s) {
  k_cell_keys<<<(g.n + 255) / 256, 256, 0, s>>>(g); note_launch();
}

// Scatter into cell ranges. The slot order inside a cell is settled later
// (octant split, then a sort of each leaf by original index), so the atomic
// cursor does not make the final order depend on timing.
__global__ void k_cell_scatter(GridArgs g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = k < g.n;
  const int c = valid ? g.cell_of[k] : -1;
  int rank;
  const unsigned peers = warp_peers(c, rank);
  int base = 0;
  if (valid && rank == 0) base = atomicAdd(&g.cursor[c], __popc(peers));
  base = __shfl_sync(0xffffffffu, base, __ffs(peers) - 1);
  if (!valid) return;
  const int pos = g.cell_start[c] + base + rank;
  g.order[pos] = k;
  g.morton_tmp[pos] = g.morton[k];
}

void launch_cell_scatter(const GridArgs &g, cudaStream_t s) {
  k_cell_scatter<<<(g.n + 255) / 256, 256, 0, s>>>(g); note_launch();
}

// ------------------------------------------------------------------ A2

__device__ __forceinline__ void reset_bounds(Node &nd) {
  for (int d = 0; d < 3; ++d) {
    nd.lo[d] = __int_as_float(0x7f800000);   // +inf
    nd.hi[d] = __int_as_float(0xff800000);   // -inf
  }
  nd.hmax = 0.f;
}

__global__ void k_init_top_nodes(Node *nodes, GridArgs g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n_cells) return;
  Node nd;
  nd.start = g.cell_start[c];
  nd.count = g.cell_count[c];
  nd.child = -1;
  nd.parent = -1;
  nd.cell = c;
  nd.leaf = -1;
  nd.level = 0;
  nd.ix = nd.iy = nd.iz = 0;
  nd.box = box_of_cell(g.boxes, g.n_boxes, c);
  reset_bounds(nd);
  nodes[c] = nd;
}

void launch_init_top_nodes(Node *nodes, const GridArgs &g, cudaStream_t s) {
  k_init_top_nodes<<<(g.n_cells + 255) / 256, 256, 0, s>>>(nodes, g); note_launch();
}

__global__ void k_frontier_top(const Node *nodes, int n_cells, int n_split, int *frontier,
                               DevCounters *ctr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  if (nodes[c].count > n_split) frontier[atomicAdd(&ctr->n_frontier, 1)] = c;
}

void launch_frontier_top(const Node *nodes, int n_cells, int n_split, int *frontier,
                         DevCounters *ctr, cudaStream_t s) {
  k_frontier_top<<<(n_cells + 255) / 256, 256, 0, s>>>(nodes, n_cells, n_split, frontier, ctr); note_launch();
}

// One block per node to split: count its particles per octant, lay the 8
// children out in octant order, move the particles into the children.
__global__ void k_split(Node *nodes, const int *frontier, int n_frontier, int child_base,
                        int level, int n_split, int *next_frontier, DevCounters *ctr,
                        GridArgs g) {
  const int f = blockIdx.x;
  if (f >= n_frontier) return;
  const int id = frontier[f];
  const Node F = nodes[id];
  __shared__ int cnt[8], beg[8], cur[8];
  if (threadIdx.x < 8) {
    cnt[threadIdx.x] = 0;
    cur[threadIdx.x] = 0;
  }
  __syncthreads();
  const int shift = 3 * (kMaxDepth - 1 - level);
  const int s0 = F.start, s1 = F.start + F.count;
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x)
    atomicAdd(&cnt[(g.morton_tmp[s] >> shift) & 7u], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = s0;
    for (int o = 0; o < 8; ++o) {
      beg[o] = run;
      run += cnt[o];
    }
    nodes[id].child = child_base + 8 * f;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int o = threadIdx.x;
    Node c;
    c.start = beg[o];
    c.count = cnt[o];
    c.child = -1;
    c.parent = id;
    c.cell = F.cell;
    c.leaf = -1;
    c.level = level + 1;
    c.ix = 2 * F.ix + ((o >> 2) & 1);
    c.iy = 2 * F.iy + ((o >> 1) & 1);
    c.iz = 2 * F.iz + (o & 1);
    c.box = F.box;
    reset_bounds(c);
    nodes[child_base + 8 * f + o] = c;
    if (c.count > n_split && c.level < kMaxDepth)
      next_frontier[atomicAdd(&ctr->n_frontier, 1)] = child_base + 8 * f + o;
  }
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const unsigned mk = g.morton_tmp[s];
    const int o = (mk >> shift) & 7u;
    const int pos = beg[o] + atomicAdd(&cur[o], 1);
    g.order_tmp[pos] = g.order[s];
    g.morton_scr[pos] = mk;
  }
  __syncthreads();
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    g.order[s] = g.order_tmp[s];
    g.morton_tmp[s] = g.morton_scr[s];
  }
}

void launch_split_level(Node *nodes, const int *frontier, int n_frontier, int child_base,
                        int level, int n_split, int *next_frontier, DevCounters *ctr,
                        const GridArgs &g, cudaStream_t s) {
  if (n_frontier <= 0) return;
  k_split<<<n_frontier, 256, 0, s>>>(nodes, frontier, n_frontier, child_base, level, n_split,
                                     next_frontier, ctr, g); note_launch();
}

__global__ void k_mark_leaves(const Node *nodes, int n_nodes, int *flag) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_nodes) return;
  const Node &nd = nodes[id];
  if (nd.child < 0 && nd.count > 0) flag[nd.start] = 1;
}

void launch_mark_leaves(const Node *nodes, int n_nodes, int *flag, cudaStream_t s) {
  k_mark_leaves<<<(n_nodes + 255) / 256, 256, 0, s>>>(nodes, n_nodes, flag); note_launch();
}

__global__ void k_fill_leaves(Node *nodes, int n_nodes, const int *excl, Leaf *leaves,
                              const BoxDev *boxes, int n_boxes) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_nodes) return;
  Node &nd = nodes[id];
  if (!(nd.child < 0 && nd.count > 0)) return;
  const int li = excl[nd.start];
  nd.leaf = li;
  const BoxDev &B = boxes[nd.box];
  const double scale = 1.0 / (double)(1 << nd.level);
  Leaf L;
  L.start = nd.start;
  L.count = nd.count;
  L.node = id;
  L.box = nd.box;
  L.o[0] = (double)nd.ix * (B.w[0] * scale);
  L.o[1] = (double)nd.iy * (B.w[1] * scale);
  L.o[2] = (double)nd.iz * (B.w[2] * scale);
  for (int d = 0; d < 3; ++d) L.of[d] = (float)L.o[d];
  L.pad = 0;
  leaves[li] = L;
}

void launch_fill_leaves(Node *nodes, int n_nodes, const int *leaf_idx_excl, Leaf *leaves,
                        const BoxDev *boxes, int n_boxes, cudaStream_t s) {
  k_fill_leaves<<<(n_nodes + 255) / 256, 256, 0, s>>>(nodes, n_nodes, leaf_idx_excl, leaves,
                                                      boxes, n_boxes); note_launch();
}

// Order each leaf's particles by (Morton code inside the top cell, original
// index) (insertion sort; leaves are small): the slot order never depends on
// atomic timing, and consecutive slots stay spatially close, so the batched
// kernels' groups of 32 consecutive particles are compact.
__global__ void k_sort_leaves(const Leaf *leaves, int n_leaves, int *order, const int *orig,
                              const unsigned *morton) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= n_leaves) return;
  const Leaf L = leaves[li];
  if (L.count > 512) return;
  int *o = order + L.start;
  auto key_of = [&](int v) {
    return ((unsigned long long)morton[v] << 32) | (unsigned)orig[v];
  };
  for (int a = 1; a < L.count; ++a) {
    const int v = o[a];
    const unsigned long long key = key_of(v);
    int b = a - 1;
    while (b >= 0 && key_of(o[b]) > key) {
      o[b + 1] = o[b];
      --b;
    }
    o[b + 1] = v;
  }
}

void launch_sort_leaves(const Leaf *leaves, int n_leaves, int *order, const int *orig,
                        const unsigned *morton, cudaStream_t s) {
  k_sort_leaves<<<(n_leaves + 127) / 128, 128, 0, s>>>(leaves, n_leaves, order, orig, morton);
  note_launch();
}

// --------------------------------------------------- leaf geometry / hmax

__device__ __forceinline__ void atomic_max_pos(float *a, float v) {  // a, v >= 0
  atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
}
// Float min / max of any sign by integer atomics: non-negative floats order
// like their bits as signed ints, negative ones inversely as unsigned ints.
__device__ __forceinline__ void atomic_min_f(float *a, float v) {
  if (v >= 0.f)
    atomicMin(reinterpret_cast<int *>(a), __float_as_int(v));
  else
    atomicMax(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float *a, float v) {
  if (v >= 0.f)
    atomicMax(reinterpret_cast<int *>(a), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned *>(a), __float_as_uint(v));
}

// One warp per leaf: leaf-relative FP32 positions (cell-relative precision)
// and the leaf bounding box (top-cell-relative), pushed up the tree. Each
// position is taken at the periodic image nearest its top cell, so after a
// drift without a regrid a particle that crossed the box boundary stays
// beside its cell; *a.maxout (if given) receives the largest distance by
// which a particle lies outside its top cell (float bits).
__global__ void k_leaf_geometry(GeomArgs a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.n_leaves) return;
  const Leaf L = a.leaves[warp];
  const BoxDev &B = a.boxes[L.box];
  const Node &nd = a.nodes[L.node];
  int c[3];
  cell_coords(B, nd.cell - B.cell_base, c);
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  float out = 0.f;
  for (int k = lane; k < L.count; k += 32) {
    const int s = L.start + k;
    const double x[3] = {a.x0[s], a.x1[s], a.x2[s]};
    float p[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // the periodic image nearest the top cell; the FP32 copy decides (a
      // particle lies within about one cell of its own, far from L/2)
      double rel = x[d] - (double)c[d] * B.w[d];
      float rf = (float)rel;
      if (fabsf(rf) > 0.5f * (float)B.L[d]) {
        rel += rf > 0.f ? -B.L[d] : B.L[d];
        rf = (float)rel;
      }
      p[d] = (float)(rel - L.o[d]);
      lo[d] = fminf(lo[d], rf);
      hi[d] = fmaxf(hi[d], rf);
      out = fmaxf(out, fmaxf(-rf, rf - B.wf[d]));
    }
    a.pm[s] = make_float4(p[0], p[1], p[2], a.m[s]);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  }
  for (int o = 16; o; o >>= 1) out = fmaxf(out, __shfl_xor_sync(0xffffffffu, out, o));
  if (lane == 0) {
    // up the tree until a node's box already holds this leaf's: the leaf that
    // gave it those bounds takes them further up itself (a node's lo only
    // falls and hi only rises within the launch, so a stale read can only
    // cost an extra atomic, never skip a needed one)
    int id = L.node;
    while (id >= 0) {
      Node *n = &a.nodes[id];
      bool held = true;
      for (int d = 0; d < 3; ++d) {
        if (lo[d] < n->lo[d]) {
          atomic_min_f(&n->lo[d], lo[d]);
          held = false;
        }
        if (hi[d] > n->hi[d]) {
          atomic_max_f(&n->hi[d], hi[d]);
          held = false;
        }
      }
      if (held) break;
      id = n->parent;
    }
    if (a.maxout && out > 0.f) atomicMax(&a.maxout[L.box], __float_as_uint(out));
  }
}

// Empty bounding boxes for every node (before k_leaf_geometry refills them).
__global__ void k_reset_boxes(Node *nodes, int n_nodes) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_nodes) return;
  for (int d = 0; d < 3; ++d) {
    nodes[id].lo[d] = __int_as_float(0x7f800000);
    nodes[id].hi[d] = __int_as_float(0xff800000);
  }
}

void launch_refresh_geometry(const GeomArgs &a, int n_nodes, cudaStream_t s) {
  if (n_nodes > 0) {
    k_reset_boxes<<<(n_nodes + 255) / 256, 256, 0, s>>>(a.nodes, n_nodes);
    note_launch();
  }
  if (a.n_leaves <= 0) return;
  k_leaf_geometry<<<(a.n_leaves * 32 + 255) / 256, 256, 0, s>>>(a);
  note_launch();
}

__global__ void k_reset_hmax(Node *nodes, int n_nodes) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id < n_nodes) nodes[id].hmax = 0.f;
}

__global__ void k_leaf_hmax(GeomArgs a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.n_leaves) return;
  const Leaf L = a.leaves[warp];
  float hm = 0.f;
  for (int k = lane; k < L.count; k += 32) hm = fmaxf(hm, a.hf[L.start + k]);
  for (int o = 16; o; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
  if (lane == 0) {  // up the tree until a node already holds hm (as in k_leaf_geometry)
    int id = L.node;
    while (id >= 0 && hm > a.nodes[id].hmax) {
      atomic_max_pos(&a.nodes[id].hmax, hm);
      id = a.nodes[id].parent;
    }
  }
}

void launch_leaf_geometry(const GeomArgs &a, int n_nodes, cudaStream_t s) {
  if (a.n_leaves <= 0) return;
  k_leaf_geometry<<<(a.n_leaves * 32 + 255) / 256, 256, 0, s>>>(a); note_launch();
}

void launch_leaf_hmax(const GeomArgs &a, int n_nodes, cudaStream_t s) {
  k_reset_hmax<<<(n_nodes + 255) / 256, 256, 0, s>>>(a.nodes, n_nodes); note_launch();
  if (a.n_leaves <= 0) return;
  k_leaf_hmax<<<(a.n_leaves * 32 + 255) / 256, 256, 0, s>>>(a); note_launch();
}

// Is the grid still valid for the h just computed? A pair in range is
// found among the 27 top cells around the target's cell as long as
// h_max (1 + 1e-6) + 2 out <= w for every box, with `out` the largest
// distance by which a particle lies outside its top cell (k_leaf_geometry);
// otherwise kErrHGrid asks for a regrid. hext[b] holds box b's largest h
// (k_h_extremes bit patterns).
__global__ void k_grid_check(const BoxDev *boxes, int nb, const unsigned long long *hext,
                             const unsigned *boxout, int *status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const BoxDev &B = boxes[b];
  const double hmax = __longlong_as_double((long long)hext[b]);
  const double out = (double)__uint_as_float(boxout[b]);
  const double wmin = fmin(B.w[0], fmin(B.w[1], B.w[2]));
  if (B.count > 0 && hmax * (1.0 + 1e-6) + 2.0 * out > wmin) atomicOr(status, kErrHGrid);
}

// hext = {0 for every box, ~0 (minimum), 0 (maximum)} on the device.
__global__ void k_hext_init(unsigned long long *hext, int nb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nb + 2) hext[k] = k == nb ? ~0ull : 0ull;
}

void launch_grid_check(const double *h, int n, const BoxDev *boxes, int nb,
                       unsigned long long *hext, const unsigned *boxout, int *status,
                       cudaStream_t s) {
  k_hext_init<<<(nb + 2 + 255) / 256, 256, 0, s>>>(hext, nb);
  note_launch();
  launch_h_extremes(h, n, boxes, nb, hext, hext + nb, s);
  k_grid_check<<<(nb + 255) / 256, 256, 0, s>>>(boxes, nb, hext, boxout, status);
  note_launch();
}

// Starting guess for the h iteration from the number density of each octree
// leaf cell, n = count / cell volume: h_est = (3 n_ngb / (4 pi n))^(1/3),
// capped below the top-cell width and L/3. A particle keeps its own h unless
// that is more than 2x away from h_est (the root does not depend on where the
// iteration starts; a near guess, e.g. the previous step's h, is kept).
__global__ void k_h_guess(GeomArgs a, double n_ngb, double *h, float *hf) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= a.n_leaves) return;
  const Leaf L = a.leaves[li];
  const Node &nd = a.nodes[L.node];
  const BoxDev &B = a.boxes[L.box];
  const double scale = 1.0 / (double)(1 << nd.level);
  const double vol = B.w[0] * scale * B.w[1] * scale * B.w[2] * scale;
  const double n = (double)L.count / vol;
  double est = cbrt(3.0 * n_ngb / (4.0 * 3.14159265358979323846 * n));
  const double wmin = fmin(B.w[0], fmin(B.w[1], B.w[2]));
  const double lmin = fmin(B.L[0], fmin(B.L[1], B.L[2]));
  est = fmin(est, fmin(wmin, lmin / 3.0) / (1.0 + 1e-5));
  for (int k = 0; k < L.count; ++k) {
    const int s = L.start + k;
    const double hs = h[s];
    if (hs > 2.0 * est || hs < 0.5 * est) {
      h[s] = est;
      hf[s] = (float)est;
    }
  }
}

void launch_h_guess(const GeomArgs &a, double n_ngb, double *h, float *hf, cudaStream_t s) {
  if (a.n_leaves <= 0) return;
  k_h_guess<<<(a.n_leaves + 127) / 128, 128, 0, s>>>(a, n_ngb, h, hf);
  note_launch();
}

// ------------------------------------------------------------ task lists

constexpr int kWalkStack = 96;

// One thread per target leaf. Walks the octrees of the 27 neighbouring top
// cells (periodic), keeping every source leaf whose bounding box is closer
// than the interaction radius: cap_T = cap_factor * hmax_T for the density
// gather, max(hmax_T, hmax_S) for the force. Count pass when a.tasks is null,
// fill pass otherwise (same walk, same order).
__global__ void k_lists(ListArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_targets) return;
  if (!a.flag[t]) return;  // the warp walk handled this target
  const int T = a.active ? a.active[t] : t;
  const Leaf LT = a.leaves[T];
  const Node NT = a.nodes[LT.node];
  const BoxDev &B = a.boxes[LT.box];
  int c[3];
  cell_coords(B, NT.cell - B.cell_base, c);
  const float capT = a.force ? NT.hmax : NT.hmax * a.cap_factor;
  const float eps = B.eps;
  const bool fill = a.tasks != nullptr;
  int cnt = 0;
  const int base = fill ? a.offset[t] : 0;
  int stack[kWalkStack];
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        const int nc[3] = {(c[0] + dx + B.n[0]) % B.n[0], (c[1] + dy + B.n[1]) % B.n[1],
                           (c[2] + dz + B.n[2]) % B.n[2]};
        const int cellS = B.cell_base + (nc[0] * B.n[1] + nc[1]) * B.n[2] + nc[2];
        const double shd[3] = {dx * B.w[0], dy * B.w[1], dz * B.w[2]};
        const float sh[3] = {(float)shd[0], (float)shd[1], (float)shd[2]};
        int top = 0;
        stack[top++] = cellS;
        while (top > 0) {
          const int id = stack[--top];
          const Node &S = a.nodes[id];
          if (S.count == 0) continue;
          float d2 = 0.f;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float slo = S.lo[d] + sh[d], shi = S.hi[d] + sh[d];
            const float g = fmaxf(0.f, fmaxf(slo - NT.hi[d], NT.lo[d] - shi));
            d2 = fmaf(g, g, d2);
          }
          const float crit = (a.force ? fmaxf(capT, S.hmax) : capT) + eps;
          if (d2 >= crit * crit) continue;
          if (S.child < 0) {
            if (fill) {
              const Leaf &LS = a.leaves[S.leaf];
              Task tk;
              tk.sx = (float)(LS.o[0] + shd[0] - LT.o[0]);
              tk.sy = (float)(LS.o[1] + shd[1] - LT.o[1]);
              tk.sz = (float)(LS.o[2] + shd[2] - LT.o[2]);
              tk.src = S.leaf;
              a.tasks[base + cnt] = tk;
            }
            ++cnt;
          } else if (top + 8 <= kWalkStack) {
            for (int o = 7; o >= 0; --o) stack[top++] = S.child + o;
          } else {
            atomicOr(a.status, kErrListOverflow);  // cannot happen for depth <= 10
          }
        }
      }
  if (!fill) a.count[t] = cnt;
}

constexpr int kLWarps = 4;
constexpr int kLFront = 512;

// One warp per target leaf: the walk of k_lists (the 27 neighbouring top-cell
// octrees, every leaf whose box lies within reach of the target leaf's box),
// breadth first, the lanes testing 32 frontier nodes at a time; passing
// leaves are appended by ballot in walk order. A frontier beyond kLFront
// marks the target (flag) for k_lists instead.
__global__ void __launch_bounds__(kLWarps * 32) k_lists_warp(ListArgs a) {
  __shared__ int2 front_all[kLWarps][2][kLFront];  // (node, neighbour code 0..26)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned ltmask = (1u << lane) - 1u;
  const int t = blockIdx.x * kLWarps + warp;
  if (t >= a.n_targets) return;  // warp-uniform
  const bool fill = a.tasks != nullptr;
  if (fill && a.flag[t]) return;
  int2 *cur = front_all[warp][0], *nxt = front_all[warp][1];
  const int T = a.active ? a.active[t] : t;
  const Leaf LT = a.leaves[T];
  const Node NT = a.nodes[LT.node];
  const BoxDev &B = a.boxes[LT.box];
  int c[3];
  cell_coords(B, NT.cell - B.cell_base, c);
  const float capT = a.force ? NT.hmax : NT.hmax * a.cap_factor;
  const int base = fill ? a.offset[t] : 0;
  int n = 0;
  {
    const bool in = lane < 27;
    int2 e = make_int2(0, lane);
    if (in) {
      const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
      const int nc[3] = {(c[0] + dx + B.n[0]) % B.n[0], (c[1] + dy + B.n[1]) % B.n[1],
                         (c[2] + dz + B.n[2]) % B.n[2]};
      e.x = B.cell_base + (nc[0] * B.n[1] + nc[1]) * B.n[2] + nc[2];
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (in) cur[__popc(m & ltmask)] = e;
    n = __popc(m);
  }
  __syncwarp();
  int ntask = 0;
  bool overflow = false;
  while (n > 0) {
    int nn = 0;
    for (int b0 = 0; b0 < n; b0 += 32) {
      const int idx = b0 + lane;
      bool leaf_in = false, inner_in = false;
      int code = 0, child = 0, leaf = 0;
      if (idx < n) {
        const int2 e = cur[idx];
        code = e.y;
        const Node &S = a.nodes[e.x];
        if (S.count > 0) {
          const int dx = code / 9 - 1, dy = (code / 3) % 3 - 1, dz = code % 3 - 1;
          const float sh[3] = {dx * B.wf[0], dy * B.wf[1], dz * B.wf[2]};
          float d2 = 0.f;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float g = fmaxf(0.f, fmaxf((S.lo[d] + sh[d]) - NT.hi[d], NT.lo[d] - (S.hi[d] + sh[d])));
            d2 = fmaf(g, g, d2);
          }
          const float crit = (a.force ? fmaxf(capT, S.hmax) : capT) + B.eps;
          if (d2 < crit * crit) {
            child = S.child;
            leaf = S.leaf;
            leaf_in = child < 0;
            inner_in = child >= 0;
          }
        }
      }
      const unsigned ml = __ballot_sync(0xffffffffu, leaf_in);
      if (leaf_in && fill) {
        const int dx = code / 9 - 1, dy = (code / 3) % 3 - 1, dz = code % 3 - 1;
        const Leaf &LS = a.leaves[leaf];
        Task tk;
        tk.sx = (float)(LS.o[0] + dx * B.w[0] - LT.o[0]);
        tk.sy = (float)(LS.o[1] + dy * B.w[1] - LT.o[1]);
        tk.sz = (float)(LS.o[2] + dz * B.w[2] - LT.o[2]);
        tk.src = leaf;
        a.tasks[base + ntask + __popc(ml & ltmask)] = tk;
      }
      ntask += __popc(ml);
      const unsigned mi = __ballot_sync(0xffffffffu, inner_in);
      if (inner_in) {
        const int pos = nn + 8 * __popc(mi & ltmask);
        for (int o = 0; o < 8; ++o)
          if (pos + o < kLFront) nxt[pos + o] = make_int2(child + o, code);
      }
      nn += 8 * __popc(mi);
    }
    __syncwarp();
    if (nn > kLFront) {
      overflow = true;
      break;
    }
    int2 *tmp = cur;
    cur = nxt;
    nxt = tmp;
    n = nn;
  }
  if (lane == 0 && !fill) {
    a.flag[t] = overflow ? 1 : 0;
    if (!overflow) a.count[t] = ntask;
  }
}

void launch_build_lists(const ListArgs &a, cudaStream_t s) {
  if (a.n_targets <= 0) return;
  k_lists_warp<<<(a.n_targets + kLWarps - 1) / kLWarps, kLWarps * 32, 0, s>>>(a);
  note_launch();
  k_lists<<<(a.n_targets + 127) / 128, 128, 0, s>>>(a);  // flagged targets only
  note_launch();
}

// ---------------------------------------------------------------- getters

// Per particle (caller order): the integer coordinates of its top cell in its
// box and the level of its octree leaf (out4[4 k ...]), and the leaf cell's
// integer coordinates at that level inside the top cell (out3[3 k ...]).
__global__ void k_get_cells(const int *orig, const int *leaf_of, const Leaf *leaves,
                            const Node *nodes, const BoxDev *boxes, int n, int *out4,
                            int *out3) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const Node nd = nodes[leaves[leaf_of[s]].node];
  const BoxDev &B = boxes[nd.box];
  int c[3];
  cell_coords(B, nd.cell - B.cell_base, c);
  const size_t k = (size_t)orig[s];
  if (out4) {
    out4[4 * k] = c[0];
    out4[4 * k + 1] = c[1];
    out4[4 * k + 2] = c[2];
    out4[4 * k + 3] = nd.level;
  }
  if (out3) {
    out3[3 * k] = nd.ix;
    out3[3 * k + 1] = nd.iy;
    out3[3 * k + 2] = nd.iz;
  }
}

void launch_get_cells(const int *orig, const int *leaf_of, const Leaf *leaves, const Node *nodes,
                      const BoxDev *boxes, int n, int *out4, int *out3, cudaStream_t s) {
  if (n <= 0) return;
  k_get_cells<<<(n + 255) / 256, 256, 0, s>>>(orig, leaf_of, leaves, nodes, boxes, n, out4, out3);
  note_launch();
}

}  // namespace sph
