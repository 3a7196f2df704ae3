// batched.cu -- the batched interaction form: one block of 4 warps per target
// group of up to 32 consecutive particles of a top cell, candidates staged
// once in shared memory, per-lane compacted neighbour lists, and the
// smoothing-length iteration run inside the kernel (Section 2 density and
// force, with the ghost task of Section 3.1 fused into the density kernel).
//
// Per group:
//   1. walk the octrees of the 27 neighbouring top cells for the source leaves
//      whose box lies within the group's radius (the refined pair tasks);
//   2. stage, into shared memory, every source particle within that radius of
//      the group's bounding box, shifted into the group's frame;
//   3. each warp keeps the staged particles within reach of its sub-cluster of
//      8 targets, and each lane keeps its share of its target's neighbours in
//      a list of 16-bit stage indices, so the passes over h, and the force,
//      touch only those;
//   4. density: sums, Newton step on ln N(ln h) (h in FP32, acceptance test in
//      FP64), repeated until every lane converged (candidates and lists rebuilt
//      from the stage when an h outgrows them); force: one pass over the lists.
// Groups whose stage overflows are staged again by each target's own radius
// (second tier, larger stage); targets that overflow that, or whose h outgrows
// the staged radius, are finished one warp per target by a direct walk of the
// octrees (third tier). Only a target the third tier cannot finish is left to
// the per-pass form, so results never depend on the capacities.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kGroup = 32;

__device__ __forceinline__ void cell_xyz(const BoxDev &B, int local, int c[3]) {
  c[2] = local % B.n[2];
  c[1] = (local / B.n[2]) % B.n[1];
  c[0] = local / (B.n[1] * B.n[2]);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_max_int(int v) {
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void add_comp(float &s, float &c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

}  // namespace

// ------------------------------------------------------------- groups

// Groups owned by node `id`: a top cell that is itself a leaf is cut into
// equal chunks of <= 32; an internal node packs runs of consecutive leaf
// children (siblings, hence spatially adjacent and contiguous in memory) into
// groups of <= 32 and cuts any larger leaf child into equal chunks. Other
// leaves belong to their parent's packing. `emit(start, count)` is called per
// group; returns the number of groups.
template <class Emit>
__device__ int pack_node(const Node *nodes, int id, Emit emit) {
  const Node &nd = nodes[id];
  int ng = 0;
  auto chunk = [&](int start, int count) {
    const int parts = (count + kGroup - 1) / kGroup;
    const int base = count / parts, rem = count % parts;
    for (int p = 0; p < parts; ++p) {
      const int sz = base + (p < rem ? 1 : 0);
      emit(start, sz);
      start += sz;
      ++ng;
    }
  };
  if (nd.child < 0) {
    if (nd.parent < 0 && nd.count > 0) chunk(nd.start, nd.count);
    return ng;
  }
  int run_start = 0, run_count = 0;
  for (int o = 0; o < 8; ++o) {
    const Node &ch = nodes[nd.child + o];
    if (ch.count == 0) continue;
    const bool big = ch.child >= 0 || ch.count > kGroup;
    if (big || run_count + ch.count > kGroup) {
      if (run_count > 0) {
        emit(run_start, run_count);
        ++ng;
      }
      run_count = 0;
    }
    if (ch.child >= 0) continue;  // an internal child packs its own leaves
    if (ch.count > kGroup) {
      chunk(ch.start, ch.count);
      continue;
    }
    if (run_count == 0) run_start = ch.start;
    run_count += ch.count;
  }
  if (run_count > 0) {
    emit(run_start, run_count);
    ++ng;
  }
  return ng;
}

__global__ void k_group_count(GroupBuildArgs a) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id < a.n_nodes) a.gcount[id] = pack_node(a.nodes, id, [](int, int) {});
}

void launch_group_count(const GroupBuildArgs &a, cudaStream_t s) {
  k_group_count<<<(a.n_nodes + 255) / 256, 256, 0, s>>>(a);
  note_launch();
}

// gcount holds the exclusive offsets here.
__global__ void k_group_fill(GroupBuildArgs a) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.n_nodes) return;
  const Node &nd = a.nodes[id];
  int k = a.gcount[id];
  pack_node(a.nodes, id, [&](int start, int count) {
    Group G;
    G.start = start;
    G.count = count;
    G.cell = nd.cell;
    G.box = nd.box;
    for (int d = 0; d < 3; ++d) {
      G.o[d] = 0.0;
      G.tlo[d] = G.thi[d] = G.flo[d] = G.fhi[d] = 0.f;
    }
    G.hmax = 0.f;
    G.pad = 0;
    a.groups[k++] = G;
  });
}

void launch_group_fill(const GroupBuildArgs &a, cudaStream_t s) {
  k_group_fill<<<(a.n_nodes + 255) / 256, 256, 0, s>>>(a);
  note_launch();
}

// One warp per group: frame origin (leaf-cell origin of its first particle)
// and the bounding boxes in the group frame and relative to the top cell.
__global__ void k_group_geometry(GroupBuildArgs a) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= a.n_groups) return;
  Group *G = &a.groups[g];
  const int start = G->start, count = G->count;
  const int leaf0 = a.leaf_of[start];
  const Leaf &L0 = a.leaves[leaf0];
  const double o[3] = {L0.o[0], L0.o[1], L0.o[2]};
  float flo[3] = {3e38f, 3e38f, 3e38f}, fhi[3] = {-3e38f, -3e38f, -3e38f};
  float tlo[3] = {3e38f, 3e38f, 3e38f}, thi[3] = {-3e38f, -3e38f, -3e38f};
  if (lane < count) {
    const int i = start + lane;
    const int li = a.leaf_of[i];
    const Leaf &L = a.leaves[li];
    const float4 q = a.pm[i];
    const float pq[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // group frame: the leaf offset from the group's first leaf, formed in
      // FP64 and rounded once; top-cell frame (the walk's box, which has a
      // pruning margin) in FP32
      const float f = li == leaf0 ? pq[d] : pq[d] + (float)(L.o[d] - o[d]);
      const float t = L.of[d] + pq[d];
      flo[d] = fhi[d] = f;
      tlo[d] = thi[d] = t;
    }
    a.gpos[i] = make_float4(flo[0], flo[1], flo[2], q.w);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int s = 16; s; s >>= 1) {
      flo[d] = fminf(flo[d], __shfl_xor_sync(0xffffffffu, flo[d], s));
      fhi[d] = fmaxf(fhi[d], __shfl_xor_sync(0xffffffffu, fhi[d], s));
      tlo[d] = fminf(tlo[d], __shfl_xor_sync(0xffffffffu, tlo[d], s));
      thi[d] = fmaxf(thi[d], __shfl_xor_sync(0xffffffffu, thi[d], s));
    }
  if (lane == 0) {
    for (int d = 0; d < 3; ++d) {
      G->o[d] = o[d];
      G->flo[d] = flo[d];
      G->fhi[d] = fhi[d];
      G->tlo[d] = tlo[d];
      G->thi[d] = thi[d];
    }
  }
}

void launch_group_geometry(const GroupBuildArgs &a, cudaStream_t s) {
  if (a.n_groups <= 0) return;
  k_group_geometry<<<(a.n_groups * 32 + 255) / 256, 256, 0, s>>>(a);
  note_launch();
}

__global__ void k_group_hmax(GroupBuildArgs a) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= a.n_groups) return;
  Group *G = &a.groups[g];
  float hm = lane < G->count ? a.hf[G->start + lane] : 0.f;
  for (int s = 16; s; s >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, s));
  if (lane == 0) G->hmax = hm;
}

void launch_group_hmax(const GroupBuildArgs &a, cudaStream_t s) {
  if (a.n_groups <= 0) return;
  k_group_hmax<<<(a.n_groups * 32 + 255) / 256, 256, 0, s>>>(a);
  note_launch();
}

// One warp per group: the source leaves within the group's radius, found by
// a breadth-first walk of the octrees of the 27 neighbouring top cells
// (periodic). The lanes test 32 frontier nodes at a time; passing leaves are
// written, in walk order, straight into the group's task slots, passing
// inner nodes put their 8 children on the next frontier. Radius: for the
// density, min(skin hmax_G, top-cell width); for the force, max(hmax_G,
// hmax_S), both from the group's bounding box. A group whose walk overflows
// (more than tcap leaves, or a frontier beyond kFront) is queued, and the
// second, tight walk tests every node against each target's own sphere
// instead (density: min(skin h_i, top-cell width); force: max(h_i, hmax_S)):
// a group of large-h particles next to a dense clump keeps only what its
// particles reach. count[g] > tcap still marks an overflow (the group is then
// left to the per-pass form).
constexpr int kWalkWarps = 4;
constexpr int kFront = 512;

// Walk modes: the plain walk of every group (with the neighbour cache: only
// the groups that need one), the tight walk of the groups it queued, and the
// far-reacher walk of the force (below).
enum { kWalkPlain = 0, kWalkTight = 1, kWalkFar = 2 };

// Largest over the lanes of a warp.
__device__ __forceinline__ float warp_max_f(float v) {
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// delta of the neighbour cache: the largest path length since the epoch
// began over the particles of the 27 top cells around `cell` (every lane of
// the warp gets it; lanes 0..26 read one cell each).
__device__ __forceinline__ float cell_motion(const CacheArgs &C, const BoxDev &B, int cell,
                                             int lane) {
  int c[3];
  cell_xyz(B, cell - B.cell_base, c);
  float m = 0.f;
  if (lane < 27) {
    const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
    const int nc = B.cell_base + (((c[0] + dx + B.n[0]) % B.n[0]) * B.n[1] +
                                  (c[1] + dy + B.n[1]) % B.n[1]) * B.n[2] +
                   (c[2] + dz + B.n[2]) % B.n[2];
    m = __uint_as_float(C.dmax_cell[nc]);
  }
  return warp_max_f(m);
}

// Far-reacher walk (force, neighbour cache): a group whose density finished
// in the first tier on per-lane lists can take its force pairs from the
// stored stage and lists, unless some particle outside the stage has an h
// that reaches the group. Outside the stage means at distance >= Reff =
// Rg - max_i dpath_i - delta from every target now, so only nodes whose
// largest h exceeds Reff and that lie within that h of the group box can
// hold one: the walk follows only those and stops at the first leaf.
// fuse[g] = 1 when none exists.
template <int MODE>
__global__ void __launch_bounds__(kWalkWarps * 32, MODE == kWalkTight ? 4 : 10)
    k_group_walk(GroupListArgs a) {
  __shared__ int front_all[kWalkWarps][2][kFront];  // node << 5 | neighbour code (0..26)
  constexpr bool tight = MODE == kWalkTight;
  constexpr bool far = MODE == kWalkFar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned ltmask = (1u << lane) - 1u;
  const int ng = tight ? *a.walk_queued : a.n_groups;
  // the cached force is skipped in this call: fuse[] is not read (stale)
  if (far && a.cache.ctl->force_off) return;
  int n_reused = 0, n_failed = 0;
  for (int q = blockIdx.x * kWalkWarps + warp; q < ng; q += gridDim.x * kWalkWarps) {
    const int g = tight ? a.walk_queue[q] : q;
    int *cur = front_all[warp][0], *nxt = front_all[warp][1];
    const Group G = a.groups[g];
    const BoxDev &B = a.boxes[G.box];
    float far_thr = 0.f;  // far walk: the effective stage radius Reff
    if (MODE == kWalkPlain && a.cache_on && !a.force) {
      // density: is the stored stage still complete for the starting h?
      bool reuse = false;
      const GroupCache &M = a.cache.meta[g];
      if (!a.cache.ctl->build_all && M.stage_ok) {
        float hm = 0.f, need = 0.f;
        if (lane < G.count) {
          hm = a.hf[G.start + lane];
          need = hm + a.cache.dpath[G.start + lane];
        }
        hm = warp_max_f(hm);
        need = warp_max_f(need) + cell_motion(a.cache, B, G.cell, lane);
        reuse = need <= M.Rg;
        // failures caused by motion count toward a new epoch (one that resets
        // the path lengths); an h that outgrew the stage rebuilds regardless
        if (!reuse && hm <= M.Rg) ++n_failed;
      }
      if (lane == 0) a.cache.gmode[g] = reuse ? 1 : 0;
      if (reuse) {
        ++n_reused;
        continue;  // the stored task slots and count stay
      }
    }
    if (MODE == kWalkPlain && a.cache_on && a.force && !a.cache.ctl->force_off &&
        a.cache.fuse[g]) {
      if (lane == 0) a.count[g] = 0;  // the force reuses the density's cache: no walk
      continue;
    }
    if (far) {
      // candidates: every warp of the group finished its density on lists
      const GroupCache &M = a.cache.meta[g];
      bool ok = M.stage_ok;
      for (int w = 0; w < 4; ++w)
        if (w * 8 < G.count && !M.wok[w]) ok = false;
      if (!ok) {
        if (lane == 0) a.cache.fuse[g] = 0;
        continue;
      }
      float dt = lane < G.count ? a.cache.dpath[G.start + lane] : 0.f;
      dt = warp_max_f(dt);
      far_thr = M.Rg - dt - cell_motion(a.cache, B, G.cell, lane);
    }
    int c[3];
    cell_xyz(B, G.cell - B.cell_base, c);
    const float wmin = fminf(B.wf[0], fminf(B.wf[1], B.wf[2]));
    const float capG = a.force ? G.hmax : fminf(G.hmax * a.skin, wmin);
    Task *out = a.tasks + (size_t)g * a.tcap;
    // tight walk: this lane's target (top-cell-relative position, radius)
    float tx = 0.f, ty = 0.f, tz = 0.f, tr = -1.f;
    if (tight && lane < G.count) {
      const int i = G.start + lane;
      const Leaf &L = a.leaves[a.leaf_of[i]];
      const float4 p = a.pm[i];
      tx = (float)(L.o[0] + (double)p.x);
      ty = (float)(L.o[1] + (double)p.y);
      tz = (float)(L.o[2] + (double)p.z);
      const float h = a.hf[i];
      tr = a.force ? h : fminf(h * a.skin, wmin);
    }

    // frontier 0: the 27 neighbouring top cells
    int n = 0;
    {
      bool in = lane < 27;
      int e = lane;
      if (in) {
        const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
        const int nc[3] = {(c[0] + dx + B.n[0]) % B.n[0], (c[1] + dy + B.n[1]) % B.n[1],
                           (c[2] + dz + B.n[2]) % B.n[2]};
        e |= (B.cell_base + (nc[0] * B.n[1] + nc[1]) * B.n[2] + nc[2]) << 5;
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
      for (int base = 0; base < n; base += 32) {
        const int idx = base + lane;
        bool valid = false;
        int code = 0, child = 0, leaf = 0;
        float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f}, shm = 0.f;
        if (idx < n) {
          const int e = cur[idx];
          code = e & 31;
          const Node &S = a.nodes[e >> 5];
          if (S.count > 0) {
            const int dx = code / 9 - 1, dy = (code / 3) % 3 - 1, dz = code % 3 - 1;
            const float sh[3] = {dx * B.wf[0], dy * B.wf[1], dz * B.wf[2]};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              lo[d] = S.lo[d] + sh[d];
              hi[d] = S.hi[d] + sh[d];
            }
            shm = S.hmax;
            child = S.child;
            leaf = S.leaf;
            valid = true;
          }
        }
        bool pass = false;
        if (far) {
          float d2 = 0.f;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float gap = fmaxf(0.f, fmaxf(lo[d] - G.thi[d], G.tlo[d] - hi[d]));
            d2 = fmaf(gap, gap, d2);
          }
          const float crit = shm + B.eps;
          pass = valid && shm > far_thr && d2 < crit * crit;
        } else if (!tight) {
          float d2 = 0.f;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float gap = fmaxf(0.f, fmaxf(lo[d] - G.thi[d], G.tlo[d] - hi[d]));
            d2 = fmaf(gap, gap, d2);
          }
          const float crit = (a.force ? fmaxf(capG, shm) : capG) + B.eps;
          pass = valid && d2 < crit * crit;
        } else {
          for (int k = 0; k < G.count; ++k) {  // warp-uniform loop over the targets
            const float xk = __shfl_sync(0xffffffffu, tx, k);
            const float yk = __shfl_sync(0xffffffffu, ty, k);
            const float zk = __shfl_sync(0xffffffffu, tz, k);
            const float rk = __shfl_sync(0xffffffffu, tr, k);
            const float gx = fmaxf(0.f, fmaxf(lo[0] - xk, xk - hi[0]));
            const float gy = fmaxf(0.f, fmaxf(lo[1] - yk, yk - hi[1]));
            const float gz = fmaxf(0.f, fmaxf(lo[2] - zk, zk - hi[2]));
            const float crit = (a.force ? fmaxf(rk, shm) : rk) + B.eps;
            pass |= fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < crit * crit;
          }
          pass = pass && valid;
        }
        const bool leaf_in = pass && child < 0, inner_in = pass && child >= 0;
        const unsigned ml = __ballot_sync(0xffffffffu, leaf_in);
        if (far) {  // a far reacher exists: stop (no tasks are written)
          if (ml) {
            ntask = 1;
            nn = 0;
            break;
          }
        } else if (leaf_in) {
          const int pos = ntask + __popc(ml & ltmask);
          if (pos < a.tcap) {
            const int dx = code / 9 - 1, dy = (code / 3) % 3 - 1, dz = code % 3 - 1;
            const Leaf &LS = a.leaves[leaf];
            Task tk;
            tk.sx = (float)(LS.o[0] + dx * B.w[0] - G.o[0]);
            tk.sy = (float)(LS.o[1] + dy * B.w[1] - G.o[1]);
            tk.sz = (float)(LS.o[2] + dz * B.w[2] - G.o[2]);
            tk.src = leaf;
            out[pos] = tk;
          }
        }
        ntask += __popc(ml);
        const unsigned mi = __ballot_sync(0xffffffffu, inner_in);
        if (inner_in) {
          const int pos = nn + 8 * __popc(mi & ltmask);
          for (int o = 0; o < 8; ++o)
            if (pos + o < kFront) nxt[pos + o] = ((child + o) << 5) | code;
        }
        nn += 8 * __popc(mi);
      }
      __syncwarp();
      if (far && ntask) break;
      if (nn > kFront) {
        overflow = true;
        break;
      }
      int *t = cur;
      cur = nxt;
      nxt = t;
      n = nn;
    }
    __syncwarp();  // the frontier buffers are reused by this warp's next group
    if (far) {  // a frontier overflow counts as a far reacher (full path)
      if (lane == 0) a.cache.fuse[g] = (ntask == 0 && !overflow) ? 1 : 0;
      if (ntask == 0 && !overflow) ++n_reused;
      continue;
    }
    overflow = overflow || ntask > a.tcap;
    if (lane == 0) {
      a.count[g] = overflow ? a.tcap + 1 : ntask;
      if (overflow && !tight && a.walk_queue) a.walk_queue[atomicAdd(a.walk_queued, 1)] = g;
      if (a.wmode) a.wmode[g] = tight ? 1 : 0;
    }
  }
  if (a.cache_on && lane == 0 && (n_reused || n_failed)) {
    if (MODE == kWalkPlain && !a.force) {
      atomicAdd(&a.ctr->cache_used[0], n_reused);
      if (n_failed) atomicAdd(&a.cache.ctl->fail, n_failed);
    }
    if (far) {
      atomicAdd(&a.ctr->cache_used[1], n_reused);
      atomicAdd(&a.cache.ctl->fused, n_reused);
    }
  }
}

// The walk over every group, then the tight walk over the groups it queued
// (`*a.walk_queued` must be zero on entry; the second launch reads it on the
// device).
void launch_group_lists(const GroupListArgs &a, cudaStream_t s) {
  if (a.n_groups <= 0) return;
  const int gblocks = (a.n_groups + kWalkWarps - 1) / kWalkWarps;
  if (a.cache_on && a.force) {  // far reachers decide which groups reuse the cache
    k_group_walk<kWalkFar><<<gblocks, kWalkWarps * 32, 0, s>>>(a);
    note_launch();
  }
  k_group_walk<kWalkPlain><<<gblocks, kWalkWarps * 32, 0, s>>>(a);
  note_launch();
  if (!a.walk_queue) return;
  const int blocks = a.n_groups < 152 * 8 * kWalkWarps ? gblocks : 152 * 8;
  k_group_walk<kWalkTight><<<blocks, kWalkWarps * 32, 0, s>>>(a);
  note_launch();
}

// ------------------------------------------------------------ kernels
//
// One block of kNW warps per group. All warps stage the group's candidates
// together, in one pass, each warp into its own segment of the stage in the
// order it found them (the stage order never depends on timing). Then each
// warp works alone on a sub-cluster of 8 consecutive targets (compact:
// consecutive in octree order): it keeps the staged entries within its
// sub-cluster's radius, and gives every target 4 lanes, lane s of a target
// handling every 4th of those entries; the 4 partial sums are combined by
// shuffles in fixed order, so the 4 lanes hold identical totals and take
// identical h steps.

constexpr int kNW = 4;           // warps per block, one group per block
constexpr int kSub = 8;          // targets per warp
constexpr int kSlice = 4;        // lanes per target
constexpr int kStageD = 1152;    // density stage entries per group (6 blocks per SM)
constexpr int kStageF = 704;     // force stage entries per group (7 blocks per SM)
constexpr int kBigStageD = 4096; // second tier: groups whose stage overflowed the first
constexpr int kBigStageF = 3072;
constexpr int kCandD = 1152;     // density entries kept per warp
constexpr int kCandF = 512;      // force entries kept per warp
// Tile 1 (the autotuner's alternative for clumped inputs): larger first-tier
// stages at lower occupancy, so fewer groups need the second tier.
constexpr int kStageDL = 1792;   // 4 blocks per SM
constexpr int kStageFL = 1536;   // 4 blocks per SM
constexpr int kCandFL = 640;
constexpr int dens_min_blocks(int ns) { return ns == kStageD ? 6 : (ns == kStageDL ? 4 : 1); }
constexpr int force_min_blocks(int ns) { return ns == kStageF ? 7 : (ns == kStageFL ? 4 : 1); }
constexpr int force_cand(int ns) { return ns == kStageF ? kCandF : kCandFL; }
constexpr int kLaneD = 32;       // density list entries per lane (tile 0)
constexpr int kLaneF = 28;       // force list entries per lane (tile 0)
// list entries per lane for a first-tier stage size (tile 1 and the second
// tier hold longer lists: clumped inputs put more particles inside the list radius)
constexpr int dens_lane(int ns) { return ns == kStageD ? kLaneD : 48; }
constexpr int force_lane(int ns) { return ns == kStageF ? kLaneF : 32; }
static_assert(kLaneD % 4 == 0 && kLaneF % 4 == 0, "lists are padded to multiples of 4");

// Entry NS of a stage is a sentinel (far away, zero mass, zero A): per-lane
// lists are padded with it to a multiple of 4 entries, so the sums run in
// steps of 4 with no bounds test; it never passes r^2 < h^2 and adds an
// exact zero to the FP32 force sums (the compensated sums skip it).
constexpr float kFar = 1e18f;

static_assert(sizeof(unsigned short) * kNW * kCandD >= 12 * 384,
              "the density's cand space holds the task shifts while a cached stage loads");

template <int NS>
struct DensSmem {
  unsigned dmax_bits;                       // largest dpath of a reloaded stage (float bits)
  unsigned pad_[3];
  float4 tgt[32];                           // tight stage: target position (group frame), radius
  float4 stage[NS + 1];                     // position in the group frame, m; [NS] sentinel
  unsigned short cand[kNW][kCandD];         // each warp's pre-filtered entries
  unsigned short list[kNW][dens_lane(NS) * 32];  // [entry][lane]
  int wcount[kNW];
  int qslot[8];                             // work queue: claimed chunks (two slots), timing
};

template <int NS>
struct ForceSmem {
  float4 tgt[32];                           // tight stage: target position (group frame), h
  float4 sq[NS + 1];                        // position in the group frame, m; [NS] sentinel
  float2 sf[NS + 1];                        // A (8/pi) h^-4, h^2
  int sj[NS + 1];                           // particle index (velocity read on use)
  unsigned short cand[kNW][force_cand(NS)];
  unsigned short list[kNW][force_lane(NS) * 32];
  int wcount[kNW];
  int qslot[8];                             // work queue: claimed chunks (two slots), timing
};

// Group g of a launch: tier 0 walks every group; tier 1 the groups tier 0
// queued because their stage outgrew it (restaged by each target's own
// radius at the first tier's stage size); tier 2 those whose tight stage
// still outgrew it (the large stage). Counts are read on the device, so the
// launches need no host round trip.
__device__ __forceinline__ int tier_group(int tier, int q, const int *queue,
                                          const int *queue_big) {
  return tier == 0 ? q : (tier == 1 ? queue[q] : queue_big[q]);
}
__device__ __forceinline__ int tier_count(int tier, int n_groups, const int *queued,
                                          const int *queued_big) {
  return tier == 0 ? n_groups : (tier == 1 ? *queued : *queued_big);
}

// The block-uniform cursor of a first-tier group loop. With a work queue,
// warp 0 claims the next kClaim queue positions with one atomic (claiming
// again while every group of the claim is one this launch skips) and hands
// the groups to run over as a bit mask through two alternating shared slots
// (a slot is rewritten only two claims later, behind a barrier that every
// thread reaches after reading it); without, a grid stride. Thread 0 times
// each group run (from its fetch to the next fetch) into wq.cost.
constexpr int kClaim = 32;
// Queue positions of n groups: whole chunks when ordered by chunk.
__device__ __forceinline__ int queue_positions(const WorkQueue &wq, int n) {
  return wq.order ? (n + kClaim - 1) / kClaim * kClaim : n;
}
struct GroupCursor {
  bool dyn;
  int it;
  int base;        // queue position of the claimed chunk
  unsigned mask;   // its groups still to run
  // skip: the launch leaves group g out when sel && (sel[g] != 0) != want
  __device__ int fetch(const WorkQueue &wq, int head, const unsigned char *sel, bool want,
                       int *slot, int ng) {
    if (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      return base + b;
    }
    int *s = slot + 2 * (it++ & 1);
    if (threadIdx.x < 32) {
      int b0;
      unsigned m;
      do {
        b0 = 0;
        if (threadIdx.x == 0) b0 = atomicAdd(wq.head + head, kClaim);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
        const int p = b0 + (int)threadIdx.x;
        const int gp = p < ng ? (wq.order ? wq.order[p] : p) : -1;  // -1: past the last group
        const bool run = gp >= 0 && !(sel && (sel[gp] != 0) != want);
        m = __ballot_sync(0xffffffffu, run);
      } while (m == 0u && b0 < ng);
      if (threadIdx.x == 0) {
        s[0] = b0;
        s[1] = (int)m;
      }
    }
    __syncthreads();
    base = s[0];
    mask = (unsigned)s[1];
    if (!mask) return ng;  // the queue is empty
    const int b = __ffs(mask) - 1;
    mask &= mask - 1;
    return base + b;
  }
  // slot[4], slot[5]: thread 0's timed group (-1: none) and its start (a
  // clock64 split in two ints); only thread 0 reads or writes them
  __device__ int first(const WorkQueue &wq, int head, const unsigned char *sel, bool want,
                       int *slot, int ng) {
    it = 0;
    mask = 0u;
    if (threadIdx.x == 0) slot[4] = -1;
    return dyn ? fetch(wq, head, sel, want, slot, ng) : (int)blockIdx.x;
  }
  __device__ int next(const WorkQueue &wq, int head, const unsigned char *sel, bool want,
                      int *slot, int ng, int q) {
    if (!dyn) return q + gridDim.x;
    if (threadIdx.x == 0 && slot[4] >= 0) {
      const long long t0 = (long long)(((unsigned long long)(unsigned)slot[6] << 32) |
                                       (unsigned)slot[5]);
      wq.cost[slot[4]] = (float)(clock64() - t0);
      slot[4] = -1;
    }
    return fetch(wq, head, sel, want, slot, ng);
  }
  __device__ void run(int *slot, int group) {
    if (dyn && threadIdx.x == 0) {
      const unsigned long long t0 = (unsigned long long)clock64();
      slot[4] = group;
      slot[5] = (int)(unsigned)t0;
      slot[6] = (int)(unsigned)(t0 >> 32);
    }
  }
};

// The stage is laid out in two halves of cap / 2 entries, one per pair of
// warps: warp 0 fills the first half from its start upward and warp 1 from its
// end downward, warps 2 and 3 the second half the same way, each in the order
// it found its particles (deterministic). A pair overflows only when its two
// shares together exceed the half, so a group fits when the larger pair sum
// does (with a quarter of the stage per warp, the largest single share had
// to). A flat index t in [0, total) (warp 0's entries, then warp 1's, 2's,
// 3's) maps to its slot through the prefix counts pre[].
struct StageRange {
  int total;      // staged entries, all warps
  int over;       // some pair's shares outgrew its half (the stage is incomplete)
  int unmapped;   // (stored stage) some batch of tasks had no task map: slots not stored
  int need;       // stage slots this group needs: 2 x the larger pair sum
  int segcap;     // a quarter of the stage (a half holds 2 x segcap)
  int pre1, pre2, pre3;  // prefix counts of warps 0, 0..1, 0..2
  __device__ __forceinline__ int index(int t) const {
    if (t < pre1) return t;                              // warp 0: upward from 0
    if (t < pre2) return 2 * segcap - 1 + pre1 - t;      // warp 1: downward from the half
    if (t < pre3) return 2 * segcap + t - pre2;          // warp 2: upward from the half
    return 4 * segcap - 1 + pre3 - t;                    // warp 3: downward from the end
  }
};
__device__ __forceinline__ int stage_need(int c0, int c1, int c2, int c3) {
  return 2 * max(c0 + c1, c2 + c3);
}

constexpr int kMap = 1024;  // per-warp particle -> task map (bytes, aliases the warp's cand)
constexpr int kMapD = 2048; // the density's (its cand is larger)
static_assert(kCandD * 2 >= kMapD && kCandF * 2 >= kMap && kCandFL * 2 >= kMap,
              "task map must fit a warp's cand");
static_assert(kStageD % kNW == 0 && kStageF % kNW == 0 && kBigStageD % kNW == 0 &&
                  kBigStageF % kNW == 0 && kStageDL % kNW == 0 && kStageFL % kNW == 0,
              "stage segments");

// Stage the particles of this warp's share of the group's source leaves that
// lie within R of the group box (R = Rg, or max(Rg, h_j) for the force), in
// one pass. The warp takes 32 of its tasks at a time, one per lane; a warp
// scan of their particle counts lays the 32 leaves end to end, each lane
// marks its leaf's stretch in a shared-memory map, and the lanes then walk
// the concatenated particles 32 at a time (kU loads in flight), reading each
// particle's task from the map and the task's base and shift by shuffles.
// Passing particles are appended by ballot at the warp's end of its pair's
// half of the stage. Called by every thread of the block.
// st_j / st_slot (density, first tier, neighbour cache): each staged
// particle's index and task slot are also written there, at its stage slot.
template <bool FORCE>
__device__ StageRange stage_group(const BatchDensArgs *da, const BatchForceArgs *fa,
                                  const Group &G, int e0, int e1, int warp, int lane, float Rg,
                                  float4 *sq, float2 *sf, int *sj, int *wcount,
                                  unsigned char *tmap, int cap, const float4 *tgt,
                                  int *st_j = nullptr, unsigned short *st_slot = nullptr) {
  const unsigned ltmask = (1u << lane) - 1u;
  const Task *tasks = FORCE ? fa->tasks : da->tasks;
  const Leaf *leaves = FORCE ? fa->leaves : da->leaves;
  const float4 *pm = FORCE ? fa->pm : da->pm;
  const int ntask = e1 - e0;
  const int segcap = cap / kNW;
  const int half = 2 * segcap;
  // this warp's k-th entry goes to slot sbase + sdir * k (k < half)
  const int sdir = (warp & 1) ? -1 : 1;
  const int sbase = (warp >> 1) * half + ((warp & 1) ? half - 1 : 0);
  constexpr int map_cap = FORCE ? kMap : kMapD;
  __syncthreads();  // every warp is done with the previous group's stage
  int nst = 0;
  bool unmapped = false;
  for (int tb = warp; tb < ntask; tb += 32 * kNW) {
    const int mt = tb + lane * kNW;  // this lane's task
    int start = 0, cnt = 0;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    if (mt < ntask) {
      const Task tk = tasks[e0 + mt];
      const Leaf &LS = leaves[tk.src];
      start = LS.start;
      cnt = LS.count;
      sx = tk.sx;
      sy = tk.sy;
      sz = tk.sz;
    }
    int incl = cnt;  // inclusive scan over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int jbase = start - (incl - cnt);  // particle of flat index f: jbase_t + f
    const bool mapped = total <= map_cap;    // warp-uniform
    unmapped |= !mapped;
    if (mapped) {
      for (int f = incl - cnt; f < incl; ++f) tmap[f] = (unsigned char)lane;
      __syncwarp();
    }
    constexpr int kU = FORCE ? 4 : 8;  // chunks in flight together (fewer: the force kernel spills)
    for (int f0 = 0; f0 < total; f0 += 32 * kU) {
      float4 q[kU], fj[kU];
      int jj[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int f = f0 + 32 * u + lane;
        int t = 0;
        if (mapped) {
          t = f < total ? tmap[f] : 0;
        } else {  // first task whose inclusive count exceeds f
#pragma unroll
          for (int s = 16; s; s >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, t + s - 1);
            if (v <= f) t += s;
          }
        }
        const int tb0 = __shfl_sync(0xffffffffu, jbase, t);
        const float tx = __shfl_sync(0xffffffffu, sx, t);
        const float ty = __shfl_sync(0xffffffffu, sy, t);
        const float tz = __shfl_sync(0xffffffffu, sz, t);
        jj[u] = tb0 + f;
        q[u] = make_float4(tx, ty, tz, 0.f);
        fj[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (f < total) {
          const float4 p4 = pm[jj[u]];
          q[u].x += p4.x;
          q[u].y += p4.y;
          q[u].z += p4.z;
          q[u].w = p4.w;
          if (FORCE) fj[u] = fa->fi[jj[u]];
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int f = f0 + 32 * u + lane;
        bool in = false;
        if (f < total) {
          if (!tgt) {
            const float R = FORCE ? fmaxf(Rg, fj[u].x) : Rg;
            const float gx = fmaxf(0.f, fmaxf(G.flo[0] - q[u].x, q[u].x - G.fhi[0]));
            const float gy = fmaxf(0.f, fmaxf(G.flo[1] - q[u].y, q[u].y - G.fhi[1]));
            const float gz = fmaxf(0.f, fmaxf(G.flo[2] - q[u].z, q[u].z - G.fhi[2]));
            in = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < R * R;
          } else {  // tight: within some target's own radius (force: max(h_i, h_j))
            for (int k = 0; k < G.count; ++k) {
              const float4 t = tgt[k];
              const float dx = q[u].x - t.x, dy = q[u].y - t.y, dz = q[u].z - t.z;
              const float R = FORCE ? fmaxf(t.w, fj[u].x) : t.w;
              in |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < R * R;
            }
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        const int pos = nst + __popc(m & ltmask);
        if (in && pos < half) {  // within this pair's half (a pair that overflows is discarded)
          const int slot = sbase + sdir * pos;
          sq[slot] = q[u];
          if (FORCE) {
            sf[slot] = make_float2(fj[u].z, fj[u].w);
            sj[slot] = jj[u];
          }
          if (st_j) {  // the task of flat index f: from the map (else not stored)
            st_j[slot] = jj[u];
            const int tl = mapped ? (int)tmap[f0 + 32 * u + lane] : 0;
            st_slot[slot] = (unsigned short)(tb + tl * kNW);
          }
        }
        nst += __popc(m);
      }
    }
    if (mapped) __syncwarp();  // the map is rewritten by the next 32 tasks
  }
  if (lane == 0) wcount[warp] = nst;
  __syncthreads();
  StageRange r;
  r.segcap = segcap;
  const int c0 = wcount[0], c1 = wcount[1], c2 = wcount[2], c3 = wcount[3];
  r.pre1 = c0;
  r.pre2 = c0 + c1;
  r.pre3 = c0 + c1 + c2;
  r.total = r.pre3 + c3;
  r.need = stage_need(c0, c1, c2, c3);
  r.over = r.need > cap;
  r.unmapped = __syncthreads_or(unmapped);
  return r;
}

// Sub-cluster box of this warp's targets (lanes with has = false ignored):
// every lane gets the min / max over the warp.
__device__ __forceinline__ void sub_box(bool has, float px, float py, float pz, float lo[3],
                                        float hi[3]) {
  lo[0] = has ? px : 3e38f;
  lo[1] = has ? py : 3e38f;
  lo[2] = has ? pz : 3e38f;
  hi[0] = has ? px : -3e38f;
  hi[1] = has ? py : -3e38f;
  hi[2] = has ? pz : -3e38f;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
}

// Warp-wide filter of the stage: entries within R (R = Rsub, or for the
// force max(Rsub, h_j)) of the sub-cluster box, compacted in stage order into
// `cand`. Returns the count (> cap means overflow).
template <bool FORCE>
__device__ __forceinline__ int filter_stage(const float4 *sq, const float2 *sf,
                                            const StageRange &sr, const float lo[3],
                                            const float hi[3], float Rsub, unsigned short *cand,
                                            int cap, int lane) {
  const unsigned ltmask = (1u << lane) - 1u;
  int n = 0;
  for (int tb = 0; tb < sr.total; tb += 32) {
    const int t = tb + lane;
    bool in = false;
    int k = 0;
    if (t < sr.total) {
      k = sr.index(t);
      const float4 q = sq[k];
      const float R = FORCE ? fmaxf(Rsub, sqrtf(sf[k].y)) : Rsub;
      const float gx = fmaxf(0.f, fmaxf(lo[0] - q.x, q.x - hi[0]));
      const float gy = fmaxf(0.f, fmaxf(lo[1] - q.y, q.y - hi[1]));
      const float gz = fmaxf(0.f, fmaxf(lo[2] - q.z, q.z - hi[2]));
      in = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < R * R;
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    const int pos = n + __popc(m & ltmask);
    if (in && pos < cap) cand[pos] = (unsigned short)k;
    n += __popc(m);
  }
  __syncwarp();
  return n;
}

// The force kernel's filter in chunks: from stage entry `sp` on, entries
// within max(Rsub, h_j) of the sub-cluster box, compacted in stage order into
// `cand`, 32 entries at a time while at least 32 slots remain free. Returns
// the count (<= cap) and advances sp past the entries it examined.
__device__ __forceinline__ int filter_chunk(const float4 *sq, const float2 *sf,
                                            const StageRange &sr, int &sp, const float lo[3],
                                            const float hi[3], float Rsub,
                                            unsigned short *cand, int cap, int lane) {
  const unsigned ltmask = (1u << lane) - 1u;
  int n = 0;
  for (; sp < sr.total && n <= cap - 32; sp += 32) {
    const int t = sp + lane;
    bool in = false;
    int k = 0;
    if (t < sr.total) {
      k = sr.index(t);
      const float4 q = sq[k];
      const float R = fmaxf(Rsub, sqrtf(sf[k].y));
      const float gx = fmaxf(0.f, fmaxf(lo[0] - q.x, q.x - hi[0]));
      const float gy = fmaxf(0.f, fmaxf(lo[1] - q.y, q.y - hi[1]));
      const float gz = fmaxf(0.f, fmaxf(lo[2] - q.z, q.z - hi[2]));
      in = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < R * R;
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (in) cand[n + __popc(m & ltmask)] = (unsigned short)k;
    n += __popc(m);
  }
  __syncwarp();
  return n;
}

// Sum of a per-lane value over the kSlice lanes of one target, in fixed order.
__device__ __forceinline__ float slice_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// One lane's density sums (Eq. rho and the h-derivative terms) over its
// share of the candidates: q = r / h_i for r^2 < h2.
template <bool KAHAN>
struct DensAcc {
  float sw = 0.f, sdw = 0.f, smw = 0.f, smdh = 0.f;
  float cw = 0.f, cdw = 0.f, cmw = 0.f, cmdh = 0.f;
  int c = 0;
  __device__ __forceinline__ void add(float4 q, float px, float py, float pz, float h2,
                                      float hinv) {
    const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < h2) {
      const float r = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
      const float qq = r * hinv;
      float w, dw;
      w_and_dw(qq, w, dw);
      const float qdw = qq * dw;
      if (KAHAN) {
        add_comp(sw, cw, w);
        add_comp(sdw, cdw, qdw);
        add_comp(smw, cmw, q.w * w);
        add_comp(smdh, cmdh, q.w * fmaf(3.f, w, qdw));
      } else {
        sw += w;
        sdw += qdw;
        smw = fmaf(q.w, w, smw);
        smdh = fmaf(q.w, fmaf(3.f, w, qdw), smdh);
      }
      ++c;
    }
  }
};

// Reload a group's stored stage (neighbour cache) into shared memory at the
// current positions: the stage slot k of warp w's entries (wc[w] of them, at
// the slots of the staging layout) holds particle sj[k],
// moved into the group frame by its task's shift (the same sum as the
// staging, so the same FP32 values). The group's task shifts are first
// copied to `shift` (shared memory free at this point, >= 3 ntask floats),
// then every thread takes 8 entries at a time with their loads in flight
// together. FORCE also stages (A', h^2) and the index. Returns the stage
// range; *dmax receives the largest dpath of the staged particles (through
// *dmax_bits, shared). Called by every thread of the block.
template <bool FORCE>
__device__ StageRange load_stage_cached(const CacheArgs &C, int g, const int wc[4],
                                        const Task *tasks, int ntask, const float4 *pm,
                                        const float4 *fi, float4 *sq, float2 *sf, int *sj,
                                        int cap, float *shift, unsigned *dmax_bits,
                                        float *dmax) {
  __syncthreads();  // every warp is done with the previous group's stage and shift space
  if (threadIdx.x == 0) *dmax_bits = 0u;
  StageRange r;
  r.segcap = cap / kNW;
  r.pre1 = wc[0];
  r.pre2 = wc[0] + wc[1];
  r.pre3 = r.pre2 + wc[2];
  r.total = r.pre3 + wc[3];
  r.need = stage_need(wc[0], wc[1], wc[2], wc[3]);
  r.over = 0;
  r.unmapped = 0;
  for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
    const Task tk = tasks[t];
    shift[3 * t] = tk.sx;
    shift[3 * t + 1] = tk.sy;
    shift[3 * t + 2] = tk.sz;
  }
  const size_t base = (size_t)g * C.ns;
  constexpr int kU = 8;
  const int t0 = threadIdx.x;
  int k[kU], j[kU], sl[kU];
  // the first 8 entries' indices load while the shifts are being written
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int t = t0 + u * blockDim.x;
    k[u] = t < r.total ? r.index(t) : -1;
    j[u] = k[u] >= 0 ? C.sj[base + k[u]] : 0;
    sl[u] = k[u] >= 0 ? (int)C.slot[base + k[u]] : 0;
  }
  __syncthreads();
  float dm = 0.f;
  for (int tb = 0;; tb += kU * blockDim.x) {
    float4 p4[kU], f4[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      p4[u] = pm[j[u]];
      if (FORCE) f4[u] = fi[j[u]];
      dm = fmaxf(dm, k[u] >= 0 ? C.dpath[j[u]] : 0.f);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (k[u] < 0) continue;
      const float *sh = shift + 3 * sl[u];
      float4 q = make_float4(sh[0], sh[1], sh[2], 0.f);
      q.x += p4[u].x;
      q.y += p4[u].y;
      q.z += p4[u].z;
      q.w = p4[u].w;
      sq[k[u]] = q;
      if (FORCE) {
        sf[k[u]] = make_float2(f4[u].z, f4[u].w);
        sj[k[u]] = j[u];
      }
    }
    const int tn = tb + kU * blockDim.x;
    if (tn >= r.total) break;  // block-uniform
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int t = tn + t0 + u * blockDim.x;
      k[u] = t < r.total ? r.index(t) : -1;
      j[u] = k[u] >= 0 ? C.sj[base + k[u]] : 0;
      sl[u] = k[u] >= 0 ? (int)C.slot[base + k[u]] : 0;
    }
  }
  dm = warp_max_f(dm);
  if ((threadIdx.x & 31) == 0) atomicMax(dmax_bits, __float_as_uint(dm));
  __syncthreads();
  *dmax = __uint_as_float(*dmax_bits);
  return r;
}

// Asynchronous copy of `rows` rows of 32 list entries (64 bytes each) from
// global to shared memory, 16 bytes per request (cp.async, no registers
// held); wait with cp_async_wait_all().
__device__ __forceinline__ void cp_async_rows(unsigned short *dst, const unsigned short *src,
                                              int rows, int lane) {
  for (int t = lane; t < rows * 4; t += 32) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst + 8 * t);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(src + 8 * t)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <bool KAHAN, int NS, bool REUSE, bool MID>
__global__ void __launch_bounds__(kNW * 32, dens_min_blocks(NS))
    k_density_batched(BatchDensArgs a, int tier) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DensSmem<NS> &S = *reinterpret_cast<DensSmem<NS> *>(smem_raw);
  // the second and later tiers stage by each target's own radius
  constexpr bool TIGHT = MID || NS == kBigStageD;
  constexpr int LANE = dens_lane(NS);
  const double tol_n = a.tol * a.n_ngb;
  const float gm1 = (float)(a.gamma - 1.0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slice = lane & (kSlice - 1);
  unsigned short *cand = S.cand[warp];
  unsigned short *list = S.list[warp];
  unsigned long long ntest = 0, inter = 0;
  int max_it = 0, st_bits = 0, stage_max = 0, n_direct[2] = {0, 0}, n_built = 0, n_relist = 0;
  if (threadIdx.x == 0) S.stage[NS] = make_float4(kFar, kFar, kFar, 0.f);  // read after a barrier
  // the neighbour cache: first tier only
  const bool use_cache = !TIGHT && a.cache_on;

  const int ng = tier_count(tier, a.n_groups, &a.ctr->queued[0], &a.ctr->queued_big[0]);
  GroupCursor cur;
  // with the queue: heads [0] and [1] for the launches on stored stages and anew
  cur.dyn = tier == 0 && a.wq.head != nullptr;
  const int qn = cur.dyn ? queue_positions(a.wq, ng) : ng;
  for (int q = cur.first(a.wq, REUSE ? 0 : 1, use_cache ? a.cache.gmode : nullptr, REUSE,
                         S.qslot, qn);
       q < qn; q = cur.next(a.wq, REUSE ? 0 : 1, use_cache ? a.cache.gmode : nullptr, REUSE,
                            S.qslot, qn, q)) {
    const int g =
        cur.dyn ? (a.wq.order ? a.wq.order[q] : q) : tier_group(tier, q, a.queue, a.queue_big);
    const Group G = a.groups[g];
    const BoxDev &B = a.boxes[G.box];
    const float wmin = fminf(B.wf[0], fminf(B.wf[1], B.wf[2]));
    const float hcap = (float)B.hcap;
    const float Rg = fminf(G.hmax * a.skin_stage, wmin);
    if (use_cache && (a.cache.gmode[g] != 0) != REUSE) continue;  // the other instantiation's
    cur.run(S.qslot, g);
    // tasks from the tight walk: complete only within each target's own
    // starting radius (block-uniform; a reused stage never came from one)
    const bool tightw = !REUSE && !TIGHT && a.wmode && a.wmode[g];
    const int nt = a.tcount[g];
    const int e0 = g * a.tcap;
    GroupCache *M = use_cache ? &a.cache.meta[g] : nullptr;
    float Rgb = Rg, Dst = 0.f;   // stage radius at the build, largest staged dpath
    if (TIGHT) __syncthreads();  // the previous group's warps are done reading tgt
    if (TIGHT && threadIdx.x < 32) {  // tight stage: each target's own radius
      float4 t = make_float4(0.f, 0.f, 0.f, -1.f);
      if ((int)threadIdx.x < G.count) {
        const int it = G.start + threadIdx.x;
        const float4 pq = a.gpos[it];
        t = make_float4(pq.x, pq.y, pq.z, fminf(a.hf[it] * a.skin_stage, wmin));
      }
      S.tgt[threadIdx.x] = t;  // read after stage_group's opening barrier
    }
    StageRange sr;
    if constexpr (REUSE) {
      int wc[4];
      for (int w = 0; w < 4; ++w) wc[w] = M->wc[w];
      Rgb = M->Rg;
      // this warp's stored lists start copying to shared memory now (the
      // previous group's warps are done with them: the load's barrier
      // follows, and each warp copies only its own rows)
      const int tp = M->tpad[warp];
      if (tp > 0)
        cp_async_rows(S.list[warp],
                      a.cache.list + ((size_t)g * kNW + warp) * a.cache.lane_cap * 32, tp, lane);
      sr = load_stage_cached<false>(a.cache, g, wc, a.tasks + e0, min(nt, a.tcap), a.pm,
                                    nullptr, S.stage, nullptr, nullptr, NS,
                                    reinterpret_cast<float *>(&S.cand[0][0]), &S.dmax_bits,
                                    &Dst);
    } else {
      sr = stage_group<false>(&a, nullptr, G, e0, e0 + min(nt, a.tcap), warp, lane, Rg, S.stage,
                              nullptr, nullptr, S.wcount, (unsigned char *)cand, NS,
                              TIGHT ? S.tgt : nullptr,
                              use_cache ? a.cache.sj + (size_t)g * a.cache.ns : nullptr,
                              use_cache ? a.cache.slot + (size_t)g * a.cache.ns : nullptr);
      if (use_cache && threadIdx.x == 0) {
        for (int w = 0; w < 4; ++w) M->wc[w] = min(S.wcount[w], 2 * sr.segcap);
        M->Rg = Rg;
        M->stage_ok = !sr.over && nt <= a.tcap && !sr.unmapped && !tightw;
        ++n_built;
      }
    }
    stage_max = max(stage_max, sr.total);
    if (sr.over || nt > a.tcap) {  // block-uniform
      if (use_cache && threadIdx.x < kNW) M->wok[threadIdx.x] = 0;
      if (MID && nt <= a.tcap) {  // the tight stage outgrew this size: the large one
        if (threadIdx.x == 0) a.queue_big[atomicAdd(&a.ctr->queued_big[0], 1)] = g;
      } else if (threadIdx.x < kNW && (TIGHT || nt > a.tcap)) {  // the third tier walks them
        a.queue2[atomicAdd(&a.ctr->queued2[0], 1)] = g * kNW + threadIdx.x;
      } else if (threadIdx.x == 0 && !TIGHT && nt <= a.tcap) {  // second tier: tight stage
        a.queue[atomicAdd(&a.ctr->queued[0], 1)] = g;
      }
      continue;
    }
    // this warp's targets: lane = target * kSlice + slice
    const int tloc = warp * kSub + (lane >> 2);
    const bool has = tloc < G.count;
    const int i = G.start + tloc;
    float px = 0.f, py = 0.f, pz = 0.f;
    HIterF it;
    it.start(has ? a.hf[i] : 1.f);
    // with tasks from the tight walk, this target's own walked radius
    const float Rtight = fminf(it.h * a.skin_stage, wmin);
    if (has) {
      const float4 q = a.gpos[i];
      px = q.x;
      py = q.y;
      pz = q.z;
    }
    if (!__any_sync(0xffffffffu, has)) {  // this warp has no targets
      if (use_cache && lane == 0) M->wok[warp] = 1;
      continue;
    }
    float blo[3], bhi[3];
    sub_box(has, px, py, pz, blo, bhi);

    bool failed = false, fin = !has, need_list = has, need_filter = true;
    // 0: per-lane lists; 1: a lane's list outgrew LANE, the warp reads its
    // candidates directly; 2: the candidates outgrew kCandD, the warp reads
    // the whole stage (slower, same sums)
    int mode = 0;
    int ncand = 0, cnt = 0, passes = 0, ngb = 0, tpad = 0;
    float rsub = 0.f, rl = 0.f;
    // radius within which the stage is complete for this warp's targets: Rg
    // when staged now; with a reused stage, Rg - dpath_i - delta (minimum over
    // the warp)
    float Rgw = Rg;
    bool fresh = true;      // the per-lane lists were built in this call
    bool have_cand = true;  // cand holds the filtered stage (else a list rebuild refilters)
    if constexpr (REUSE) {
      const float dp = has ? a.cache.dpath[i] : 0.f;
      const float delta = cell_motion(a.cache, B, G.cell, lane);
      float rw = has ? Rgb - dp - delta : 3e38f;
      for (int o = 16; o; o >>= 1) rw = fminf(rw, __shfl_xor_sync(0xffffffffu, rw, o));
      Rgw = rw;
      const int tp = M->tpad[warp];
      if (tp >= 0) {  // stored lists: complete within rl_i - dpath_i - D for staged j
        cp_async_wait_all();
        __syncwarp();
        cnt = tp;
        tpad = tp;
        rl = has ? a.cache.rl[i] - dp - Dst : 0.f;
        rsub = Rgw;
        have_cand = false;  // an h beyond rl refilters the stage, then rebuilds the lists
        fresh = false;
        need_list = false;
        // the stored lists serve only if every starting h lies within them
        need_filter = __any_sync(0xffffffffu, has && it.h > rl);
        // motion (not a grown h) made them incomplete: counts toward a new epoch
        const bool grown = __any_sync(0xffffffffu, has && it.h > a.cache.rl[i]);
        if (need_filter && !grown && lane == 0) atomicAdd(&a.cache.ctl->lfail, 1);
      }
    }
    float4 fs = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int pass = 0; pass < a.max_iter; ++pass) {
      if (mode < 2 && __any_sync(0xffffffffu, need_filter)) {
        // sub-cluster radius: its largest h x the list skin, capped by Rgw
        float hm = has && !fin ? it.h : 0.f;
        for (int o = 16; o; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
        rsub = fminf(hm * a.skin_list, Rgw);
        ncand = filter_stage<false>(S.stage, nullptr, sr, blo, bhi, rsub, cand, kCandD, lane);
        need_filter = false;
        have_cand = true;
        need_list = !fin;
        if (ncand > kCandD) mode = 2;  // ncand is warp-uniform
      }
      if (mode == 0 && __any_sync(0xffffffffu, need_list)) {
        float rl2 = -1.f;
        if (need_list) {
          rl = fminf(it.h * a.skin_list, rsub);
          rl2 = rl * rl;
          cnt = 0;
          ntest += (ncand + kSlice - 1 - slice) / kSlice;
        }
#pragma unroll 4
        for (int t = slice; t < ncand; t += kSlice) {
          const int k = cand[t];
          const float4 q = S.stage[k];
          const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (r2 < rl2) {
            if (cnt < LANE) list[cnt * 32 + lane] = (unsigned short)k;
            ++cnt;
          }
        }
        need_list = false;
        fresh = true;
        if (__any_sync(0xffffffffu, cnt > LANE)) {
          mode = 1;
        } else {  // pad every lane's list with the sentinel to the warp's longest, x4
          tpad = (warp_max_int(cnt) + 3) & ~3;
          for (int t = cnt; t < tpad; ++t) list[t * 32 + lane] = (unsigned short)NS;
        }
        __syncwarp();
      }
      // partial sums over this lane's slice at the current h
      const float hf = it.h;
      const float h2 = fin ? -1.f : hf * hf;
      const float hinv = 1.f / hf;
      DensAcc<KAHAN> acc;
      if (mode == 0) {  // finished lanes have h2 < 0: nothing passes
        const int tmax = (warp_max_int(fin ? 0 : cnt) + 3) & ~3;
        for (int t = 0; t < tmax; t += 4) {
          int k[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) k[u] = list[(t + u) * 32 + lane];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc.add(S.stage[k[u]], px, py, pz, h2, hinv);
        }
        if (!fin) ntest += cnt;
      } else {
        const int nsrc = mode == 1 ? ncand : sr.total;
        for (int t = slice; t < nsrc; t += kSlice)
          acc.add(S.stage[mode == 1 ? (int)cand[t] : sr.index(t)], px, py, pz, h2, hinv);
        if (!fin) ntest += (nsrc + kSlice - 1 - slice) / kSlice;
      }
      const float4 tot = make_float4(slice_sum(acc.sw), slice_sum(acc.sdw), slice_sum(acc.smw),
                                     slice_sum(acc.smdh));
      int ctot = acc.c;
      ctot += __shfl_xor_sync(0xffffffffu, ctot, 1);
      ctot += __shfl_xor_sync(0xffffffffu, ctot, 2);
      if (!fin) {
        ++passes;
        int st = 0;
        const bool conv = h_newton_step_f(it, tot.x, tot.y, a.n_ngb, tol_n, hcap, &st);
        st_bits |= st;
        if (conv) {
          fin = true;
          fs = tot;
          ngb = ctot - 1;  // the self term is always inside
        } else if (it.h > rsub || (it.h > rl && !have_cand)) {
          need_filter = true;
        } else if (it.h > rl) {
          need_list = true;
        }
      }
      // this target's staged radius
      const float Rown = TIGHT && has ? S.tgt[tloc].w : (tightw ? Rtight : Rgw);
      if (__any_sync(0xffffffffu, !fin && it.h > Rown)) {
        failed = true;  // beyond the staged radius
        break;
      }
      if (__all_sync(0xffffffffu, fin)) break;
    }
    if (lane == 0 && mode) ++n_direct[mode - 1];
    if (REUSE && fresh && lane == 0) ++n_relist;
    if (failed || !__all_sync(0xffffffffu, fin)) {
      // this warp's unfinished targets go to the third tier (done is not set)
      if (lane == 0) {
        a.queue2[atomicAdd(&a.ctr->queued2[0], 1)] = g * kNW + warp;
        if (use_cache) M->wok[warp] = 0;
      }
      continue;
    }
    if (use_cache) {  // keep this warp's lists for the force and later calls
      if (mode == 0 && fresh) {
        const size_t lrow = ((size_t)g * kNW + warp) * a.cache.lane_cap * 32;
        for (int t = 0; t < tpad; ++t) a.cache.list[lrow + t * 32 + lane] = list[t * 32 + lane];
        if (has && slice == 0) a.cache.rl[i] = rl;
      }
      if (lane == 0) {
        if (mode != 0)
          M->tpad[warp] = -1;
        else if (fresh)
          M->tpad[warp] = tpad;
        M->wok[warp] = mode == 0 && !tightw;  // the force needs the stage complete within Rg
      }
    }
    if (has && slice == 0) {
      float rho, omega, P;
      float4 fi;
      const bool ok = finalise_density(it.h, fs, a.vu[i].w, gm1, &rho, &omega, &P, &fi);
      if (!ok) st_bits |= kErrNonPhysical;
      a.h[i] = (double)it.h;
      a.hf[i] = it.h;
      a.rho[i] = rho;
      a.omega[i] = omega;
      a.P[i] = P;
      a.fi[i] = fi;
      a.nngb[i] = ngb;
      a.niter[i] = passes;
      a.done[i] = 1;
      inter += (unsigned long long)ngb;
      max_it = max(max_it, passes);
    }
  }
  ntest = warp_sum(ntest);
  inter = warp_sum(inter);
  max_it = warp_max_int(max_it);
  for (int o = 16; o; o >>= 1) st_bits |= __shfl_xor_sync(0xffffffffu, st_bits, o);
  if (lane == 0) {
    if (ntest) atomicAdd(&a.ctr->dens_cand, ntest);
    if (inter) atomicAdd(&a.ctr->dens_inter, inter);
    if (max_it) atomicMax(&a.ctr->max_iter_used, max_it);
    if (st_bits) atomicOr(&a.ctr->status, st_bits);
    atomicMax(&a.ctr->stage_max[0], stage_max);
    if (n_direct[0]) atomicAdd(&a.ctr->direct[0], n_direct[0]);
    if (n_direct[1]) atomicAdd(&a.ctr->direct[1], n_direct[1]);
  }
  if (n_built) atomicAdd(&a.ctr->cache_built, n_built);
  if (n_relist) atomicAdd(&a.ctr->cache_relist, n_relist);
}

// One lane's force sums (Eqs. dvdt, dudt) over its share of the staged
// particles. hi2 < 0: the entry is a listed neighbour (accepted); otherwise
// the pair is tested, r > 0 and r^2 < max(h_i^2, h_j^2).
template <bool KAHAN>
struct ForceAcc {
  float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
  float cx = 0.f, cy = 0.f, cz = 0.f, cu = 0.f;  // Kahan compensations
  int c = 0;
  // k == skip (the stage sentinel) adds exact zeros; it is not counted and
  // the compensated sums leave it out.
  template <class SM>
  __device__ __forceinline__ void add(const SM &S, int k, const float4 *vu, float px,
                                      float py, float pz, float4 fi, float4 vi, float hi2,
                                      int skip = -1) {
    const float4 q = S.sq[k];
    const float2 f = S.sf[k];
    const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (hi2 >= 0.f && !(r2 > 0.f && r2 < fmaxf(hi2, f.y))) return;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float ti = fi.z * dw_only(r * fi.y);         // A_i dW/dr(r, h_i)
    const float tj = f.x * dw_only(r * rsqrtf(f.y));   // A_j dW/dr(r, h_j)
    const float fac = q.w * (ti + tj) * rinv;
    const float4 vj = vu[S.sj[k]];
    const float dvdx = (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
    if (KAHAN && k == skip) return;
    accumulate(fac, dx, dy, dz, q.w * ti * rinv * dvdx);
    if (!KAHAN && k == skip) --c;
  }
  // a -= fac (x_i - x_j), du/dt += the energy term
  __device__ __forceinline__ void accumulate(float fac, float dx, float dy, float dz, float dui) {
    if (KAHAN) {
      add_comp(ax, cx, -fac * dx);
      add_comp(ay, cy, -fac * dy);
      add_comp(az, cz, -fac * dz);
      add_comp(du, cu, dui);
    } else {
      ax = fmaf(-fac, dx, ax);
      ay = fmaf(-fac, dy, ay);
      az = fmaf(-fac, dz, az);
      du += dui;
    }
    ++c;
  }
};

// ---------------------------------------------------------------- third tier
//
// Targets whose group outgrew both stages or its task slots (a large-h
// particle beside a dense clump can have thousands of particles inside its h
// while its weighted neighbour number is 48), or whose h outgrew the staged
// radius, are done one warp per target: the warp walks the octrees of the 27
// neighbouring top cells with the target's own sphere and streams the
// particles of every leaf it reaches from global memory (kU loads in flight
// per lane), reducing its lanes' partial sums by shuffles in fixed order. No
// stage and no task slots, so no capacity limit but the frontier's.

constexpr int kSWarps = 4;       // warps per third-tier block
constexpr int kSStack = 1536;    // node stack entries per warp

// Calls f(q, j) for every particle j (q: position shifted into the group
// frame, mass) of every leaf whose box lies within reach of the point xt
// (top-cell-relative): reach = R, or max(R, hmax_S) when FORCE. The walk is
// depth first with a warp-wide stack: each round pops up to 32 nodes (fewer
// when the stack is nearly full, so 8 children per popped node always fit),
// streams the passing leaves and pushes the passing inner nodes' children.
// Deterministic order. Returns false if the stack overflowed anyway (the
// sums are then incomplete).
template <bool FORCE, class F>
__device__ bool walk_stream(const Node *nodes, const Leaf *leaves, const float4 *pm,
                            const BoxDev &B, const Group &G, const float xt[3], float R,
                            int lane, int2 *stk, F &&f) {
  const unsigned ltmask = (1u << lane) - 1u;
  int c[3];
  cell_xyz(B, G.cell - B.cell_base, c);
  if (lane < 27) {
    const int dx = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dz = lane % 3 - 1;
    const int nc[3] = {(c[0] + dx + B.n[0]) % B.n[0], (c[1] + dy + B.n[1]) % B.n[1],
                       (c[2] + dz + B.n[2]) % B.n[2]};
    stk[26 - lane] = make_int2(B.cell_base + (nc[0] * B.n[1] + nc[1]) * B.n[2] + nc[2], lane);
  }
  __syncwarp();
  int n = 27;
  bool ok = true;
  while (n > 0) {
    int k = min(32, n);
    const int room = (kSStack - n) / 7;  // pops whose 8 children fit after the pop
    if (k > room) k = room > 0 ? room : 1;
    bool leaf_in = false, inner_in = false;
    int code = 0, child = 0, leaf = 0;
    if (lane < k) {
      const int2 e = stk[n - 1 - lane];
      code = e.y;
      const Node &S = nodes[e.x];
      if (S.count > 0) {
        const int dx = code / 9 - 1, dy = (code / 3) % 3 - 1, dz = code % 3 - 1;
        const float sh[3] = {dx * B.wf[0], dy * B.wf[1], dz * B.wf[2]};
        float d2 = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float gap = fmaxf(0.f, fmaxf(S.lo[d] + sh[d] - xt[d], xt[d] - S.hi[d] - sh[d]));
          d2 = fmaf(gap, gap, d2);
        }
        const float crit = (FORCE ? fmaxf(R, S.hmax) : R) + B.eps;
        if (d2 < crit * crit) {
          child = S.child;
          leaf = S.leaf;
          leaf_in = child < 0;
          inner_in = child >= 0;
        }
      }
    }
    __syncwarp();
    n -= k;
    // stream the passing leaves, one at a time, all lanes on its particles
    unsigned ml = __ballot_sync(0xffffffffu, leaf_in);
    while (ml) {
      const int src = __ffs(ml) - 1;
      ml &= ml - 1;
      const int lf = __shfl_sync(0xffffffffu, leaf, src);
      const int cd = __shfl_sync(0xffffffffu, code, src);
      const Leaf &LS = leaves[lf];
      const int dx = cd / 9 - 1, dy = (cd / 3) % 3 - 1, dz = cd % 3 - 1;
      const float sx = (float)(LS.o[0] + dx * B.w[0] - G.o[0]);
      const float sy = (float)(LS.o[1] + dy * B.w[1] - G.o[1]);
      const float sz = (float)(LS.o[2] + dz * B.w[2] - G.o[2]);
      for (int kk = lane; kk < LS.count; kk += 32) {
        const int j = LS.start + kk;
        float4 q = pm[j];
        q.x += sx;
        q.y += sy;
        q.z += sz;
        f(q, j);
      }
    }
    // push the children of passing inner nodes (last pushed is popped first)
    const unsigned mi = __ballot_sync(0xffffffffu, inner_in);
    if (inner_in) {
      const int pos = n + 8 * __popc(mi & ltmask);
      for (int o = 0; o < 8; ++o)
        if (pos + o < kSStack) stk[pos + o] = make_int2(child + 7 - o, code);
    }
    n += 8 * __popc(mi);
    if (n > kSStack) {
      ok = false;
      break;
    }
    __syncwarp();
  }
  __syncwarp();
  return ok;
}

// Warp-wide sum in fixed (xor-tree) order: every lane gets the same total.
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Top-cell-relative position of particle i and its position in the group frame.
__device__ __forceinline__ void target_pos(const Leaf *leaves, const int *leaf_of,
                                           const float4 *pm, const Group &G, int i, float xt[3],
                                           float p[3]) {
  const Leaf &L = leaves[leaf_of[i]];
  const float4 q = pm[i];
  const float qq[3] = {q.x, q.y, q.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xt[d] = (float)(L.o[d] + (double)qq[d]);
    p[d] = qq[d] + (float)(L.o[d] - G.o[d]);
  }
}

template <bool KAHAN>
__global__ void __launch_bounds__(kSWarps * 32) k_density_stream(BatchDensArgs a) {
  __shared__ int2 stack[kSWarps][kSStack];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nq = a.ctr->queued2[0];
  unsigned long long ntest = 0, inter = 0;
  int fallback = 0, max_it = 0, st_bits = 0;
  int why[2] = {0, 0};
  for (int e = blockIdx.x * kSWarps + warp; e < nq * kSub; e += gridDim.x * kSWarps) {
    const int code = a.queue2[e / kSub];
    const int g = code / kNW, tloc = (code % kNW) * kSub + e % kSub;
    const Group G = a.groups[g];
    if (tloc >= G.count) continue;
    const int i = G.start + tloc;
    if (a.done[i]) continue;  // finished by an earlier tier
    const BoxDev &B = a.boxes[G.box];
    const float wmin = fminf(B.wf[0], fminf(B.wf[1], B.wf[2]));
    const float hcap = (float)B.hcap;
    float xt[3], p[3];
    target_pos(a.leaves, a.leaf_of, a.pm, G, i, xt, p);
    HIterF it;
    it.start(a.hf[i]);
    bool fin = false, failed = false;
    int passes = 0, ngb = 0;
    float4 fs = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int pass = 0; pass < a.max_iter; ++pass) {
      const float hf = it.h;
      if (hf * (1.f + 1e-6f) > wmin) {  // the 27 neighbouring top cells no longer cover h:
        failed = true;                   // keep the grown h for the regrid, which the
        st_bits |= kErrHGrid;            // caller runs before the next attempt
        if (lane == 0) {
          a.h[i] = (double)hf;
          a.hf[i] = hf;
        }
        break;
      }
      const float h2 = hf * hf, hinv = 1.f / hf;
      DensAcc<KAHAN> acc;
      int seen = 0;
      const bool ok = walk_stream<false>(a.nodes, a.leaves, a.pm, B, G, xt, hf, lane,
                                         stack[warp], [&](float4 q, int) {
                                           acc.add(q, p[0], p[1], p[2], h2, hinv);
                                           ++seen;
                                         });
      ntest += seen;
      if (!ok) {
        failed = true;
        break;
      }
      const float4 tot = make_float4(warp_sum_f(acc.sw), warp_sum_f(acc.sdw),
                                     warp_sum_f(acc.smw), warp_sum_f(acc.smdh));
      int ctot = acc.c;
      for (int o = 16; o; o >>= 1) ctot += __shfl_xor_sync(0xffffffffu, ctot, o);
      ++passes;
      int st = 0;
      const bool conv = h_newton_step_f(it, tot.x, tot.y, a.n_ngb, a.tol * a.n_ngb, hcap, &st);
      st_bits |= st;
      if (conv) {
        fin = true;
        fs = tot;
        ngb = ctot - 1;
        break;
      }
    }
    if (!fin) {  // left to the per-pass form
      if (lane == 0) {
        ++fallback;
        ++why[failed ? 0 : 1];
      }
      continue;
    }
    if (lane == 0) {
      float rho, omega, P;
      float4 fi;
      if (!finalise_density(it.h, fs, a.vu[i].w, (float)(a.gamma - 1.0), &rho, &omega, &P, &fi))
        st_bits |= kErrNonPhysical;
      a.h[i] = (double)it.h;
      a.hf[i] = it.h;
      a.rho[i] = rho;
      a.omega[i] = omega;
      a.P[i] = P;
      a.fi[i] = fi;
      a.nngb[i] = ngb;
      a.niter[i] = passes;
      a.done[i] = 1;
      inter += (unsigned long long)ngb;
      max_it = max(max_it, passes);
    }
  }
  ntest = warp_sum(ntest);
  inter = warp_sum(inter);
  fallback = (int)warp_sum((unsigned long long)fallback);
  max_it = warp_max_int(max_it);
  for (int o = 16; o; o >>= 1) st_bits |= __shfl_xor_sync(0xffffffffu, st_bits, o);
  const int w1 = (int)warp_sum((unsigned long long)why[0]);
  const int w2 = (int)warp_sum((unsigned long long)why[1]);
  if (lane == 0) {
    if (ntest) atomicAdd(&a.ctr->dens_cand, ntest);
    if (inter) atomicAdd(&a.ctr->dens_inter, inter);
    if (fallback) {
      atomicAdd(&a.ctr->unconverged, fallback);
      atomicAdd(&a.ctr->fallback, fallback);
    }
    if (w1) atomicAdd(&a.ctr->why[0], w1);
    if (w2) atomicAdd(&a.ctr->why[1], w2);
    if (max_it) atomicMax(&a.ctr->max_iter_used, max_it);
    if (st_bits) atomicOr(&a.ctr->status, st_bits);
  }
}

template <bool KAHAN>
__global__ void __launch_bounds__(kSWarps * 32) k_force_stream(BatchForceArgs a) {
  __shared__ int2 stack[kSWarps][kSStack];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nq = a.ctr->queued2[1];
  unsigned long long ntest = 0, inter = 0;
  int fallback = 0;
  for (int e = blockIdx.x * kSWarps + warp; e < nq * kSub; e += gridDim.x * kSWarps) {
    const int code = a.queue2[e / kSub];
    const int g = code / kNW, tloc = (code % kNW) * kSub + e % kSub;
    const Group G = a.groups[g];
    if (tloc >= G.count) continue;
    const int i = G.start + tloc;
    const BoxDev &B = a.boxes[G.box];
    float xt[3], p[3];
    target_pos(a.leaves, a.leaf_of, a.pm, G, i, xt, p);
    const float4 fi = a.fi[i], vi = a.vu[i];
    ForceAcc<KAHAN> acc;
    int seen = 0;
    const bool ok = walk_stream<true>(
        a.nodes, a.leaves, a.pm, B, G, xt, fi.x, lane, stack[warp],
        [&](float4 q, int j) {
          ++seen;
          const float dx = p[0] - q.x, dy = p[1] - q.y, dz = p[2] - q.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (!(r2 > 0.f)) return;
          const float4 fj = a.fi[j];
          if (!(r2 < fmaxf(fi.w, fj.w))) return;
          const float rinv = rsqrtf(r2);
          const float r = r2 * rinv;
          const float ti = fi.z * dw_only(r * fi.y);  // A_i dW/dr(r, h_i)
          const float tj = fj.z * dw_only(r * fj.y);  // A_j dW/dr(r, h_j)
          const float fac = q.w * (ti + tj) * rinv;
          const float4 vj = a.vu[j];
          const float dvdx = (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
          acc.accumulate(fac, dx, dy, dz, q.w * ti * rinv * dvdx);
        });
    ntest += seen;
    if (!ok) {  // left to the per-pass form
      if (lane == 0) ++fallback;
      continue;
    }
    const float ax = warp_sum_f(acc.ax), ay = warp_sum_f(acc.ay), az = warp_sum_f(acc.az),
                du = warp_sum_f(acc.du);
    int c = acc.c;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
      a.acc[i] = make_float4(ax, ay, az, du);
      a.nforce[i] = c;
      a.fdone[i] = 1;
      inter += (unsigned long long)c;
    }
  }
  ntest = warp_sum(ntest);
  inter = warp_sum(inter);
  fallback = (int)warp_sum((unsigned long long)fallback);
  if (lane == 0) {
    if (ntest) atomicAdd(&a.ctr->force_cand, ntest);
    if (inter) atomicAdd(&a.ctr->force_inter, inter);
    if (fallback) {
      atomicAdd(&a.ctr->unconverged, fallback);
      atomicAdd(&a.ctr->fallback, fallback);
      atomicAdd(&a.ctr->why[2], fallback);
    }
  }
}

// ---------------------------------------------------- task cost ordering
//
// The queue is ordered by chunks of kClaim consecutive groups (one claim
// each), so that a block still runs neighbouring groups one after another
// (their stages overlap in L1) while the chunks go costliest first.

__device__ __forceinline__ float group_cost(const Group *groups, const int *tcount,
                                            const float *cost, int g) {
  const float c = cost[g];
  return c > 0.f ? c : 64.f * (float)groups[g].count * (float)max(tcount[g], 1);
}

// c > 0: its bits order like an unsigned integer; exponent and the top three
// mantissa bits give eight bins per octave, the costliest first.
__device__ __forceinline__ int cost_bin(float c) {
  const unsigned k = min(__float_as_uint(c) >> 20, (unsigned)(kCostBins - 1));
  return kCostBins - 1 - (int)k;
}

// One warp per chunk: its summed cost's bin into cbin[chunk] and the
// histogram.
__global__ void k_chunk_cost(const Group *groups, int n, const int *tcount, const float *cost,
                             int *cbin, int *bins) {
  __shared__ int h[kCostBins];
  for (int b = threadIdx.x; b < kCostBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int n_chunks = (n + kClaim - 1) / kClaim;
  for (int ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < n_chunks;
       ch += (gridDim.x * blockDim.x) >> 5) {
    const int g = ch * kClaim + lane;
    float c = g < n ? group_cost(groups, tcount, cost, g) : 0.f;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
      const int b = cost_bin(fmaxf(c, 1.f));
      cbin[ch] = b;
      atomicAdd(&h[b], 1);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kCostBins; b += blockDim.x)
    if (h[b]) atomicAdd(&bins[b], h[b]);
}

// One block of kCostBins / 2 threads: bins become their exclusive prefix
// sums (the first queue chunk of each bin); the queue heads are zeroed.
__global__ void k_cost_scan(int *bins, int *heads, int n_heads) {
  __shared__ int wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int v0 = bins[2 * t], v1 = bins[2 * t + 1];
  int incl = v0 + v1;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;  // inclusive over the warps
  }
  __syncthreads();
  const int ex = incl - v0 - v1 + (warp ? wsum[warp - 1] : 0);
  bins[2 * t] = ex;
  bins[2 * t + 1] = ex + v0;
  if (t < n_heads) heads[t] = 0;
}

// One warp per chunk: the chunk takes its bin's next queue chunk and lays
// its groups out there (-1 past the last group).
__global__ void k_chunk_scatter(int n, const int *cbin, int *bins, int *order) {
  const int lane = threadIdx.x & 31;
  const int n_chunks = (n + kClaim - 1) / kClaim;
  for (int ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < n_chunks;
       ch += (gridDim.x * blockDim.x) >> 5) {
    int pos = 0;
    if (lane == 0) pos = atomicAdd(&bins[cbin[ch]], 1);
    pos = __shfl_sync(0xffffffffu, pos, 0);
    const int g = ch * kClaim + lane;
    order[pos * kClaim + lane] = g < n ? g : -1;
  }
}

void launch_cost_order(const Group *groups, int n_groups, const int *tcount, const float *cost,
                       int *order, int *bins, int *cbin, int *heads, int n_heads,
                       cudaStream_t s) {
  static_assert(kCostBins == 2048, "k_cost_scan holds two bins per thread of one block");
  static_assert(kClaim == 32, "a chunk is one warp's lanes");
  if (n_groups <= 0) return;
  cudaMemsetAsync(bins, 0, sizeof(int) * kCostBins, s);
  const int n_chunks = (n_groups + kClaim - 1) / kClaim;
  const int blocks = std::min((n_chunks + 7) / 8, 152 * 8);
  k_chunk_cost<<<blocks, 256, 0, s>>>(groups, n_groups, tcount, cost, cbin, bins);
  note_launch();
  k_cost_scan<<<1, kCostBins / 2, 0, s>>>(bins, heads, n_heads);
  note_launch();
  k_chunk_scatter<<<blocks, 256, 0, s>>>(n_groups, cbin, bins, order);
  note_launch();
}

// ------------------------------------------------------ tile 2 partition

__global__ void k_bin_flag(const int *gstage, int n, int fit, int *flag) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) flag[g] = gstage[g] >= 0 && gstage[g] <= fit ? 1 : 0;
  if (g == n) flag[g] = 0;
}

__global__ void k_bin_scatter(int n, const int *flag, const int *excl, int *order, int *split) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int ns = excl[n];
  order[flag[g] ? excl[g] : ns + g - excl[g]] = g;
  if (g == 0) *split = ns;
}

void launch_force_bins(const int *gstage, int n_groups, int fit, int *flag, int *excl,
                       void *scan_tmp, size_t scan_tmp_bytes, int *order, int *split,
                       cudaStream_t s) {
  if (n_groups <= 0) return;
  const int nb = (n_groups + 1 + 255) / 256;
  k_bin_flag<<<nb, 256, 0, s>>>(gstage, n_groups, fit, flag);
  note_launch();
  exclusive_scan_int(flag, excl, n_groups + 1, scan_tmp, scan_tmp_bytes, s);
  k_bin_scatter<<<nb, 256, 0, s>>>(n_groups, flag, excl, order, split);
  note_launch();
}

// Blocks of `kernel` resident on the whole GPU at once (the grid of a
// launch that claims its groups from a work queue).
template <class K>
int resident_blocks(K kernel, int bytes) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kNW * 32, bytes);
  return std::max(per, 1) * std::max(sms, 1);
}

template <bool KAHAN, int NS, bool REUSE = false, bool MID = false>
void launch_density_tier(const BatchDensArgs &a, int tier, int blocks, cudaStream_t s) {
  static bool attr = false;
  static int resident = 0;
  const int bytes = (int)sizeof(DensSmem<NS>);
  if (!attr) {
    cudaFuncSetAttribute(k_density_batched<KAHAN, NS, REUSE, MID>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    resident = resident_blocks(k_density_batched<KAHAN, NS, REUSE, MID>, bytes);
    attr = true;
  }
  if (tier == 0 && a.wq.head) blocks = std::min(a.n_groups, resident);
  k_density_batched<KAHAN, NS, REUSE, MID><<<blocks, kNW * 32, bytes, s>>>(a, tier);
  note_launch();
}

// The first tier: with the neighbour cache, the groups on their stored stage
// first, then those that stage anew.
template <bool KAHAN, int NS>
void launch_density_first(const BatchDensArgs &a, int blocks, cudaStream_t s) {
  if (a.cache_on) launch_density_tier<KAHAN, NS, true>(a, 0, blocks, s);
  launch_density_tier<KAHAN, NS, false>(a, 0, blocks, s);
}

__global__ void k_cache_init(CacheCtl *ctl, int n_groups) {
  ctl->build_all = 1;
  ctl->fail = 0;
  ctl->n_groups = n_groups;
  ctl->lfail = 0;
  ctl->force_off = 0;
  ctl->fused = n_groups;  // the first force call tries
  ctl->probe = 0;
}

__global__ void k_force_gate(CacheCtl *ctl) {
  if (ctl->force_off) {  // skipping: count down to the next try
    if (--ctl->probe <= 0) ctl->force_off = 0;
  } else if (ctl->fused * 8 < ctl->n_groups) {  // the last try paid too little
    ctl->force_off = 1;
    ctl->probe = 15;
  }
  if (!ctl->force_off) ctl->fused = 0;  // counted afresh by this call's far walk
}

void launch_force_gate(CacheCtl *ctl, cudaStream_t s) {
  k_force_gate<<<1, 1, 0, s>>>(ctl);
  note_launch();
}

void launch_cache_init(CacheCtl *ctl, int n_groups, cudaStream_t s) {
  k_cache_init<<<1, 1, 0, s>>>(ctl, n_groups);
  note_launch();
}

__global__ void k_cache_decide(CacheCtl *ctl) {
  ctl->build_all = (ctl->fail * 8 > ctl->n_groups || ctl->lfail * 2 > ctl->n_groups) ? 1 : 0;
  ctl->fail = 0;
  ctl->lfail = 0;
}

void launch_cache_decide(CacheCtl *ctl, cudaStream_t s) {
  k_cache_decide<<<1, 1, 0, s>>>(ctl);
  note_launch();
}

int cache_stage_slots(int tile) { return tile ? kStageDL : kStageD; }
int cache_lane_cap(int tile) { return dens_lane(tile ? kStageDL : kStageD); }

// Tier 0 over every group; tier 1 over the groups tier 0 queued, restaged by
// each target's own radius at the first tier's stage size (same occupancy);
// tier 2 (large stage, 2 blocks per SM) over those whose tight stage still
// outgrew it; then the third tier. `a.ctr` queue counts must be zeroed and
// the queues sized for n_groups by the caller.
template <bool KAHAN>
void launch_density_tiers(const BatchDensArgs &a, int blocks, int big, cudaStream_t s) {
  if (a.tile) {
    launch_density_first<KAHAN, kStageDL>(a, blocks, s);
    launch_density_tier<KAHAN, kStageDL, false, true>(a, 1, blocks, s);
  } else {
    launch_density_first<KAHAN, kStageD>(a, blocks, s);
    launch_density_tier<KAHAN, kStageD, false, true>(a, 1, blocks, s);
  }
  launch_density_tier<KAHAN, kBigStageD>(a, 2, big, s);
  k_density_stream<KAHAN><<<152 * 8, 128, 0, s>>>(a);
  note_launch();
}

void launch_density_batched(const BatchDensArgs &a, cudaStream_t s) {
  if (a.n_groups <= 0) return;
  const int blocks = a.n_groups < 152 * 64 ? a.n_groups : 152 * 64;
  const int big = a.n_groups < 152 * 2 ? a.n_groups : 152 * 2;
  if (a.kahan)
    launch_density_tiers<true>(a, blocks, big, s);
  else
    launch_density_tiers<false>(a, blocks, big, s);
}


template <bool KAHAN, int NS, bool MID>
__global__ void __launch_bounds__(kNW * 32, force_min_blocks(NS))
    k_force_batched(BatchForceArgs a, int tier) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ForceSmem<NS> &S = *reinterpret_cast<ForceSmem<NS> *>(smem_raw);
  // the second and later tiers stage by each target's own radius
  constexpr bool TIGHT = MID || NS == kBigStageF;
  constexpr int CANDF = force_cand(NS);
  constexpr int LANE = force_lane(NS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slice = lane & (kSlice - 1);
  unsigned short *cand = S.cand[warp];
  unsigned short *list = S.list[warp];
  unsigned long long ntest = 0, inter = 0;
  int stage_max = 0, n_direct[2] = {0, 0};
  if (threadIdx.x == 0) {  // read after a barrier
    S.sq[NS] = make_float4(kFar, kFar, kFar, 0.f);
    S.sf[NS] = make_float2(0.f, 1.f);
    S.sj[NS] = 0;
  }

  const int ng = tier_count(tier, a.n_groups, &a.ctr->queued[1], &a.ctr->queued_big[1]);
  GroupCursor cur;
  cur.dyn = tier == 0 && a.wq.head != nullptr;
  // tile 2: this launch's part of the partitioned groups (with its own queue head)
  const bool binned = tier == 0 && a.bin > 0;
  const int blo = binned ? (a.bin == 2 ? *a.bsplit : 0) : 0;
  const int bhi = binned ? (a.bin == 2 ? a.n_groups : *a.bsplit) : 0;
  WorkQueue wq = a.wq;
  if (binned) {
    wq.order = a.border + blo;
    if (wq.head) wq.head += a.bin - 1;
  }
  const int qn = binned ? bhi - blo : (cur.dyn ? queue_positions(a.wq, ng) : ng);
  // groups done on the cache (fuse[g], unless the cached force is off in this call)
  const unsigned char *fuse =
      tier == 0 && a.cache_on && !a.cache.ctl->force_off ? a.cache.fuse : nullptr;
  for (int q = cur.first(wq, 0, fuse, false, S.qslot, qn); q < qn;
       q = cur.next(wq, 0, fuse, false, S.qslot, qn, q)) {
    const int g = binned ? a.border[blo + q]
                         : (cur.dyn ? (wq.order ? wq.order[q] : q)
                                    : tier_group(tier, q, a.queue, a.queue_big));
    if (fuse && fuse[g]) continue;  // done on the cache
    cur.run(S.qslot, g);
    const Group G = a.groups[g];
    const int nt = a.tcount[g];
    const int e0 = g * a.tcap;
    if (TIGHT) __syncthreads();  // the previous group's warps are done with the smem
    if (TIGHT && threadIdx.x < 32) {  // tight stage: each target's own h
      float4 t = make_float4(0.f, 0.f, 0.f, -1.f);
      if ((int)threadIdx.x < G.count) {
        const int it = G.start + threadIdx.x;
        const float4 pq = a.gpos[it];
        t = make_float4(pq.x, pq.y, pq.z, a.fi[it].x);
      }
      S.tgt[threadIdx.x] = t;  // read after stage_group's opening barrier
    }
    const StageRange sr =
        stage_group<true>(nullptr, &a, G, e0, e0 + min(nt, a.tcap), warp, lane, G.hmax, S.sq,
                          S.sf, S.sj, S.wcount, (unsigned char *)cand, NS,
                          TIGHT ? S.tgt : nullptr);
    // for tile 2: the stage this group needs (2 x the larger pair of warp shares)
    if (tier == 0 && a.gstage && threadIdx.x == 0) a.gstage[g] = sr.need;
    stage_max = max(stage_max, sr.total);
    if (sr.over || nt > a.tcap) {  // block-uniform
      if (MID && nt <= a.tcap) {  // the tight stage outgrew this size: the large one
        if (threadIdx.x == 0) a.queue_big[atomicAdd(&a.ctr->queued_big[1], 1)] = g;
      } else if (threadIdx.x < kNW && (TIGHT || nt > a.tcap)) {  // the third tier walks them
        a.queue2[atomicAdd(&a.ctr->queued2[1], 1)] = g * kNW + threadIdx.x;
      } else if (threadIdx.x == 0 && !TIGHT && nt <= a.tcap) {  // second tier: tight stage
        a.queue[atomicAdd(&a.ctr->queued[1], 1)] = g;
      }
      continue;
    }
    const int tloc = warp * kSub + (lane >> 2);
    const bool has = tloc < G.count;
    const int i = G.start + tloc;
    float px = 0.f, py = 0.f, pz = 0.f;
    float4 fi = make_float4(1.f, 1.f, 0.f, -1.f), vi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (has) {
      const float4 q = a.gpos[i];
      px = q.x;
      py = q.y;
      pz = q.z;
      fi = a.fi[i];
      vi = a.vu[i];
    }
    if (!__any_sync(0xffffffffu, has)) continue;
    float blo[3], bhi[3];
    sub_box(has, px, py, pz, blo, bhi);
    float hm = has ? fi.x : 0.f;
    for (int o = 16; o; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
    const float hi2 = has ? fi.w : -1.f;
    ForceAcc<KAHAN> acc;
    if constexpr (NS == kStageF) {
      // tile 0 (inputs without strong clumps): one filter of the stage into
      // cand, one list per lane; a warp whose list outgrows LANE reads its
      // candidates directly, one whose candidates outgrow CANDF reads the
      // whole stage (rare here; the lean loop keeps this tile's registers)
      const int ncand = filter_stage<true>(S.sq, S.sf, sr, blo, bhi, hm, cand, CANDF, lane);
      int mode = ncand > CANDF ? 2 : 0;  // ncand is warp-uniform
      int cnt = 0;
      if (mode == 0) {
#pragma unroll 4
        for (int t = slice; t < ncand; t += kSlice) {
          const int k = cand[t];
          const float4 q = S.sq[k];
          const float hj2 = S.sf[k].y;
          const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          if (has && r2 > 0.f && r2 < fmaxf(hi2, hj2)) {
            if (cnt < LANE) list[cnt * 32 + lane] = (unsigned short)k;
            ++cnt;
          }
        }
        if (has) ntest += (ncand + kSlice - 1 - slice) / kSlice;
        if (__any_sync(0xffffffffu, cnt > LANE)) {
          mode = 1;
        } else {  // pad every lane's list with the sentinel to the warp's longest, x4
          const int tpad = (warp_max_int(cnt) + 3) & ~3;
          for (int t = cnt; t < tpad; ++t) list[t * 32 + lane] = (unsigned short)NS;
        }
        __syncwarp();
      }
      if (mode == 0) {
        const int tmax = (warp_max_int(has ? cnt : 0) + 3) & ~3;
        for (int t = 0; t < tmax; t += 4) {
          int k[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) k[u] = list[(t + u) * 32 + lane];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc.add(S, k[u], a.vu, px, py, pz, fi, vi, -1.f, NS);
        }
        if (has) ntest += cnt;
      } else {
        const int nsrc = mode == 1 ? ncand : sr.total;
        if (has)
          for (int t = slice; t < nsrc; t += kSlice)
            acc.add(S, mode == 1 ? (int)cand[t] : sr.index(t), a.vu, px, py, pz, fi, vi, hi2);
        if (has) ntest += (nsrc + kSlice - 1 - slice) / kSlice;
      }
      if (lane == 0 && mode) ++n_direct[mode - 1];
    } else {
      // tile 1 and the second tier (clumped inputs): the stage is filtered
      // in chunks of at most CANDF candidates, and each chunk's per-lane
      // lists are built and summed in rounds of at most LANE entries per
      // lane (a lane resumes its scan where its last round stopped). The
      // common case is one chunk and one round; every case sums the same
      // pairs in the same per-lane order.
      int sp = 0, chunks = 0, rounds = 0;  // sp: next stage entry to filter (warp-uniform)
      while (sp < sr.total) {
        const int ncand = filter_chunk(S.sq, S.sf, sr, sp, blo, bhi, hm, cand, CANDF, lane);
        ++chunks;
        int tpos = has ? slice : ncand;  // this lane's next candidate
        bool first = true;
        do {
          const int t0 = tpos;
          int cnt = 0;
          if (first) {  // scan every candidate; note where the list filled up
            int tres = ncand;
  #pragma unroll 4
            for (; tpos < ncand; tpos += kSlice) {
              const int k = cand[tpos];
              const float4 q = S.sq[k];
              const float hj2 = S.sf[k].y;
              const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              if (r2 > 0.f && r2 < fmaxf(hi2, hj2)) {
                if (cnt < LANE)
                  list[cnt * 32 + lane] = (unsigned short)k;
                else if (cnt == LANE)
                  tres = tpos;  // the first neighbour left out: the next round starts here
                ++cnt;
              }
            }
            if (cnt > LANE) {
              cnt = LANE;
              tpos = tres;
            }
            first = false;
          } else {  // later rounds stop as soon as the list is full
  #pragma unroll 4
            for (; tpos < ncand; tpos += kSlice) {
              const int k = cand[tpos];
              const float4 q = S.sq[k];
              const float hj2 = S.sf[k].y;
              const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              if (r2 > 0.f && r2 < fmaxf(hi2, hj2)) {
                list[cnt * 32 + lane] = (unsigned short)k;
                if (++cnt == LANE) {
                  tpos += kSlice;
                  break;
                }
              }
            }
          }
          ntest += (max(tpos, t0) - t0) / kSlice + cnt;
          // pad every lane's list with the sentinel to the warp's longest, x4
          const int tmax = (warp_max_int(cnt) + 3) & ~3;
          for (int t = cnt; t < tmax; ++t) list[t * 32 + lane] = (unsigned short)NS;
          __syncwarp();
          for (int t = 0; t < tmax; t += 4) {
            int k[4];
  #pragma unroll
            for (int u = 0; u < 4; ++u) k[u] = list[(t + u) * 32 + lane];
  #pragma unroll
            for (int u = 0; u < 4; ++u) acc.add(S, k[u], a.vu, px, py, pz, fi, vi, -1.f, NS);
          }
          ++rounds;
          __syncwarp();  // the next round rewrites the lists
        } while (__any_sync(0xffffffffu, tpos < ncand));
      }
      if (lane == 0) {
        n_direct[0] += rounds > chunks;
        n_direct[1] += chunks > 1;
      }
    }
    int cnt = acc.c;
    float ax = acc.ax, ay = acc.ay, az = acc.az, du = acc.du;
    ax = slice_sum(ax);
    ay = slice_sum(ay);
    az = slice_sum(az);
    du = slice_sum(du);
    int ctot = cnt;
    ctot += __shfl_xor_sync(0xffffffffu, ctot, 1);
    ctot += __shfl_xor_sync(0xffffffffu, ctot, 2);
    if (has && slice == 0) {
      a.acc[i] = make_float4(ax, ay, az, du);
      a.nforce[i] = ctot;
      a.fdone[i] = 1;
      inter += (unsigned long long)ctot;
    }
  }
  ntest = warp_sum(ntest);
  inter = warp_sum(inter);
  if (lane == 0) {
    if (ntest) atomicAdd(&a.ctr->force_cand, ntest);
    if (inter) atomicAdd(&a.ctr->force_inter, inter);
    atomicMax(&a.ctr->stage_max[1], stage_max);
    if (n_direct[0]) atomicAdd(&a.ctr->direct[0], n_direct[0]);
    if (n_direct[1]) atomicAdd(&a.ctr->direct[1], n_direct[1]);
  }

}

// ------------------------------------------------- force on the cache
//
// Groups whose density finished in the first tier on per-lane lists, with no
// particle outside their stage able to reach them (fuse[g], set by the
// far-reacher walk), take the force from the density's stored stage and
// lists: no walk, no staging tests, no filter, no list build. A target's
// pairs r < max(h_i, h_j) are (a) its listed entries, each tested, and (b)
// staged j whose own h reaches it from beyond its list: a staged j missing
// from i's list lies at r >= rl_i - dpath_i - D >= thr (the list's radius
// less the motion since it was built), so only j with h_j > thr can add a
// pair; those are taken from the stage 32 at a time, and a per-target bitmap
// of the listed entries keeps each pair once.
template <int NSD>
struct ForceReuseSmem {
  unsigned dmax_bits;
  unsigned pad_[3];
  float4 sq[NSD + 1];                  // position in the group frame, m; [NSD] sentinel
  float2 sf[NSD + 1];                  // A (8/pi) h^-4, h^2
  int sj[NSD + 1];                     // particle index
  unsigned bm[kNW][kSub][(NSD + 32) / 32];  // listed stage entries per target
};

constexpr int force_reuse_min_blocks(int nsd) { return nsd == kStageD ? 6 : 4; }
static_assert(sizeof(unsigned) * kNW * kSub * ((kStageD + 32) / 32) >= 12 * 384,
              "the force-on-cache bitmap space holds the task shifts while the stage loads");

template <bool KAHAN, int NSD>
__global__ void __launch_bounds__(kNW * 32, force_reuse_min_blocks(NSD))
    k_force_reuse(BatchForceArgs a) {
  if (a.cache.ctl->force_off) return;  // the cached force is skipped in this call
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ForceReuseSmem<NSD> &S = *reinterpret_cast<ForceReuseSmem<NSD> *>(smem_raw);
  constexpr int BMW = (NSD + 32) / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slice = lane & (kSlice - 1);
  unsigned long long ntest = 0, inter = 0;
  if (threadIdx.x == 0) {  // read after a barrier
    S.sq[NSD] = make_float4(kFar, kFar, kFar, 0.f);
    S.sf[NSD] = make_float2(0.f, 1.f);
    S.sj[NSD] = 0;
  }
  const CacheArgs &C = a.cache;
  for (int g = blockIdx.x; g < a.n_groups; g += gridDim.x) {
    if (!C.fuse[g]) continue;  // block-uniform
    const Group G = a.groups[g];
    const GroupCache &M = C.meta[g];
    int wc[4];
    for (int w = 0; w < 4; ++w) wc[w] = M.wc[w];
    const int ntask = min(C.tcount[g], a.tcap);
    float Dst;
    const StageRange sr = load_stage_cached<true>(
        C, g, wc, C.tasks + (size_t)g * a.tcap, ntask, a.pm, a.fi, S.sq, S.sf, S.sj, NSD,
        reinterpret_cast<float *>(&S.bm[0][0][0]), &S.dmax_bits, &Dst);
    const int tloc = warp * kSub + (lane >> 2);
    const bool has = tloc < G.count;
    if (!__any_sync(0xffffffffu, has)) continue;
    const int i = G.start + tloc;
    float px = 0.f, py = 0.f, pz = 0.f, thr = 3e38f;
    float4 fi = make_float4(1.f, 1.f, 0.f, -1.f), vi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (has) {
      const float4 q = a.gpos[i];
      px = q.x;
      py = q.y;
      pz = q.z;
      fi = a.fi[i];
      vi = a.vu[i];
      thr = C.rl[i] - C.dpath[i] - Dst;
    }
    for (int o = 16; o; o >>= 1) thr = fminf(thr, __shfl_xor_sync(0xffffffffu, thr, o));
    const float thr2 = thr > 0.f ? thr * thr : -1.f;
    unsigned *bm = S.bm[warp][lane >> 2];
    for (int t = lane; t < kSub * BMW; t += 32) S.bm[warp][t / BMW][t % BMW] = 0u;
    __syncwarp();
    const int tp = M.tpad[warp];
    const size_t lrow = ((size_t)g * kNW + warp) * C.lane_cap * 32;
    ForceAcc<KAHAN> acc;
    // (a) listed entries (sentinel padded, x4), 8 rows per round trip
    for (int t = 0; t < tp; t += 8) {
      int k[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) k[u] = t + u < tp ? C.list[lrow + (t + u) * 32 + lane] : NSD;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (!has || t + u >= tp) continue;
        if (k[u] < NSD) atomicOr(&bm[k[u] >> 5], 1u << (k[u] & 31));
        acc.add(S, k[u], a.vu, px, py, pz, fi, vi, fi.w, NSD);
      }
    }
    if (has) ntest += tp;
    __syncwarp();
    // (b) staged j with h_j > thr, not listed for the target, r < h_j
    int turn = 0;
    for (int tb = 0; tb < sr.total; tb += 32) {
      const int t = tb + lane;
      int k = NSD;
      bool in = false;
      if (t < sr.total) {
        k = sr.index(t);
        in = S.sf[k].y > thr2;
      }
      unsigned m = __ballot_sync(0xffffffffu, in);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int kk = __shfl_sync(0xffffffffu, k, src);
        const bool listed = (bm[kk >> 5] >> (kk & 31)) & 1u;
        if (has && !listed && slice == (turn & 3)) {
          acc.add(S, kk, a.vu, px, py, pz, fi, vi, fi.w, NSD);
          ++ntest;
        }
        ++turn;
      }
    }
    const float ax = slice_sum(acc.ax), ay = slice_sum(acc.ay), az = slice_sum(acc.az),
                du = slice_sum(acc.du);
    int ctot = acc.c;
    ctot += __shfl_xor_sync(0xffffffffu, ctot, 1);
    ctot += __shfl_xor_sync(0xffffffffu, ctot, 2);
    if (has && slice == 0) {
      a.acc[i] = make_float4(ax, ay, az, du);
      a.nforce[i] = ctot;
      a.fdone[i] = 1;
      inter += (unsigned long long)ctot;
    }
  }
  ntest = warp_sum(ntest);
  inter = warp_sum(inter);
  if (lane == 0) {
    if (ntest) atomicAdd(&a.ctr->force_cand, ntest);
    if (inter) atomicAdd(&a.ctr->force_inter, inter);
  }
}

template <bool KAHAN, int NSD>
void launch_force_reuse(const BatchForceArgs &a, int blocks, cudaStream_t s) {
  static bool attr = false;
  const int bytes = (int)sizeof(ForceReuseSmem<NSD>);
  if (!attr) {
    cudaFuncSetAttribute(k_force_reuse<KAHAN, NSD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes);
    attr = true;
  }
  k_force_reuse<KAHAN, NSD><<<blocks, kNW * 32, bytes, s>>>(a);
  note_launch();
}

template <bool KAHAN, int NS, bool MID = false>
void launch_force_tier(const BatchForceArgs &a, int tier, int blocks, cudaStream_t s) {
  static bool attr = false;
  static int resident = 0;
  const int bytes = (int)sizeof(ForceSmem<NS>);
  if (!attr) {
    cudaFuncSetAttribute(k_force_batched<KAHAN, NS, MID>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    resident = resident_blocks(k_force_batched<KAHAN, NS, MID>, bytes);
    attr = true;
  }
  if (tier == 0 && a.wq.head) blocks = std::min(a.n_groups, resident);
  k_force_batched<KAHAN, NS, MID><<<blocks, kNW * 32, bytes, s>>>(a, tier);
  note_launch();
}

// The force's tiers, as the density's: first tier, the tight tier at the
// first tier's stage size, the large-stage tier, the third tier.
template <bool KAHAN>
void launch_force_tiers(const BatchForceArgs &a, int blocks, int big, cudaStream_t s) {
  if (a.tile == 2) {  // per group: the small stage where the last one fitted, else the large
    BatchForceArgs a0 = a, a1 = a;
    a0.bin = 1;
    a1.bin = 2;
    launch_force_tier<KAHAN, kStageF>(a0, 0, blocks, s);
    launch_force_tier<KAHAN, kStageFL>(a1, 0, blocks, s);
    launch_force_tier<KAHAN, kStageFL, true>(a, 1, blocks, s);
  } else if (a.tile) {
    launch_force_tier<KAHAN, kStageFL>(a, 0, blocks, s);
    launch_force_tier<KAHAN, kStageFL, true>(a, 1, blocks, s);
  } else {
    launch_force_tier<KAHAN, kStageF>(a, 0, blocks, s);
    launch_force_tier<KAHAN, kStageF, true>(a, 1, blocks, s);
  }
  launch_force_tier<KAHAN, kBigStageF>(a, 2, big, s);
  k_force_stream<KAHAN><<<152 * 8, 128, 0, s>>>(a);
  note_launch();
}

void launch_force_batched(const BatchForceArgs &a, cudaStream_t s) {
  if (a.n_groups <= 0) return;
  const int blocks = a.n_groups < 152 * 64 ? a.n_groups : 152 * 64;
  const int big = a.n_groups < 152 * 2 ? a.n_groups : 152 * 2;
  if (a.cache_on) {  // groups on the density's cache first (fuse[g]); the tiers skip them
    if (a.kahan) {
      if (a.tile)
        launch_force_reuse<true, kStageDL>(a, blocks, s);
      else
        launch_force_reuse<true, kStageD>(a, blocks, s);
    } else {
      if (a.tile)
        launch_force_reuse<false, kStageDL>(a, blocks, s);
      else
        launch_force_reuse<false, kStageD>(a, blocks, s);
    }
  }
  if (a.kahan)
    launch_force_tiers<true>(a, blocks, big, s);
  else
    launch_force_tiers<false>(a, blocks, big, s);
}

}  // namespace sph
