// axis_sort.cu -- pair-axis sorts of the particles of every octree leaf
// (Section 3.1: before a cell's density tasks run, its particles are sorted
// along the axes that join it to its neighbours, so that a pair task need only
// visit the particles of the source cell that project within reach of the
// target cell's).
//
// For each leaf and each of the 13 directions e_k joining a cell to half of
// its 26 neighbours (the other 13 are their negatives and share the order),
// the key of particle p is d_k(p) = x_p . e_k, with x_p the leaf-relative FP32
// position. The leaf's particles are ranked by (key, local index), so the
// order is a permutation and does not depend on scheduling:
//   skey[k * N + start + r] = key of the particle of rank r,
//   sidx[k * N + start + r] = its index within the leaf.
// A pair task along e_k then takes, from the source leaf, the contiguous
// sorted range whose keys fall inside [min_i d_i - R, max_i d_i + R] (shifted
// into the source frame); |d_i - d_j| <= |x_i - x_j| makes the cut exact.
//
// One warp per leaf; every particle counts the keys below its own (ranks,
// O(count^2) compares). A leaf of at most kSortMax particles (every leaf but
// those at the depth limit) has its positions read once into shared memory
// and each direction's keys formed once there; larger leaves are ranked
// against tiles of keys read from global memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

constexpr int kSortWarps = 4;
constexpr int kSortTile = 256;
constexpr int kSortMax = 256;  // leaves ranked from shared memory

__global__ void __launch_bounds__(kSortWarps * 32) k_axis_sort(AxisSortArgs a) {
  __shared__ float4 pos_all[kSortWarps][kSortMax];
  __shared__ float tile_all[kSortWarps][kSortTile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = blockIdx.x * kSortWarps + warp;
  if (li >= a.n_leaves) return;  // warp-uniform
  const Leaf L = a.leaves[li];
  float *tile = tile_all[warp];
  if (L.count <= kSortMax) {
    float4 *pos = pos_all[warp];
    for (int p = lane; p < L.count; p += 32) pos[p] = a.pm[L.start + p];
    for (int k = 0; k < kAxes; ++k) {
      const float3 e = axis_vec(k);
      __syncwarp();  // pos written; the previous direction's ranking is done with tile
      for (int p = lane; p < L.count; p += 32) tile[p] = axis_key(pos[p], e);
      __syncwarp();
      float *key_out = a.skey + (size_t)k * a.n + L.start;
      int *idx_out = a.sidx + (size_t)k * a.n + L.start;
      for (int p = lane; p < L.count; p += 32) {
        const float kp = tile[p];
        int rank = 0;
        for (int q = 0; q < L.count; ++q) {
          const float kq = tile[q];
          rank += (kq < kp || (kq == kp && q < p)) ? 1 : 0;
        }
        key_out[rank] = kp;
        idx_out[rank] = p;
      }
    }
    return;
  }
  for (int k = 0; k < kAxes; ++k) {
    const float3 e = axis_vec(k);
    float *key_out = a.skey + (size_t)k * a.n + L.start;
    int *idx_out = a.sidx + (size_t)k * a.n + L.start;
    for (int pb = 0; pb < L.count; pb += 32) {
      const int p = pb + lane;
      float kp = 0.f;
      if (p < L.count) kp = axis_key(a.pm[L.start + p], e);
      int rank = 0;
      for (int qb = 0; qb < L.count; qb += kSortTile) {
        const int nq = min(kSortTile, L.count - qb);
        __syncwarp();
        for (int q = lane; q < nq; q += 32) tile[q] = axis_key(a.pm[L.start + qb + q], e);
        __syncwarp();
        for (int q = 0; q < nq; ++q) {
          const float kq = tile[q];
          rank += (kq < kp || (kq == kp && qb + q < p)) ? 1 : 0;
        }
      }
      if (p < L.count) {
        key_out[rank] = kp;
        idx_out[rank] = p;
      }
    }
  }
}

void launch_axis_sort(const AxisSortArgs &a, cudaStream_t s) {
  if (a.n_leaves <= 0) return;
  k_axis_sort<<<(a.n_leaves + kSortWarps - 1) / kSortWarps, kSortWarps * 32, 0, s>>>(a);
  note_launch();
}

// Slot s of leaf l: leaf_out[s] = l, order_out[s] = caller index of the
// particle of rank s - start(l) along `axis`.
__global__ void k_get_pair_order(const Leaf *leaves, const int *leaf_of, const int *sidx,
                                 const int *orig, int n, int axis, int *order_out,
                                 int *leaf_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int l = leaf_of[s];
  const int start = leaves[l].start;
  order_out[s] = orig[start + sidx[(size_t)axis * n + s]];
  leaf_out[s] = l;
}

void launch_get_pair_order(const Leaf *leaves, const int *leaf_of, const int *sidx,
                           const int *orig, int n, int axis, int *order_out, int *leaf_out,
                           cudaStream_t s) {
  if (n <= 0) return;
  k_get_pair_order<<<(n + 255) / 256, 256, 0, s>>>(leaves, leaf_of, sidx, orig, n, axis,
                                                    order_out, leaf_out);
  note_launch();
}

}  // namespace sph
