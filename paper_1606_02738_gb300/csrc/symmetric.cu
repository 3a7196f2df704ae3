// Symmetric force form (SPH_MODE_SYMMETRIC): every unordered pair is
// evaluated once and updates both particles.
//
// Section 3.1 builds the interactions from pair tasks between neighbouring
// cells that update the particles of both cells, exploiting the symmetry of
// the pair terms, with conflicts between tasks that touch the same cell
// resolved by the scheduler. Here a pair task is a pair of octree leaves
// (A, B), B >= A by leaf index, taken from the force task lists of the
// per-pass form (leaf boxes within max(hmax_A, hmax_B) of each other). One
// block owns one top cell and runs the tasks of the cell's leaves one after
// another; the cells are coloured so that two cells of one colour are at
// least three cells apart along some axis (periodically), so the 27-cell
// neighbourhoods of the cells that run at once are disjoint and every
// particle a launch touches belongs to one block: no atomics on the
// results, and the order of every sum is fixed (colour, cell, leaf, task).
//
// Within a task the block's warps take 32 particles of A each (one per
// lane) and step through B's particles together: a lane adds the pair's
// term to its own particle, and the warp sums the 32 lanes' terms for the
// B particle by shuffles in fixed order. The B sums of the warps are then
// added in warp order. Pair terms of Eqs. (dvdt) and (dudt) for r_ij <
// max(h_i, h_j):
//   a_i -= m_j (A_i W'(r, h_i) + A_j W'(r, h_j)) (x_i - x_j) / r
//   a_j += m_i (A_i W'(r, h_i) + A_j W'(r, h_j)) (x_i - x_j) / r
//   du_i/dt += m_j A_i W'(r, h_i) (v_i - v_j).(x_i - x_j) / r
//   du_j/dt += m_i A_j W'(r, h_j) (v_i - v_j).(x_i - x_j) / r
// with A_k = P_k / (Omega_k rho_k^2) and W' = dW/dr (the force record).
// FP32 sums (no compensated variant).

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kSymWarps = 4;
constexpr int kSymChunk = 256;  // particles of a leaf held at once (a larger leaf is cut)

struct SymSmem {
  float4 pa[kSymChunk], fa[kSymChunk], va[kSymChunk];  // A chunk: position, force record, (v, u)
  float4 pb[kSymChunk], fb[kSymChunk], vb[kSymChunk];  // B chunk, shifted into A's frame
  float4 acca[kSymChunk];                              // A chunk's sums over the cell's tasks
  int cnta[kSymChunk];
  float4 jpart[kSymWarps][kSymChunk];                  // each warp's sums for the B chunk
  int jcnt[kSymWarps][kSymChunk];
};

__device__ __forceinline__ void load_chunk(const float4 *pm, const float4 *fi, const float4 *vu,
                                           int start, int n, float sx, float sy, float sz,
                                           float4 *p, float4 *f, float4 *v) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    float4 q = pm[start + k];
    q.x += sx;
    q.y += sy;
    q.z += sz;
    p[k] = q;
    f[k] = fi[start + k];
    v[k] = vu[start + k];
  }
}

__global__ void __launch_bounds__(kSymWarps * 32) k_force_sym(SymArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SymSmem &S = *reinterpret_cast<SymSmem *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long tests = 0, inter = 0;
  for (int ci = blockIdx.x; ci < a.n_cells; ci += gridDim.x) {
    const int cell = a.cells[ci];
    const int l0 = a.cell_leaf[cell], l1 = a.cell_leaf[cell + 1];
    for (int A = l0; A < l1; ++A) {
      const Leaf LA = a.leaves[A];
      const int e0 = a.list_off[A], e1 = a.list_off[A + 1];
      for (int ca = 0; ca < LA.count; ca += kSymChunk) {
        const int na = min(kSymChunk, LA.count - ca);
        __syncthreads();  // the previous chunk's sums are out of shared memory
        load_chunk(a.pm, a.fi, a.vu, LA.start + ca, na, 0.f, 0.f, 0.f, S.pa, S.fa, S.va);
        for (int k = threadIdx.x; k < na; k += blockDim.x) {
          S.acca[k] = make_float4(0.f, 0.f, 0.f, 0.f);
          S.cnta[k] = 0;
        }
        for (int e = e0; e < e1; ++e) {
          const Task tk = a.tasks[e];
          const int B = tk.src;
          if (B < A) continue;  // that pair is B's task
          const Leaf LB = a.leaves[B];
          for (int cb = (B == A ? ca : 0); cb < LB.count; cb += kSymChunk) {
            const int nb = min(kSymChunk, LB.count - cb);
            const bool same = B == A && cb == ca;  // pairs i < j of the A chunk
            __syncthreads();  // the previous B chunk and its sums are done with
            if (!same)
              load_chunk(a.pm, a.fi, a.vu, LB.start + cb, nb, tk.sx, tk.sy, tk.sz, S.pb, S.fb,
                         S.vb);
            for (int k = threadIdx.x; k < kSymWarps * nb; k += blockDim.x) {
              S.jpart[k / nb][k % nb] = make_float4(0.f, 0.f, 0.f, 0.f);
              S.jcnt[k / nb][k % nb] = 0;
            }
            __syncthreads();
            const float4 *pb = same ? S.pa : S.pb;
            const float4 *fb = same ? S.fa : S.fb;
            const float4 *vb = same ? S.va : S.vb;
            for (int ib = warp * 32; ib < na; ib += kSymWarps * 32) {
              const int i = ib + lane;
              const bool has = i < na;
              const float4 pi = has ? S.pa[i] : make_float4(0.f, 0.f, 0.f, 0.f);
              const float4 fi = has ? S.fa[i] : make_float4(1.f, 1.f, 0.f, -1.f);
              const float4 vi = has ? S.va[i] : make_float4(0.f, 0.f, 0.f, 0.f);
              float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
              int c = 0;
              // for the A chunk with itself, j runs over the pairs j > i of this
              // warp's rows only (j from ib: the rows below are earlier warps')
              for (int j = same ? ib : 0; j < nb; ++j) {
                const float4 q = pb[j];
                const float4 fj = fb[j];
                const float dx = pi.x - q.x, dy = pi.y - q.y, dz = pi.z - q.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float bx = 0.f, by = 0.f, bz = 0.f, bu = 0.f;
                int bc = 0;
                if (has && (!same || j > i) && r2 > 0.f && r2 < fmaxf(fi.w, fj.w)) {
                  const float rinv = rsqrtf(r2);
                  const float r = r2 * rinv;
                  const float ti = fi.z * dw_only(r * fi.y);  // A_i dW/dr(r, h_i)
                  const float tj = fj.z * dw_only(r * fj.y);  // A_j dW/dr(r, h_j)
                  const float s = (ti + tj) * rinv;
                  const float4 vj = vb[j];
                  const float dvdx =
                      (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
                  const float fac_i = q.w * s, fac_j = pi.w * s;
                  ax = fmaf(-fac_i, dx, ax);
                  ay = fmaf(-fac_i, dy, ay);
                  az = fmaf(-fac_i, dz, az);
                  du += q.w * ti * rinv * dvdx;
                  ++c;
                  bx = fac_j * dx;
                  by = fac_j * dy;
                  bz = fac_j * dz;
                  bu = pi.w * tj * rinv * dvdx;
                  bc = 1;
                }
                // j's terms from the warp's 32 rows, summed in fixed order
                for (int o = 16; o; o >>= 1) {
                  bx += __shfl_xor_sync(0xffffffffu, bx, o);
                  by += __shfl_xor_sync(0xffffffffu, by, o);
                  bz += __shfl_xor_sync(0xffffffffu, bz, o);
                  bu += __shfl_xor_sync(0xffffffffu, bu, o);
                  bc += __shfl_xor_sync(0xffffffffu, bc, o);
                }
                if (lane == 0 && bc) {
                  float4 &jp = S.jpart[warp][j];
                  jp.x += bx;
                  jp.y += by;
                  jp.z += bz;
                  jp.w += bu;
                  S.jcnt[warp][j] += bc;
                }
              }
              if (has) {
                const int rows = same ? max(0, nb - ib) : nb;
                tests += (unsigned long long)(same ? max(0, rows - lane - 1) : rows);
                float4 &acc = S.acca[i];
                acc.x += ax;
                acc.y += ay;
                acc.z += az;
                acc.w += du;
                S.cnta[i] += c;
              }
            }
            __syncthreads();
            // the B chunk's sums, the warps' parts in warp order
            for (int k = threadIdx.x; k < nb; k += blockDim.x) {
              float4 t = S.jpart[0][k];
              int tc = S.jcnt[0][k];
              for (int w = 1; w < kSymWarps; ++w) {
                t.x += S.jpart[w][k].x;
                t.y += S.jpart[w][k].y;
                t.z += S.jpart[w][k].z;
                t.w += S.jpart[w][k].w;
                tc += S.jcnt[w][k];
              }
              if (same) {
                float4 &acc = S.acca[k];
                acc.x += t.x;
                acc.y += t.y;
                acc.z += t.z;
                acc.w += t.w;
                S.cnta[k] += tc;
              } else if (tc) {  // this launch owns B's particles: a plain update
                const int jg = LB.start + cb + k;
                float4 g = a.acc[jg];
                g.x += t.x;
                g.y += t.y;
                g.z += t.z;
                g.w += t.w;
                a.acc[jg] = g;
                a.nforce[jg] += tc;
                inter += (unsigned long long)tc;
              }
            }
          }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < na; k += blockDim.x) {
          const int ig = LA.start + ca + k;
          float4 g = a.acc[ig];
          const float4 t = S.acca[k];
          g.x += t.x;
          g.y += t.y;
          g.z += t.z;
          g.w += t.w;
          a.acc[ig] = g;
          a.nforce[ig] += S.cnta[k];
          inter += (unsigned long long)S.cnta[k];
        }
      }
    }
  }
  // interactions: ordered pairs (each unordered pair counts for both particles)
  for (int o = 16; o; o >>= 1) {
    tests += __shfl_xor_sync(0xffffffffu, tests, o);
    inter += __shfl_xor_sync(0xffffffffu, inter, o);
  }
  if (lane == 0) {
    if (tests) atomicAdd(&a.ctr->force_cand, tests);
    if (inter) atomicAdd(&a.ctr->force_inter, inter);
  }
}

// Per leaf: its global top cell.
__global__ void k_leaf_cells(const Leaf *leaves, const Node *nodes, int n_leaves, int *out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n_leaves) out[l] = nodes[leaves[l].node].cell;
}

}  // namespace

void launch_leaf_cells(const Leaf *leaves, const Node *nodes, int n_leaves, int *out,
                       cudaStream_t s) {
  if (n_leaves <= 0) return;
  k_leaf_cells<<<(n_leaves + 255) / 256, 256, 0, s>>>(leaves, nodes, n_leaves, out);
  note_launch();
}

void launch_force_sym(const SymArgs &a, cudaStream_t s) {
  if (a.n_cells <= 0) return;
  static bool attr = false;
  static int resident = 0;
  const int bytes = (int)sizeof(SymSmem);
  if (!attr) {
    cudaFuncSetAttribute(k_force_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_force_sym, kSymWarps * 32, bytes);
    resident = std::max(per, 1) * std::max(sms, 1);
    attr = true;
  }
  const int blocks = std::min(a.n_cells, resident);
  k_force_sym<<<blocks, kSymWarps * 32, bytes, s>>>(a);
  note_launch();
}

// Colour classes of the top cells that hold leaves: per axis, cells below
// the largest multiple of three take the coordinate mod 3, the one or two
// cells above it a class of their own (3, 4), so two cells of one class are
// at least three cells apart along that axis, also across the periodic
// wrap; the colour combines the three axes (at most 125). cell_leaf[c] is
// the first leaf of cell c (leaves are stored by cell), cell_leaf[n_cells]
// the leaf count.
void sym_colours(const std::vector<BoxDev> &boxes, int n_cells, const std::vector<int> &leaf_cell,
                 std::vector<int> &cell_leaf, std::vector<int> &colour_cells,
                 std::vector<int> &colour_off) {
  const int nl = (int)leaf_cell.size();
  cell_leaf.assign((size_t)n_cells + 1, nl);
  for (int l = nl - 1; l >= 0; --l) cell_leaf[leaf_cell[l]] = l;
  for (int c = n_cells - 1; c >= 0; --c) cell_leaf[c] = std::min(cell_leaf[c], cell_leaf[c + 1]);
  std::vector<std::vector<int>> cls(125);
  for (const BoxDev &B : boxes) {
    const int nc = B.n[0] * B.n[1] * B.n[2];
    for (int local = 0; local < nc; ++local) {
      const int cell = B.cell_base + local;
      if (cell_leaf[cell] == cell_leaf[cell + 1]) continue;  // no leaf
      const int c[3] = {local / (B.n[1] * B.n[2]), (local / B.n[2]) % B.n[1], local % B.n[2]};
      int col = 0;
      for (int d = 2; d >= 0; --d) {
        const int full = B.n[d] / 3 * 3;
        const int v = c[d] < full ? c[d] % 3 : 3 + (c[d] - full);
        col = col * 5 + v;
      }
      cls[col].push_back(cell);
    }
  }
  colour_cells.clear();
  colour_off.assign(1, 0);
  for (const auto &v : cls) {
    if (v.empty()) continue;
    colour_cells.insert(colour_cells.end(), v.begin(), v.end());
    colour_off.push_back((int)colour_cells.size());
  }
}

}  // namespace sph
