// interact.cu -- the SPH interaction loops (Section 2 of the paper).
//
// Density (Eq. rho), gather form: every target particle i sums over the
// particles j of the source leaves in its leaf's task list,
//   sum_j w(q), sum_j q w'(q), sum_j m_j w(q), sum_j m_j (3 w(q) + q w'(q)),
// q = r_ij / h_i, r_ij < h_i (self term included). These give the weighted
// neighbour number N_i = (32/3) sum w, dN/dh = -(32/(3h)) sum q w',
// rho_i = (8/pi) h^-3 sum m w and drho/dh = -(8/pi) h^-4 sum m (3w + q w').
//
// Ghost (the per-cell barrier task between density and force): FP64 update of
// h toward N_i(h) = n_ngb (safeguarded Newton inside a bisection bracket) and,
// once converged, rho, Omega = 1 + h/(3 rho) drho/dh, P = (gamma-1) rho u.
//
// Force (Eqs. dvdt, dudt), gather form over r_ij < max(h_i, h_j):
//   a_i   -= m_j [A_i dW/dr(r,h_i) + A_j dW/dr(r,h_j)] (x_i - x_j) / r
//   du_i  += m_j A_i dW/dr(r,h_i) (v_i - v_j).(x_i - x_j) / r
// with A = P / (Omega rho^2) and dW/dr = (8/pi) w'(q) / h^4. Each i is owned
// by one lane, so results need no atomics.
//
// Layout: one warp per target leaf; the i particles sit in lanes, the j
// particles of each source leaf are staged in shared memory (shifted into the
// target leaf's frame) and read as warp-wide broadcasts. For a pair task only
// the source particles whose key along the pair's sort axis lies within reach
// of the warp's targets are staged (pair-axis sorts, Section 3.1).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

constexpr int kWarpsPerBlock = 4;
constexpr int kStage = 64;

__device__ __forceinline__ void add_comp(float &s, float &c, float v) {
  // compensated (Kahan) summation
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pair-axis pruning of one task for the warp's 32 targets: the rank range
// [r0, r1) of the source leaf's particles, sorted along the direction nearest
// the task's shift, whose keys lie within reach R of some active target's key
// (|d_i - d_j| <= r_ij, so no neighbour is cut). `ix` maps a rank to the
// leaf-local index; it is null (whole leaf, unsorted) for the self task or
// when no sorts are given.
__device__ __forceinline__ void source_range(const float *skey, const int *sidx, int n,
                                             const Task &tk, int T, const Leaf &LS, bool act,
                                             float4 pi, float R, int &r0, int &r1,
                                             const int *&ix) {
  r0 = 0;
  r1 = LS.count;
  ix = nullptr;
  if (!skey || (tk.src == T && tk.sx == 0.f && tk.sy == 0.f && tk.sz == 0.f)) return;
  const int k = warp_best_axis(tk.sx, tk.sy, tk.sz);
  const float3 e = axis_vec(k);
  const float sd = fmaf(tk.sx, e.x, fmaf(tk.sy, e.y, tk.sz * e.z));
  float lo, hi;
  if (!warp_key_window(act, axis_key(pi, e), R, sd, lo, hi)) {
    r1 = 0;  // no active target in the warp
    return;
  }
  const size_t base = (size_t)k * n + LS.start;
  warp_key_range(skey + base, LS.count, lo, hi, r0, r1);
  ix = sidx + base;
}

// ---------------------------------------------------------------- density

template <bool KAHAN>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_density(DensArgs a) {
  __shared__ float4 sj[kWarpsPerBlock][kStage];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long cand = 0;
  for (int t = blockIdx.x * kWarpsPerBlock + warp; t < a.n_active;
       t += gridDim.x * kWarpsPerBlock) {
    const int T = a.active[t];
    const Leaf LT = a.leaves[T];
    const int e0 = a.list_off[t], e1 = a.list_off[t + 1];
    for (int ib = 0; ib < LT.count; ib += 32) {
      const int i = LT.start + ib + lane;
      const bool has = ib + lane < LT.count;
      bool act = false;
      float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
      float hi = 1.f;
      if (has) {
        act = !a.done[i];
        pi = a.pm[i];
        hi = a.hf[i];
      }
      const float h2 = act ? hi * hi : -1.f;  // inactive lanes accept nothing
      const float hinv = 1.f / hi;
      float sw = 0.f, sdw = 0.f, smw = 0.f, smdh = 0.f;
      float cw = 0.f, cdw = 0.f, cmw = 0.f, cmdh = 0.f;
      int c = 0;
      for (int e = e0; e < e1; ++e) {
        const Task tk = a.tasks[e];
        const Leaf LS = a.leaves[tk.src];
        int r0, r1;
        const int *ix;
        source_range(a.skey, a.sidx, a.n, tk, T, LS, act, pi, hi, r0, r1, ix);
        for (int jb = r0; jb < r1; jb += kStage) {
          const int nj = min(kStage, r1 - jb);
          __syncwarp();
          for (int k = lane; k < nj; k += 32) {
            float4 q = a.pm[LS.start + (ix ? ix[jb + k] : jb + k)];
            q.x += tk.sx;
            q.y += tk.sy;
            q.z += tk.sz;
            sj[warp][k] = q;
          }
          __syncwarp();
          for (int k = 0; k < nj; ++k) {
            const float4 q = sj[warp][k];
            const float dx = pi.x - q.x, dy = pi.y - q.y, dz = pi.z - q.z;
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
          if (act) cand += nj;
        }
      }
      if (act) {
        a.sums[i] = make_float4(sw, sdw, smw, smdh);
        a.cnt[i] = c - 1;  // the self term is always inside
      }
    }
  }
  cand = warp_sum_u64(cand);
  if (lane == 0 && cand) atomicAdd(&a.ctr->dens_cand, cand);
}

void launch_density(const DensArgs &a, cudaStream_t s) {
  if (a.n_active <= 0) return;
  int blocks = (a.n_active + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (a.kahan)
    k_density<true><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
  else
    k_density<false><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
  note_launch();
}

// ------------------------------------------------------------------ ghost

__global__ void k_ghost(GhostArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool finished_now = false;
  int ngb = 0;
  if (i < a.n && !a.done[i]) {
    const float4 s = a.sums[i];
    const int it = a.niter[i] + 1;
    a.niter[i] = it;
    HIter hs;
    hs.start(a.h[i], a.hlo[i], a.hhi[i], a.fprev[i]);
    const Leaf &L = a.leaves[a.leaf_of[i]];
    const BoxDev &B = a.boxes[L.box];
    const double wmin = fmin(B.w[0], fmin(B.w[1], B.w[2]));
    const double hcap = B.hcap;
    int st = 0;
    const double h = hs.h;
    const bool conv = h_newton_step(hs, s.x, s.y, a.n_ngb, a.tol * a.n_ngb, hcap, &st);
    if (!conv) {
      a.h[i] = hs.h;
      a.hf[i] = hs.hf;
      a.hlo[i] = hs.lo;
      a.hhi[i] = hs.hi;
      a.fprev[i] = hs.fprev;
      if (hs.h * (1.0 + 1e-6) > wmin) st |= kErrHGrid;
      if (it >= a.max_iter) st |= kErrNotConverged;
      atomicAdd(&a.ctr->unconverged, 1);
    } else {
      float rho, omega, P;
      float4 fi;
      if (!finalise_density((float)h, s, a.vu[i].w, (float)(a.gamma - 1.0), &rho, &omega, &P,
                            &fi))
        st |= kErrNonPhysical;
      a.rho[i] = rho;
      a.omega[i] = omega;
      a.P[i] = P;
      a.force_i[i] = fi;
      a.done[i] = 1;
      a.nngb[i] = a.cnt[i];
      ngb = a.cnt[i];
      finished_now = true;
      atomicMax(&a.ctr->max_iter_used, it);
    }
    if (st) atomicOr(&a.ctr->status, st);
  }
  unsigned long long v = finished_now ? (unsigned long long)ngb : 0ull;
  v = warp_sum_u64(v);
  if (lane == 0 && v) atomicAdd(&a.ctr->dens_inter, v);
}

void launch_ghost(const GhostArgs &a, cudaStream_t s) {
  k_ghost<<<(a.n + 255) / 256, 256, 0, s>>>(a); note_launch();
}

__global__ void k_active_leaves(const Leaf *leaves, int n_leaves, const unsigned char *done,
                                int *active, DevCounters *ctr) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= n_leaves) return;
  const Leaf L = leaves[li];
  bool any = false;
  for (int k = 0; k < L.count && !any; ++k) any = !done[L.start + k];
  if (any) active[atomicAdd(&ctr->n_active, 1)] = li;
}

void launch_active_leaves(const Leaf *leaves, int n_leaves, const unsigned char *done,
                          int *active, DevCounters *ctr, cudaStream_t s) {
  k_active_leaves<<<(n_leaves + 255) / 256, 256, 0, s>>>(leaves, n_leaves, done, active, ctr); note_launch();
}

// ------------------------------------------------------------------ force

template <bool KAHAN>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_force(ForceArgs a) {
  __shared__ float4 sp[kWarpsPerBlock][kStage];
  __shared__ float4 sf[kWarpsPerBlock][kStage];
  __shared__ float4 sv[kWarpsPerBlock][kStage];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long cand = 0, inter = 0;
  for (int t = blockIdx.x * kWarpsPerBlock + warp; t < a.n_targets;
       t += gridDim.x * kWarpsPerBlock) {
    const int T = a.active ? a.active[t] : t;
    const Leaf LT = a.leaves[T];
    const int e0 = a.list_off[t], e1 = a.list_off[t + 1];
    for (int ib = 0; ib < LT.count; ib += 32) {
      const int i = LT.start + ib + lane;
      const bool has = ib + lane < LT.count;
      float4 pi = make_float4(0.f, 0.f, 0.f, 0.f), fi = make_float4(1.f, 1.f, 0.f, -1.f),
             vi = make_float4(0.f, 0.f, 0.f, 0.f);
      if (has) {
        pi = a.pm[i];
        fi = a.fi[i];
        vi = a.vu[i];
      }
      float ax = 0.f, ay = 0.f, az = 0.f, du = 0.f;
      float cx = 0.f, cy = 0.f, cz = 0.f, cu = 0.f;
      int c = 0;
      for (int e = e0; e < e1; ++e) {
        const Task tk = a.tasks[e];
        const Leaf LS = a.leaves[tk.src];
        int r0, r1;
        const int *ix;
        const float reach = a.skey ? fmaxf(fi.x, a.nodes[LS.node].hmax) : 0.f;
        source_range(a.skey, a.sidx, a.n, tk, T, LS, has, pi, reach, r0, r1, ix);
        for (int jb = r0; jb < r1; jb += kStage) {
          const int nj = min(kStage, r1 - jb);
          __syncwarp();
          for (int k = lane; k < nj; k += 32) {
            const int j = LS.start + (ix ? ix[jb + k] : jb + k);
            float4 q = a.pm[j];
            q.x += tk.sx;
            q.y += tk.sy;
            q.z += tk.sz;
            sp[warp][k] = q;
            sf[warp][k] = a.fi[j];
            sv[warp][k] = a.vu[j];
          }
          __syncwarp();
          for (int k = 0; k < nj; ++k) {
            const float4 q = sp[warp][k];
            const float4 fj = sf[warp][k];
            const float dx = pi.x - q.x, dy = pi.y - q.y, dz = pi.z - q.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float hij2 = has ? fmaxf(fi.w, fj.w) : -1.f;
            if (r2 < hij2 && r2 > 0.f) {
              const float rinv = rsqrtf(r2);
              const float r = r2 * rinv;
              const float ti = fi.z * dw_only(r * fi.y);  // A_i dW/dr(r, h_i)
              const float tj = fj.z * dw_only(r * fj.y);  // A_j dW/dr(r, h_j)
              const float fac = q.w * (ti + tj) * rinv;
              const float4 vj = sv[warp][k];
              const float dvdx = (vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz;
              const float dui = q.w * ti * rinv * dvdx;
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
          }
          if (has) cand += nj;
        }
      }
      if (has && !(a.skip && a.skip[i])) {
        a.acc[i] = make_float4(ax, ay, az, du);
        a.nforce[i] = c;
        inter += c;
      }
    }
  }
  cand = warp_sum_u64(cand);
  inter = warp_sum_u64(inter);
  if (lane == 0) {
    if (cand) atomicAdd(&a.ctr->force_cand, cand);
    if (inter) atomicAdd(&a.ctr->force_inter, inter);
  }
}

void launch_force(const ForceArgs &a, cudaStream_t s) {
  if (a.n_targets <= 0) return;
  int blocks = (a.n_targets + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (a.kahan)
    k_force<true><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
  else
    k_force<false><<<blocks, kWarpsPerBlock * 32, 0, s>>>(a);
  note_launch();
}

}  // namespace sph
