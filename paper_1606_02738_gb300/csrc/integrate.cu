// integrate.cu -- particle-store movement and the integrator task.
//
// Section 3.1 of the paper: once all force tasks on a cell are done, the
// integrator task updates particle positions and velocities. The scheme here
// is kick-drift-kick with one global time step: half kick of v and u, drift of
// the FP64 positions (periodic wrap), prediction of v and u to the end of the
// step for the next force evaluation, and the closing half kick after it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"
#include "sph_internal.cuh"

namespace sph {

__device__ __forceinline__ int box_of_slot(const BoxDev *b, int nb, int k) {
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

__device__ __forceinline__ double wrap1(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y -= L;
  if (y < 0.0) y = 0.0;
  return y;
}

// The drift of one step moves a particle by much less than a box length: one
// conditional add brings it back, and only a coordinate still outside [0, L)
// pays for the general form's FP64 division (FP64 runs at 1/64 of the FP32
// rate here).
__device__ __forceinline__ double wrap_near(double x, double L) {
  double y = x;
  if (y >= L)
    y -= L;
  else if (y < 0.0)
    y += L;
  if (y >= L || y < 0.0) y = wrap1(x, L);
  return y;
}

// caller x [N][3] -> wrapped SoA copy (caller order)
__global__ void k_wrap_from_caller(const double *x, const BoxDev *boxes, int nb, int n,
                                   double *x0, double *x1, double *x2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const BoxDev &B = boxes[box_of_slot(boxes, nb, k)];
  x0[k] = wrap1(x[3 * (size_t)k], B.L[0]);
  x1[k] = wrap1(x[3 * (size_t)k + 1], B.L[1]);
  x2[k] = wrap1(x[3 * (size_t)k + 2], B.L[2]);
}

void launch_wrap_cell_keys_from_caller(const double *x, const BoxDev *boxes, int n_boxes, int n,
                                       double *x0, double *x1, double *x2, cudaStream_t s) {
  k_wrap_from_caller<<<(n + 255) / 256, 256, 0, s>>>(x, boxes, n_boxes, n, x0, x1, x2); note_launch();
}

// Sorted store <- caller arrays; `order[s]` is the caller index of slot s.
struct LoadArgs {
  StoreArrays dst;
  const int *order;
  int n;
  const double *wx0, *wx1, *wx2;  // wrapped positions, caller order
  const float *v, *m, *u;
  const double *h;
};

__global__ void k_load(LoadArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const int k = a.order[s];
  a.dst.x0[s] = a.wx0[k];
  a.dst.x1[s] = a.wx1[k];
  a.dst.x2[s] = a.wx2[k];
  const float4 vu = make_float4(a.v[3 * (size_t)k], a.v[3 * (size_t)k + 1],
                                a.v[3 * (size_t)k + 2], a.u[k]);
  a.dst.vu[s] = vu;
  a.dst.vu_pred[s] = vu;
  a.dst.acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  a.dst.m[s] = a.m[k];
  a.dst.h[s] = a.h[k];
  a.dst.hlo[s] = 0.0;
  a.dst.hhi[s] = 1e308;
  a.dst.orig[s] = k;
}

void launch_load_caller(const StoreArrays &dst, const int *order, int n, const double *wx,
                        const float *v, const float *m, const float *u, const double *h,
                        cudaStream_t s) {
  LoadArgs a{dst, order, n, wx, wx + n, wx + 2 * (size_t)n, v, m, u, h};
  k_load<<<(n + 255) / 256, 256, 0, s>>>(a); note_launch();
}

__global__ void k_permute(StoreArrays d, StoreArrays src, const int *order, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int k = order[s];
  d.x0[s] = src.x0[k];
  d.x1[s] = src.x1[k];
  d.x2[s] = src.x2[k];
  d.h[s] = src.h[k];
  d.hlo[s] = src.hlo[k];
  d.hhi[s] = src.hhi[k];
  d.vu[s] = src.vu[k];
  d.vu_pred[s] = src.vu_pred[k];
  d.acc[s] = src.acc[k];
  d.m[s] = src.m[k];
  d.orig[s] = src.orig[k];
}

void launch_permute(const StoreArrays &dst, const StoreArrays &src, const int *order, int n,
                    cudaStream_t s) {
  k_permute<<<(n + 255) / 256, 256, 0, s>>>(dst, src, order, n); note_launch();
}

// First half kick, drift, prediction of v and u, and the starting guess of
// the next h iteration: with a constant neighbour number h varies as
// rho^(-1/3), and in the adiabatic flow d ln rho / dt = (du/dt) / ((gamma-1) u)
// (the same velocity-divergence sum as du/dt), so h is carried to the end of
// the step as h exp(-dt (du/dt) / (3 (gamma-1) u)). Only the guess moves: the
// density stage still iterates h to its own root (Section 2, constant
// neighbour number), so results do not depend on it beyond the tolerance.
template <bool SAVE>
__global__ void k_kick_drift(StoreArrays st, int n, double dt, const BoxDev *boxes, int nb,
                             float gm1, float *hf, StoreArrays save, unsigned char *done,
                             unsigned char *fdone, DevCounters *ctr, DriftCache dc) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  // neighbour-cache bookkeeping: path length since the epoch began (an upper
  // bound of the displacement) and its largest value per top cell, one
  // atomic per warp where the warp's particles share a cell (the usual case
  // in the cell-sorted store)
  float dp = 0.f;
  int cell = -1;
  if (s < n && dc.dpath) {
    const float4 a = st.acc[s];
    const float4 v = st.vu[s];
    const float hdt = (float)(0.5 * dt);
    const float vx = fmaf(a.x, hdt, v.x), vy = fmaf(a.y, hdt, v.y), vz = fmaf(a.z, hdt, v.z);
    const float step = sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz))) * (float)dt;
    // rounding of |v dt| and of the sum: a relative 1e-6 keeps it an upper bound
    dp = dc.ctl->build_all ? 0.f : (dc.dpath[s] + step * (1.f + 1e-6f)) * (1.f + 1e-6f);
    dc.dpath[s] = dp;
    cell = dc.nodes[dc.leaves[dc.leaf_of[s]].node].cell;
  }
  if (dc.dpath) {  // dp >= 0: its bit pattern orders like an unsigned integer
    const int c0 = __shfl_sync(0xffffffffu, cell, 0);
    if (__all_sync(0xffffffffu, cell == c0 || cell < 0)) {
      float m = dp;
      for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0 && c0 >= 0 && m > 0.f) atomicMax(&dc.dmax_cell[c0], __float_as_uint(m));
    } else if (cell >= 0 && dp > 0.f) {
      atomicMax(&dc.dmax_cell[cell], __float_as_uint(dp));
    }
  }
  if (s >= n) return;
  if (done) done[s] = 0;
  if (fdone) fdone[s] = 0;
  const float hdt = (float)(0.5 * dt);
  const float4 a = st.acc[s];
  float4 v = st.vu[s];
  if (SAVE) {
    save.x0[s] = st.x0[s];
    save.x1[s] = st.x1[s];
    save.x2[s] = st.x2[s];
    save.h[s] = st.h[s];
    save.vu[s] = v;
    save.acc[s] = a;
  }
  if (v.w > 0.f && a.w != 0.f) {
    const float e = fminf(fmaxf(-(float)dt * a.w / (3.f * gm1 * v.w), -0.2f), 0.2f);
    const double h = st.h[s] * (double)expf(e);
    st.h[s] = h;
    hf[s] = (float)h;
  }
  v.x = fmaf(a.x, hdt, v.x);
  v.y = fmaf(a.y, hdt, v.y);
  v.z = fmaf(a.z, hdt, v.z);
  v.w = fmaf(a.w, hdt, v.w);
  st.vu[s] = v;  // v and u at the half step
  const BoxDev &B = boxes[box_of_slot(boxes, nb, s)];
  st.x0[s] = wrap_near(st.x0[s] + (double)v.x * dt, B.L[0]);
  st.x1[s] = wrap_near(st.x1[s] + (double)v.y * dt, B.L[1]);
  st.x2[s] = wrap_near(st.x2[s] + (double)v.z * dt, B.L[2]);
  const float4 p = make_float4(fmaf(a.x, hdt, v.x), fmaf(a.y, hdt, v.y), fmaf(a.z, hdt, v.z),
                               fmaf(a.w, hdt, v.w));
  st.vu_pred[s] = p;
  if (!(p.w > 0.f) || !(v.w > 0.f)) atomicOr(&ctr->step_status, kErrNonPhysical);
}

void launch_kick_drift(StoreArrays st, int n, double dt, const BoxDev *boxes, int n_boxes,
                       double gamma, float *hf, const StoreArrays *save, unsigned char *done,
                       unsigned char *fdone, DevCounters *ctr, cudaStream_t s,
                       const DriftCache *dcp) {
  const float gm1 = (float)(gamma - 1.0);
  const DriftCache dc = dcp ? *dcp : DriftCache{};
  if (save)
    k_kick_drift<true><<<(n + 255) / 256, 256, 0, s>>>(st, n, dt, boxes, n_boxes, gm1, hf, *save,
                                                       done, fdone, ctr, dc);
  else
    k_kick_drift<false><<<(n + 255) / 256, 256, 0, s>>>(st, n, dt, boxes, n_boxes, gm1, hf,
                                                        StoreArrays{}, done, fdone, ctr, dc);
  note_launch();
}

// Closing half kick with the new accelerations.
__global__ void k_kick(StoreArrays st, int n, double dt, DevCounters *ctr) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float hdt = (float)(0.5 * dt);
  const float4 a = st.acc[s];
  float4 v = st.vu[s];
  v.x = fmaf(a.x, hdt, v.x);
  v.y = fmaf(a.y, hdt, v.y);
  v.z = fmaf(a.z, hdt, v.z);
  v.w = fmaf(a.w, hdt, v.w);
  st.vu[s] = v;
  st.vu_pred[s] = v;
  if (!(v.w > 0.f)) atomicOr(&ctr->step_status, kErrNonPhysical);
}

void launch_kick(StoreArrays st, int n, double dt, DevCounters *ctr, cudaStream_t s) {
  k_kick<<<(n + 255) / 256, 256, 0, s>>>(st, n, dt, ctr); note_launch();
}

__global__ void k_h_to_float(const double *h, float *hf, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) hf[s] = (float)h[s];
}

void launch_h_to_float(const double *h, float *hf, int n, cudaStream_t s) {
  k_h_to_float<<<(n + 255) / 256, 256, 0, s>>>(h, hf, n); note_launch();
}

constexpr int kExtItems = 8;

// Non-negative doubles order like their bit patterns, so the extremes are
// reduced on the bits. Each thread takes kExtItems consecutive slots, the
// warp reduces, and one lane per warp issues the atomics (per-box maxima: one
// atomic per warp when the whole warp lies in one box, else one per lane).
__global__ void k_h_extremes(const double *h, int n, const BoxDev *boxes, int nb,
                             unsigned long long *dmax, unsigned long long *dminmax) {
  const int lane = threadIdx.x & 31;
  const int base = (blockIdx.x * blockDim.x + threadIdx.x) * kExtItems;
  unsigned long long mn = ~0ull, mx = 0ull, bmax = 0ull;
  int box = -1;
  for (int k = 0; k < kExtItems; ++k) {
    const int s = base + k;
    if (s >= n) break;
    const unsigned long long b = (unsigned long long)__double_as_longlong(h[s]);
    mn = b < mn ? b : mn;
    mx = b > mx ? b : mx;
    const int bs = box_of_slot(boxes, nb, s);
    if (bs != box) {
      if (box >= 0) atomicMax(&dmax[box], bmax);
      box = bs;
      bmax = b;
    } else if (b > bmax) {
      bmax = b;
    }
  }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, mn, o);
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, mx, o);
    mn = a < mn ? a : mn;
    mx = c > mx ? c : mx;
  }
  if (lane == 0 && mx > 0ull) {
    atomicMin(&dminmax[0], mn);
    atomicMax(&dminmax[1], mx);
  }
  const int box0 = __shfl_sync(0xffffffffu, box, 0);
  if (__all_sync(0xffffffffu, box == box0 || box < 0)) {
    for (int o = 16; o; o >>= 1) {
      const unsigned long long c = __shfl_xor_sync(0xffffffffu, bmax, o);
      bmax = c > bmax ? c : bmax;
    }
    if (lane == 0 && box0 >= 0) atomicMax(&dmax[box0], bmax);
  } else if (box >= 0) {
    atomicMax(&dmax[box], bmax);
  }
}

void launch_h_extremes(const double *h, int n, const BoxDev *boxes, int n_boxes,
                       unsigned long long *dmax, unsigned long long *dminmax, cudaStream_t s) {
  const int threads = (n + kExtItems - 1) / kExtItems;
  k_h_extremes<<<(threads + 255) / 256, 256, 0, s>>>(h, n, boxes, n_boxes, dmax, dminmax);
  note_launch();
}

__global__ void k_validate(const double *x, const float *v, const float *m, const float *u,
                           const double *h, int n, int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  bool ok = m[k] > 0.f && isfinite(m[k]) && u[k] >= 0.f && isfinite(u[k]) && h[k] > 0.0 &&
            isfinite(h[k]);
  for (int d = 0; d < 3; ++d)
    ok = ok && isfinite(x[3 * (size_t)k + d]) && isfinite(v[3 * (size_t)k + d]);
  if (!ok) atomicOr(status, kErrInvalidInput);
}

void launch_validate(const double *x, const float *v, const float *m, const float *u,
                     const double *h, int n, int *status, cudaStream_t s) {
  k_validate<<<(n + 255) / 256, 256, 0, s>>>(x, v, m, u, h, n, status); note_launch();
}

__global__ void k_reset_iteration(unsigned char *done, int *niter, double *hlo, double *hhi,
                                  float *fprev, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  done[s] = 0;
  niter[s] = 0;
  hlo[s] = 0.0;
  hhi[s] = 1e308;
  fprev[s] = __int_as_float(0x7f800000);
}

void launch_reset_iteration(unsigned char *done, int *niter, double *hlo, double *hhi,
                            float *fprev, int n, cudaStream_t s) {
  k_reset_iteration<<<(n + 255) / 256, 256, 0, s>>>(done, niter, hlo, hhi, fprev, n);
  note_launch();
}

__global__ void k_leaf_of(const Leaf *leaves, int n_leaves, int *leaf_of) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= n_leaves) return;
  const Leaf L = leaves[li];
  for (int k = 0; k < L.count; ++k) leaf_of[L.start + k] = li;
}

void launch_leaf_of(const Leaf *leaves, int n_leaves, int *leaf_of, cudaStream_t s) {
  k_leaf_of<<<(n_leaves + 255) / 256, 256, 0, s>>>(leaves, n_leaves, leaf_of); note_launch();
}

struct GetArgs {
  int field;
  void *out;
  const int *orig;
  int n;
  StoreArrays st;
  const float *rho, *omega, *P;
  const int *nngb, *niter, *nforce;
};

__global__ void k_get(GetArgs a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n) return;
  const size_t k = (size_t)a.orig[s];
  switch (a.field) {
    case SPH_X: {
      double *o = (double *)a.out;
      o[3 * k] = a.st.x0[s];
      o[3 * k + 1] = a.st.x1[s];
      o[3 * k + 2] = a.st.x2[s];
    } break;
    case SPH_V: {
      float *o = (float *)a.out;
      const float4 v = a.st.vu[s];
      o[3 * k] = v.x;
      o[3 * k + 1] = v.y;
      o[3 * k + 2] = v.z;
    } break;
    case SPH_U: ((float *)a.out)[k] = a.st.vu[s].w; break;
    case SPH_H: ((double *)a.out)[k] = a.st.h[s]; break;
    case SPH_RHO: ((float *)a.out)[k] = a.rho[s]; break;
    case SPH_OMEGA: ((float *)a.out)[k] = a.omega[s]; break;
    case SPH_P: ((float *)a.out)[k] = a.P[s]; break;
    case SPH_A: {
      float *o = (float *)a.out;
      const float4 v = a.st.acc[s];
      o[3 * k] = v.x;
      o[3 * k + 1] = v.y;
      o[3 * k + 2] = v.z;
    } break;
    case SPH_DUDT: ((float *)a.out)[k] = a.st.acc[s].w; break;
    case SPH_NNGB: ((int *)a.out)[k] = a.nngb[s]; break;
    case SPH_NITER: ((int *)a.out)[k] = a.niter[s]; break;
    case SPH_NFORCE: ((int *)a.out)[k] = a.nforce[s]; break;
    case SPH_M: ((float *)a.out)[k] = a.st.m[s]; break;
    default: break;
  }
}

void launch_get(int field, void *out, const int *orig, int n, const StoreArrays &st,
                const float *rho, const float *omega, const float *P, const int *nngb,
                const int *niter, const int *nforce, cudaStream_t s) {
  GetArgs a{field, out, orig, n, st, rho, omega, P, nngb, niter, nforce};
  k_get<<<(n + 255) / 256, 256, 0, s>>>(a); note_launch();
}

}  // namespace sph
