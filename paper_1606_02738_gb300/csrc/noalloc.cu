// noalloc.cu -- sph_density_noalloc: the h-iterated density stage for one
// small periodic box, using no device allocation at all.
//
// Who needs it: callers that must not allocate device memory on the calls
// they make -- a host framework that owns every byte of the GPU through its
// own pool and forbids foreign cudaMalloc/cudaFree (a call that can also
// synchronise the device at an awkward moment), or code that runs where a new
// allocation would fail or stall. The regular entry points allocate their
// particle store and task lists; this one keeps its per-particle scratch in a
// fixed, file-scope __device__ array instead.
//
// Method: the same sums and the same smoothing-length update as the regular
// density stage, but neighbours are found by scanning every particle of the
// box (all pairs, minimum image), which is what makes a fixed-size scratch
// possible; hence the particle cap SPH_NOALLOC_MAX_PARTICLES.
//
// Scratch: `g_na` below (about 0.9 MB) is allocated by the CUDA runtime when
// the library is loaded, on every device that loads it, and lives until the
// process exits. It is shared by all calls: the kernels clear what must start
// at zero, and two calls whose work overlaps on the GPU (different streams,
// or different host threads without ordering) race on it and give wrong
// results. Host code cannot use the symbol as a device address, so the
// first call on each device asks the runtime for the array's device address
// (cudaGetSymbolAddress) and caches it; make that first call before any
// stream capture begins.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/sph.h"
#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr int kNaMax = SPH_NOALLOC_MAX_PARTICLES;
constexpr int kNaThreads = 128;

struct NaScratch {
  float4 sums[kNaMax];  // sum w, sum q w', sum m w, sum m (3 w + q w')
  double h[kNaMax];     // current smoothing length
  double lo[kNaMax];    // root bracket
  double hi[kNaMax];
  float fprev[kNaMax];  // |N - n_ngb| of the previous pass
  int done[kNaMax];
  int status;           // kErr* bits
  int unconverged;      // particles still iterating after the last pass
};

static __device__ __align__(256) NaScratch g_na;

struct NaArgs {
  int n;
  double L[3];
  const double *x;
  const float *m;
  double n_ngb, tol;
  int max_iter;
  NaScratch *s;  // device address of g_na
  double *h_out;
  float *rho_out, *omega_out;
};

__global__ void k_na_init(NaArgs a, const double *h0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    a.s->status = 0;
    a.s->unconverged = 0;
  }
  if (i >= a.n) return;
  a.s->h[i] = h0[i];
  a.s->lo[i] = 0.0;
  a.s->hi[i] = 1e308;
  a.s->fprev[i] = __int_as_float(0x7f800000);
  a.s->done[i] = 0;
}

// All-pairs density sums at the current h of every unfinished particle.
__global__ void __launch_bounds__(kNaThreads) k_na_sums(NaArgs a) {
  __shared__ double sx[kNaThreads], sy[kNaThreads], sz[kNaThreads];
  __shared__ float sm[kNaThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < a.n && !a.s->done[i];
  double xi = 0, yi = 0, zi = 0, h = 1.0;
  if (i < a.n) {
    xi = a.x[3 * (size_t)i];
    yi = a.x[3 * (size_t)i + 1];
    zi = a.x[3 * (size_t)i + 2];
    h = a.s->h[i];
  }
  const float hf = (float)h, hinv = 1.f / hf, h2 = act ? hf * hf : -1.f;
  float sw = 0.f, sdw = 0.f, smw = 0.f, smdh = 0.f;
  for (int base = 0; base < a.n; base += kNaThreads) {
    const int j = base + threadIdx.x;
    __syncthreads();
    if (j < a.n) {
      sx[threadIdx.x] = a.x[3 * (size_t)j];
      sy[threadIdx.x] = a.x[3 * (size_t)j + 1];
      sz[threadIdx.x] = a.x[3 * (size_t)j + 2];
      sm[threadIdx.x] = a.m[j];
    }
    __syncthreads();
    const int nj = min(kNaThreads, a.n - base);
    for (int k = 0; k < nj; ++k) {
      double d0 = xi - sx[k], d1 = yi - sy[k], d2 = zi - sz[k];
      d0 -= a.L[0] * rint(d0 / a.L[0]);
      d1 -= a.L[1] * rint(d1 / a.L[1]);
      d2 -= a.L[2] * rint(d2 / a.L[2]);
      const float dx = (float)d0, dy = (float)d1, dz = (float)d2;
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (r2 < h2) {
        const float r = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
        const float q = r * hinv;
        float w, dw;
        w_and_dw(q, w, dw);
        const float qdw = q * dw;
        sw += w;
        sdw += qdw;
        smw = fmaf(sm[k], w, smw);
        smdh = fmaf(sm[k], fmaf(3.f, w, qdw), smdh);
      }
    }
  }
  if (act) a.s->sums[i] = make_float4(sw, sdw, smw, smdh);
}

// Smoothing-length update (the same rule as the regular ghost step) and,
// once converged, rho and Omega.
__global__ void k_na_update(NaArgs a, int pass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n || a.s->done[i]) return;
  const double h = a.s->h[i];
  const float4 s = a.s->sums[i];
  const double N = (32.0 / 3.0) * (double)s.x;
  const double dN = -(32.0 / (3.0 * h)) * (double)s.y;
  const double f = N - a.n_ngb;
  bool conv = fabs(f) <= a.tol * a.n_ngb;
  if (!conv) {
    double lo = a.s->lo[i], hi = a.s->hi[i];
    if (f < 0.0)
      lo = h;
    else
      hi = h;
    const double s_ln = (N > 0.0 && dN > 0.0) ? h * dN / N : 0.0;
    double hn = s_ln > 0.0 ? h * exp(log(a.n_ngb / N) / s_ln) : 2.0 * h;
    hn = fmin(fmax(hn, 0.125 * h), 2.0 * h);
    if (hi < 1e300 && (!(hn > lo && hn < hi) || fabs(f) > 0.5 * (double)a.s->fprev[i]))
      hn = 0.5 * (lo + hi);
    a.s->fprev[i] = (float)fabs(f);
    const double hcap = fmin(a.L[0], fmin(a.L[1], a.L[2])) / (3.0 * (1.0 + 1e-6));
    if (hn > hcap) {
      if (h >= hcap * (1.0 - 1e-12) && f < 0.0) atomicOr(&a.s->status, kErrBoxTooSmall);
      hn = hcap;
    }
    if (fabs(hn - h) <= 5e-7 * h) {
      conv = true;
    } else {
      a.s->h[i] = hn;
      a.s->lo[i] = lo;
      a.s->hi[i] = hi;
      if (pass + 1 >= a.max_iter) atomicOr(&a.s->status, kErrNotConverged);
      atomicAdd(&a.s->unconverged, 1);
    }
  }
  if (conv) {
    const double h2 = h * h;
    const double rho = 8.0 / 3.14159265358979323846 * (double)s.z / (h2 * h);
    const double drho = -8.0 / 3.14159265358979323846 * (double)s.w / (h2 * h2);
    const double omega = 1.0 + h / (3.0 * rho) * drho;
    a.h_out[i] = h;
    a.rho_out[i] = (float)rho;
    a.omega_out[i] = (float)omega;
    a.s->done[i] = 1;
    if (!(rho > 0.0) || !(omega > 0.0)) atomicOr(&a.s->status, kErrNonPhysical);
  }
}

__global__ void k_na_clear_counter(NaScratch *s) { s->unconverged = 0; }

// Device address of g_na, looked up once per device.
std::mutex g_na_mutex;
void *g_na_addr[64] = {};

}  // namespace
}  // namespace sph

using namespace sph;

extern "C" int sph_density_noalloc(int n, const double *box_len, const double *x,
                                   const float *m, const double *h0, double n_ngb, double h_tol,
                                   int max_iter, double *h_out, float *rho_out, float *omega_out,
                                   void *cuda_stream) {
  if (n < 1 || n > SPH_NOALLOC_MAX_PARTICLES) return SPH_EINVAL;  // beyond the fixed scratch
  if (!box_len || !x || !m || !h0 || !h_out || !rho_out || !omega_out) return SPH_EINVAL;
  if (!(n_ngb > 32.0 / 3.0) || !(h_tol > 0.0) || max_iter < 1) return SPH_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!(box_len[d] > 0.0) || !std::isfinite(box_len[d])) return SPH_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPH_ECUDA;
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_na) != cudaSuccess || !p) {
        cudaGetLastError();
        return SPH_ECUDA;
      }
      g_na_addr[dev] = p;
    }
    addr = g_na_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  NaArgs a;
  a.n = n;
  for (int d = 0; d < 3; ++d) a.L[d] = box_len[d];
  a.x = x;
  a.m = m;
  a.n_ngb = n_ngb;
  a.tol = h_tol;
  a.max_iter = max_iter;
  a.s = reinterpret_cast<NaScratch *>(addr);
  a.h_out = h_out;
  a.rho_out = rho_out;
  a.omega_out = omega_out;
  const int blocks = (n + kNaThreads - 1) / kNaThreads;
  k_na_init<<<blocks, kNaThreads, 0, st>>>(a, h0);
  int status = 0;
  for (int pass = 0; pass < max_iter; ++pass) {
    k_na_clear_counter<<<1, 1, 0, st>>>(a.s);
    k_na_sums<<<blocks, kNaThreads, 0, st>>>(a);
    k_na_update<<<blocks, kNaThreads, 0, st>>>(a, pass);
    int counters[2] = {0, 0};
    if (cudaMemcpyAsync(counters, &a.s->status, sizeof counters, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SPH_ECUDA;
    status = counters[0];
    if (status & kErrBoxTooSmall) return SPH_EBOXTOOSMALL;
    if (status & kErrNonPhysical) return SPH_ENONPHYSICAL;
    if (counters[1] == 0) return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ECUDA;
  }
  return SPH_ENOTCONVERGED;
}
