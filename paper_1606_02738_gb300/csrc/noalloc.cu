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
// Method: the same sums and the same smoothing-length update rule as the
// per-pass density form (h_newton_step, FP64 h and bracket), but neighbours
// are found by scanning every particle of the box (all pairs, minimum image),
// which is what makes a fixed-size scratch possible; hence the particle cap
// SPH_NOALLOC_MAX_PARTICLES.
//
// Scratch: `g_na` below (about 0.9 MB) belongs to this library's CUDA module.
// The module, and with it the array, is loaded into a device's context when
// that context first needs it: at context creation when the process runs with
// CUDA_MODULE_LOADING=EAGER, otherwise (lazy loading, the default of recent
// CUDA releases) at the first use of anything in the module on that device,
// which may be this entry point's first call. That first load is the one
// allocation involved, made by the CUDA runtime; a caller that must see no
// allocation at all makes one warm-up call per device (or sets
// CUDA_MODULE_LOADING=EAGER) before it relies on that. The array then lives
// until the process exits. It is shared by all calls: the kernels clear what
// must start at zero, and two calls whose work overlaps on the GPU (different
// streams, or different host threads without ordering) race on it and give
// wrong results. Host code cannot use the symbol as a device address, so the
// first call on each device asks the runtime for the array's device address
// (cudaGetSymbolAddress) and caches it.
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
  double iL[3];  // 1 / L (minimum image by a product, no FP64 division per pair)
  double hcap;   // largest allowed h: min(L) / (3 (1 + 1e-6)), as the regular path
  const double *x;
  const float *m;
  double n_ngb, tol;
  int max_iter;
  NaScratch *s;  // device address of g_na
  double *h_out;
  float *rho_out, *omega_out;
};

// Iteration state from the caller's guesses; h0 <= 0, m <= 0 or a
// non-finite x, h0 or m raises kErrInvalidInput (the call then returns
// SPH_EINVAL before any density pass).
__global__ void k_na_init(NaArgs a, const double *h0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    a.s->status = 0;
    a.s->unconverged = 0;
  }
  if (i >= a.n) return;
  const double h = h0[i];
  const float m = a.m[i];
  const double x0 = a.x[3 * (size_t)i], x1 = a.x[3 * (size_t)i + 1], x2 = a.x[3 * (size_t)i + 2];
  const bool ok = h > 0.0 && isfinite(h) && m > 0.f && isfinite(m) && isfinite(x0) &&
                  isfinite(x1) && isfinite(x2);
  if (!ok) atomicOr(&a.s->status, kErrInvalidInput);
  a.s->h[i] = ok ? h : 1.0;
  a.s->lo[i] = 0.0;
  a.s->hi[i] = 1e308;  // open bracket, as HIter expects
  a.s->fprev[i] = __int_as_float(0x7f800000);
  a.s->done[i] = ok ? 0 : 1;
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
      d0 = fma(-a.L[0], rint(d0 * a.iL[0]), d0);
      d1 = fma(-a.L[1], rint(d1 * a.iL[1]), d1);
      d2 = fma(-a.L[2], rint(d2 * a.iL[2]), d2);
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

// Smoothing-length update by h_newton_step (the rule of the per-pass ghost
// kernel: Newton on ln N(ln h) inside the bisection bracket, FP64 h) and,
// once converged, rho and Omega (FP64 from the FP32 sums).
__global__ void k_na_update(NaArgs a, int pass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n || a.s->done[i]) return;
  const float4 s = a.s->sums[i];
  HIter it;
  it.start(a.s->h[i], a.s->lo[i], a.s->hi[i], a.s->fprev[i]);
  const double h = it.h;
  int st = 0;
  const bool conv = h_newton_step(it, s.x, s.y, a.n_ngb, a.tol * a.n_ngb, a.hcap, &st);
  if (st) atomicOr(&a.s->status, st);
  if (!conv) {
    a.s->h[i] = it.h;
    a.s->lo[i] = it.lo;
    a.s->hi[i] = it.hi;
    a.s->fprev[i] = it.fprev;
    if (pass + 1 >= a.max_iter) atomicOr(&a.s->status, kErrNotConverged);
    atomicAdd(&a.s->unconverged, 1);
    return;
  }
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
  for (int d = 0; d < 3; ++d) {
    a.L[d] = box_len[d];
    a.iL[d] = 1.0 / box_len[d];
  }
  a.hcap = std::fmin(box_len[0], std::fmin(box_len[1], box_len[2])) / (3.0 * (1.0 + 1e-6));
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
  // each launch is checked as it is made, so an error reported here is one
  // of this call's launches
  k_na_init<<<blocks, kNaThreads, 0, st>>>(a, h0);
  if (cudaGetLastError() != cudaSuccess) return SPH_ECUDA;
  for (int pass = 0; pass < max_iter; ++pass) {
    k_na_clear_counter<<<1, 1, 0, st>>>(a.s);
    if (cudaGetLastError() != cudaSuccess) return SPH_ECUDA;
    k_na_sums<<<blocks, kNaThreads, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return SPH_ECUDA;
    k_na_update<<<blocks, kNaThreads, 0, st>>>(a, pass);
    if (cudaGetLastError() != cudaSuccess) return SPH_ECUDA;
    int counters[2] = {0, 0};
    if (cudaMemcpyAsync(counters, &a.s->status, sizeof counters, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SPH_ECUDA;
    const int status = counters[0];
    if (status & kErrInvalidInput) return SPH_EINVAL;
    if (status & kErrBoxTooSmall) return SPH_EBOXTOOSMALL;
    if (status & kErrNonPhysical) return SPH_ENONPHYSICAL;
    if (counters[1] == 0) return SPH_OK;
  }
  return SPH_ENOTCONVERGED;
}
