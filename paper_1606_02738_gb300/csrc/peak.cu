// peak.cu -- sph_fp32_peak: the FP32 rate this device sustains on fused
// multiply-adds, measured, as a second denominator beside the one derived
// from SM count x 128 FP32 lanes x 2 flops x the maximum SM clock (the
// interaction kernels are FP32-ALU work, not a dense contraction).
//
// Every thread runs kChains independent FFMA chains (enough independent work
// to cover the pipeline latency at full occupancy); the loop is unrolled so
// that loop control takes about 1% of the issue slots. Chain values stay
// finite (|b| < 1) and are written only under a condition that never holds,
// which keeps the work live without memory traffic.
#include <cuda_runtime.h>

#include "../../include/sph.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;  // 2048 threads per SM
constexpr int kIters = 8192;     // per thread, a multiple of kUnroll

__global__ void __launch_bounds__(kThreads) k_ffma_peak(float *sink, int iters, float b,
                                                        float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)threadIdx.x + (float)k;
  for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.f) sink[blockIdx.x] = s;  // the chains converge to c / (1 - b) > 0
}

}  // namespace

extern "C" int sph_fp32_peak(int device, double *tflops_out, double *ms_out) {
  if (!tflops_out) return SPH_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return SPH_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return SPH_EINVAL;
  }
  int rc = SPH_OK;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float *sink = nullptr;
  int sms = 0;
  float best = 1e30f;
  do {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = SPH_ECUDA;
      break;
    }
    const int blocks = sms * kBlocksPerSM;
    if (cudaMalloc(&sink, sizeof(float) * (size_t)blocks) != cudaSuccess) {
      rc = SPH_ENOMEM;
      break;
    }
    for (int r = 0; r < 6 && rc == SPH_OK; ++r) {  // the first run warms up, best of 5
      cudaEventRecord(e0, s);
      k_ffma_peak<<<blocks, kThreads, 0, s>>>(sink, kIters, 0.999f, 1e-3f);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        rc = SPH_ECUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && ms < best) best = ms;
    }
    if (rc == SPH_OK) {
      const double flops = 2.0 * kChains * (double)kIters * kThreads * (double)blocks;
      *tflops_out = flops / (best * 1e-3) / 1e12;
      if (ms_out) *ms_out = best;
    }
  } while (false);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return rc;
}
