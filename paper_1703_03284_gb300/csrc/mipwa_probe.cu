// Throughput probes of the arithmetic pipes the likelihood kernels run on
// (mipwa_probe_peak): the peaks their roofline fractions are quoted against,
// measured on the GPU at hand instead of taken from unit counts.
//
// Each probe is a grid of SMs x 4 blocks x 256 threads (32 warps per SM), every
// thread running eight independent dependency chains of one instruction kind
// for a given number of iterations, so that the pipe, not latency, limits the
// rate. The host times it with CUDA events and reports operations per second
// (one fused multiply-add = 2 flops; a packed f32x2 one = 4; a special-function
// approximation = 1 operation).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mipwa.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 4;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_ffma(float* out, int iters, float m,
                                                            float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma2(float* out, int iters, float m,
                                                             float c) {
  unsigned long long a[kChains];
  unsigned long long mm, cc;
  asm("mov.b64 %0, {%1, %1};" : "=l"(mm) : "f"(m));
  asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    const float x = (float)(threadIdx.x + k) * 1e-3f, y = x + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(x), "f"(y));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(mm), "l"(cc));
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[k]));
    s += x + y;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dfma(float* out, int iters, float m,
                                                            float c) {
  double a[kChains];
  const double md = m, cd = c;
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], md, cd);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// Special-function unit: rsqrt.approx.ftz.f32 (the FP32 kernels' square roots
// and, via rcp.approx, their reciprocals run on the same unit). The chain
// x <- rsqrt(x) * m + c keeps x positive and finite; it costs one FMA per
// approximation, which the FMA pipe absorbs.
__global__ void __launch_bounds__(kProbeThreads) probe_mufu(float* out, int iters, float m,
                                                            float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0f + (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      float r;
      asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
      a[k] = fmaf(r, m, c);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_probe(int kind, int grid, float* out, int iters) {
  // m, c keep every chain bounded: x -> 0.5 x + 0.25 (FMA), x -> rsqrt(x) + 0.5
  switch (kind) {
    case MIPWA_PROBE_FFMA: probe_ffma<<<grid, kProbeThreads>>>(out, iters, 0.5f, 0.25f); break;
    case MIPWA_PROBE_FFMA2: probe_ffma2<<<grid, kProbeThreads>>>(out, iters, 0.5f, 0.25f); break;
    case MIPWA_PROBE_DFMA: probe_dfma<<<grid, kProbeThreads>>>(out, iters, 0.5f, 0.25f); break;
    case MIPWA_PROBE_MUFU: probe_mufu<<<grid, kProbeThreads>>>(out, iters, 1.0f, 0.5f); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

double ops_per_iteration(int kind) {
  switch (kind) {
    case MIPWA_PROBE_FFMA: return 2.0 * kChains;
    case MIPWA_PROBE_FFMA2: return 4.0 * kChains;
    case MIPWA_PROBE_DFMA: return 2.0 * kChains;
    default: return 1.0 * kChains;
  }
}

}  // namespace

extern "C" int mipwa_probe_peak(int device, int kind, double target_ms, double* ops_per_s,
                                double* ms) {
  if (!ops_per_s || kind < MIPWA_PROBE_FFMA || kind > MIPWA_PROBE_MUFU || !(target_ms > 0) ||
      target_ms > 10000.0)
    return MIPWA_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return MIPWA_ECUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return MIPWA_ECUDA;
  }
  const int grid = sms * kProbeBlocksPerSM;
  float* out = nullptr;
  if (cudaMalloc(&out, (size_t)grid * kProbeThreads * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return MIPWA_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MIPWA_OK;
  float t = 0.0f;
  int iters = 1024;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MIPWA_ECUDA;
  // calibrate: grow the iteration count until one launch takes a tenth of the
  // target, then time one launch of target_ms (capped at 2^30 iterations)
  for (int pass = 0; rc == MIPWA_OK && pass < 24; ++pass) {
    if (launch_probe(kind, grid, out, iters) != cudaSuccess ||
        cudaEventRecord(e0) != cudaSuccess || launch_probe(kind, grid, out, iters) != cudaSuccess ||
        cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      rc = MIPWA_ECUDA;
      break;
    }
    if (t >= 0.1 * target_ms || iters >= (1 << 26)) {
      const double scale = target_ms / (t > 1e-3f ? t : 1e-3f);
      const double want = iters * scale;
      iters = (int)(want < (double)(1 << 30) ? (want > 1.0 ? want : 1.0) : (double)(1 << 30));
      if (cudaEventRecord(e0) != cudaSuccess ||
          launch_probe(kind, grid, out, iters) != cudaSuccess ||
          cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        rc = MIPWA_ECUDA;
      break;
    }
    iters *= 4;
  }
  if (rc == MIPWA_OK) {
    const double ops = (double)grid * kProbeThreads * (double)iters * ops_per_iteration(kind);
    *ops_per_s = ops / (t * 1e-3);
    if (ms) *ms = t;
  } else {
    cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
