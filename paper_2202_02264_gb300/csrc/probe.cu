// probe.cu -- arithmetic unit rates of the device (MUFU ex2, FP32 FFMA, packed FFMA2,
// FADD, FP64 DFMA), measured with CUDA events on the caller's stream.  The fused exponential kernels
// are bound by these units, not by HBM, so their roofline denominators come from here
// (results per clock per SM) and the device's clock.
#include <cuda_runtime.h>

#include "dsmc.h"

namespace {

__device__ __forceinline__ float ex2_unit(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Eight independent dependency chains per thread; MODE 0 ex2, 1 FFMA, 2 FFMA2, 3 FADD,
// 4 DFMA.
// The sink store never happens for these inputs; it keeps the chains alive.
template <int MODE>
__global__ void unit_rate_kernel(float* sink, int iters) {
  float a[8];
  float2 b[8];
  double c[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = -1.0f - 0.001f * (float)(threadIdx.x + k);
    b[k] = make_float2(a[k], 0.5f * a[k]);
    c[k] = (double)a[k];
  }
  const float2 m2 = make_float2(0.999f, 0.998f), c2 = make_float2(1e-3f, 2e-3f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (MODE == 0) a[k] = ex2_unit(-a[k]);
      else if (MODE == 1) a[k] = fmaf(a[k], 0.999f, 1e-3f);
      else if (MODE == 2) b[k] = __ffma2_rn(b[k], m2, c2);
      else if (MODE == 3) a[k] = a[k] + 1e-3f;
      else c[k] = fma(c[k], 0.999, 1e-3);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k] + b[k].x + b[k].y + (float)c[k];
  if (s == 123.456f) sink[0] = s;
}

template <int MODE>
cudaError_t time_mode(float* sink, int sms, cudaStream_t st, double* ops_per_s) {
  constexpr int kThreads = 256, kPerSm = 4, kIters = 4096;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
    cudaEventRecord(e0, st);
    unit_rate_kernel<MODE><<<sms * kPerSm, kThreads, 0, st>>>(sink, kIters);
    e = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double ops = (double)sms * kPerSm * kThreads * kIters * 8;
  *ops_per_s = e == cudaSuccess ? ops / (best * 1e-3) : 0.0;
  return e;
}

}  // namespace

extern "C" dsmc_status_t dsmc_profile_unit_rates(float* sink, double ops_per_s[5], void* stream) {
  if (!sink || !ops_per_s) return DSMC_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DSMC_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DSMC_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (time_mode<0>(sink, sms, st, &ops_per_s[0]) != cudaSuccess) return DSMC_ERR_CUDA;
  if (time_mode<1>(sink, sms, st, &ops_per_s[1]) != cudaSuccess) return DSMC_ERR_CUDA;
  if (time_mode<2>(sink, sms, st, &ops_per_s[2]) != cudaSuccess) return DSMC_ERR_CUDA;
  if (time_mode<3>(sink, sms, st, &ops_per_s[3]) != cudaSuccess) return DSMC_ERR_CUDA;
  if (time_mode<4>(sink, sms, st, &ops_per_s[4]) != cudaSuccess) return DSMC_ERR_CUDA;
  return DSMC_OK;
}
