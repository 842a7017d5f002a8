// unit_rates.cu -- standalone GB300 throughput probe (not part of libdsmc): MUFU ex2, FP32
// FFMA, packed FFMA2 and FADD, in results per clock per SM from wall time at the sampled
// clock.  These rates set the roofline of the fused exp kernels.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o unit_rates unit_rates.cu && ./unit_rates
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int MODE>
__global__ void probe(float* out, int iters) {
  float a[8];
  float2 b[8];
  for (int k = 0; k < 8; ++k) {
    a[k] = -1.0f - 0.001f * (threadIdx.x + k);
    b[k] = make_float2(a[k], a[k] * 0.5f);
  }
  const float2 m2 = make_float2(0.999f, 0.998f), c2 = make_float2(1e-3f, 2e-3f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (MODE == 0) a[k] = ex2(-a[k]);
      else if (MODE == 1) a[k] = fmaf(a[k], 0.999f, 1e-3f);
      else if (MODE == 2) b[k] = __ffma2_rn(b[k], m2, c2);
      else a[k] = a[k] + 1e-3f;
    }
  }
  float s = 0.f;
  for (int k = 0; k < 8; ++k) s += a[k] + b[k].x + b[k].y;
  if (s == 123.456f) out[0] = s;
}

int main() {
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, 0);
  const int sms = p.multiProcessorCount, threads = 256, per_sm = 4, iters = 4096;
  float* out;
  cudaMalloc(&out, 4);
  const char* names[] = {"ex2 (MUFU)", "ffma", "ffma2 (lane-ops)", "fadd"};
  printf("device %s, %d SMs\n", p.name, sms);
  for (int mode = 0; mode < 4; ++mode) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0);
      if (mode == 0) probe<0><<<sms * per_sm, threads>>>(out, iters);
      if (mode == 1) probe<1><<<sms * per_sm, threads>>>(out, iters);
      if (mode == 2) probe<2><<<sms * per_sm, threads>>>(out, iters);
      if (mode == 3) probe<3><<<sms * per_sm, threads>>>(out, iters);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    const double ops = (double)sms * per_sm * threads * iters * 8;
    printf("%-18s %.3f ms  %.3e ops/s  %.1f ops/clk/SM at 2070 MHz, %.1f at 1950 MHz\n", names[mode], best,
           ops / (best * 1e-3), ops / (best * 1e-3) / sms / 2.07e9, ops / (best * 1e-3) / sms / 1.95e9);
  }
  cudaError_t e = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
