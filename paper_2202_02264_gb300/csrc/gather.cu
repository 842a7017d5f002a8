// gather.cu -- trajectory storage: resolution of the output trajectories from the stored
// pairs and the coalesced gather, with the smoothing moments fused in.
//
// The output trajectory n at time t is X_t[sigma_t(n)], where sigma_t(n) composes the
// resampling arrays of the Remark in Section 3.1 from the root down to the leaf t: at
// every level whose combination covers t, n <- l_n (t in the left block) or r_n (right).
// Algorithm 1 copies the trajectories at every level instead; the result is the same
// (the tests check it bit for bit against the oracle's explicit copies), but this form
// moves O(K N (d + L)) bytes once instead of O(K N d L).
#include "kernels.cuh"

namespace dsmc {

namespace {

constexpr int kGatherThreads = 256;

template <int D>
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(GatherArgs a) {
  constexpr int NW = kGatherThreads / 32;
  const int t = blockIdx.x;
  const int N = a.N, d = a.d, K = a.K;
  __shared__ int path_g[32];
  __shared__ int path_side[32];
  __shared__ int np_s;
  if (threadIdx.x == 0) {
    int np = 0;
    for (int l = a.L - 1; l >= 0; --l) {
      const int size = 1 << l;
      const int p = (t / (2 * size)) * 2 * size;
      if (p + size < K) {
        path_g[np] = a.level_off[l] + p / (2 * size);
        path_side[np] = t >= p + size ? 1 : 0;
        ++np;
      }
    }
    np_s = np;
  }
  __syncthreads();
  const int np = np_s;
  const float* Xt = a.X + (size_t)t * N * d;
  const bool weighted = (a.L == 0);  // K == 1: the root is the weighted leaf
  float s1[D], s2[D];
#pragma unroll
  for (int k = 0; k < D; ++k) s1[k] = s2[k] = 0.f;
  bool corrupt = false;
  // four independent walks per thread keep several dependent loads in flight
  constexpr int W = 4;
  for (int n0 = threadIdx.x; n0 < N; n0 += W * kGatherThreads) {
    int sidx[W];
#pragma unroll
    for (int q = 0; q < W; ++q) sidx[q] = min(n0 + q * kGatherThreads, N - 1);
    for (int p = 0; p < np; ++p) {
      const int32_t* pp = a.pairs + ((size_t)path_g[p] * 2 + path_side[p]) * N;
#pragma unroll
      for (int q = 0; q < W; ++q) sidx[q] = checked_index(pp[sidx[q]], N, corrupt);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int n = n0 + q * kGatherThreads;
      if (n >= N) continue;
      const float* xp = Xt + (size_t)sidx[q] * d;
      const float w = weighted ? expf(a.logw[n]) : 1.f;
      float x[D];
#pragma unroll
      for (int k = 0; k < D; ++k) x[k] = k < d ? xp[k] : 0.f;
      if (a.traj) {
        float* o = a.traj + ((size_t)t * N + n) * d;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k < d) o[k] = x[k];
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        s1[k] = fmaf(w, x[k], s1[k]);
        s2[k] = fmaf(w * x[k], x[k], s2[k]);
      }
    }
  }
  if (corrupt) record_status(a.status, DSMC_ERR_INVALID_ARG);
  // moments: FP32 within each warp (butterfly), FP64 across the warps by d threads only
  // (FP64 is slow on this part)
  __shared__ float red1[NW][D], red2[NW][D];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    float v1 = s1[k], v2 = s2[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v1 += __shfl_xor_sync(0xffffffffu, v1, o);
      v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    if (lane == 0) {
      red1[warp][k] = v1;
      red2[warp][k] = v2;
    }
  }
  __syncthreads();
  if (threadIdx.x < d) {
    double v1 = 0.0, v2 = 0.0;
    for (int w = 0; w < NW; ++w) {
      v1 += (double)red1[w][threadIdx.x];
      v2 += (double)red2[w][threadIdx.x];
    }
    const double scale = weighted ? 1.0 : 1.0 / (double)N;
    a.mean[(size_t)t * d + threadIdx.x] = v1 * scale;
    if (a.m2) a.m2[(size_t)t * d + threadIdx.x] = v2 * scale;
  }
  // conditional mode: the next reference, from the extra root draw (I*, J*)
  if (a.x_star && threadIdx.x == 0) {
    int sidx;
    if (np == 0) {
      sidx = checked_index(a.star[0], N, corrupt);  // K == 1: the draw from the weighted leaf
    } else {
      sidx = checked_index(a.star[path_side[0]], N, corrupt);
      for (int q = 1; q < np; ++q)
        sidx = checked_index(a.pairs[((size_t)path_g[q] * 2 + path_side[q]) * N + sidx], N, corrupt);
    }
    if (corrupt) record_status(a.status, DSMC_ERR_INVALID_ARG);
    for (int k = 0; k < d; ++k) a.x_star[(size_t)t * d + k] = Xt[(size_t)sidx * d + k];
  }
}

__global__ void philox_kernel(const uint4* ctr, int64_t n, uint64_t seed, uint4* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], (uint32_t)seed, (uint32_t)(seed >> 32));
}

// K == 1 in conditional mode: the next reference is one draw from the weighted leaf at
// t = 0 (slot N of the dense purpose, 53-bit uniform, FP64 inverse CDF).  One thread.
__global__ void k1_star_kernel(const float* logw, int N, uint64_t seed, uint32_t base, int32_t* star) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const uint4 w = draw(seed, (uint32_t)N, 0u, kPurposeDense, base, 0u);
  const unsigned long long m = ((unsigned long long)w.x << 21) | (unsigned long long)(w.y >> 11);
  const double u = ((double)m + 0.5) * 0x1p-53;
  double S = 0.0;
  for (int n = 0; n < N; ++n) S += exp((double)logw[n]);
  const double target = u * S;
  double c = 0.0;
  int pick = -1, last_pos = 0;
  for (int n = 0; n < N; ++n) {
    const double e = exp((double)logw[n]);
    c += e;
    if (e > 0.0) last_pos = n;
    if (c > target) { pick = n; break; }
  }
  star[0] = pick < 0 ? last_pos : pick;
  star[1] = star[0];
}

template <int D>
cudaError_t gather_t(const GatherArgs& a, cudaStream_t s) {
  gather_kernel<D><<<a.K, kGatherThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather(int D, const GatherArgs& a, cudaStream_t s) {
  switch (D) {
    case 1: return gather_t<1>(a, s);
    case 2: return gather_t<2>(a, s);
    case 4: return gather_t<4>(a, s);
    case 8: return gather_t<8>(a, s);
    case 16: return gather_t<16>(a, s);
    case 32: return gather_t<32>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_k1_star(const float* logw, int N, uint64_t seed, uint32_t base, int32_t* star,
                           cudaStream_t s) {
  k1_star_kernel<<<1, 32, 0, s>>>(logw, N, seed, base, star);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int th = 256;
  philox_kernel<<<(unsigned)((n + th - 1) / th), th, 0, s>>>(
      reinterpret_cast<const uint4*>(ctr), n, seed, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace dsmc
