// gather.cu -- trajectory storage: resolution of the output trajectories from the stored
// pairs and the coalesced gather, with the smoothing moments fused in.
//
// The output trajectory n at time t is X_t[sigma_t(n)], where sigma_t(n) composes the
// resampling arrays of the Remark in Section 3.1 from the root down to the leaf t: at
// every level whose combination covers t, n <- l_n (t in the left block) or r_n (right).
// The composition runs top-down, one level per launch (all combinations of the level, of
// every sequence of a batch, together): for a combination with blocks starting at a and c,
// S[a][n] <- l[S[a][n]] and S[c][n] <- r[S[a][n]] (at the root S[a][n] = n).  After level
// 0, S[t][n] is sigma_t(n) for every t (every t starts a block at the level where it is a
// right child, or is 0).  Slot N of S carries the extra root draw (I*, J*) of a
// conditional sweep down the same way.  Algorithm 1 copies the trajectories at every level
// instead; the result is the same (the tests check it bit for bit against the oracle's
// explicit copies), but this form moves O(K N (d + L)) bytes once instead of O(K N d L).
#include "kernels.cuh"

namespace dsmc {

namespace {

constexpr int kGatherThreads = 256;
constexpr int kResolveThreads = 256;

// One level of the top-down composition.  S is the sequence's first-map buffer ([2][K][N]
// int32, free once every level is merged), used as [K][N+1].
__global__ void __launch_bounds__(kResolveThreads) resolve_level_kernel(MergeArgs a, int chunks) {
  const int s = blockIdx.x / chunks, ch = blockIdx.x - s * chunks;
  const Comb cb = comb_of(a, s);
  const int N = a.N;
  const size_t W = (size_t)N + 1;
  int32_t* S = cb.first;
  const int32_t* pl = cb.pairs + (size_t)cb.gid * 2 * N;
  const int32_t* pr = pl + N;
  bool corrupt = false;
  for (int n = ch * kResolveThreads + threadIdx.x; n <= N; n += chunks * kResolveThreads) {
    int l, r;
    if (n == N && cb.root) {   // the root draw of a conditional sweep (0 otherwise)
      l = checked_index(cb.star[0], N, corrupt);
      r = checked_index(cb.star[1], N, corrupt);
    } else {
      const int sg = cb.root ? n : checked_index(S[(size_t)cb.at * W + n], N, corrupt);
      l = checked_index(pl[sg], N, corrupt);
      r = checked_index(pr[sg], N, corrupt);
    }
    S[(size_t)cb.at * W + n] = l;
    S[(size_t)cb.c * W + n] = r;
  }
  if (corrupt) record_status(a.ws.status, DSMC_ERR_INVALID_ARG);
}

// The gather of time t (one CTA): X_t[S[t][n]] for every n, the moments, the trajectories
// and the next reference.
template <int D>
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(GatherArgs a) {
  constexpr int NW = kGatherThreads / 32;
  int t = blockIdx.x;
  const int N = a.N, d = a.d;
  const size_t W = (size_t)N + 1;
  // this block's sequence: the call's own, or one of a batch
  const float *X = a.X, *logw = a.logw;
  const int32_t *S = a.S, *star = a.star;
  float *traj = a.traj, *x_star = a.x_star;
  double *mean = a.mean, *m2 = a.m2, *logL_out = nullptr;
  const double* logL = nullptr;
  int L = a.L;
  if (a.seqs != nullptr) {
    int seq;
    batch_time(a.kstart, a.n_seq, blockIdx.x, seq, t);
    const SeqDesc& q = a.seqs[seq];
    X = q.X;
    logw = q.logw;
    S = q.first;
    star = q.star;
    traj = nullptr;
    x_star = q.conditional ? q.x_star : nullptr;
    mean = q.mean;
    m2 = q.m2;
    logL_out = q.logL_out;
    logL = q.logL;
    L = q.L;
  }
  const float* Xt = X + (size_t)t * N * d;
  const int32_t* St = S + (size_t)t * W;
  const bool leaf = (L == 0);  // K == 1: the root is the weighted leaf, sigma = identity
  if (logL_out && t == 0 && threadIdx.x == 0) *logL_out = logL[0];
  float s1[D], s2[D];
#pragma unroll
  for (int k = 0; k < D; ++k) s1[k] = s2[k] = 0.f;
  bool corrupt = false;
  for (int n = threadIdx.x; n < N; n += kGatherThreads) {
    const int idx = leaf ? n : checked_index(St[n], N, corrupt);
    const float* xp = Xt + (size_t)idx * d;
    const float w = leaf ? expf(logw[n]) : 1.f;
    float x[D];
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = k < d ? xp[k] : 0.f;
    if (traj) {
      float* o = traj + ((size_t)t * N + n) * d;
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
    const double scale = leaf ? 1.0 : 1.0 / (double)N;
    mean[(size_t)t * d + threadIdx.x] = v1 * scale;
    if (m2) m2[(size_t)t * d + threadIdx.x] = v2 * scale;
  }
  // conditional mode: the next reference, from the extra root draw (I*, J*)
  if (x_star && threadIdx.x == 0) {
    const int sidx = leaf ? checked_index(star[0], N, corrupt)  // K == 1: the draw from the weighted leaf
                          : checked_index(St[N], N, corrupt);
    if (corrupt) record_status(a.status, DSMC_ERR_INVALID_ARG);
    for (int k = 0; k < d; ++k) x_star[(size_t)t * d + k] = Xt[(size_t)sidx * d + k];
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
  // a.K blocks: the call's time steps, or every time step of a batch (sum of its K)
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

cudaError_t launch_resolve_level(const MergeArgs& a, cudaStream_t s) {
  const int chunks = (a.N + 1 + kResolveThreads - 1) / kResolveThreads;
  resolve_level_kernel<<<(unsigned)((size_t)a.mc * chunks), kResolveThreads, 0, s>>>(a, chunks);
  return cudaGetLastError();
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
