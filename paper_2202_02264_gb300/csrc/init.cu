// init.cu -- Algorithm 2 (smoother initialisation), and its conditional form (Section 3.2).
//
// One CTA per time step t.  Each thread draws particles x_t^n ~ q_t from Philox normals
// (Box-Muller; uniform proposals from the uniforms themselves), writes them, and computes
// the leaf log-weight
//   t = 0:  log h_0(y_0 | x) + log P_0(x) - log q_0(x)
//   t >= 1: log nu_t(x) - log q_t(x)          (exactly 0 when nu_t = q_t)
// The CTA then normalises the N weights of its t by a log-sum-exp and stores
// log L_t = LSE - log N.  HBM-bound: writes K N (d + 1) floats.
#include "kernels.cuh"

namespace dsmc {

namespace {

constexpr int kInitThreads = 256;

// UNIF: the uniform proposal (a separate instance, so the Gaussian proposals' instance keeps
// its registers and four CTAs per SM for D <= 4).
template <int D, bool UNIF>
__global__ void __launch_bounds__(kInitThreads, D <= 4 ? 4 : 1) init_kernel(InitArgs a, ModelParams<D> mp) {
  int t = blockIdx.x;
  const int N = a.N, d = a.d;
  // this block's sequence: the call's own, or one of a batch
  uint64_t seed = a.seed;
  uint32_t base = a.base;
  const float *y = a.y, *x_ref = a.x_ref, *pmean = mp.prop_mean, *pstd = mp.prop_std;
  float *X = a.X, *logw = a.logw;
  double* logL = a.logL;
  if (a.seqs != nullptr) {
    int seq;
    batch_time(a.kstart, a.n_seq, blockIdx.x, seq, t);
    const SeqDesc& q = a.seqs[seq];
    seed = q.seed;
    base = q.base;
    y = q.y;
    x_ref = q.x_ref;
    pmean = q.prop_mean;
    pstd = q.prop_std;
    X = q.X;
    logw = q.logw;
    logL = q.logL;
  }
  float yt[D], qm[D], qs[D];
#pragma unroll
  for (int k = 0; k < D; ++k) yt[k] = k < d ? y[(size_t)t * d + k] : 0.f;
  proposal_at<D>(mp, y, pmean, pstd, t, qm, qs);
  float qinv[D];
  const float qnorm = proposal_consts<D>(d, qs, qinv);
  float logsd = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (k < d) logsd += logf(qs[k]);

  float* lw = logw + (size_t)t * N;
  float lmax = -INFINITY;
  bool bad = false;
  const bool uniform = (t > 0 && mp.nu == DSMC_NU_EQ_Q);
  constexpr bool unif = UNIF;
  for (int n = threadIdx.x; n < N; n += kInitThreads) {
    float x[D], z[D];
    if (unif) {  // q_t = U([-s, s]^d): x = s (2 u - 1) from the words of counter j = k / 4
#pragma unroll
      for (int k = 0; k < D; ++k) z[k] = 0.f;
      if (x_ref != nullptr && n == 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = k < d ? x_ref[(size_t)t * d + k] : 0.f;
      } else {
#pragma unroll
        for (int j = 0; j < (D + 3) / 4; ++j) {
          if (4 * j < d) {
            const uint4 w = draw(seed, (uint32_t)n, (uint32_t)t, kPurposeInit, base, (uint32_t)j);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int k = 4 * j + p;
              if (k < D) x[k] = k < d ? mp.prop_scale * fmaf(2.f, u23(ws[p]), -1.f) : 0.f;
            }
          }
        }
      }
    } else if (x_ref != nullptr && n == 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        x[k] = k < d ? x_ref[(size_t)t * d + k] : 0.f;
        z[k] = k < d ? (x[k] - qm[k]) / qs[k] : 0.f;
      }
    } else {
#pragma unroll
      for (int j = 0; j < (D + 3) / 4; ++j) {
        if (4 * j < d) {
          const uint4 w = draw(seed, (uint32_t)n, (uint32_t)t, kPurposeInit, base, (uint32_t)j);
          const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const float r = sqrtf(-2.f * logf(u23(ws[2 * p])));
            float sn, cs;
            sincospif(2.f * u23(ws[2 * p + 1]), &sn, &cs);
            const int k0 = 4 * j + 2 * p;
            if (k0 < D) z[k0] = r * cs;
            if (k0 + 1 < D) z[k0 + 1] = r * sn;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (k >= d) z[k] = 0.f;
        x[k] = k < d ? fmaf(qs[k], z[k], qm[k]) : 0.f;
      }
    }
    float* xo = X + ((size_t)t * N + n) * d;
    if ((D % 4) == 0 && d == D) {  // 16-byte vector stores (rows of D floats)
#pragma unroll
      for (int k4 = 0; k4 < D / 4; ++k4)
        reinterpret_cast<float4*>(xo)[k4] = make_float4(x[4 * k4], x[4 * k4 + 1], x[4 * k4 + 2], x[4 * k4 + 3]);
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (k < d) xo[k] = x[k];
    }
    float lq = 0.f;
    if (unif) {
      lq = log_q_uniform<D>(mp, x);
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (k < d) lq = fmaf(-0.5f * z[k], z[k], lq);
      lq -= logsd + (float)d * kHalfLog2Pi;
    }
    float l;
    if (t == 0) {
      l = log_h<D>(mp, yt, x) + log_p0<D>(mp, x) - lq;
    } else if (mp.nu == DSMC_NU_EQ_Q) {
      l = 0.f;
    } else {
      l = log_nu<D>(mp, yt, qm, qinv, qnorm, x) - lq;
    }
    if (isnan(l)) bad = true;
    lw[n] = uniform ? -a.logN : l;
    lmax = fmaxf(lmax, l);
  }
  // nu_t = q_t at t >= 1: every log-weight is exactly 0, so the normalised weights are
  // exactly -log N and log L_t = 0 (what the general path below computes, without it)
  if (uniform) {
    if (threadIdx.x == 0) logL[t] = 0.0;
    return;
  }

  __shared__ float red[kInitThreads / 32];
  __shared__ float reds[kInitThreads / 32];
  __shared__ float lse_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // block max
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if (lane == 0) red[warp] = lmax;
  __syncthreads();
  float M = red[0];
#pragma unroll
  for (int w = 1; w < kInitThreads / 32; ++w) M = fmaxf(M, red[w]);
  // block sum of exp(l - M): FP32 within each warp (a few terms per thread, then a
  // butterfly), FP64 across the warps and for the log, by one thread (FP64 is slow here)
  float s = 0.f;
  for (int n = threadIdx.x; n < N; n += kInitThreads) s += expf(lw[n] - M);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) reds[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
#pragma unroll
    for (int w = 0; w < kInitThreads / 32; ++w) S += (double)reds[w];
    const double lse = (double)M + log(S);
    lse_s = (float)lse;
    logL[t] = lse - log((double)N);
  }
  __syncthreads();
  const float lsef = lse_s;
  for (int n = threadIdx.x; n < N; n += kInitThreads) lw[n] = lw[n] - lsef;
  if (bad || !(M > -INFINITY)) record_status(a.status, bad ? DSMC_ERR_NONFINITE : DSMC_ERR_DEGENERATE);
}

template <int D>
cudaError_t launch_init_t(const InitArgs& a, const void* mp, cudaStream_t s) {
  const ModelParams<D>& p = *static_cast<const ModelParams<D>*>(mp);
  if (p.prop_kind == DSMC_PROP_UNIFORM)
    init_kernel<D, true><<<a.K, kInitThreads, 0, s>>>(a, p);
  else
    init_kernel<D, false><<<a.K, kInitThreads, 0, s>>>(a, p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init(int D, const InitArgs& a, const void* mp, cudaStream_t s) {
  switch (D) {
    case 1: return launch_init_t<1>(a, mp, s);
    case 2: return launch_init_t<2>(a, mp, s);
    case 4: return launch_init_t<4>(a, mp, s);
    case 8: return launch_init_t<8>(a, mp, s);
    case 16: return launch_init_t<16>(a, mp, s);
    case 32: return launch_init_t<32>(a, mp, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dsmc
