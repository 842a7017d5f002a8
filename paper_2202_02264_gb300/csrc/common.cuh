// common.cuh -- device-side building blocks of the dSMC library (sm_103a).
//
// Philox4x32-10 (Salmon et al., SC'11), the uniform conversion, the model log-densities of
// Eq. (ssm) in base-agnostic FP32, and the parameter blocks the kernels receive by value.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dsmc.h"

namespace dsmc {

constexpr uint32_t kPurposeInit = 1u;
constexpr uint32_t kPurposeDense = 2u;
constexpr uint32_t kPurposeRS = 3u;
constexpr uint32_t kPurposeMH = 4u;
constexpr uint32_t kPurposeSys = 5u;   // systematic offset, one per combination (slot 0)
constexpr uint32_t kPurposeRSF = 6u;   // factorised proposals: the pair's two 64-bit uniforms
constexpr uint32_t kPurposeRSU = 7u;   // factorised proposals: the acceptance uniform

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kHalfLog2Pi = 0.91893853320467274f;
constexpr double kLn2d = 0.69314718055994530942;
constexpr double kLog2ed = 1.4426950408889634074;

// Philox4x32-10: ten rounds of two 32x32 -> 64-bit products with the round multipliers;
// the high halves are xor-ed with the other words and the round key, and the round key
// advances by the Weyl increments before each round after the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// The counter layout of every draw: (slot, id, purpose | base << 4, j), key = seed.
__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t slot, uint32_t id, uint32_t purpose,
                                      uint32_t base, uint32_t j) {
  return philox4x32_10(make_uint4(slot, id, purpose | (base << 4), j), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// u23(w) = ((w >> 9) + 0.5) * 2^-23: 23 random bits, exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float u23(uint32_t w) {
  return __fmul_rn(__fadd_rn(__uint2float_rn(w >> 9), 0.5f), 0x1p-23f);
}

// 2^x on the MUFU unit (flush-to-zero below 2^-126).
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Model parameters, pre-computed on the host in FP64 and rounded once to FP32.  D is the
// padded state dimension (zero rows/columns beyond d).  The transition is N(m(x), Q) with
// m(x) = A x + c (LGSSM; SV and COX with A = phi (lam), c = mu (1 - phi); CRW with A = 1,
// c = 0) or m(x) = x + tau0 - tau1 exp(tau2 x) (THETA_LOGISTIC).
template <int D>
struct ModelParams {
  int kind;         // DSMC_MODEL_*
  int d;            // true dimension
  int prop_kind;    // DSMC_PROP_OBS or DSMC_PROP_GAUSS
  int nu;           // DSMC_NU_EQ_Q or DSMC_NU_PROP_H
  float A[D * D];
  float c[D];
  float Qi[D * D];  // Q^{-1}
  float Ri[D * D];  // R^{-1} (LGSSM)
  float P0i[D * D]; // P0^{-1}
  float m0[D];
  float log_f_max;  // -1/2 log |2 pi Q|, the maximum of log p_t(x' | x)
  float log_h_norm; // -1/2 log |2 pi R| (LGSSM) or -1/2 log(2 pi) (SV)
  float log_p0_norm;// -1/2 log |2 pi P0|
  float prop_scale;
  float log_prop_scale;
  float tau0, tau1, tau2;  // THETA_LOGISTIC: transition mean x + tau0 - tau1 exp(tau2 x)
  float bound;             // CRW: constraint half-width
  const float* prop_mean;  // DEVICE [K][d] (DSMC_PROP_GAUSS)
  const float* prop_std;   // DEVICE [K][d]
};

// x^T M x for a padded D x D matrix.
template <int D>
__device__ __forceinline__ float quad_form(const float* M, const float* x) {
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) r = fmaf(M[i * D + k], x[k], r);
    s = fmaf(x[i], r, s);
  }
  return s;
}

// The transition mean m(x) of the model (see ModelParams).
template <int D>
__device__ __forceinline__ void transition_mean(const ModelParams<D>& mp, const float* x, float* m) {
  if (mp.kind == DSMC_MODEL_THETA_LOGISTIC) {
    m[0] = x[0] + mp.tau0 - mp.tau1 * expf(mp.tau2 * x[0]);
#pragma unroll
    for (int r = 1; r < D; ++r) m[r] = 0.f;
    return;
  }
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float acc = mp.c[r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc = fmaf(mp.A[r * D + k], x[k], acc);
    m[r] = acc;
  }
}

// log h_t(y_t | x): N(y; x, R) for the linear-Gaussian and theta-logistic models,
// N(y; 0, exp(x)) for SV, Poisson(y; exp(x)) for COX, the indicator of |x| <= bound for CRW.
template <int D>
__device__ __forceinline__ float log_h(const ModelParams<D>& mp, const float* yt, const float* x) {
  if (mp.kind == DSMC_MODEL_SV) {
    return mp.log_h_norm - 0.5f * x[0] - 0.5f * yt[0] * yt[0] * expf(-x[0]);
  }
  if (mp.kind == DSMC_MODEL_COX) {
    return yt[0] * x[0] - expf(x[0]) - lgammaf(yt[0] + 1.f);
  }
  if (mp.kind == DSMC_MODEL_CRW) {
    return fabsf(x[0]) <= mp.bound ? 0.f : -INFINITY;
  }
  float r[D];
#pragma unroll
  for (int k = 0; k < D; ++k) r[k] = yt[k] - x[k];
  return mp.log_h_norm - 0.5f * quad_form<D>(mp.Ri, r);
}

// log q_t(x) for the diagonal Gaussian proposal with mean qm and standard deviation s_k,
// given the per-t constants qinv_k = 1 / s_k and qnorm = -sum_k log s_k - d/2 log(2 pi).
template <int D>
__device__ __forceinline__ float log_q(int d, const float* qm, const float* qinv, float qnorm, const float* x) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k < d) {
      const float z = (x[k] - qm[k]) * qinv[k];
      s = fmaf(z, z, s);
    }
  }
  return fmaf(-0.5f, s, qnorm);
}

// log q_t(x) of the uniform proposal on [-scale, scale]^d.
template <int D>
__device__ __forceinline__ float log_q_uniform(const ModelParams<D>& mp, const float* x) {
  bool in = true;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (k < mp.d) in &= fabsf(x[k]) <= mp.prop_scale;
  return in ? -(float)mp.d * (kLn2 + mp.log_prop_scale) : -INFINITY;
}

// log nu_t(x) (Definition 1): q_t itself, or h_t(y_t | .) normalised over x
// (N(x; y_t, R) for the linear-Gaussian and theta-logistic models; h_t * |y_t| for SV; the
// uniform law on [-bound, bound] for CRW).
template <int D>
__device__ __forceinline__ float log_nu(const ModelParams<D>& mp, const float* yt, const float* qm,
                                        const float* qinv, float qnorm, const float* x) {
  if (mp.nu == DSMC_NU_EQ_Q)
    return mp.prop_kind == DSMC_PROP_UNIFORM ? log_q_uniform<D>(mp, x) : log_q<D>(mp.d, qm, qinv, qnorm, x);
  const float lh = log_h<D>(mp, yt, x);
  if (mp.kind == DSMC_MODEL_SV) return lh + logf(fabsf(yt[0]));
  if (mp.kind == DSMC_MODEL_CRW) return lh - logf(2.f * mp.bound);
  return lh;
}

// log P_0(x): N(m0, P0).
template <int D>
__device__ __forceinline__ float log_p0(const ModelParams<D>& mp, const float* x) {
  float r[D];
#pragma unroll
  for (int k = 0; k < D; ++k) r[k] = x[k] - mp.m0[k];
  return mp.log_p0_norm - 0.5f * quad_form<D>(mp.P0i, r);
}

// Proposal mean / std of time t into registers (zero / one beyond d).
template <int D>
__device__ __forceinline__ void proposal_at(const ModelParams<D>& mp, const float* y, const float* prop_mean,
                                            const float* prop_std, int t, float* qm, float* qs) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k < mp.d) {
      if (mp.prop_kind == DSMC_PROP_OBS) {
        qm[k] = y[(size_t)t * mp.d + k];
        qs[k] = mp.prop_scale;
      } else if (mp.prop_kind == DSMC_PROP_UNIFORM) {  // not a Gaussian: log_q_uniform applies
        qm[k] = 0.f;
        qs[k] = mp.prop_scale;
      } else {
        qm[k] = prop_mean[(size_t)t * mp.d + k];
        qs[k] = prop_std[(size_t)t * mp.d + k];
      }
    } else {
      qm[k] = 0.f;
      qs[k] = 1.f;
    }
  }
}

// The per-t constants of log_q from the proposal standard deviations.
template <int D>
__device__ __forceinline__ float proposal_consts(int d, const float* qs, float* qinv) {
  float lsum = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    qinv[k] = 1.f / qs[k];
    if (k < d) lsum += logf(qs[k]);
  }
  return -lsum - (float)d * kHalfLog2Pi;
}

__device__ __forceinline__ void record_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

// An index read from the state (maps, pairs) is kept inside [0, N): a state that was not
// produced by the calls in order (e.g. a level skipped) records an error instead of
// reading out of bounds.
__device__ __forceinline__ int checked_index(int v, int N, bool& bad) {
  if ((unsigned)v < (unsigned)N) return v;
  bad = true;
  return 0;
}

// ceil(log2(s)) for s >= 1.
__host__ __device__ __forceinline__ int ceil_log2(int s) {
  int l = 0;
  while ((1 << l) < s) ++l;
  return l;
}

}  // namespace dsmc
