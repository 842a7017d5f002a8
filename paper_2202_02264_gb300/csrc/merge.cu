// merge.cu -- one level of Algorithm 6: Combine (Algorithm 1), ConditionalCombine
// (Algorithm 5) and the lazy rejection sampler (Algorithm 8) for every adjacent block pair.
//
// For a combination of left block [a, c-1] and right block [c, b] the log-weights of
// Eq. (normalized-weights) with the stitching weight of Proposition 2 are
//   logW_ij = log p_c(xR_j | xL_i) + a_i + b'_j,
//   a_i = logw_L[i],  b'_j = logw_R[j] + log h_c(y_c | xR_j) - log nu_c(xR_j),
// with xL_i the left block's state at c-1 and xR_j the right block's state at c.  For the
// Gaussian transition N(A x + c, Q), with a centre mu, w_i = A xL_i + c - mu, v_j = xR_j - mu:
//   log p = log f_max - 1/2 w_i' Q^-1 w_i - 1/2 v_j' Q^-1 v_j + (Q^-1 w_i)' v_j.
// With B* = max_j b'_j and the per-row bound shift_i = a_i + log f_max + B*, the base-2
// exponent of every pair is <= 0:
//   (logW_ij - shift_i) log2(e) = alpha_i + beta_j + u_i . v_j,
//   u_i = log2(e) Q^-1 w_i,  alpha_i = -log2(e) 1/2 w_i' Q^-1 w_i,
//   beta_j = log2(e) (b'_j - B* - 1/2 v_j' Q^-1 v_j).
// The N x N matrix is never stored: the row-sum kernel evaluates the exponents, takes
// 2^x on MUFU and keeps per-row and per-tile (32..512 columns) sums.  The sampler draws
// each pair in three inverse-CDF stages (row, tile, column), recomputing only the
// chosen tile's columns.
#include <algorithm>
#include <cfloat>

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace dsmc {

namespace {

constexpr int kEpiThreads = 256;
constexpr int kRsThreads = 128;

// The base-2 exponent of pair (i, j): (alpha_i + beta_j) then u_i . v_j by FMAs in
// ascending k.  Every kernel that evaluates a pair uses this one function, so the
// row-sum pass and the sampler's recomputation agree bit for bit.
template <int D>
__device__ __forceinline__ float pair_exponent(const float* u, float al, const float* v, float be) {
  float acc = __fadd_rn(al, be);
#pragma unroll
  for (int k = 0; k < D; ++k) acc = __fmaf_rn(u[k], v[k], acc);
  return acc;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One row of a tensor-core operand: element k of row r at (r/8)*256 + (k/epc)*128 +
// (r%8)*16 + (k%epc)*eb bytes (8-row x 16-byte core matrices, K = 32 bytes: 16 BF16 or 8
// TF32 values; entries beyond D are zero).  TF32 is rounded to nearest.
template <int D>
__device__ __forceinline__ void store_mma_row(unsigned char* base, int r, const float* x, int compute) {
  unsigned char* row = base + (size_t)(r / 8) * 256 + (size_t)(r % 8) * 16;
  if (compute == DSMC_BF16) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float v = k < D ? x[k] : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(row + (k / 8) * 128 + (k % 8) * 2) = __float2bfloat16_rn(v);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float v = k < D ? x[k] : 0.f;
      uint32_t t;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
      *reinterpret_cast<uint32_t*>(row + (k / 4) * 128 + (k % 4) * 4) = t;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Prologue: endpoint states through the block index maps, column / row terms, bound.
// One CTA per combination.
// ---------------------------------------------------------------------------------------
template <int D>
__host__ __device__ constexpr int prologue_threads() {
  return D <= 8 ? 512 : 256;
}

template <int D>
__global__ void __launch_bounds__(prologue_threads<D>()) prologue_kernel(MergeArgs a, ModelParams<D> mp) {
  constexpr int kProThreads = prologue_threads<D>();
  constexpr int NW = kProThreads / 32;
  const int s = blockIdx.x;
  const int m = a.m0 + s;
  int at, c, b;
  merge_geom(a.K, a.level, m, at, c, b);
  const int N = a.N, d = a.d;
  const bool left_leaf = (a.level == 0);
  const int sR = b - c + 1;
  const bool right_leaf = (sR == 1);
  const int bufL = a.level & 1;
  const int bufR = ceil_log2(sR) & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  float yc[D], qm[D], qs[D];
#pragma unroll
  for (int k = 0; k < D; ++k) yc[k] = k < d ? a.y[(size_t)c * d + k] : 0.f;
  proposal_at<D>(mp, a.y, c, qm, qs);

  float* V = a.ws.V + (size_t)s * N * D;
  float* beta = a.ws.beta + (size_t)s * N;
  float* U = a.ws.U + (size_t)s * N * D;
  float* alpha = a.ws.alpha + (size_t)s * N;
  double* shift = a.ws.shift + (size_t)s * N;
  const int32_t* firstR = a.ws.first + ((size_t)bufR * a.K + c) * N;
  const int32_t* lastL = a.ws.last + ((size_t)bufL * a.K + at) * N;

  __shared__ float red_v[NW][D];
  __shared__ float red_s[NW];
  __shared__ float mu_s[D];
  __shared__ float bstar_s;

  // pass 1: right block at time c
  float sx[D];
#pragma unroll
  for (int k = 0; k < D; ++k) sx[k] = 0.f;
  float bmax = -INFINITY;
  bool bad = false, corrupt = false;
  for (int j = threadIdx.x; j < N; j += kProThreads) {
    const int idx = right_leaf ? j : checked_index(firstR[j], N, corrupt);
    const float* xp = a.X + ((size_t)c * N + idx) * d;
    float x[D];
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = k < d ? xp[k] : 0.f;
    const float bj = right_leaf ? a.logw[(size_t)c * N + j] : -a.logN;
    const float g = log_h<D>(mp, yc, x) - log_nu<D>(mp, yc, qm, qs, x);
    const float bp = bj + g;
    bad |= isnan(bp);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      V[(size_t)j * D + k] = x[k];
      sx[k] += x[k];
    }
    beta[j] = bp;
    bmax = fmaxf(bmax, bp);
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float v = warp_sum(sx[k]);
    if (lane == 0) red_v[warp][k] = v;
  }
  bmax = warp_max(bmax);
  if (lane == 0) red_s[warp] = bmax;
  __syncthreads();
  if (threadIdx.x < D) {
    float t = 0.f;
    for (int w = 0; w < NW; ++w) t += red_v[w][threadIdx.x];
    mu_s[threadIdx.x] = t / (float)N;
  }
  if (threadIdx.x == 0) {
    float t = red_s[0];
    for (int w = 1; w < NW; ++w) t = fmaxf(t, red_s[w]);
    bstar_s = t;
  }
  __syncthreads();
  float mu[D];
#pragma unroll
  for (int k = 0; k < D; ++k) mu[k] = mu_s[k];
  const float bstar = bstar_s;

  // pass 2a: columns  v_j = xR_j - mu,  beta_j = log2(e) (b'_j - B* - 1/2 v' Q^-1 v)
  for (int j = threadIdx.x; j < N; j += kProThreads) {
    float v[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = V[(size_t)j * D + k] - mu[k];
#pragma unroll
    for (int k = 0; k < D; ++k) V[(size_t)j * D + k] = v[k];
    beta[j] = kLog2e * (beta[j] - bstar - 0.5f * quad_form<D>(mp.Qi, v));
    if (a.compute != DSMC_FP32) {
      store_mma_row<D>(a.ws.Vb + (size_t)s * a.Nr * 32, j, v, a.compute);
      a.ws.betap[(size_t)s * a.Nr + j] = beta[j];
    }
  }
  if (a.compute != DSMC_FP32) {  // zero the padding rows of the tensor-core operands
    const float zero[D] = {};
    for (int j = N + threadIdx.x; j < a.Nr; j += kProThreads) {
      store_mma_row<D>(a.ws.Vb + (size_t)s * a.Nr * 32, j, zero, a.compute);
      store_mma_row<D>(a.ws.Ub + (size_t)s * a.Nr * 32, j, zero, a.compute);
      a.ws.betap[(size_t)s * a.Nr + j] = 0.f;
    }
  }
  // pass 2b: rows  w_i = A xL_i + c - mu,  u_i = log2(e) Q^-1 w_i,
  //                alpha_i = -log2(e) 1/2 w_i' Q^-1 w_i  (B* is folded into beta)
  float amax = -INFINITY;
  for (int i = threadIdx.x; i < N; i += kProThreads) {
    const int idx = left_leaf ? i : checked_index(lastL[i], N, corrupt);
    const float* xp = a.X + ((size_t)(c - 1) * N + idx) * d;
    float x[D], w[D], u[D];
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = k < d ? xp[k] : 0.f;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      float acc = mp.c[r];
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(mp.A[r * D + k], x[k], acc);
      w[r] = acc - mu[r];
    }
    float q = 0.f;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(mp.Qi[r * D + k], w[k], acc);
      u[r] = acc;
      q = fmaf(w[r], acc, q);
    }
    const float ai = left_leaf ? a.logw[(size_t)(c - 1) * N + i] : -a.logN;
    bad |= isnan(ai);
#pragma unroll
    for (int k = 0; k < D; ++k) U[(size_t)i * D + k] = kLog2e * u[k];
    if (a.compute != DSMC_FP32) {
      float ul[D];
#pragma unroll
      for (int k = 0; k < D; ++k) ul[k] = kLog2e * u[k];
      store_mma_row<D>(a.ws.Ub + (size_t)s * a.Nr * 32, i, ul, a.compute);
    }
    alpha[i] = -0.5f * kLog2e * q;
    shift[i] = (double)ai + (double)mp.log_f_max + (double)bstar;
    amax = fmaxf(amax, ai);
  }
  amax = warp_max(amax);
  __syncthreads();
  if (lane == 0) red_s[warp] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = red_s[0];
    for (int w = 1; w < NW; ++w) t = fmaxf(t, red_s[w]);
    a.ws.logbar[s] = (double)mp.log_f_max + (double)t + (double)bstar;
  }
  if (corrupt) record_status(a.ws.status, DSMC_ERR_INVALID_ARG);
  if (bad) record_status(a.ws.status, DSMC_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------------------
// Tile sums: for rows of one combination and one column chunk, t_ik = sum over the
// columns j of tile k of 2^{e_ij}, accumulated sequentially over j (the row total is the
// sequential sum of its tiles, so no result depends on how columns are chunked).  Thread-per-row with R rows
// per thread; the chunk's v_j / beta_j are staged in shared memory and read as
// broadcasts.  FP32 FMA + MUFU ex2; the N x N exponents never leave registers.
// ---------------------------------------------------------------------------------------
template <int D, int R>
__global__ void __launch_bounds__(128) rowsum_kernel(MergeArgs a, int SC) {
  const int NT = blockDim.x;
  const int s = blockIdx.z, ch = blockIdx.x;
  const int N = a.N, B = a.B;
  const float* U = a.ws.U + (size_t)s * N * D;
  const float* alpha = a.ws.alpha + (size_t)s * N;
  const float* V = a.ws.V + (size_t)s * N * D;
  const float* beta = a.ws.beta + (size_t)s * N;
  float* T = a.ws.T + (size_t)s * N * a.nTp;
  const int j0 = ch * a.CW;
  const int j1 = min(j0 + a.CW, N);
  const int ibase = blockIdx.y * a.rows_per_cta + threadIdx.x;

  float u[R][D], al[R];
  int rowi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = ibase + r * NT;
    rowi[r] = i;
    if (i < N) {
#pragma unroll
      for (int k = 0; k < D; ++k) u[r][k] = U[(size_t)i * D + k];
      al[r] = alpha[i];
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) u[r][k] = 0.f;
      al[r] = -INFINITY;
    }
  }
  float ts[R];
#pragma unroll
  for (int r = 0; r < R; ++r) ts[r] = 0.f;

  extern __shared__ float4 sm4[];
  float* sv = reinterpret_cast<float*>(sm4);  // [SC][D]
  float* sb = sv + (size_t)SC * D;            // [SC]

  for (int jc = j0; jc < j1; jc += SC) {
    const int je = min(jc + SC, j1);
    __syncthreads();
    if ((D % 4) == 0) {
      const float4* src = reinterpret_cast<const float4*>(V + (size_t)jc * D);
      float4* dst = reinterpret_cast<float4*>(sv);
      for (int q = threadIdx.x; q < (je - jc) * D / 4; q += NT) dst[q] = src[q];
    } else {
      for (int q = threadIdx.x; q < (je - jc) * D; q += NT) sv[q] = V[(size_t)jc * D + q];
    }
    for (int q = threadIdx.x; q < je - jc; q += NT) sb[q] = beta[jc + q];
    __syncthreads();
    int j = jc;
    while (j < je) {
      const int tile_end = min((j / B + 1) * B, N);
      const int seg_end = min(tile_end, je);
      int jj = j;
#pragma unroll 2
      for (; jj + 4 <= seg_end; jj += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float* vj = sv + (size_t)(jj + q - jc) * D;
          const float bj = sb[jj + q - jc];
#pragma unroll
          for (int r = 0; r < R; ++r) ts[r] = __fadd_rn(ts[r], ex2(pair_exponent<D>(u[r], al[r], vj, bj)));
        }
      }
      for (; jj < seg_end; ++jj) {
        const float* vj = sv + (size_t)(jj - jc) * D;
        const float bj = sb[jj - jc];
#pragma unroll
        for (int r = 0; r < R; ++r) ts[r] = __fadd_rn(ts[r], ex2(pair_exponent<D>(u[r], al[r], vj, bj)));
      }
      j = seg_end;
      if (seg_end == tile_end) {
        const int kt = (tile_end - 1) / B;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (rowi[r] < N) T[(size_t)rowi[r] * a.nTp + kt] = ts[r];
          ts[r] = 0.f;
        }
      }
    }
  }
}

// Block-wide inclusive scan of N uint64 values in shared memory (in place).
__device__ void block_scan_u64(unsigned long long* v, int N, unsigned long long* warp_tot) {
  const int NT = blockDim.x;
  const int per = (N + NT - 1) / NT;
  const int lo = min(threadIdx.x * per, N), hi = min(lo + per, N);
  unsigned long long run = 0;
  for (int i = lo; i < hi; ++i) run += v[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int w = 0; w < NT / 32; ++w) {
      const unsigned long long t = warp_tot[w];
      warp_tot[w] = acc;
      acc += t;
    }
  }
  __syncthreads();
  unsigned long long pre = warp_tot[warp] + incl - run;
  for (int i = lo; i < hi; ++i) {
    pre += v[i];
    v[i] = pre;
  }
  __syncthreads();
}

// Exact-max recomputation of one row (rare: used when the bound-shifted row total fell
// below 2^-64).  One warp; writes the row's tile sums relative to the new shift, returns
// the row total (lane-local sums, then a butterfly) and the extra base-2 shift.
template <int D>
__device__ void recompute_row(const MergeArgs& a, int s, int i, float* out_sum, float* out_delta) {
  const int N = a.N, B = a.B;
  const int lane = threadIdx.x & 31;
  const float* U = a.ws.U + (size_t)s * N * D;
  const float* V = a.ws.V + (size_t)s * N * D;
  const float* beta = a.ws.beta + (size_t)s * N;
  float u[D];
#pragma unroll
  for (int k = 0; k < D; ++k) u[k] = U[(size_t)i * D + k];
  const float al = a.ws.alpha[(size_t)s * N + i];
  float mx = -INFINITY;
  for (int j = lane; j < N; j += 32) mx = fmaxf(mx, pair_exponent<D>(u, al, V + (size_t)j * D, beta[j]));
  mx = warp_max(mx);
  if (!(mx > -INFINITY)) mx = 0.f;  // all -inf: the row keeps weight zero
  float* T = a.ws.T + ((size_t)s * N + i) * a.nTp;
  float tot = 0.f;
  for (int kt = lane; kt < a.nT; kt += 32) {
    const int jb = kt * B, je = min(jb + B, N);
    float ts = 0.f;
    for (int j = jb; j < je; ++j)
      ts = __fadd_rn(ts, ex2(pair_exponent<D>(u, al, V + (size_t)j * D, beta[j]) - mx));
    T[kt] = ts;
    tot += ts;
  }
  tot = warp_sum(tot);
  *out_sum = tot;
  *out_delta = mx;
}

// The fixed-point image floor(x 2^(40 - E)) of a weight x below twice its reference
// (2^(E-2) <= ref < 2^(E-1), ref_be = the reference's biased exponent + 1):
// (significand << 16) >> (ref_be - be), the shift clamped to [0, 63].  Exact, order-free and
// branch-free; zero, negative, subnormal and non-finite x give 0.
__device__ __forceinline__ unsigned long long q40(float x, int ref_be) {
  const uint32_t b = __float_as_uint(x);
  const int be = (int)((b >> 23) & 0xFFu);
  const bool zero = (b >> 31) || be == 0 || be == 0xFF;
  const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u) << 16;
  const int r = min(max(ref_be - be, 0), 63);
  return zero ? 0ull : (m >> r);
}

__device__ __forceinline__ int ref_exponent(float ref) {
  return (int)((__float_as_uint(ref) >> 23) & 0xFFu) + 1;
}

// Sum of a row's tile weights in ascending tile order (vector loads).
__device__ __forceinline__ float row_total(const float* row, int nT, int nTp) {
  const float4* t4 = reinterpret_cast<const float4*>(row);
  float t = 0.f;
  for (int k4 = 0; k4 < nTp / 4; ++k4) {
    const float4 v = t4[k4];
    const int k = 4 * k4;
    if (k < nT) t = __fadd_rn(t, v.x);
    if (k + 1 < nT) t = __fadd_rn(t, v.y);
    if (k + 2 < nT) t = __fadd_rn(t, v.z);
    if (k + 3 < nT) t = __fadd_rn(t, v.w);
  }
  return t;
}

// ---------------------------------------------------------------------------------------
// Row CDF of one combination (one CTA):
//   row totals s_i = sum of the row's tile weights in ascending tile order (thread per row,
//   independent vector loads; no result depends on how the tile-sum kernel chunked the
//   columns); a row whose total fell below 2^-64 of its bound is recomputed with its exact
//   maximum as shift (rare; tiles rewritten, extra base-2 shift kept in delta);
//   row weights r_i = 2^(l_i - max l) in FP32 with l_i = shift_i log2(e) + delta_i + log2 s_i;
//   their exact 2^40 fixed-point prefix sums (the row stage of the sampler);
//   the FP64 log normalising-constant increment of Eq. (Lab) and log L_{a:b}.
// ---------------------------------------------------------------------------------------
constexpr int kCdfThreads = 512;

template <int D>
__global__ void __launch_bounds__(kCdfThreads) rowcdf_kernel(MergeArgs a) {
  constexpr int NW = kCdfThreads / 32;
  const int s = blockIdx.x;
  const int N = a.N, nT = a.nT, nTp = a.nTp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned long long* cum = reinterpret_cast<unsigned long long*>(smraw);      // [N]
  float* l2 = reinterpret_cast<float*>(smraw + (size_t)N * 8);                 // [N]
  int* under = reinterpret_cast<int*>(cum);  // rows that underflowed (before cum is built)
  __shared__ unsigned long long warp_tot[NW];
  __shared__ double redd[NW];
  __shared__ double M_s;
  __shared__ int n_under, nonfinite_s;
  if (threadIdx.x == 0) {
    n_under = 0;
    nonfinite_s = 0;
  }
  __syncthreads();
  const float* Tt = a.ws.T + (size_t)s * N * nTp;
  const double* shift = a.ws.shift + (size_t)s * N;
  float* delta = a.ws.delta + (size_t)s * N;
  float* rowsum = a.ws.rowsum + (size_t)s * N;
  for (int i = threadIdx.x; i < N; i += kCdfThreads) {
    float t = row_total(Tt + (size_t)i * nTp, nT, nTp);
    if (isnan(t)) {
      nonfinite_s = 1;
      t = 0.f;
    }
    l2[i] = t;
    delta[i] = 0.f;
    if (t < 0x1p-64f) under[atomicAdd(&n_under, 1)] = i;
  }
  __syncthreads();
  for (int q = warp; q < n_under; q += NW) {
    const int i = under[q];
    float si, dl;
    recompute_row<D>(a, s, i, &si, &dl);
    __syncwarp();
    if (lane == 0) {
      si = row_total(Tt + (size_t)i * nTp, nT, nTp);
      l2[i] = isnan(si) ? 0.f : si;
      delta[i] = dl;
    }
  }
  __syncthreads();
  double mloc = -INFINITY;
  for (int i = threadIdx.x; i < N; i += kCdfThreads) {
    const float t = l2[i];
    rowsum[i] = t;
    const float v = t > 0.f ? (float)(shift[i] * kLog2ed + (double)delta[i] + (double)log2f(t)) : -INFINITY;
    l2[i] = v;
    mloc = fmax(mloc, (double)v);
  }
  mloc = warp_max(mloc);
  if (lane == 0) redd[warp] = mloc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = redd[0];
    for (int w = 1; w < NW; ++w) t = fmax(t, redd[w]);
    M_s = t;
  }
  __syncthreads();
  const double M = M_s;
  const bool degenerate = !(M > -INFINITY) || isnan(M);
  float* rw = a.ws.rw + (size_t)s * N;
  double sr = 0.0;
  for (int i = threadIdx.x; i < N; i += kCdfThreads) {
    float r = degenerate ? 0.f : ex2(__fsub_rn(l2[i], (float)M));
    if (!(r > 0.f)) r = 0.f;
    if (r > 1.f) r = 1.f;
    rw[i] = r;
    sr += (double)r;
    cum[i] = (unsigned long long)__float2ull_rz(r * 0x1p40f);
  }
  __syncthreads();
  sr = warp_sum(sr);
  if (lane == 0) redd[warp] = sr;
  block_scan_u64(cum, N, warp_tot);
  unsigned long long* gcum = a.ws.cum + (size_t)s * N;
  for (int i = threadIdx.x; i < N; i += kCdfThreads) gcum[i] = cum[i];
  if (threadIdx.x == 0) {
    int at, c, b;
    merge_geom(a.K, a.level, a.m0 + s, at, c, b);
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += redd[w];
    const double inc = degenerate ? (double)NAN : M * kLn2d + log(t);
    a.ws.inc[s] = inc;
    a.logL[at] = a.logL[at] + a.logL[c] + inc;
    if (degenerate || cum[N - 1] == 0ull) record_status(a.ws.status, DSMC_ERR_DEGENERATE);
    if (nonfinite_s) record_status(a.ws.status, DSMC_ERR_NONFINITE);
  }
}

// Fixed-point pick over n <= 32 weights held in registers: q_k = q40(x_k; ref), Q = sum q,
// T = w Q >> 32 (w a 32-bit uniform word), the first k whose prefix sum exceeds T.  The
// images are recomputed in the second pass (cheap) rather than kept (64 registers).
__device__ __forceinline__ int pick_regs(const float* x, int n, uint32_t w, int ref_be) {
  unsigned long long Q = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) Q += (k < n) ? q40(x[k], ref_be) : 0ull;
  if (Q == 0ull) return 0;
  const unsigned long long T = __umul64hi((unsigned long long)w << 32, Q);
  unsigned long long c = 0;
  int idx = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    c += (k < n) ? q40(x[k], ref_be) : 0ull;
    idx += (c <= T) ? 1 : 0;
  }
  return min(idx, n - 1);
}

// D floats of a row of U or V into registers (vector loads when D is a multiple of 4; the
// rows are then 16-byte aligned).
template <int D>
__device__ __forceinline__ void load_row(const float* p, float* r) {
  if ((D % 4) == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < D / 4; ++k) {
      const float4 v = p4[k];
      r[4 * k] = v.x;
      r[4 * k + 1] = v.y;
      r[4 * k + 2] = v.z;
      r[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) r[k] = p[k];
  }
}

// ---------------------------------------------------------------------------------------
// Pair draws (one thread per slot, many small CTAs per combination):
//   row:    T = U64 * S >> 64 against the exact prefix sums (binary search, L1-cached);
//   tile:   fixed-point tile weights of the row (reference: its largest tile), T = w2 Q >> 32;
//   column: the chosen tile's columns recomputed (pair_exponent + ex2), fixed point
//           (reference: the tile weight t_ik), w3;
// then the pair and the new block's first / last index maps (the composition of the
// Remark in Section 3.1) into the other map buffer.  REG = 1 keeps the row's tiles and the
// tile's exponentials in registers (nT <= 32 and B = 32, i.e. N <= 1024).
// ---------------------------------------------------------------------------------------
constexpr int kSlotThreads = 128;

template <int D, int REG>
__global__ void __launch_bounds__(kSlotThreads) slots_kernel(MergeArgs a, int cum_in_smem) {
  const int s = blockIdx.x;
  const int gid = a.gid0 + s;
  const int N = a.N, B = a.B, nT = a.nT, nTp = a.nTp;
  // the row prefix sums: copied to shared memory in one round trip when they fit
  extern __shared__ unsigned long long scum[];
  const unsigned long long* gcum = a.ws.cum + (size_t)s * N;
  if (cum_in_smem) {
    for (int q = threadIdx.x; q < N; q += kSlotThreads) scum[q] = gcum[q];
    __syncthreads();
    gcum = scum;
  }
  const float* Tt = a.ws.T + (size_t)s * N * nTp;
  int at, c, b;
  merge_geom(a.K, a.level, a.m0 + s, at, c, b);
  int32_t* pl = a.pairs + (size_t)gid * 2 * N;
  int32_t* pr = pl + N;
  const int n_lo = a.conditional ? 1 : 0;
  const int n_hi = N + ((a.conditional && a.root) ? 1 : 0);
  const bool left_leaf = (a.level == 0);
  const int sR = b - c + 1;
  const bool right_leaf = (sR == 1);
  const int bufL = a.level & 1, bufR = ceil_log2(sR) & 1, bufO = (a.level + 1) & 1;
  int32_t* first_out = a.ws.first + ((size_t)bufO * a.K + at) * N;
  int32_t* last_out = a.ws.last + ((size_t)bufO * a.K + at) * N;
  const int32_t* first_L = a.ws.first + ((size_t)bufL * a.K + at) * N;
  const int32_t* last_R = a.ws.last + ((size_t)bufR * a.K + c) * N;
  if (a.conditional && blockIdx.y == 0 && threadIdx.x == 0) {
    pl[0] = 0;
    pr[0] = 0;
    first_out[0] = left_leaf ? 0 : first_L[0];
    last_out[0] = right_leaf ? 0 : last_R[0];
  }
  const int n = n_lo + blockIdx.y * kSlotThreads + threadIdx.x;
  if (n >= n_hi) return;
  const unsigned long long S = gcum[N - 1];
  int i, j;
  if (S == 0ull) {
    i = n % N;
    j = n % N;
  } else {
    const uint4 w = draw(a.seed, (uint32_t)n, (uint32_t)gid, kPurposeDense, a.base, 0u);
    const unsigned long long Uw = ((unsigned long long)w.x << 32) | (unsigned long long)w.y;
    const unsigned long long Tg = __umul64hi(Uw, S);
    int lo = 0, hi = N - 1;  // first i with cum[i] > Tg (cum[N-1] = S > Tg)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (gcum[mid] > Tg) hi = mid; else lo = mid + 1;
    }
    i = lo;
    const float* Ti = Tt + (size_t)i * nTp;
    const float4* Ti4 = reinterpret_cast<const float4*>(Ti);
    float u[D];
    load_row<D>(a.ws.U + ((size_t)s * N + i) * D, u);
    const float al = __fsub_rn(a.ws.alpha[(size_t)s * N + i], a.ws.delta[(size_t)s * N + i]);
    const float* V = a.ws.V + (size_t)s * N * D;
    const float* beta = a.ws.beta + (size_t)s * N;
    int kt;
    if (REG) {
      float t[32];
#pragma unroll
      for (int k4 = 0; k4 < 8; ++k4) {
        const float4 v = (4 * k4 < nTp) ? Ti4[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
        t[4 * k4] = v.x;
        t[4 * k4 + 1] = v.y;
        t[4 * k4 + 2] = v.z;
        t[4 * k4 + 3] = v.w;
      }
      float tmax = 0.f;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < nT) tmax = fmaxf(tmax, t[k]);
      kt = pick_regs(t, nT, w.z, ref_exponent(tmax));
    } else {
      float tmax = 0.f;
      for (int k = 0; k < nT; ++k) tmax = fmaxf(tmax, Ti[k]);
      const int rbe = ref_exponent(tmax);
      unsigned long long Q = 0;
      for (int k = 0; k < nT; ++k) Q += q40(Ti[k], rbe);
      kt = 0;
      if (Q != 0ull) {
        const unsigned long long Tq = __umul64hi((unsigned long long)w.z << 32, Q);
        unsigned long long cc = 0;
        for (int k = 0; k < nT; ++k) {
          cc += q40(Ti[k], rbe);
          kt += (cc <= Tq) ? 1 : 0;
        }
        kt = min(kt, nT - 1);
      }
    }
    const int tbe = ref_exponent(Ti[kt]);
    const int jb = kt * B, je = min(jb + B, N);
    if (REG) {
      // the tile's 32 columns: beta as 8 vector loads, each v_j as D/4 vector loads
      float bt[32], e[32];
      // vector loads only when the tile is full and its beta run is 16-byte aligned (the
      // per-combination stride N need not be a multiple of 4)
      if (je - jb == 32 && ((reinterpret_cast<uintptr_t>(beta + jb) & 15u) == 0)) {
        const float4* b4 = reinterpret_cast<const float4*>(beta + jb);
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4) {
          const float4 v = b4[q4];
          bt[4 * q4] = v.x;
          bt[4 * q4 + 1] = v.y;
          bt[4 * q4 + 2] = v.z;
          bt[4 * q4 + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) bt[q] = beta[min(jb + q, N - 1)];
      }
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        float v[D];
        load_row<D>(V + (size_t)min(jb + q, N - 1) * D, v);
        e[q] = (jb + q < je) ? ex2(pair_exponent<D>(u, al, v, bt[q])) : 0.f;
      }
      j = jb + pick_regs(e, je - jb, w.w, tbe);
    } else {
      unsigned long long Qc = 0;
      for (int jj = jb; jj < je; ++jj)
        Qc += q40(ex2(pair_exponent<D>(u, al, V + (size_t)jj * D, beta[jj])), tbe);
      j = jb;
      if (Qc != 0ull) {
        const unsigned long long Tc = __umul64hi((unsigned long long)w.w << 32, Qc);
        unsigned long long cc = 0;
        int cnt = 0;
        for (int jj = jb; jj < je; ++jj) {
          cc += q40(ex2(pair_exponent<D>(u, al, V + (size_t)jj * D, beta[jj])), tbe);
          cnt += (cc <= Tc) ? 1 : 0;
        }
        j = jb + min(cnt, je - jb - 1);
      }
    }
  }
  if (n < N) {
    pl[n] = i;
    pr[n] = j;
    first_out[n] = left_leaf ? i : first_L[i];
    last_out[n] = right_leaf ? j : last_R[j];
  } else {
    a.ws.star[0] = i;
    a.ws.star[1] = j;
  }
}

// ---------------------------------------------------------------------------------------
// Lazy rejection sampler (Algorithm 8): per slot, attempts (I, J, u) until u < ratio(I, J),
// ratio = exp(logW_IJ - log omega-bar); (I, J, u) are redrawn at every attempt.  Only the
// proposed pairs are evaluated.  One thread per slot; capped at rs_max attempts.
// ---------------------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ float rs_ratio(const MergeArgs& a, int s, int I, int J, double logbar) {
  const int N = a.N;
  const float* U = a.ws.U + ((size_t)s * N + I) * D;
  const float* V = a.ws.V + ((size_t)s * N + J) * D;
  float u[D], v[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    u[k] = U[k];
    v[k] = V[k];
  }
  const float off = (float)((a.ws.shift[(size_t)s * N + I] - logbar) * kLog2ed);
  const float e = pair_exponent<D>(u, a.ws.alpha[(size_t)s * N + I], v, a.ws.beta[(size_t)s * N + J]);
  return ex2(__fadd_rn(e, off));
}

template <int D>
__global__ void __launch_bounds__(kRsThreads) sample_rs_kernel(MergeArgs a) {
  const int s = blockIdx.y;
  const int gid = a.gid0 + s;
  const int N = a.N;
  const int n_lo = a.conditional ? 1 : 0;
  const int n_hi = N + ((a.conditional && a.root) ? 1 : 0);
  const int n = n_lo + blockIdx.x * kRsThreads + threadIdx.x;
  const double logbar = a.ws.logbar[s];
  int32_t* pl = a.pairs + (size_t)gid * 2 * N;
  int32_t* pr = pl + N;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ws.inc[s] = (double)NAN;  // the lazy sampler never forms the N x N sum
    if (a.conditional) {
      pl[0] = 0;
      pr[0] = 0;
    }
  }
  if (n >= n_hi) return;
  int I = 0, J = 0;
  bool ok = false;
  for (uint32_t att = 0; att < a.rs_max; ++att) {
    const uint4 w = draw(a.seed, (uint32_t)n, (uint32_t)gid, kPurposeRS, a.base, att);
    I = (int)__umulhi(w.x, (uint32_t)N);
    J = (int)__umulhi(w.y, (uint32_t)N);
    if (u23(w.z) < rs_ratio<D>(a, s, I, J, logbar)) {
      ok = true;
      break;
    }
  }
  if (!ok) record_status(a.ws.status, DSMC_ERR_RS_LIMIT);
  if (n < N) {
    pl[n] = I;
    pr[n] = J;
  } else {
    a.ws.star[0] = I;
    a.ws.star[1] = J;
  }
}

// ---------------------------------------------------------------------------------------
// Epilogue: the new block's first/last index maps (the composition of the Remark in
// Section 3.1) into the other map buffer, and log L_{a:b} = log L_{a:c-1} + log L_{c:b} +
// increment (Eq. rec-loglik, weighted form).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kEpiThreads) epilogue_kernel(MergeArgs a) {
  const int s = blockIdx.x;
  const int m = a.m0 + s;
  const int gid = a.gid0 + s;
  int at, c, b;
  merge_geom(a.K, a.level, m, at, c, b);
  const int N = a.N;
  const bool left_leaf = (a.level == 0);
  const int sR = b - c + 1;
  const bool right_leaf = (sR == 1);
  const int bufL = a.level & 1, bufR = ceil_log2(sR) & 1, bufO = (a.level + 1) & 1;
  const int n = blockIdx.y * kEpiThreads + threadIdx.x;
  const int32_t* pl = a.pairs + (size_t)gid * 2 * N;
  const int32_t* pr = pl + N;
  if (n < N) {
    bool corrupt = false;
    const int l = checked_index(pl[n], N, corrupt), r = checked_index(pr[n], N, corrupt);
    a.ws.first[((size_t)bufO * a.K + at) * N + n] =
        left_leaf ? l : a.ws.first[((size_t)bufL * a.K + at) * N + l];
    a.ws.last[((size_t)bufO * a.K + at) * N + n] =
        right_leaf ? r : a.ws.last[((size_t)bufR * a.K + c) * N + r];
    if (corrupt) record_status(a.ws.status, DSMC_ERR_INVALID_ARG);
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) a.logL[at] = a.logL[at] + a.logL[c] + a.ws.inc[s];
}

// ---------------------------------------------------------------------------------------
// Inspection: the device's own weights of one combination, for the parity tests.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void debug_weights_kernel(MergeArgs a, int s, float* logW, float* r, float* rowsum,
                                     float* tiles, float* e, float* ratio) {
  const int i = blockIdx.x;
  const int N = a.N;
  const float* U = a.ws.U + (size_t)s * N * D;
  const float* V = a.ws.V + (size_t)s * N * D;
  const float* alpha = a.ws.alpha + (size_t)s * N;
  const float* beta = a.ws.beta + (size_t)s * N;
  const double sh = a.ws.shift[(size_t)s * N + i];
  const float dl = a.ws.delta[(size_t)s * N + i];
  const double logbar = a.ws.logbar[s];
  float u[D];
#pragma unroll
  for (int k = 0; k < D; ++k) u[k] = U[(size_t)i * D + k];
  const float al = __fsub_rn(alpha[i], dl);
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float x = pair_exponent<D>(u, alpha[i], V + (size_t)j * D, beta[j]);
    if (logW) logW[(size_t)i * N + j] = (float)(sh + (double)x * kLn2d);
    if (e) e[(size_t)i * N + j] = ex2(pair_exponent<D>(u, al, V + (size_t)j * D, beta[j]));
    if (ratio) ratio[(size_t)i * N + j] = rs_ratio<D>(a, s, i, j, logbar);
  }
  if (threadIdx.x == 0 && r) r[i] = a.ws.rw[(size_t)s * N + i];
  if (threadIdx.x == 0 && rowsum) rowsum[i] = a.ws.rowsum[(size_t)s * N + i];
  if (tiles)
    for (int k = threadIdx.x; k < a.nT; k += blockDim.x)
      tiles[(size_t)i * a.nT + k] = a.ws.T[((size_t)s * N + i) * a.nTp + k];
}

// ------------------------------------------------------------------- launch wrappers
template <int D>
cudaError_t prologue_t(const MergeArgs& a, const void* mp, cudaStream_t st) {
  prologue_kernel<D><<<a.mc, prologue_threads<D>(), 0, st>>>(a, *static_cast<const ModelParams<D>*>(mp));
  return cudaGetLastError();
}

template <int D>
__host__ __device__ constexpr int rows_per_thread() {
  return D <= 8 ? 4 : (D <= 16 ? 2 : 1);
}

template <int D>
cudaError_t rowsum_t(const MergeArgs& a, cudaStream_t st) {
  constexpr int R = rows_per_thread<D>();
  const int NT = a.rows_per_cta / R;
  const int SC = D <= 8 ? 512 : 256;
  const size_t smem = (size_t)SC * (D + 1) * sizeof(float);
  dim3 grid(a.CH, (a.N + a.rows_per_cta - 1) / a.rows_per_cta, a.mc);
  rowsum_kernel<D, R><<<grid, NT, smem, st>>>(a, SC);
  return cudaGetLastError();
}

template <int D>
cudaError_t sample_dense_t(const MergeArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)a.N * (sizeof(unsigned long long) + sizeof(float));
  if (smem > 40 * 1024) {  // static shared memory counts against the 48 KB default
    cudaError_t e = cudaFuncSetAttribute(rowcdf_kernel<D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  rowcdf_kernel<D><<<a.mc, kCdfThreads, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int slots = a.N + ((a.conditional && a.root) ? 1 : 0) - (a.conditional ? 1 : 0);
  dim3 grid(a.mc, (slots + kSlotThreads - 1) / kSlotThreads);
  const int cum_in_smem = a.N <= 4096 ? 1 : 0;   // <= 32 KB: several CTAs per SM
  const size_t smem_slot = cum_in_smem ? (size_t)a.N * sizeof(unsigned long long) : 0;
  if (a.nT <= 32 && a.B == 32)
    slots_kernel<D, 1><<<grid, kSlotThreads, smem_slot, st>>>(a, cum_in_smem);
  else
    slots_kernel<D, 0><<<grid, kSlotThreads, smem_slot, st>>>(a, cum_in_smem);
  return cudaGetLastError();
}

template <int D>
cudaError_t sample_rs_t(const MergeArgs& a, cudaStream_t st) {
  const int slots = a.N + ((a.conditional && a.root) ? 1 : 0) - (a.conditional ? 1 : 0);
  dim3 grid((slots + kRsThreads - 1) / kRsThreads, a.mc);
  sample_rs_kernel<D><<<grid, kRsThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t debug_t(const MergeArgs& a, int s, float* logW, float* r, float* rowsum, float* tiles,
                    float* e, float* ratio, cudaStream_t st) {
  debug_weights_kernel<D><<<a.N, 128, 0, st>>>(a, s, logW, r, rowsum, tiles, e, ratio);
  return cudaGetLastError();
}

}  // namespace

#define DSMC_DISPATCH(D, CALL)            \
  switch (D) {                            \
    case 1: { constexpr int DD = 1; return CALL; }   \
    case 2: { constexpr int DD = 2; return CALL; }   \
    case 4: { constexpr int DD = 4; return CALL; }   \
    case 8: { constexpr int DD = 8; return CALL; }   \
    case 16: { constexpr int DD = 16; return CALL; } \
    case 32: { constexpr int DD = 32; return CALL; } \
  }                                       \
  return cudaErrorInvalidValue;

cudaError_t launch_prologue(int D, const MergeArgs& a, const void* mp, cudaStream_t s) {
  DSMC_DISPATCH(D, prologue_t<DD>(a, mp, s))
}

cudaError_t launch_rowsum(int D, const MergeArgs& a, cudaStream_t s) {
  DSMC_DISPATCH(D, rowsum_t<DD>(a, s))
}

cudaError_t launch_sample_dense(int D, const MergeArgs& a, cudaStream_t s) {
  DSMC_DISPATCH(D, sample_dense_t<DD>(a, s))
}

cudaError_t launch_sample_rs(int D, const MergeArgs& a, cudaStream_t s) {
  DSMC_DISPATCH(D, sample_rs_t<DD>(a, s))
}

cudaError_t launch_epilogue(const MergeArgs& a, cudaStream_t s) {
  dim3 grid(a.mc, (a.N + kEpiThreads - 1) / kEpiThreads);
  epilogue_kernel<<<grid, kEpiThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_debug_weights(int D, const MergeArgs& a, int s_local, float* logW, float* r,
                                 float* rowsum, float* tiles, float* e, float* ratio,
                                 cudaStream_t s) {
  DSMC_DISPATCH(D, debug_t<DD>(a, s_local, logW, r, rowsum, tiles, e, ratio, s))
}

int rowsum_rows_per_thread(int D) {
  switch (D) {
    case 1: return rows_per_thread<1>();
    case 2: return rows_per_thread<2>();
    case 4: return rows_per_thread<4>();
    case 8: return rows_per_thread<8>();
    case 16: return rows_per_thread<16>();
    default: return rows_per_thread<32>();
  }
}

}  // namespace dsmc
