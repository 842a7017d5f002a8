// merge_parts.cuh -- the per-pair, per-column, per-row and per-slot arithmetic of one
// combination of Algorithm 1 / Algorithm 5, shared by the split per-level kernels
// (merge.cu) and the fused single-launch level kernel (level_fused.cu), so that both paths
// produce the same bits from the same inputs.
//
// Notation (Section 3.1): left block [a, c-1], right block [c, b]; xL_i = left state at c-1,
// xR_j = right state at c; a_i = logw_L[i]; b'_j = logw_R[j] + log h_c(y_c|xR_j) - log nu_c(xR_j).
// For the Gaussian transition N(m(x), Q) (m(x) = A x + c, or the theta-logistic mean) with
// centre mu (mean of the xR_j):
//   w_i = m(xL_i) - mu,  v_j = xR_j - mu,  u_i = log2(e) Q^-1 w_i,
//   alpha_i = -log2(e) 1/2 w_i' Q^-1 w_i,  beta_j = log2(e) (b'_j - B* - 1/2 v_j' Q^-1 v_j),
// and the base-2 exponent of pair (i, j) relative to the row bound
// shift_i = a_i + log f_max + B* is alpha_i + beta_j + u_i . v_j <= 0.
#pragma once

#include "kernels.cuh"

namespace dsmc {
namespace parts {

// The base-2 exponent of pair (i, j): (alpha_i + beta_j) then u_i . v_j by FMAs in
// ascending k.  Every kernel that evaluates a pair on the CUDA cores uses this function.
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

// Column-term layouts.  In global memory v_j is row j of [N][D] and beta_j element j.
// Shared-memory copies (PAD = true) insert a gap after every 32 columns (one tile at
// B = 32): kVPad<D> floats for v, one float for beta.  Threads that read column q of
// different tiles then hit different banks instead of all hitting the same one.
template <int D>
constexpr int kVPad = D >= 4 ? 4 : D;

template <int D, bool PAD>
__host__ __device__ __forceinline__ int vidx(int j) {
  return PAD ? j * D + (j >> 5) * kVPad<D> : j * D;
}

template <bool PAD>
__host__ __device__ __forceinline__ int bidx(int j) {
  return PAD ? j + (j >> 5) : j;
}

// Floats of a padded shared-memory copy of N columns.
template <int D>
__host__ __device__ __forceinline__ int vpad_floats(int N) {
  return N * D + ((N + 31) >> 5) * kVPad<D>;
}
__host__ __device__ __forceinline__ int bpad_floats(int N) { return N + ((N + 31) >> 5); }

// ---------------------------------------------------------------- column and row terms
// Column j, first pass: the right block's state xR_j (particle map[j] of the time-c slice
// Xs [N][d], or particle j when the right block is a leaf, map = nullptr) and
// b'_j = b_j + log h - log nu, where b_j is the leaf's log-weight lw[j] (lw = nullptr:
// a merged block, b_j = -log N).  Returns b'_j; x receives the padded state.
template <int D>
__device__ __forceinline__ float column_bprime(const ModelParams<D>& mp, int N, int d, float logN,
                                               const float* yc, const float* qm, const float* qinv,
                                               float qnorm, const float* Xs, const int32_t* map,
                                               const float* lw, int j, float* x, bool& corrupt) {
  const int idx = map != nullptr ? checked_index(map[j], N, corrupt) : j;
  const float* xp = Xs + (size_t)idx * d;
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = k < d ? xp[k] : 0.f;
  const float bj = lw != nullptr ? lw[j] : -logN;
  const float g = log_h<D>(mp, yc, x) - log_nu<D>(mp, yc, qm, qinv, qnorm, x);
  return bj + g;
}

// The column pass with the column mean mu reduced in a fixed order that does not depend on
// the block size.  Columns fall into G <= 32 groups of 32 Q consecutive columns, where
// Q = ceil(N / 1024); warp w of NW takes the groups g = w, w + NW, ...; in a group, lane l
// adds its columns 32 (Q g + c) + l in order of c, then the lanes are summed by a butterfly
// into gsum[g][k]; the group sums are added in group order.  `col(j, x)` evaluates column
// j (j < N) into x[D] and returns b'_j.  Returns mu (every thread) and B* = max_j b'_j.
constexpr int kMaxColumnGroups = 32;

template <int D, typename ColFn>
__device__ __forceinline__ void column_pass(int N, float* gsum, float* red_s, float* mu_s, float* bstar_s,
                                            float* mu, float& bstar, bool& bad, ColFn col) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int Q = (N + 1023) / 1024, Wd = 32 * Q;
  const int G = (N + Wd - 1) / Wd;
  float bmax = -INFINITY;
  for (int g = warp; g < G; g += NW) {
    float acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = 0.f;
    for (int c = 0; c < Q; ++c) {
      const int j = Wd * g + 32 * c + lane;
      if (j < N) {
        float x[D];
        const float bp = col(j, x);
        bad |= isnan(bp);
        bmax = fmaxf(bmax, bp);
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] += x[k];
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float t = warp_sum(acc[k]);
      if (lane == 0) gsum[g * D + k] = t;
    }
  }
  bmax = warp_max(bmax);
  if (lane == 0) red_s[warp] = bmax;
  __syncthreads();
  if (threadIdx.x < D) {
    float t = 0.f;
    for (int g = 0; g < G; ++g) t += gsum[g * D + threadIdx.x];
    mu_s[threadIdx.x] = t / (float)N;
  }
  if (threadIdx.x == 0) {
    float t = red_s[0];
    for (int w = 1; w < NW; ++w) t = fmaxf(t, red_s[w]);
    *bstar_s = t;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < D; ++k) mu[k] = mu_s[k];
  bstar = *bstar_s;
}

// Column j, second pass: v_j = xR_j - mu (in place) and beta_j.
template <int D>
__device__ __forceinline__ float column_beta(const ModelParams<D>& mp, float* v, const float* mu,
                                             float bprime, float bstar) {
#pragma unroll
  for (int k = 0; k < D; ++k) v[k] = v[k] - mu[k];
  return kLog2e * (bprime - bstar - 0.5f * quad_form<D>(mp.Qi, v));
}

// Row i: the left block's state xL_i (particle map[i] of the time-(c - 1) slice Xs, or
// particle i when the left block is a leaf, map = nullptr), u_i (already scaled by
// log2(e)), alpha_i, and a_i (the leaf's log-weight lw[i], or -log N).  Returns alpha_i.
template <int D>
__device__ __forceinline__ float row_terms(const ModelParams<D>& mp, int N, int d, float logN,
                                           const float* Xs, const int32_t* map, const float* lw, int i,
                                           const float* mu, float* ul, float& ai, bool& corrupt) {
  const int idx = map != nullptr ? checked_index(map[i], N, corrupt) : i;
  const float* xp = Xs + (size_t)idx * d;
  float x[D], w[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = k < d ? xp[k] : 0.f;
  transition_mean<D>(mp, x, w);
#pragma unroll
  for (int r = 0; r < D; ++r) w[r] = w[r] - mu[r];
  float q = 0.f;
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) acc = fmaf(mp.Qi[r * D + k], w[k], acc);
    ul[r] = kLog2e * acc;
    q = fmaf(w[r], acc, q);
  }
  ai = lw != nullptr ? lw[i] : -logN;
  return -0.5f * kLog2e * q;
}

// A block's copy of n 32-bit words from global to shared memory (16-byte vector loads when
// both ends are 16-byte aligned).  The caller synchronises.
template <typename T>
__device__ __forceinline__ void stage_words(T* dst, const T* src, int n) {
  static_assert(sizeof(T) == 4, "32-bit words");
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const int n4 = n >> 2;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (int t = threadIdx.x; t < n4; t += blockDim.x) d4[t] = __ldg(s4 + t);
    for (int t = 4 * n4 + threadIdx.x; t < n; t += blockDim.x) dst[t] = __ldg(src + t);
  } else {
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = __ldg(src + t);
  }
}

// Row i's base-2 shift delta_i: the largest exponent over a fixed sample of 8 columns
// (j = k N / 8), floored at -96.  The row's pairs are evaluated relative to
// shift_i + delta_i ln 2 (alpha_i - delta_i in base 2): the sampled best column then weighs
// about 1, so the row total cannot underflow, while every pair stays below 2^96 (the
// exponents relative to the bound are <= 0), so no tile sum overflows.  In high dimension
// the bound log f_max is far above every pair of a row; without this shift whole rows fall
// below FP32's range.
template <int D, bool PAD>
__device__ __forceinline__ float row_shift(const float* u, float al, const float* V, const float* beta, int N) {
  constexpr int S = 8;
  float mx = -INFINITY;
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int j = N >= S ? (int)(((long long)k * N) / S) : (k < N ? k : N - 1);
    mx = fmaxf(mx, pair_exponent<D>(u, al, V + vidx<D, PAD>(j), beta[bidx<PAD>(j)]));
  }
  return fmaxf(mx, -96.f);
}

// ---------------------------------------------------------------- row totals and CDF
// The row total, every path's definition: the tile weights summed in pairs
// q_p = t_{2p} + t_{2p+1} (t_{2p+1} = 0 past the last tile), the even pairs and the odd pairs
// each accumulated in ascending p, then the two sums added (FP32, round to nearest).  A
// tensor-core epilogue warp that holds the even (or odd) pairs of a row accumulates its
// half as it goes; vector loads here (the row is 16-byte aligned, nTp a multiple of 4).
__device__ __forceinline__ float row_total(const float* row, int nT, int nTp) {
  const float4* t4 = reinterpret_cast<const float4*>(row);
  float se = 0.f, so = 0.f;
  for (int k4 = 0; k4 < nTp / 4; ++k4) {
    const float4 v = t4[k4];
    const int k = 4 * k4;  // pairs 2 k4 (even) and 2 k4 + 1 (odd)
    if (k < nT) se = __fadd_rn(se, __fadd_rn(v.x, k + 1 < nT ? v.y : 0.f));
    if (k + 2 < nT) so = __fadd_rn(so, __fadd_rn(v.z, k + 3 < nT ? v.w : 0.f));
  }
  return __fadd_rn(se, so);
}

// row_total of a row of nT <= 16 tiles that is only 8-byte aligned: the same sums in the
// same order.
__device__ __forceinline__ float row_total_small(const float* row, int nT) {
  float se = 0.f, so = 0.f;
#pragma unroll
  for (int p = 0; p < 8; ++p) {  // pair p = tiles 2p, 2p + 1; even p into se, odd p into so
    if (2 * p < nT) {
      const float q = __fadd_rn(row[2 * p], 2 * p + 1 < nT ? row[2 * p + 1] : 0.f);
      if (p & 1) so = __fadd_rn(so, q); else se = __fadd_rn(se, q);
    }
  }
  return __fadd_rn(se, so);
}

// The row's natural-log shift a_i + log f_max + B* + dl_i ln 2 in FP64, in that order (the
// lazy samplers' acceptance terms and the inspection entry points): shift_base gives the first
// three terms; a merged left block has a_i = -log N on every row, so its base is computed
// once per combination with the same bits.
__device__ __forceinline__ double shift_base(float ai, float log_f_max, float bstar) {
  return (double)ai + (double)log_f_max + (double)bstar;
}
__device__ __forceinline__ double row_shift_total(double base, float dl) { return base + (double)dl * kLn2d; }

// The dense samplers split the same shift into a combination base C (natural log, FP64, once
// per combination) and a per-row base-2 offset g_i (FP32), shift_i = C + g_i ln 2:
//   C = log f_max + B*, less log N for a merged left block (whose a_i = -log N on every row);
//   g_i = a_i log2(e) + dl_i for a leaf left block (lw = its log-weights), dl_i for a merged one.
// Only differences between rows reach the row weights, and C enters only the increment of
// Eq. (Lab), so no per-row arithmetic is FP64 (GB300 issues under 2 DFMA per clock per SM).
__device__ __forceinline__ double comb_base(bool left_leaf, float logN, float log_f_max, float bstar) {
  return shift_base(left_leaf ? 0.f : -logN, log_f_max, bstar);
}
__device__ __forceinline__ float row_offset(bool left_leaf, float ai, float dl) {
  return left_leaf ? __fmaf_rn(ai, kLog2e, dl) : dl;
}

// The row's base-2 log weight relative to C: l_i = (g_i + delta_i) + log2 s_i in FP32
// (-inf when s_i = 0); delta_i is the extra shift of a row recomputed after underflow (else 0).
__device__ __forceinline__ float row_log2_weight(float g, float delta, float total) {
  if (!(total > 0.f)) return -INFINITY;
  return __fadd_rn(__fadd_rn(g, delta), log2f(total));
}

// The increment of Eq. (Lab): log sum_ij omega_ij = C + M ln 2 + ln(S 2^-40), with M the
// largest row log weight and S the row weights' exact fixed-point total.
__device__ __forceinline__ double lab_increment(double C, float M, double log_total) {
  return (C + (double)M * kLn2d) + log_total;
}

// The row weight r_i = 2^(l_i - M) in FP32, clamped to [0, 1].
__device__ __forceinline__ float row_weight(float l, float M, bool degenerate) {
  float r = degenerate ? 0.f : ex2(__fsub_rn(l, M));
  if (!(r > 0.f)) r = 0.f;
  if (r > 1.f) r = 1.f;
  return r;
}

// Natural log of the row-weight total from its exact fixed-point image S = sum_i
// floor(r_i 2^40) (r_i <= 1, so the truncation is below N 2^-40 of a total >= 1):
// ln(S 2^-40) with S = m 2^e, m in [1, 2) taken from the top 24 bits, log2 m in FP32.
__device__ __forceinline__ double log_fixed_total(unsigned long long S) {
  if (S == 0ull) return (double)NAN;
  const int e = 63 - __clzll(S);
  const unsigned long long top = e >= 23 ? (S >> (e - 23)) : (S << (23 - e));
  const float m = (float)(uint32_t)top * 0x1p-23f;
  return ((double)(e - 40) + (double)log2f(m)) * kLn2d;
}

// Block-wide inclusive scan of N uint64 values in shared memory (in place); warp_tot holds
// blockDim.x / 32 entries.  Integer: the result does not depend on the thread count.
__device__ __forceinline__ void block_scan_u64(unsigned long long* v, int N, unsigned long long* warp_tot) {
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
// below 2^-64).  One warp; rewrites the row's tile sums relative to the new shift, returns
// the row total (lane-local sums, then a butterfly) and the extra base-2 shift.
template <int D, bool PAD>
__device__ void recompute_row(const float* u, float al, const float* V, const float* beta, int N,
                              int B, int nT, float* Trow, float* out_sum, float* out_delta) {
  const int lane = threadIdx.x & 31;
  float mx = -INFINITY;
  for (int j = lane; j < N; j += 32)
    mx = fmaxf(mx, pair_exponent<D>(u, al, V + vidx<D, PAD>(j), beta[bidx<PAD>(j)]));
  mx = warp_max(mx);
  if (!(mx > -INFINITY)) mx = 0.f;  // all -inf: the row keeps weight zero
  float tot = 0.f;
  for (int kt = lane; kt < nT; kt += 32) {
    const int jb = kt * B, je = min(jb + B, N);
    float ts = 0.f;
    for (int j = jb; j < je; ++j)
      ts = __fadd_rn(ts, ex2(pair_exponent<D>(u, al, V + vidx<D, PAD>(j), beta[bidx<PAD>(j)]) - mx));
    Trow[kt] = ts;
    tot += ts;
  }
  tot = warp_sum(tot);
  *out_sum = tot;
  *out_delta = mx;
}

// ---------------------------------------------------------------- fixed-point draws
// The fixed-point image q24(x; ref) = floor(x 2^(24 - E)) of a weight x >= 0, where
// 2^(E-2) <= ref < 2^(E-1) (ref_be = the reference's biased exponent + 1, E = ref_be - 126),
// saturated at 2^32 - 1; negative and NaN x give 0.  Computed as one exact power-of-two
// scaling and a truncating conversion (the scale exponent is clamped to 127, which no
// chosen tile reaches: a chosen tile weighs at least 2^-24 of its row's largest tile and
// that one at least 2^-70 of the row bound).  A weight equal to its reference keeps 23
// significant bits, as many as the FP32 weight carries; below twice the reference the
// image is < 2^24.
__device__ __forceinline__ uint32_t q24(float x, int ref_be) {
  const int k = min(150 - ref_be, 127);
  const float scale = __uint_as_float((uint32_t)(k + 127) << 23);
  return __float2uint_rz(x * scale);
}

__device__ __forceinline__ int ref_exponent(float ref) {
  return (int)((__float_as_uint(ref) >> 23) & 0xFFu) + 1;
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

// The inputs of one combination's pair draws.  Each pair is drawn in three fixed-point
// inverse-CDF stages:
//   row:    T = U64 * S >> 64 against the exact prefix sums of trunc(r_i 2^40);
//   tile:   24-bit fixed-point images of the row's tile weights (reference: its largest
//           tile), T = floor(w2 Q / 2^32);
//   column: the chosen tile's columns recomputed (pair_exponent + ex2), images relative to
//           the tile weight t_ik, w3.
struct DrawIn {
  int sys;                        // systematic positions (k + U) / N instead of iid uniforms
  const unsigned long long* cum;  // [N] exact prefix sums of the row weights
  const float* T;                 // [N][nTp] tile weights
  const float* U;                 // [N][D]
  const float* alpha;             // [N]
  const float* delta;             // [N]
  const float* V;                 // [N][D]
  const float* beta;              // [N]
  int N, B, nT, nTp;
};

// Fixed-point pick over n <= W <= 32 weights held in registers: q_k = q24(x_k; ref),
// Q = sum q (< 2^29 for tile weights below their maximum, < 2^29 for columns below twice
// their tile weight), T = floor(w Q / 2^32) (w a 32-bit uniform word), the number of prefix
// sums <= T, clamped to n - 1; 0 when Q = 0.  Entries past n add nothing to Q and never
// count (their prefix sum is Q > T), so every W >= n gives the same index.
// The systematic sampler's next uniform word: the target's position inside the chosen
// interval [bef, aft) as a fraction of its length, trunc((T - bef) / (aft - bef) 2^32), with a
// correctly rounded FP64 quotient (the oracle's checker computes the same bits).
__device__ __forceinline__ uint32_t remainder_word(unsigned long long T, unsigned long long bef,
                                                   unsigned long long aft) {
  return __double2uint_rz(__ddiv_rn((double)(T - bef), (double)(aft - bef)) * 4294967296.0);
}

// When wrem is not null it receives remainder_word of the target inside the chosen entry.
template <int W>
__device__ __forceinline__ int pick_w(const float* x, int n, uint32_t w, int ref_be, uint32_t* wrem = nullptr) {
  uint32_t c[W];  // the prefix sums, formed as Q is summed
  uint32_t Q = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    Q += (k < n) ? q24(x[k], ref_be) : 0u;
    c[k] = Q;
  }
  if (Q == 0u) {
    if (wrem) *wrem = w;
    return 0;
  }
  const uint32_t T = __umulhi(w, Q);
  uint32_t bef = 0, aft = 0xFFFFFFFFu;
  int idx = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    idx += (c[k] <= T) ? 1 : 0;
    if (wrem) {
      bef = (c[k] <= T) ? c[k] : bef;
      aft = (c[k] > T) ? min(aft, c[k]) : aft;
    }
  }
  if (wrem) *wrem = remainder_word(T, bef, aft);
  return min(idx, n - 1);
}
__device__ __forceinline__ int pick32(const float* x, int n, uint32_t w, int ref_be) {
  return pick_w<32>(x, n, w, ref_be);
}

// The tile stage over nT <= W tiles of a row held in registers: the largest tile is the
// reference.  The row is read as float4 (16-byte aligned rows) or, with T2, as float2
// (8-byte aligned rows); entries past nT are ignored.
template <int W, bool T2 = false>
__device__ __forceinline__ int pick_tile(const float* Ti, int nT, uint32_t w, uint32_t* wrem = nullptr) {
  float t[W];
  if (T2) {
    const float2* Ti2 = reinterpret_cast<const float2*>(Ti);
#pragma unroll
    for (int k2 = 0; k2 < W / 2; ++k2) {
      const float2 v = (2 * k2 < nT) ? Ti2[k2] : make_float2(0.f, 0.f);
      t[2 * k2] = v.x;
      t[2 * k2 + 1] = v.y;
    }
  } else {
    const float4* Ti4 = reinterpret_cast<const float4*>(Ti);
#pragma unroll
    for (int k4 = 0; k4 < W / 4; ++k4) {
      const float4 v = (4 * k4 < nT) ? Ti4[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
      t[4 * k4] = v.x;
      t[4 * k4 + 1] = v.y;
      t[4 * k4 + 2] = v.z;
      t[4 * k4 + 3] = v.w;
    }
  }
  float tmax = 0.f;
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (k < nT) tmax = fmaxf(tmax, t[k]);
  return pick_w<W>(t, nT, w, ref_exponent(tmax), wrem);
}

// The same pick over n weights in memory (any n; 64-bit sums).
__device__ __forceinline__ int pick_mem(const float* x, int n, uint32_t w, int ref_be, uint32_t* wrem = nullptr) {
  unsigned long long Q = 0;
  for (int k = 0; k < n; ++k) Q += q24(x[k], ref_be);
  if (Q == 0ull) {
    if (wrem) *wrem = w;
    return 0;
  }
  const unsigned long long T = __umul64hi((unsigned long long)w << 32, Q);
  unsigned long long c = 0, bef = 0, aft = ~0ull;
  int idx = 0;
  for (int k = 0; k < n; ++k) {
    c += q24(x[k], ref_be);
    idx += (c <= T) ? 1 : 0;
    bef = (c <= T) ? c : bef;
    aft = (c > T) ? min(aft, c) : aft;
  }
  if (wrem) *wrem = remainder_word(T, bef, aft);
  return min(idx, n - 1);
}

// The tile stage over 32 < nT <= 64 tiles of a row in memory (16-byte aligned, nTp >= nT
// floats, entries past nT ignored): the largest tile is the reference; both halves' image
// sums, then the chosen half once more (the same index as one pass over all tiles).
__device__ __forceinline__ int pick_tile64(const float* Ti, int nT, uint32_t w, uint32_t* wrem = nullptr) {
  const float4* T4 = reinterpret_cast<const float4*>(Ti);
  auto at = [&](const float4& v, int k, int c) {  // element c of the float4 at tile 4k
    const float x = c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
    return 4 * k + c < nT ? x : 0.f;
  };
  float tmax = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (4 * k < nT) {
      const float4 v = T4[k];
#pragma unroll
      for (int c = 0; c < 4; ++c) tmax = fmaxf(tmax, at(v, k, c));
    }
  }
  const int be = ref_exponent(tmax);
  unsigned long long Q1 = 0, Q2 = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (4 * k < nT) {
      const float4 v = T4[k];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const uint32_t q = q24(at(v, k, c), be);
        if (k < 8) Q1 += q; else Q2 += q;
      }
    }
  }
  const unsigned long long Q = Q1 + Q2;
  if (Q == 0ull) {
    if (wrem) *wrem = w;
    return 0;
  }
  const unsigned long long T = __umul64hi((unsigned long long)w << 32, Q);
  const bool second = T >= Q1;
  const int k0 = second ? 8 : 0;
  unsigned long long c = second ? Q1 : 0ull;
  unsigned long long bef = c, aft = ~0ull;
  int cnt = second ? 32 : 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (4 * (k0 + k) < nT) {
      const float4 v = T4[k0 + k];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        c += q24(at(v, k0 + k, e), be);
        const bool in = 4 * (k0 + k) + e < nT;
        cnt += (in && c <= T) ? 1 : 0;
        if (wrem && in) {
          bef = (c <= T) ? c : bef;
          aft = (c > T) ? min(aft, c) : aft;
        }
      }
    }
  }
  if (wrem) *wrem = remainder_word(T, bef, aft);
  return min(cnt, nT - 1);
}

// Slot n's pair (i, j) of combination gid, one thread:
//   row:    binary search of T = U64 * S >> 64 in the exact prefix sums;
//   tile:   pick over the row's tile weights (reference: the largest), word w2;
//   column: the chosen tile's columns recomputed (pair_exponent + ex2), pick with the
//           tile weight t_ik as reference, word w3.
// Systematic mode (in.sys): one 64-bit uniform U of the combination (counter (0, gid, SYS))
// gives V = floor(U S / 2^64), slot k's row target is T_k = floor((k S + V) / N) =
// k q + floor((k r + V) / N) with S = q N + r, and w2 / w3 are the remainder words of the
// row and tile targets inside their chosen entries, so that every slot sits at its own
// position of the flattened fixed-point CDF, S / N apart.
// The tiles are held in registers when nT <= 32, the columns when the tile has <= 32.
// SMALL: the caller guarantees nT <= 16 and tiles of <= 32 columns (N <= 512 at B = 32),
// and only those paths are compiled (the same decisions as the general form).  T2: the tile
// rows are only 8-byte aligned (SMALL only).
template <int D, bool PAD, bool SMALL = false, bool T2 = false>
__device__ __forceinline__ void draw_pair(const DrawIn& in, uint64_t seed, uint32_t base, int gid, int n,
                                          int& i, int& j) {
  const int N = in.N, B = in.B, nT = in.nT, nTp = in.nTp;
  const unsigned long long S = in.cum[N - 1];
  if (S == 0ull) {
    i = n % N;
    j = n % N;
    return;
  }
  unsigned long long Tg;
  uint32_t w2, w3;
  if (in.sys) {
    const uint4 w0 = draw(seed, 0u, (uint32_t)gid, kPurposeSys, base, 0u);
    const unsigned long long V = __umul64hi(((unsigned long long)w0.x << 32) | (unsigned long long)w0.y, S);
    const unsigned long long q = S / (unsigned long long)N, r = S % (unsigned long long)N;
    Tg = (unsigned long long)n * q + ((unsigned long long)n * r + V) / (unsigned long long)N;
    w2 = w3 = 0u;
  } else {
    const uint4 w = draw(seed, (uint32_t)n, (uint32_t)gid, kPurposeDense, base, 0u);
    Tg = __umul64hi(((unsigned long long)w.x << 32) | (unsigned long long)w.y, S);
    w2 = w.z;
    w3 = w.w;
  }
  int lo = 0, hi = N - 1;  // first i with cum[i] > Tg (cum[N-1] = S > Tg)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (in.cum[mid] > Tg) hi = mid; else lo = mid + 1;
  }
  i = lo;
  uint32_t* wr = nullptr;
  if (in.sys) {
    const unsigned long long prev = i > 0 ? in.cum[i - 1] : 0ull;
    w2 = remainder_word(Tg, prev, in.cum[i]);
    wr = &w3;
  }
  const float* Ti = in.T + (size_t)i * nTp;
  int kt;
  if (SMALL || nT <= 16) {
    kt = pick_tile<16, T2>(Ti, nT, w2, wr);
  } else if (nT <= 32) {
    kt = pick_tile<32>(Ti, nT, w2, wr);
  } else if (nT <= 64) {
    kt = pick_tile64(Ti, nT, w2, wr);
  } else {
    float tmax = 0.f;
    for (int k = 0; k < nT; ++k) tmax = fmaxf(tmax, Ti[k]);
    kt = pick_mem(Ti, nT, w2, ref_exponent(tmax), wr);
  }
  const int tbe = ref_exponent(Ti[kt]);
  const int jb = kt * B, ncol = min(jb + B, N) - jb;
  float u[D];
  load_row<D>(in.U + (size_t)i * D, u);
  const float al = __fsub_rn(in.alpha[i], in.delta[i]);
  const float* V = in.V;
  const float* beta = in.beta;
  if (ncol == 32) {  // a full tile: the columns sit at fixed offsets from the tile's first
    const float* Vt = V + vidx<D, PAD>(jb);
    const float* bt = beta + bidx<PAD>(jb);
    float e[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      float v[D];
      load_row<D>(Vt + q * D, v);
      e[q] = ex2(pair_exponent<D>(u, al, v, bt[q]));
    }
    j = jb + pick32(e, 32, w3, tbe);
  } else if (SMALL || ncol <= 32) {
    float e[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int jj = jb + min(q, ncol - 1);
      float v[D];
      load_row<D>(V + vidx<D, PAD>(jj), v);
      e[q] = (q < ncol) ? ex2(pair_exponent<D>(u, al, v, beta[bidx<PAD>(jj)])) : 0.f;
    }
    j = jb + pick32(e, ncol, w3, tbe);
  } else if (ncol <= 64) {
    // two halves of 32 columns: both image sums, then the chosen half once more.  This is
    // the index of one pass over all columns: every prefix sum of the other half lies on
    // the far side of T (the first half's are <= Q1 <= T, the second's >= Q1 > T).
    const int n2 = ncol - 32;
    unsigned long long Q1 = 0, Q2 = 0;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      float v[D];
      load_row<D>(V + vidx<D, PAD>(jb + q), v);
      Q1 += q24(ex2(pair_exponent<D>(u, al, v, beta[bidx<PAD>(jb + q)])), tbe);
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int jj = jb + 32 + min(q, n2 - 1);
      float v[D];
      load_row<D>(V + vidx<D, PAD>(jj), v);
      const float x = ex2(pair_exponent<D>(u, al, v, beta[bidx<PAD>(jj)]));
      Q2 += (q < n2) ? q24(x, tbe) : 0u;
    }
    const unsigned long long Qc = Q1 + Q2;
    j = jb;
    if (Qc != 0ull) {
      const unsigned long long Tc = __umul64hi((unsigned long long)w3 << 32, Qc);
      const bool second = Tc >= Q1;
      const int h0 = second ? jb + 32 : jb, hn = second ? n2 : 32;
      unsigned long long cc = second ? Q1 : 0ull;
      int cnt = second ? 32 : 0;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int jj = h0 + min(q, hn - 1);
        float v[D];
        load_row<D>(V + vidx<D, PAD>(jj), v);
        const float x = ex2(pair_exponent<D>(u, al, v, beta[bidx<PAD>(jj)]));
        cc += (q < hn) ? q24(x, tbe) : 0u;
        cnt += (q < hn && cc <= Tc) ? 1 : 0;
      }
      j = jb + min(cnt, ncol - 1);
    }
  } else {
    unsigned long long Qc = 0;
    for (int jj = jb; jj < jb + ncol; ++jj)
      Qc += q24(ex2(pair_exponent<D>(u, al, V + vidx<D, PAD>(jj), beta[bidx<PAD>(jj)])), tbe);
    j = jb;
    if (Qc != 0ull) {
      const unsigned long long Tc = __umul64hi((unsigned long long)w3 << 32, Qc);
      unsigned long long cc = 0;
      int cnt = 0;
      for (int jj = jb; jj < jb + ncol; ++jj) {
        cc += q24(ex2(pair_exponent<D>(u, al, V + vidx<D, PAD>(jj), beta[bidx<PAD>(jj)])), tbe);
        cnt += (cc <= Tc) ? 1 : 0;
      }
      j = jb + min(cnt, ncol - 1);
    }
  }
}

// ---------------------------------------------------------------- outputs of a combination
// The pair of slot n, and the new block's first / last index maps (the composition of the
// Remark in Section 3.1) into the other map buffer; slot N (a conditional root's extra draw)
// goes to the next reference's root pair.
struct SlotOut {
  int32_t *pl, *pr, *first_out, *last_out;
  const int32_t *first_L, *last_R;
  bool left_leaf, right_leaf;
  int N;
  int32_t* star;
  __device__ __forceinline__ void put(int n, int i, int j) const {
    if (n < N) {
      pl[n] = i;
      pr[n] = j;
      first_out[n] = left_leaf ? i : first_L[i];
      last_out[n] = right_leaf ? j : last_R[j];
    } else {
      star[0] = i;
      star[1] = j;
    }
  }
  // put in two halves: the composed map entries (global loads for merged blocks), and the
  // stores, which a caller can place after other work while the loads are in flight
  __device__ __forceinline__ void maps(int i, int j, int32_t& fi, int32_t& lj) const {
    fi = left_leaf ? i : first_L[i];
    lj = right_leaf ? j : last_R[j];
  }
  __device__ __forceinline__ void store(int n, int i, int j, int32_t fi, int32_t lj) const {
    if (n < N) {
      pl[n] = i;
      pr[n] = j;
      first_out[n] = fi;
      last_out[n] = lj;
    } else {
      star[0] = i;
      star[1] = j;
    }
  }
};

// The output maps of combination cb (and slot 0 of a conditional combination).
__device__ __forceinline__ SlotOut slot_out(const MergeArgs& a, const Comb& cb, bool write_slot0) {
  const int at = cb.at, c = cb.c, b = cb.b, K = cb.K;
  const int N = a.N;
  const int sR = b - c + 1;
  const int bufL = cb.level & 1, bufR = ceil_log2(sR) & 1, bufO = (cb.level + 1) & 1;
  SlotOut o;
  o.pl = cb.pairs + (size_t)cb.gid * 2 * N;
  o.pr = o.pl + N;
  o.first_out = cb.first + ((size_t)bufO * K + at) * N;
  o.last_out = cb.last + ((size_t)bufO * K + at) * N;
  o.first_L = cb.first + ((size_t)bufL * K + at) * N;
  o.last_R = cb.last + ((size_t)bufR * K + c) * N;
  o.left_leaf = (cb.level == 0);
  o.right_leaf = (sR == 1);
  o.N = N;
  o.star = cb.star;
  if (cb.conditional && write_slot0) {
    o.pl[0] = 0;
    o.pr[0] = 0;
    o.first_out[0] = o.left_leaf ? 0 : o.first_L[0];
    o.last_out[0] = o.right_leaf ? 0 : o.last_R[0];
  }
  return o;
}

}  // namespace parts
}  // namespace dsmc
