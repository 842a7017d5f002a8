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
#include "merge_parts.cuh"
#include "tc_ops.cuh"

namespace dsmc {

namespace {

using namespace parts;
using namespace tc;

constexpr int kEpiThreads = 256;
constexpr int kRsThreads = 128;

// ---------------------------------------------------------------------------------------
// Prologue: endpoint states through the block index maps, column / row terms, bound.
// One CTA per combination.
// ---------------------------------------------------------------------------------------
template <int D>
__host__ __device__ constexpr int prologue_threads() {
  return D <= 8 ? 256 : 128;   // several combinations per SM: the pass is latency-bound
}

// Shared-memory staging of the prologue (floats, each array rounded up to 4): the two
// particle slices X_c and X_{c-1} [N][d], one index map or leaf log-weight row per side
// [N], and the column terms v [N][D] and beta [N].  Staged when it fits kProStageMax bytes;
// otherwise every read goes to global memory.
constexpr size_t kProStageMax = 112 * 1024;
__host__ __device__ constexpr int round4(int n) { return (n + 3) & ~3; }
template <int D>
__host__ __device__ constexpr size_t prologue_stage_bytes(int N, int d) {
  return sizeof(float) * (2 * (size_t)round4(N * d) + 3 * (size_t)round4(N) + (size_t)round4(N * D));
}
template <int D>
__host__ __device__ constexpr bool prologue_staged(int N, int d) {
  return prologue_stage_bytes<D>(N, d) <= kProStageMax;
}

template <int D>
__host__ __device__ constexpr int prologue_min_blocks() {
  return D <= 4 ? 6 : 0;   // 0: no minimum (larger D would spill)
}

template <int D>
__global__ void __launch_bounds__(prologue_threads<D>(), prologue_min_blocks<D>())
    prologue_kernel(MergeArgs a, ModelParams<D> mp) {
  constexpr int kProThreads = prologue_threads<D>();
  constexpr int NW = kProThreads / 32;
  const int s = blockIdx.x;
  const Comb cb = comb_of(a, s);
  const int at = cb.at, c = cb.c, b = cb.b;
  const int N = a.N, d = a.d;
  const bool left_leaf = (cb.level == 0);
  const int sR = b - c + 1;
  const bool right_leaf = (sR == 1);
  const int bufL = cb.level & 1;
  const int bufR = ceil_log2(sR) & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the dense samplers' row CDF takes the shift as a combination base and FP32 row offsets
  const bool dense = a.resampler == DSMC_MULTINOMIAL || a.resampler == DSMC_SYSTEMATIC;

  float* V = a.ws.V + (size_t)s * N * D;
  float* beta = a.ws.beta + (size_t)s * N;
  float* U = a.ws.U + (size_t)s * N * D;
  float* alpha = a.ws.alpha + (size_t)s * N;
  double* shift = a.ws.shift + (size_t)s * N;
  const int32_t* firstR = right_leaf ? nullptr : cb.first + ((size_t)bufR * cb.K + c) * N;
  const int32_t* lastL = left_leaf ? nullptr : cb.last + ((size_t)bufL * cb.K + at) * N;
  const float* Xc = cb.X + (size_t)c * N * d;
  const float* Xl = cb.X + (size_t)(c - 1) * N * d;
  const float* lwc = right_leaf ? cb.logw + (size_t)c * N : nullptr;
  const float* lwl = left_leaf ? cb.logw + (size_t)(c - 1) * N : nullptr;
  // the column terms as pass 2 and the row shift read them back
  float* Vs = V;
  float* Bs = beta;
  const bool staged = prologue_staged<D>(N, d);
  if (staged) {  // every input of the combination in one round of coalesced loads
    extern __shared__ float4 pro_smem4[];
    float* sXc = reinterpret_cast<float*>(pro_smem4);
    float* sXl = sXc + round4(N * d);
    float* sR0 = sXl + round4(N * d);
    float* sL0 = sR0 + round4(N);
    Bs = sL0 + round4(N);
    Vs = Bs + round4(N);
    stage_words(sXc, Xc, N * d);
    stage_words(sXl, Xl, N * d);
    if (right_leaf)
      stage_words(sR0, lwc, N);
    else
      stage_words(reinterpret_cast<int32_t*>(sR0), firstR, N);
    if (left_leaf)
      stage_words(sL0, lwl, N);
    else
      stage_words(reinterpret_cast<int32_t*>(sL0), lastL, N);
    Xc = sXc;
    Xl = sXl;
    if (right_leaf) lwc = sR0; else firstR = reinterpret_cast<const int32_t*>(sR0);
    if (left_leaf) lwl = sL0; else lastL = reinterpret_cast<const int32_t*>(sL0);
  }

  float yc[D], qm[D], qs[D];
#pragma unroll
  for (int k = 0; k < D; ++k) yc[k] = k < d ? cb.y[(size_t)c * d + k] : 0.f;
  proposal_at<D>(mp, cb.y, cb.prop_mean, cb.prop_std, c, qm, qs);
  float qinv[D];
  const float qnorm = proposal_consts<D>(d, qs, qinv);

  __shared__ float gsum[kMaxColumnGroups * D];
  __shared__ float red_s[NW];
  __shared__ float red2_s[NW];
  __shared__ float mu_s[D];
  __shared__ float bstar_s;
  if (staged) __syncthreads();

  // One-dimensional states, lazy sampler: the hull [m_lo, m_hi] of the transition means
  // m_i = m(x_i) over the whole time-(c - 1) slice (a superset of the left block's end
  // states) bounds every pair: f(x_j | x_i) <= f_max exp(-dist_j^2 Q^-1 / 2) with dist_j
  // the distance from x_j to the hull, so log omega-bar = log f_max + max_i a_i +
  // max_j (b'_j - dist_j^2 Q^-1 / 2) is a valid bound of the combination's pair weights
  // (Algorithm 8 needs any bound; a particle far outside the hull otherwise sets it).
  const bool hull = (D == 1) && a.resampler != DSMC_MULTINOMIAL && a.resampler != DSMC_SYSTEMATIC;
  float m_lo = 0.f, m_hi = 0.f, bhull = -INFINITY;
  if (hull) {
    float lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < N; i += kProThreads) {
      float xi[D], mi[D];
#pragma unroll
      for (int k = 0; k < D; ++k) xi[k] = 0.f;
      xi[0] = Xl[i];
      transition_mean<D>(mp, xi, mi);
      const float m = mi[0];
      lo = fminf(lo, m);
      hi = fmaxf(hi, m);
    }
    lo = -warp_max(-lo);
    hi = warp_max(hi);
    if (lane == 0) {
      red_s[warp] = lo;
      red2_s[warp] = hi;
    }
    __syncthreads();
    lo = red_s[0];
    hi = red2_s[0];
    for (int w = 1; w < NW; ++w) {
      lo = fminf(lo, red_s[w]);
      hi = fmaxf(hi, red2_s[w]);
    }
    m_lo = lo;
    m_hi = hi;
    __syncthreads();  // red_s is reused by the column pass
  }

  // pass 1: right block at time c (column states, b'_j; the mean mu and B*)
  bool bad = false, corrupt = false;
  float mu[D], bstar;
  column_pass<D>(N, gsum, red_s, mu_s, &bstar_s, mu, bstar, bad, [&](int j, float* x) {
    const float bp = column_bprime<D>(mp, N, d, a.logN, yc, qm, qinv, qnorm, Xc, firstR, lwc, j, x, corrupt);
#pragma unroll
    for (int k = 0; k < D; ++k) Vs[(size_t)j * D + k] = x[k];
    Bs[j] = bp;
    return bp;
  });

  // pass 2a: columns  v_j = xR_j - mu,  beta_j = log2(e) (b'_j - B* - 1/2 v' Q^-1 v)
  const bool factored = a.resampler == DSMC_RS_FACTORED;
  for (int j = threadIdx.x; j < N; j += kProThreads) {
    float v[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = Vs[(size_t)j * D + k];
    const float bp = Bs[j];
    float dist2h = 0.f;  // dist_j^2 Q^-1 / 2
    if (hull) {  // v is still x_j here
      const float dist = fmaxf(0.f, fmaxf(v[0] - m_hi, m_lo - v[0]));
      dist2h = 0.5f * mp.Qi[0] * dist * dist;
      bhull = fmaxf(bhull, bp - dist2h);
    }
    const float bj = column_beta<D>(mp, v, mu, bp, bstar);
    if (factored) {  // column proposal weight (log) and acceptance term
      a.ws.pc[(size_t)s * N + j] = bp - dist2h;
      a.ws.kappa[(size_t)s * N + j] = kLog2e * (dist2h - 0.5f * quad_form<D>(mp.Qi, v));
    }
    beta[j] = bj;
#pragma unroll
    for (int k = 0; k < D; ++k) V[(size_t)j * D + k] = v[k];
    if (staged) {
      Bs[j] = bj;
#pragma unroll
      for (int k = 0; k < D; ++k) Vs[(size_t)j * D + k] = v[k];
    }
    if (a.compute != DSMC_FP32) {
      float ext[4];
      ext[0] = 1.f;
      ext[1] = 1.f;
      split_mma(bj, a.compute, &ext[2], &ext[3]);
      store_mma_row<D>(a.ws.Vb + (size_t)s * a.Nr * a.mma_planes * 32, a.Nr, j, v, ext, a.compute);
    }
  }
  if (a.compute != DSMC_FP32) {  // zero the padding rows of the tensor-core operands
    const float zero[D] = {};
    const float zext[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j = N + threadIdx.x; j < a.Nr; j += kProThreads) {
      store_mma_row<D>(a.ws.Vb + (size_t)s * a.Nr * a.mma_planes * 32, a.Nr, j, zero, zext, a.compute);
      store_mma_row<D>(a.ws.Ub + (size_t)s * a.Nr * a.mma_planes * 32, a.Nr, j, zero, zext, a.compute);
    }
  }
  __syncthreads();  // the column terms are written: the rows read a sample of them
  // pass 2b: rows  w_i = A xL_i + c - mu,  u_i = log2(e) Q^-1 w_i,
  //                alpha_i = -log2(e) 1/2 w_i' Q^-1 w_i - delta_i  (B* is folded into beta,
  //                delta_i, the row's sampled shift, into shift_i)
  float amax = -INFINITY;
  const double base_m = shift_base(-a.logN, mp.log_f_max, bstar);  // a merged left block's
  for (int i = threadIdx.x; i < N; i += kProThreads) {
    float ul[D], ai;
    const float al0 = row_terms<D>(mp, N, d, a.logN, Xl, lastL, lwl, i, mu, ul, ai, corrupt);
    const float dl = row_shift<D, false>(ul, al0, Vs, Bs, N);
    const float al = __fsub_rn(al0, dl);
    bad |= isnan(ai);
    if (factored) {  // row proposal weight (log) and the unshifted row term
      a.ws.pa[(size_t)s * N + i] = ai;
      a.ws.alpha0[(size_t)s * N + i] = al0;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) U[(size_t)i * D + k] = ul[k];
    if (a.compute != DSMC_FP32) {
      float ext[4];
      split_mma(al, a.compute, &ext[0], &ext[1]);
      ext[2] = 1.f;
      ext[3] = 1.f;
      store_mma_row<D>(a.ws.Ub + (size_t)s * a.Nr * a.mma_planes * 32, a.Nr, i, ul, ext, a.compute);
    }
    alpha[i] = al;
    shift[i] = row_shift_total(lwl != nullptr ? shift_base(ai, mp.log_f_max, bstar) : base_m, dl);
    if (dense) a.ws.g[(size_t)s * N + i] = row_offset(left_leaf, ai, dl);
    amax = fmaxf(amax, ai);
  }
  amax = warp_max(amax);
  bhull = warp_max(bhull);
  __syncthreads();
  if (lane == 0) {
    red_s[warp] = amax;
    red2_s[warp] = bhull;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = red_s[0], bh = red2_s[0];
    for (int w = 1; w < NW; ++w) {
      t = fmaxf(t, red_s[w]);
      bh = fmaxf(bh, red2_s[w]);
    }
    a.ws.logbar[s] = (double)mp.log_f_max + (double)t + (double)(hull ? bh : bstar);
    if (dense) a.ws.cbase[s] = comb_base(left_leaf, a.logN, mp.log_f_max, bstar);
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

// ---------------------------------------------------------------------------------------
// Row CDF of one combination (one CTA):
//   row totals s_i = row_total of the row's tile weights (even / odd pair sums; thread per row,
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
  __shared__ float redf[NW];
  __shared__ float M_s;
  __shared__ int n_under, nonfinite_s;
  if (threadIdx.x == 0) {
    n_under = 0;
    nonfinite_s = 0;
  }
  __syncthreads();
  const float* Tt = a.ws.T + (size_t)s * N * nTp;
  const float* g = a.ws.g + (size_t)s * N;
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
    {
      const float* U = a.ws.U + (size_t)s * N * D;
      recompute_row<D, false>(U + (size_t)i * D, a.ws.alpha[(size_t)s * N + i], a.ws.V + (size_t)s * N * D,
                       a.ws.beta + (size_t)s * N, N, a.B, nT, a.ws.T + ((size_t)s * N + i) * nTp, &si, &dl);
    }
    __syncwarp();
    if (lane == 0) {
      si = row_total(Tt + (size_t)i * nTp, nT, nTp);
      l2[i] = isnan(si) ? 0.f : si;
      delta[i] = dl;
    }
  }
  __syncthreads();
  float mloc = -INFINITY;
  for (int i = threadIdx.x; i < N; i += kCdfThreads) {
    const float t = l2[i];
    rowsum[i] = t;
    const float v = row_log2_weight(g[i], delta[i], t);
    l2[i] = v;
    mloc = fmaxf(mloc, v);
  }
  mloc = warp_max(mloc);
  if (lane == 0) redf[warp] = mloc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = redf[0];
    for (int w = 1; w < NW; ++w) t = fmaxf(t, redf[w]);
    M_s = t;
  }
  __syncthreads();
  const float M = M_s;
  const bool degenerate = !(M > -INFINITY) || isnan(M);
  float* rw = a.ws.rw + (size_t)s * N;
  for (int i = threadIdx.x; i < N; i += kCdfThreads) {
    const float r = row_weight(l2[i], M, degenerate);
    rw[i] = r;
    cum[i] = (unsigned long long)__float2ull_rz(r * 0x1p40f);
  }
  __syncthreads();
  block_scan_u64(cum, N, warp_tot);
  unsigned long long* gcum = a.ws.cum + (size_t)s * N;
  for (int i = threadIdx.x; i < N; i += kCdfThreads) gcum[i] = cum[i];
  if (threadIdx.x == 0) {
    const Comb cb = comb_of(a, s);
    // Eq. (Lab): log of sum_ij exp(logW_ij) = M ln 2 + ln(sum_i r_i), the row-weight total
    // taken from its exact fixed-point image
    const double inc = degenerate ? (double)NAN : lab_increment(a.ws.cbase[s], M, log_fixed_total(cum[N - 1]));
    a.ws.inc[s] = inc;
    cb.logL[cb.at] = cb.logL[cb.at] + cb.logL[cb.c] + inc;
    if (degenerate || cum[N - 1] == 0ull) record_status(a.ws.status, DSMC_ERR_DEGENERATE);
    if (nonfinite_s) record_status(a.ws.status, DSMC_ERR_NONFINITE);
  }
}

// ---------------------------------------------------------------------------------------
// Pair draws (one thread per slot, many small CTAs per combination; used when a
// combination's operands do not fit one CTA's shared memory): draw_pair, then the pair and
// the new block's first / last index maps (the composition of the Remark in Section 3.1)
// into the other map buffer.
// ---------------------------------------------------------------------------------------
constexpr int kSlotThreads = 128;

template <int D>
__global__ void __launch_bounds__(kSlotThreads) slots_kernel(MergeArgs a) {
  const int s = blockIdx.x;
  const Comb cb = comb_of(a, s);
  const int gid = cb.gid;
  const int N = a.N;
  const SlotOut o = slot_out(a, cb, blockIdx.y == 0 && threadIdx.x == 0);
  const int n_lo = cb.conditional ? 1 : 0;
  const int n_hi = N + ((cb.conditional && cb.root) ? 1 : 0);
  const int n = n_lo + blockIdx.y * kSlotThreads + threadIdx.x;
  if (n >= n_hi) return;
  DrawIn in;
  in.sys = (a.resampler == DSMC_SYSTEMATIC && !cb.conditional) ? 1 : 0;
  in.cum = a.ws.cum + (size_t)s * N;
  in.T = a.ws.T + (size_t)s * N * a.nTp;
  in.U = a.ws.U + (size_t)s * N * D;
  in.alpha = a.ws.alpha + (size_t)s * N;
  in.delta = a.ws.delta + (size_t)s * N;
  in.V = a.ws.V + (size_t)s * N * D;
  in.beta = a.ws.beta + (size_t)s * N;
  in.N = N;
  in.B = a.B;
  in.nT = a.nT;
  in.nTp = a.nTp;
  int i, j;
  draw_pair<D, false>(in, cb.seed, cb.base, gid, n, i, j);
  o.put(n, i, j);
}

// ---------------------------------------------------------------------------------------
// Row CDF and pair draws of one combination in one 256-thread CTA (when its operands fit
// shared memory; four CTAs per SM for d <= 8): the column terms v_j, beta_j, the row terms
// u_i, alpha_i and the row shifts delta_i are staged in shared memory, the row totals, the
// row CDF and the increment are computed as in rowcdf_kernel, then every slot is drawn
// (one thread per slot, N / 256 slots each) against the shared-memory copies.
// ---------------------------------------------------------------------------------------
constexpr int kCdfSlotThreads = 256;

// Shared-memory layout of the row CDF + draws kernel: padded v [vpad_floats], u [N][D],
// padded beta, l [N], prefix sums [N], alpha and delta [2][N].  The tile sums T are staged
// too (row
// stride nTs = nTp, plus 4 when nTp / 4 is even, so that the rows of 8 consecutive threads
// fall in distinct 16-byte bank groups) when the whole fits kCdfStageMax (four CTAs of 256
// threads per SM: more combinations in flight beat staging T at larger N).
constexpr size_t kCdfStageMax = 56 * 1024;
struct CdfSlotsSmem {
  size_t v, u, b, l, c, ad, t, total;
  int nTs;  // staged row stride of T, 0 when T stays in global memory
};

__host__ __device__ __forceinline__ int staged_tile_stride(int nTp) {
  return ((nTp / 4) % 2 == 0) ? nTp + 4 : nTp;
}

template <int D>
__host__ __device__ __forceinline__ CdfSlotsSmem cdf_slots_smem(int N, int nTp) {
  const auto r16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  CdfSlotsSmem f;
  size_t o = 0;
  f.v = o; o = r16(o + (size_t)vpad_floats<D>(N) * 4);
  f.u = o; o = r16(o + (size_t)N * D * 4);
  f.b = o; o = r16(o + (size_t)bpad_floats(N) * 4);
  f.l = o; o = r16(o + (size_t)N * 4);
  f.c = o; o = r16(o + (size_t)N * 8);
  f.ad = o; o = r16(o + (size_t)N * 8);   // alpha_i and delta_i (row offsets of the draws)
  f.t = o;
  const int nTs = staged_tile_stride(nTp);
  const size_t with_t = r16(o + (size_t)N * nTs * 4);
  if (with_t <= kCdfStageMax) {
    f.nTs = nTs;
    o = with_t;
  } else {
    f.nTs = 0;
  }
  f.total = o;
  return f;
}

// SMALL: nT <= 16 tiles of 32 columns (N <= 512), only the draw paths of that shape compiled.
template <int D, bool SMALL>
__global__ void __launch_bounds__(kCdfSlotThreads, D <= 8 ? 4 : 1) cdf_slots_kernel(MergeArgs a) {
  constexpr int NT = kCdfSlotThreads;
  constexpr int NW = NT / 32;
  const int s = blockIdx.x;
  const Comb cb = comb_of(a, s);
  const int gid = cb.gid;
  const int N = a.N, nT = a.nT, nTp = a.nTp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ __align__(16) unsigned char smraw[];
  const CdfSlotsSmem L = cdf_slots_smem<D>(N, nTp);
  float* sV = reinterpret_cast<float*>(smraw + L.v);
  float* sT = L.nTs ? reinterpret_cast<float*>(smraw + L.t) : nullptr;
  float* sU = reinterpret_cast<float*>(smraw + L.u);
  float* sB = reinterpret_cast<float*>(smraw + L.b);
  float* sL = reinterpret_cast<float*>(smraw + L.l);
  unsigned long long* sC = reinterpret_cast<unsigned long long*>(smraw + L.c);
  float* sAl = reinterpret_cast<float*>(smraw + L.ad);
  float* sDl = sAl + N;
  int* under = reinterpret_cast<int*>(sC);
  __shared__ unsigned long long warp_tot[NW];
  __shared__ float redf[NW];
  __shared__ float M_s;
  __shared__ int n_under, nonfinite_s;
  if (threadIdx.x == 0) {
    n_under = 0;
    nonfinite_s = 0;
  }
  __syncthreads();  // the counters are zero before any thread adds to them
  const float* U = a.ws.U + (size_t)s * N * D;
  const float* V = a.ws.V + (size_t)s * N * D;
  const float* beta = a.ws.beta + (size_t)s * N;
  const float* alpha = a.ws.alpha + (size_t)s * N;
  float* Tt = a.ws.T + (size_t)s * N * nTp;
  const float* g = a.ws.g + (size_t)s * N;
  float* delta = a.ws.delta + (size_t)s * N;
  float* rowsum = a.ws.rowsum + (size_t)s * N;
  // stage the operands (vector copies when D % 4 == 0: rows and pads are 16-byte aligned)
  if constexpr ((D % 4) == 0) {
    const float4* V4 = reinterpret_cast<const float4*>(V);
    const float4* U4 = reinterpret_cast<const float4*>(U);
    for (int q = threadIdx.x; q < N * D / 4; q += NT) {
      const int j = q / (D / 4), k4 = q - j * (D / 4);
      reinterpret_cast<float4*>(sV + vidx<D, true>(j))[k4] = V4[q];
      reinterpret_cast<float4*>(sU)[q] = U4[q];
    }
  } else {
    for (int q = threadIdx.x; q < N * D; q += NT) {
      const int j = q / D, k = q - j * D;
      sV[vidx<D, true>(j) + k] = V[q];
      sU[q] = U[q];
    }
  }
  for (int q = threadIdx.x; q < N; q += NT) {
    sB[bidx<true>(q)] = beta[q];
    sAl[q] = alpha[q];
  }
  // row totals (and the staged copy of the tile sums)
  for (int i = threadIdx.x; i < N; i += NT) {
    if (sT) {
      const float4* src = reinterpret_cast<const float4*>(Tt + (size_t)i * nTp);
      float4* dst = reinterpret_cast<float4*>(sT + (size_t)i * L.nTs);
      for (int k4 = 0; k4 < nTp / 4; ++k4) dst[k4] = src[k4];
    }
    // the row total: row_total's even / odd pair sums (every path's definition)
    float t = sT ? row_total(sT + (size_t)i * L.nTs, nT, nTp) : row_total(Tt + (size_t)i * nTp, nT, nTp);
    if (isnan(t)) {
      nonfinite_s = 1;
      t = 0.f;
    }
    sL[i] = t;
    delta[i] = 0.f;
    sDl[i] = 0.f;
    if (t < 0x1p-64f) under[atomicAdd(&n_under, 1)] = i;
  }
  __syncthreads();
  for (int q = warp; q < n_under; q += NW) {
    const int i = under[q];
    float si, dl;
    recompute_row<D, true>(sU + (size_t)i * D, sAl[i], sV, sB, N, a.B, nT, Tt + (size_t)i * nTp, &si, &dl);
    __syncwarp();
    if (sT) {  // the rewritten row into the staged copy
      for (int k = lane; k < nT; k += 32) sT[(size_t)i * L.nTs + k] = Tt[(size_t)i * nTp + k];
      __syncwarp();
    }
    if (lane == 0) {
      si = row_total(Tt + (size_t)i * nTp, nT, nTp);
      sL[i] = isnan(si) ? 0.f : si;
      delta[i] = dl;
      sDl[i] = dl;
    }
  }
  __syncthreads();
  // row CDF
  float mloc = -INFINITY;
  for (int i = threadIdx.x; i < N; i += NT) {
    const float t = sL[i];
    rowsum[i] = t;
    const float v = row_log2_weight(g[i], sDl[i], t);
    sL[i] = v;
    mloc = fmaxf(mloc, v);
  }
  mloc = warp_max(mloc);
  if (lane == 0) redf[warp] = mloc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = redf[0];
    for (int w = 1; w < NW; ++w) t = fmaxf(t, redf[w]);
    M_s = t;
  }
  __syncthreads();
  const float M = M_s;
  const bool degenerate = !(M > -INFINITY) || isnan(M);
  float* rw = a.ws.rw + (size_t)s * N;
  for (int i = threadIdx.x; i < N; i += NT) {
    const float r = row_weight(sL[i], M, degenerate);
    rw[i] = r;
    sC[i] = (unsigned long long)__float2ull_rz(r * 0x1p40f);
  }
  __syncthreads();
  block_scan_u64(sC, N, warp_tot);
  unsigned long long* gcum = a.ws.cum + (size_t)s * N;
  for (int i = threadIdx.x; i < N; i += NT) gcum[i] = sC[i];
  if (threadIdx.x == 0) {
    const double inc = degenerate ? (double)NAN : lab_increment(a.ws.cbase[s], M, log_fixed_total(sC[N - 1]));
    a.ws.inc[s] = inc;
    cb.logL[cb.at] = cb.logL[cb.at] + cb.logL[cb.c] + inc;
    if (degenerate || sC[N - 1] == 0ull) record_status(a.ws.status, DSMC_ERR_DEGENERATE);
    if (nonfinite_s) record_status(a.ws.status, DSMC_ERR_NONFINITE);
  }
  // pair draws
  const SlotOut o = slot_out(a, cb, threadIdx.x == 0);
  DrawIn in;
  in.sys = (a.resampler == DSMC_SYSTEMATIC && !cb.conditional) ? 1 : 0;
  in.cum = sC;
  in.T = sT ? sT : Tt;
  in.U = sU;
  in.alpha = sAl;
  in.delta = sDl;
  in.V = sV;
  in.beta = sB;
  in.N = N;
  in.B = a.B;
  in.nT = nT;
  in.nTp = sT ? L.nTs : nTp;
  const int n_lo = cb.conditional ? 1 : 0;
  const int n_hi = N + ((cb.conditional && cb.root) ? 1 : 0);
  for (int n = n_lo + threadIdx.x; n < n_hi; n += NT) {
    int i, j;
    draw_pair<D, true, SMALL>(in, cb.seed, cb.base, gid, n, i, j);
    o.put(n, i, j);
  }
}

// ---------------------------------------------------------------------------------------
// Lazy rejection samplers.  Only the proposed pairs are evaluated; (I, J, u) are redrawn
// at every attempt; each slot stops at its first acceptance or after rs_max attempts.
//   Algorithm 8 (DSMC_RS): I, J uniform (words x, y of the counter (n, gid, RS, attempt)),
//     accept iff u23(z) < exp(logW_IJ - log omega-bar).
//   Factorised proposals (DSMC_RS_FACTORED): I with probability Rq_I / SA and J with
//     probability Cq_J / SC (64-bit uniforms from words x:y and z:w of the counter
//     (n, gid, RSF, attempt), binary search of the exact prefix sums), accept iff
//     u23(x of (n, gid, RSU, attempt)) < f(x_J | x_I) / f_max (times e^{dist_J^2 / 2Q}).
// Each warp owns a contiguous range of kRsSlotsPerWarp slots; a lane that finishes its slot
// takes the range's next one (warp-compacted retry), so a slot with a low acceptance rate
// holds one lane, not its warp.  A slot that reaches the cap keeps (-1, -1) and records
// DSMC_ERR_RS_LIMIT; a ratio above 1 + 2^-10 records DSMC_ERR_BOUND.
// ---------------------------------------------------------------------------------------
constexpr int kRsSlotsPerWarp = 64;
constexpr float kBoundSlack = 1.0009765625f;  // 1 + 2^-10: FP32 rounding of a valid bound stays below

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

// The factorised sampler's acceptance ratio of pair (I, J): 2^(alpha0_I + kappa_J + u_I . v_J).
template <int D>
__device__ __forceinline__ float rsf_ratio(const MergeArgs& a, int s, int I, int J) {
  const int N = a.N;
  const float* U = a.ws.U + ((size_t)s * N + I) * D;
  const float* V = a.ws.V + ((size_t)s * N + J) * D;
  float u[D], v[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    u[k] = U[k];
    v[k] = V[k];
  }
  return ex2(pair_exponent<D>(u, a.ws.alpha0[(size_t)s * N + I], v, a.ws.kappa[(size_t)s * N + J]));
}

// First index with cum[idx] > T (cum[N-1] > T), through the read-only cache.
__device__ __forceinline__ int search_cum(const unsigned long long* cum, int N, unsigned long long T) {
  int lo = 0, hi = N - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(cum + mid) > T) hi = mid; else lo = mid + 1;
  }
  return lo;
}

template <int D, bool FACT>
__global__ void __launch_bounds__(kRsThreads) sample_rs_kernel(MergeArgs a) {
  const int s = blockIdx.y;
  const Comb cb = comb_of(a, s);
  const int gid = cb.gid;
  const int N = a.N;
  const int n_lo = cb.conditional ? 1 : 0;
  const int n_hi = N + ((cb.conditional && cb.root) ? 1 : 0);
  int32_t* pl = cb.pairs + (size_t)gid * 2 * N;
  int32_t* pr = pl + N;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ws.inc[s] = (double)NAN;  // the lazy sampler never forms the N x N sum
    if (cb.conditional) {
      pl[0] = 0;
      pr[0] = 0;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w0 = n_lo + (blockIdx.x * (kRsThreads / 32) + warp) * kRsSlotsPerWarp;
  const int w1 = min(w0 + kRsSlotsPerWarp, n_hi);
  if (w0 >= n_hi) return;  // warp-uniform
  const double logbar = FACT ? 0.0 : a.ws.logbar[s];
  const unsigned long long* cumA = a.ws.cumA + (size_t)s * N;
  const unsigned long long* cumC = a.ws.cumC + (size_t)s * N;
  const unsigned long long SA = FACT ? cumA[N - 1] : 0ull, SC = FACT ? cumC[N - 1] : 0ull;
  const bool degenerate = FACT && (SA == 0ull || SC == 0ull);
  auto put = [&](int n, int I, int J) {
    if (n < N) {
      pl[n] = I;
      pr[n] = J;
    } else {
      cb.star[0] = I;
      cb.star[1] = J;
    }
  };
  int slot = w0 + lane < w1 ? w0 + lane : -1;
  int next = w0 + 32;
  uint32_t att = 0;
  unsigned long long total = 0;
  bool capped = false, over = false;
  while (__any_sync(0xffffffffu, slot >= 0)) {
    bool fin = false;
    if (slot >= 0) {
      int I = -1, J = -1;
      bool acc = false;
      if (!degenerate) {
        float u, r;
        if (FACT) {
          const uint4 w = draw(cb.seed, (uint32_t)slot, (uint32_t)gid, kPurposeRSF, cb.base, att);
          const uint4 v = draw(cb.seed, (uint32_t)slot, (uint32_t)gid, kPurposeRSU, cb.base, att);
          I = search_cum(cumA, N, __umul64hi(((unsigned long long)w.x << 32) | w.y, SA));
          J = search_cum(cumC, N, __umul64hi(((unsigned long long)w.z << 32) | w.w, SC));
          u = u23(v.x);
          r = rsf_ratio<D>(a, s, I, J);
        } else {
          const uint4 w = draw(cb.seed, (uint32_t)slot, (uint32_t)gid, kPurposeRS, cb.base, att);
          I = (int)__umulhi(w.x, (uint32_t)N);
          J = (int)__umulhi(w.y, (uint32_t)N);
          u = u23(w.z);
          r = rs_ratio<D>(a, s, I, J, logbar);
        }
        over |= r > kBoundSlack;
        acc = u < r;
        ++att;
        ++total;
      }
      if (acc || att >= a.rs_max || degenerate) {
        fin = true;
        capped |= !acc;
        put(slot, acc ? I : -1, acc ? J : -1);
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, fin);
    if (fin) {
      const int k = next + __popc(m & ((1u << lane) - 1u));
      slot = k < w1 ? k : -1;
      att = 0;
    }
    next += __popc(m);
  }
  total = warp_sum(total);
  if (lane == 0) atomicAdd(a.ws.attempts_total, total);
  if (degenerate) {
    if (lane == 0) record_status(a.ws.status, DSMC_ERR_DEGENERATE);
  } else if (capped) {
    record_status(a.ws.status, DSMC_ERR_RS_LIMIT);
  }
  if (over) record_status(a.ws.status, DSMC_ERR_BOUND);
}

// The factorised proposals of one combination (one CTA): the row and column log-weights
// the prologue left in pa / pc become weights relative to their maxima, 2^((l - max) log2 e)
// in FP32 clamped to [0, 1], and their exact 2^40 fixed-point prefix sums (chunks of
// kCumChunk, exact u64 scans with a running carry).
constexpr int kRsfCdfThreads = 512;
constexpr int kCumChunk = 2048;

__device__ void relative_weights_and_cum(float* w, unsigned long long* cum, int N, unsigned long long* chunk,
                                         unsigned long long* warp_tot, float* redf, bool& bad) {
  constexpr int NW = kRsfCdfThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float m = -INFINITY;
  for (int i = threadIdx.x; i < N; i += kRsfCdfThreads) {
    const float x = w[i];
    bad |= isnan(x);
    m = fmaxf(m, x);
  }
  m = warp_max(m);
  if (lane == 0) redf[warp] = m;
  __syncthreads();
  float M = redf[0];
  for (int k = 1; k < NW; ++k) M = fmaxf(M, redf[k]);
  __syncthreads();  // redf is reused by the next call
  unsigned long long carry = 0;
  for (int c0 = 0; c0 < N; c0 += kCumChunk) {
    const int n = min(kCumChunk, N - c0);
    for (int k = threadIdx.x; k < n; k += kRsfCdfThreads) {
      float r = M > -INFINITY ? ex2(__fmul_rn(__fsub_rn(w[c0 + k], M), kLog2e)) : 0.f;
      if (!(r > 0.f)) r = 0.f;
      if (r > 1.f) r = 1.f;
      w[c0 + k] = r;
      chunk[k] = (unsigned long long)__float2ull_rz(r * 0x1p40f);
    }
    __syncthreads();
    block_scan_u64(chunk, n, warp_tot);
    for (int k = threadIdx.x; k < n; k += kRsfCdfThreads) cum[c0 + k] = carry + chunk[k];
    carry += chunk[n - 1];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRsfCdfThreads) rsf_cdf_kernel(MergeArgs a) {
  const int s = blockIdx.x;
  const int N = a.N;
  __shared__ unsigned long long chunk[kCumChunk];
  __shared__ unsigned long long warp_tot[kRsfCdfThreads / 32];
  __shared__ float redf[kRsfCdfThreads / 32];
  bool bad = false;
  relative_weights_and_cum(a.ws.pa + (size_t)s * N, a.ws.cumA + (size_t)s * N, N, chunk, warp_tot, redf, bad);
  relative_weights_and_cum(a.ws.pc + (size_t)s * N, a.ws.cumC + (size_t)s * N, N, chunk, warp_tot, redf, bad);
  if (bad) record_status(a.ws.status, DSMC_ERR_NONFINITE);
}

// ---------------------------------------------------------------------------------------
// Metropolis-Hastings lazy sampler (Algorithm 7): slot n starts at (n mod N, n mod N) and
// takes B = rs_max steps; step b proposes (I*, J*) uniformly (Philox word pair) and moves
// iff u r(I, J) < r(I*, J*) in FP32, r = omega / omega-bar the pair's ratio (the bound
// cancels; a current ratio of 0 accepts any proposal of positive ratio).  Only the current
// and the proposed pairs are evaluated.  One thread per slot; biased for finite B.
// ---------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kRsThreads) sample_mh_kernel(MergeArgs a) {
  const int s = blockIdx.y;
  const Comb cb = comb_of(a, s);
  const int gid = cb.gid;
  const int N = a.N;
  const int n_lo = cb.conditional ? 1 : 0;
  const int n_hi = N + ((cb.conditional && cb.root) ? 1 : 0);
  const int n = n_lo + blockIdx.x * kRsThreads + threadIdx.x;
  const double logbar = a.ws.logbar[s];
  int32_t* pl = cb.pairs + (size_t)gid * 2 * N;
  int32_t* pr = pl + N;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ws.inc[s] = (double)NAN;  // the lazy sampler never forms the N x N sum
    if (cb.conditional) {
      pl[0] = 0;
      pr[0] = 0;
    }
  }
  if (n >= n_hi) return;
  int I = n % N, J = n % N;
  float cur = rs_ratio<D>(a, s, I, J, logbar);
  for (uint32_t b = 0; b < a.rs_max; ++b) {
    const uint4 w = draw(cb.seed, (uint32_t)n, (uint32_t)gid, kPurposeMH, cb.base, b);
    const int Is = (int)__umulhi(w.x, (uint32_t)N);
    const int Js = (int)__umulhi(w.y, (uint32_t)N);
    const float prop = rs_ratio<D>(a, s, Is, Js, logbar);
    if (__fmul_rn(u23(w.z), cur) < prop) {
      I = Is;
      J = Js;
      cur = prop;
    }
  }
  if (isnan(cur)) record_status(a.ws.status, DSMC_ERR_NONFINITE);
  if (n < N) {
    pl[n] = I;
    pr[n] = J;
  } else {
    cb.star[0] = I;
    cb.star[1] = J;
  }
}

// ---------------------------------------------------------------------------------------
// Epilogue: the new block's first/last index maps (the composition of the Remark in
// Section 3.1) into the other map buffer, and log L_{a:b} = log L_{a:c-1} + log L_{c:b} +
// increment (Eq. rec-loglik, weighted form).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kEpiThreads) epilogue_kernel(MergeArgs a) {
  const int s = blockIdx.x;
  const Comb cb = comb_of(a, s);
  const int at = cb.at, c = cb.c, b = cb.b, K = cb.K;
  const int N = a.N;
  const bool left_leaf = (cb.level == 0);
  const int sR = b - c + 1;
  const bool right_leaf = (sR == 1);
  const int bufL = cb.level & 1, bufR = ceil_log2(sR) & 1, bufO = (cb.level + 1) & 1;
  const int n = blockIdx.y * kEpiThreads + threadIdx.x;
  const int32_t* pl = cb.pairs + (size_t)cb.gid * 2 * N;
  const int32_t* pr = pl + N;
  if (n < N) {
    bool corrupt = false;
    const int l = checked_index(pl[n], N, corrupt), r = checked_index(pr[n], N, corrupt);
    cb.first[((size_t)bufO * K + at) * N + n] = left_leaf ? l : cb.first[((size_t)bufL * K + at) * N + l];
    cb.last[((size_t)bufO * K + at) * N + n] = right_leaf ? r : cb.last[((size_t)bufR * K + c) * N + r];
    if (corrupt) record_status(a.ws.status, DSMC_ERR_INVALID_ARG);
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) cb.logL[at] = cb.logL[at] + cb.logL[c] + a.ws.inc[s];
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

template <int D>
__global__ void debug_lazy_kernel(MergeArgs a, int s, float* pa, float* pc, float* acc) {
  const int i = blockIdx.x;
  const int N = a.N;
  if (threadIdx.x == 0) {
    if (pa) pa[i] = a.ws.pa[(size_t)s * N + i];
    if (pc) pc[i] = a.ws.pc[(size_t)s * N + i];
  }
  if (acc)
    for (int j = threadIdx.x; j < N; j += blockDim.x) acc[(size_t)i * N + j] = rsf_ratio<D>(a, s, i, j);
}

// ------------------------------------------------------------------- launch wrappers
// Slots per combination to cover: N, one fewer when conditional (slot 0 is fixed), one more
// at a conditional root (the next reference).  Batched launches cover N + 1 (every
// combination decides its own range).
int launch_slots(const MergeArgs& a) {
  if (a.items != nullptr) return a.N + 1;
  return a.N + ((a.conditional && a.root) ? 1 : 0) - (a.conditional ? 1 : 0);
}

template <int D>
cudaError_t prologue_t(const MergeArgs& a, const void* mp, cudaStream_t st) {
  const size_t smem = prologue_staged<D>(a.N, a.d) ? prologue_stage_bytes<D>(a.N, a.d) : 0;
  static const cudaError_t attr = cudaFuncSetAttribute(
      prologue_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProStageMax);
  if (attr != cudaSuccess) return attr;
  prologue_kernel<D><<<a.mc, prologue_threads<D>(), smem, st>>>(a, *static_cast<const ModelParams<D>*>(mp));
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
  const size_t smem_cs = cdf_slots_smem<D>(a.N, a.nTp).total;
  if (smem_cs <= 200 * 1024) {  // one CTA per combination: row CDF and draws
    const bool small = a.nT <= 16 && a.B == 32;
    cudaError_t e = small ? cudaFuncSetAttribute(cdf_slots_kernel<D, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cs)
                          : cudaFuncSetAttribute(cdf_slots_kernel<D, false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cs);
    if (e != cudaSuccess) return e;
    if (small)
      cdf_slots_kernel<D, true><<<a.mc, kCdfSlotThreads, smem_cs, st>>>(a);
    else
      cdf_slots_kernel<D, false><<<a.mc, kCdfSlotThreads, smem_cs, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)a.N * (sizeof(unsigned long long) + sizeof(float));
  if (smem > 40 * 1024) {  // static shared memory counts against the 48 KB default
    cudaError_t e = cudaFuncSetAttribute(rowcdf_kernel<D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  rowcdf_kernel<D><<<a.mc, kCdfThreads, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid(a.mc, (launch_slots(a) + kSlotThreads - 1) / kSlotThreads);
  slots_kernel<D><<<grid, kSlotThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t sample_rs_t(const MergeArgs& a, cudaStream_t st) {
  if (a.resampler == DSMC_MH) {
    dim3 grid((launch_slots(a) + kRsThreads - 1) / kRsThreads, a.mc);
    sample_mh_kernel<D><<<grid, kRsThreads, 0, st>>>(a);
    return cudaGetLastError();
  }
  constexpr int kSlotsPerCta = kRsSlotsPerWarp * (kRsThreads / 32);
  dim3 grid((launch_slots(a) + kSlotsPerCta - 1) / kSlotsPerCta, a.mc);
  if (a.resampler == DSMC_RS_FACTORED)
    sample_rs_kernel<D, true><<<grid, kRsThreads, 0, st>>>(a);
  else
    sample_rs_kernel<D, false><<<grid, kRsThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t debug_lazy_t(const MergeArgs& a, int s, float* pa, float* pc, float* acc, cudaStream_t st) {
  debug_lazy_kernel<D><<<a.N, 128, 0, st>>>(a, s, pa, pc, acc);
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

cudaError_t launch_rsf_cdf(const MergeArgs& a, cudaStream_t s) {
  rsf_cdf_kernel<<<a.mc, kRsfCdfThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_debug_lazy(int D, const MergeArgs& a, int s_local, float* pa, float* pc, float* acc,
                              cudaStream_t s) {
  DSMC_DISPATCH(D, debug_lazy_t<DD>(a, s_local, pa, pc, acc, s))
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
