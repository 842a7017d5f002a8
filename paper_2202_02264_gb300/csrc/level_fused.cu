// level_fused.cu -- one whole level of Algorithm 6 for the dense sampler in a single launch:
// for each combination (Algorithm 1, or Algorithm 5 when conditional) one thread-block
// cluster of C CTAs computes the column and row terms, the tile weights, the row CDF with
// the normalising-constant increment of Eq. (Lab), and the N pair draws with the new block's
// index maps.
//
// The split per-level path (prologue, tile sums, row CDF, slot kernels) runs one CTA per
// combination in three of its four launches; on the upper levels of the tree, with few
// combinations, those launches are bound by memory latency on a handful of SMs.  Here the
// C CTAs of a cluster share one combination:
//   - every CTA evaluates all N columns (states, b'_j, mu, B*, v_j, beta_j) into its own
//     shared memory (O(N d) work, repeated per CTA instead of exchanged);
//   - CTA r owns rows [r R, (r+1) R) with R = ceil(N / C): their u_i, alpha_i and shift_i,
//     their tile weights t_ik and their row totals;
//   - the row log-weights l_i are exchanged through distributed shared memory (one cluster
//     barrier), after which every CTA builds the same row CDF;
//   - CTA r draws slots [r S, (r+1) S) of the combination, S = ceil(slots / C).
// The arithmetic is the split path's, function for function (merge_parts.cuh), and every
// reduction is either exact (maxima, the u64 prefix sums) or in an order that does not
// depend on the block size (the column mean, the per-row tile sums), so both paths give
// the same bits.
#include <cooperative_groups.h>

#include "kernels.cuh"
#include "merge_parts.cuh"

namespace dsmc {

namespace {

namespace cg = cooperative_groups;
using namespace parts;

template <int D>
__host__ __device__ constexpr int fused_threads() {
  return D <= 8 ? 512 : 256;
}

__host__ __device__ __forceinline__ size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory layout of one CTA (byte offsets).
struct FusedSmem {
  size_t v, b, l, c, u, al, sh, total;
};

__host__ __device__ __forceinline__ FusedSmem fused_smem(int N, int D, int rows_per) {
  FusedSmem f;
  size_t o = 0;
  f.v = o;  o = round16(o + (size_t)(N * D + ((N + 31) >> 5) * (D >= 4 ? 4 : D)) * sizeof(float));  // v_j, padded
  f.b = o;  o = round16(o + (size_t)(N + ((N + 31) >> 5)) * sizeof(float));                         // beta_j, padded
  f.l = o;  o = round16(o + (size_t)N * sizeof(float));              // l_i        [N]
  f.c = o;  o = round16(o + (size_t)N * sizeof(unsigned long long)); // prefix sums [N]
  f.u = o;  o = round16(o + (size_t)rows_per * D * sizeof(float));   // own u_i    [R][D]
  f.al = o; o = round16(o + (size_t)rows_per * sizeof(float));       // own alpha_i
  f.sh = o; o = round16(o + (size_t)rows_per * sizeof(float));       // own row offsets g_i
  f.total = o;
  return f;
}

template <int D>
__global__ void __launch_bounds__(fused_threads<D>(), 1) level_fused_kernel(MergeArgs a, ModelParams<D> mp,
                                                                         int C) {
  constexpr int NT = fused_threads<D>();
  constexpr int NW = NT / 32;
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  const int s = blockIdx.x / C;           // combination within this launch
  const Comb cb = comb_of(a, s);
  const int gid = cb.gid, K = cb.K;
  const int at = cb.at, c = cb.c, b = cb.b;
  const int N = a.N, d = a.d, B = a.B, nT = a.nT, nTp = a.nTp;
  const bool left_leaf = (cb.level == 0);
  const int sR = b - c + 1;
  const bool right_leaf = (sR == 1);
  const int bufL = cb.level & 1, bufR = ceil_log2(sR) & 1, bufO = (cb.level + 1) & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rows_per = (N + C - 1) / C;
  const int lo = min(r * rows_per, N), hi = min(lo + rows_per, N);

  extern __shared__ __align__(16) unsigned char smraw[];
  const FusedSmem L = fused_smem(N, D, rows_per);
  float* sV = reinterpret_cast<float*>(smraw + L.v);
  float* sB = reinterpret_cast<float*>(smraw + L.b);
  float* sL = reinterpret_cast<float*>(smraw + L.l);
  unsigned long long* sC = reinterpret_cast<unsigned long long*>(smraw + L.c);
  float* sU = reinterpret_cast<float*>(smraw + L.u);
  float* sAl = reinterpret_cast<float*>(smraw + L.al);
  float* sG = reinterpret_cast<float*>(smraw + L.sh);  // the own rows' offsets g_i (row_offset)
  int* under = reinterpret_cast<int*>(sC);  // own rows that underflowed (before the CDF)

  __shared__ float gsum[kMaxColumnGroups * D];
  __shared__ float red_s[NW];
  __shared__ float mu_s[D];
  __shared__ float bstar_s;
  __shared__ unsigned long long warp_tot[NW];
  __shared__ float redf[NW];
  __shared__ float M_s;
  __shared__ int n_under, nonfinite_s;
  if (threadIdx.x == 0) {
    n_under = 0;
    nonfinite_s = 0;
  }

  float* V = a.ws.V + (size_t)s * N * D;
  float* beta = a.ws.beta + (size_t)s * N;
  float* U = a.ws.U + (size_t)s * N * D;
  float* alpha = a.ws.alpha + (size_t)s * N;
  double* shift = a.ws.shift + (size_t)s * N;
  float* Tt = a.ws.T + (size_t)s * N * nTp;
  float* delta = a.ws.delta + (size_t)s * N;
  const int32_t* firstR = right_leaf ? nullptr : cb.first + ((size_t)bufR * K + c) * N;
  const int32_t* lastL = left_leaf ? nullptr : cb.last + ((size_t)bufL * K + at) * N;
  const float* Xc = cb.X + (size_t)c * N * d;
  const float* Xl = cb.X + (size_t)(c - 1) * N * d;
  const float* lwc = right_leaf ? cb.logw + (size_t)c * N : nullptr;
  const float* lwl = left_leaf ? cb.logw + (size_t)(c - 1) * N : nullptr;

  // ---------------------------------------------------------------- columns (all N)
  float yc[D], qm[D], qs[D];
#pragma unroll
  for (int k = 0; k < D; ++k) yc[k] = k < d ? cb.y[(size_t)c * d + k] : 0.f;
  proposal_at<D>(mp, cb.y, cb.prop_mean, cb.prop_std, c, qm, qs);
  float qinv[D];
  const float qnorm = proposal_consts<D>(d, qs, qinv);
  bool bad = false, corrupt = false;
  float mu[D], bstar;
  column_pass<D>(N, gsum, red_s, mu_s, &bstar_s, mu, bstar, bad, [&](int j, float* x) {
    const float bp = column_bprime<D>(mp, N, d, a.logN, yc, qm, qinv, qnorm, Xc, firstR, lwc, j, x, corrupt);
#pragma unroll
    for (int k = 0; k < D; ++k) sV[vidx<D, true>(j) + k] = x[k];
    sB[bidx<true>(j)] = bp;
    return bp;
  });
  for (int j = threadIdx.x; j < N; j += NT) {
    float v[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = sV[vidx<D, true>(j) + k];
    const float bj = column_beta<D>(mp, v, mu, sB[bidx<true>(j)], bstar);
#pragma unroll
    for (int k = 0; k < D; ++k) sV[vidx<D, true>(j) + k] = v[k];
    sB[bidx<true>(j)] = bj;
    if (j >= lo && j < hi) {  // CTA r publishes its share of the column terms
#pragma unroll
      for (int k = 0; k < D; ++k) V[(size_t)j * D + k] = v[k];
      beta[j] = bj;
    }
  }

  __syncthreads();  // the column terms are in shared memory: the rows read a sample of them
  // ---------------------------------------------------------------- own rows
  const double base_m = shift_base(-a.logN, mp.log_f_max, bstar);  // a merged left block's
  for (int i = lo + threadIdx.x; i < hi; i += NT) {
    float ul[D], ai;
    const float al0 = row_terms<D>(mp, N, d, a.logN, Xl, lastL, lwl, i, mu, ul, ai, corrupt);
    const float dl = row_shift<D, true>(ul, al0, sV, sB, N);
    const float al = __fsub_rn(al0, dl);
    bad |= isnan(ai);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      U[(size_t)i * D + k] = ul[k];
      sU[(size_t)(i - lo) * D + k] = ul[k];
    }
    alpha[i] = al;
    sAl[i - lo] = al;
    const double sh = row_shift_total(lwl != nullptr ? shift_base(ai, mp.log_f_max, bstar) : base_m, dl);
    shift[i] = sh;
    sG[i - lo] = row_offset(left_leaf, ai, dl);
  }
  // column / row errors are recorded before any row CDF of the cluster can report a
  // degenerate combination (the split path's order)
  if (corrupt) record_status(a.ws.status, DSMC_ERR_INVALID_ARG);
  if (bad) record_status(a.ws.status, DSMC_ERR_NONFINITE);
  if (r == 0) {  // the matrix bound log omega-bar (read by the inspection entry point)
    float amax = -INFINITY;
    for (int i = threadIdx.x; i < N; i += NT)
      amax = fmaxf(amax, left_leaf ? cb.logw[(size_t)(c - 1) * N + i] : -a.logN);
    amax = warp_max(amax);
    __syncthreads();
    if (lane == 0) red_s[warp] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = red_s[0];
      for (int w = 1; w < NW; ++w) t = fmaxf(t, red_s[w]);
      a.ws.logbar[s] = (double)mp.log_f_max + (double)t + (double)bstar;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- own tile weights
  // unit = (tile k, row group g): rows lo + g + G r (r < R) of one tile, G = ceil(nrow / R);
  // consecutive threads take consecutive groups of the same tile, so the column terms are
  // shared-memory broadcasts, each loaded once for R rows.  Sequential sums over the tile's
  // columns.
  {
    constexpr int R = D <= 8 ? 4 : 2;
    const int nrow = hi - lo;
    const int G = (nrow + R - 1) / R;
    for (int q = threadIdx.x; q < G * nT; q += NT) {
      const int k = q / G, g = q - k * G;
      float u[R][D], al[R], ts[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int il = g + G * rr;
        const bool ok = il < nrow;
#pragma unroll
        for (int e = 0; e < D; ++e) u[rr][e] = ok ? sU[(size_t)il * D + e] : 0.f;
        al[rr] = ok ? sAl[il] : -INFINITY;
        ts[rr] = 0.f;
      }
      const int jb = k * B, je = min(jb + B, N);
      int j = jb;
      for (; j + 4 <= je; j += 4) {
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          float v[D];
          load_row<D>(sV + vidx<D, true>(j + qq), v);
          const float bj = sB[bidx<true>(j + qq)];
#pragma unroll
          for (int rr = 0; rr < R; ++rr) ts[rr] = __fadd_rn(ts[rr], ex2(pair_exponent<D>(u[rr], al[rr], v, bj)));
        }
      }
      for (; j < je; ++j) {
        float v[D];
        load_row<D>(sV + vidx<D, true>(j), v);
        const float bj = sB[bidx<true>(j)];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) ts[rr] = __fadd_rn(ts[rr], ex2(pair_exponent<D>(u[rr], al[rr], v, bj)));
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const int il = g + G * rr;
        if (il < nrow) Tt[(size_t)(lo + il) * nTp + k] = ts[rr];
      }
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- own row totals
  float* rowsum = a.ws.rowsum + (size_t)s * N;
  for (int i = lo + threadIdx.x; i < hi; i += NT) {
    float t = row_total(Tt + (size_t)i * nTp, nT, nTp);
    if (isnan(t)) {
      nonfinite_s = 1;
      t = 0.f;
    }
    sL[i] = t;
    delta[i] = 0.f;
    if (t < 0x1p-64f) under[atomicAdd(&n_under, 1)] = i;
  }
  __syncthreads();
  for (int q = warp; q < n_under; q += NW) {
    const int i = under[q];
    float si, dl;
    recompute_row<D, true>(sU + (size_t)(i - lo) * D, sAl[i - lo], sV, sB, N, B, nT, Tt + (size_t)i * nTp, &si,
                           &dl);
    __syncwarp();
    if (lane == 0) {
      si = row_total(Tt + (size_t)i * nTp, nT, nTp);
      sL[i] = isnan(si) ? 0.f : si;
      delta[i] = dl;
    }
  }
  __syncthreads();
  for (int i = lo + threadIdx.x; i < hi; i += NT) {
    const float t = sL[i];
    rowsum[i] = t;
    sL[i] = row_log2_weight(sG[i - lo], delta[i], t);
  }

  // ---------------------------------------------------------------- exchange l_i
  __threadfence();  // U, alpha, delta, V, beta, T of this CTA's share, for the slot draws
  cluster.sync();
  for (int i = threadIdx.x; i < N; i += NT) {
    const int owner = i / rows_per;
    if (owner != r) sL[i] = *cluster.map_shared_rank(sL + i, owner);
  }
  __syncthreads();

  // ---------------------------------------------------------------- row CDF (every CTA)
  float mloc = -INFINITY;
  for (int i = threadIdx.x; i < N; i += NT) mloc = fmaxf(mloc, sL[i]);
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
    const float rr = row_weight(sL[i], M, degenerate);
    if (i >= lo && i < hi) rw[i] = rr;
    sC[i] = (unsigned long long)__float2ull_rz(rr * 0x1p40f);
  }
  __syncthreads();
  block_scan_u64(sC, N, warp_tot);
  unsigned long long* gcum = a.ws.cum + (size_t)s * N;
  for (int i = lo + threadIdx.x; i < hi; i += NT) gcum[i] = sC[i];
  if (r == 0 && threadIdx.x == 0) {
    const double inc = degenerate ? (double)NAN
                                  : lab_increment(comb_base(left_leaf, a.logN, mp.log_f_max, bstar), M,
                                                  log_fixed_total(sC[N - 1]));
    a.ws.inc[s] = inc;
    cb.logL[at] = cb.logL[at] + cb.logL[c] + inc;
    if (degenerate || sC[N - 1] == 0ull) record_status(a.ws.status, DSMC_ERR_DEGENERATE);
  }
  if (threadIdx.x == 0 && nonfinite_s) record_status(a.ws.status, DSMC_ERR_NONFINITE);

  // ---------------------------------------------------------------- this CTA's slots
  int32_t* pl = cb.pairs + (size_t)gid * 2 * N;
  int32_t* pr = pl + N;
  const int n_lo = cb.conditional ? 1 : 0;
  const int n_hi = N + ((cb.conditional && cb.root) ? 1 : 0);
  int32_t* first_out = cb.first + ((size_t)bufO * K + at) * N;
  int32_t* last_out = cb.last + ((size_t)bufO * K + at) * N;
  const int32_t* first_L = cb.first + ((size_t)bufL * K + at) * N;
  const int32_t* last_R = cb.last + ((size_t)bufR * K + c) * N;
  if (cb.conditional && r == 0 && threadIdx.x == 0) {
    pl[0] = 0;
    pr[0] = 0;
    first_out[0] = left_leaf ? 0 : first_L[0];
    last_out[0] = right_leaf ? 0 : last_R[0];
  }
  DrawIn in;
  in.sys = (a.resampler == DSMC_SYSTEMATIC && !cb.conditional) ? 1 : 0;
  in.cum = sC;
  in.T = Tt;
  in.U = U;
  in.alpha = alpha;
  in.delta = delta;
  in.V = sV;
  in.beta = sB;
  in.N = N;
  in.B = B;
  in.nT = nT;
  in.nTp = nTp;
  const int per = (n_hi - n_lo + C - 1) / C;
  const int n0 = min(n_hi, n_lo + r * per), n1 = min(n_hi, n0 + per);
  for (int n = n0 + threadIdx.x; n < n1; n += NT) {
    int i, j;
    draw_pair<D, true>(in, cb.seed, cb.base, gid, n, i, j);
    if (n < N) {
      pl[n] = i;
      pr[n] = j;
      first_out[n] = left_leaf ? i : first_L[i];
      last_out[n] = right_leaf ? j : last_R[j];
    } else {
      cb.star[0] = i;
      cb.star[1] = j;
    }
  }
  // peers may still be reading this CTA's l_i
  cluster.sync();
}

template <int D>
cudaLaunchConfig_t fused_config(const MergeArgs& a, int C, cudaStream_t st, cudaLaunchAttribute* attr,
                                size_t* smem_out) {
  const int rows_per = (a.N + C - 1) / C;
  const size_t smem = fused_smem(a.N, D, rows_per).total;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.mc * C), 1, 1);
  cfg.blockDim = dim3(fused_threads<D>(), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  *smem_out = smem;
  return cfg;
}

template <int D>
cudaError_t fused_attributes(size_t smem, int C) {
  cudaError_t e = cudaFuncSetAttribute(level_fused_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && C > 8)
    e = cudaFuncSetAttribute(level_fused_kernel<D>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <int D>
cudaError_t fused_t(const MergeArgs& a, const void* mp, int C, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  size_t smem = 0;
  const cudaLaunchConfig_t cfg = fused_config<D>(a, C, st, attr, &smem);
  cudaError_t e = fused_attributes<D>(smem, C);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, level_fused_kernel<D>, a, *static_cast<const ModelParams<D>*>(mp), C);
}

template <int D>
cudaError_t fused_max_clusters(const MergeArgs& a, int C, int* n) {
  cudaLaunchAttribute attr[1];
  size_t smem = 0;
  MergeArgs one = a;
  one.mc = 1;
  const cudaLaunchConfig_t cfg = fused_config<D>(one, C, 0, attr, &smem);
  cudaError_t e = fused_attributes<D>(smem, C);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveClusters(n, level_fused_kernel<D>, &cfg);
}

}  // namespace

size_t fused_level_smem(int D, int N, int C) {
  return fused_smem(N, D, (N + C - 1) / C).total;
}

#define DSMC_DISPATCH_F(D, CALL)                      \
  switch (D) {                                        \
    case 1: { constexpr int DD = 1; return CALL; }    \
    case 2: { constexpr int DD = 2; return CALL; }    \
    case 4: { constexpr int DD = 4; return CALL; }    \
    case 8: { constexpr int DD = 8; return CALL; }    \
    case 16: { constexpr int DD = 16; return CALL; }  \
    case 32: { constexpr int DD = 32; return CALL; }  \
  }                                                   \
  return cudaErrorInvalidValue;

cudaError_t launch_level_fused(int D, const MergeArgs& a, const void* mp, int C, cudaStream_t s) {
  DSMC_DISPATCH_F(D, fused_t<DD>(a, mp, C, s))
}

cudaError_t level_fused_max_clusters(int D, const MergeArgs& a, int C, int* n) {
  DSMC_DISPATCH_F(D, fused_max_clusters<DD>(a, C, n))
}

}  // namespace dsmc
