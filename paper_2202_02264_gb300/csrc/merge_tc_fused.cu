// merge_tc_fused.cu -- one level of Algorithm 6 for the dense samplers (Algorithm 1, its
// systematic option and Algorithm 5) with the tensor-core cross term, every stage of a
// combination in one persistent, warp-specialised kernel: no operand, tile sum or row
// weight of a combination leaves the SM (only the pairs, the new block's index maps and
// log L are written).
//
// One CTA per SM walks the combinations s = blockIdx.x, blockIdx.x + gridDim.x, ... of the
// launch.  Each combination's data lives in one of two shared-memory stages:
//   - 11 core warps alternate, for k = 0, 1, ...: the draws of combination k (every slot's
//     pair in three exact inverse-CDF stages over the row CDF the epilogue built, and the
//     new block's index maps), then the operand build of combination k + 2 into the stage k
//     released (its inputs -- two particle slices and two leaf-weight or index-map rows --
//     brought into their own buffer by bulk copies issued after the build before it; the
//     column pass -- states, b'_j, mu, B*, v_j, beta_j -- and the row pass -- u_i, alpha_i,
//     the row offsets -- as FP32 copies for the draws and as the BF16 / TF32 MMA rows [u,
//     alpha_hi, alpha_lo, 1, 1] and [v, 1, 1, beta_hi, beta_lo] in the canonical K-major
//     layout).  The next build's descriptor and observation / proposal rows are read during
//     a build by the last core warp, in the second rounds it has no work in;
//   - 1 control thread issues, for combination k + 1, one tcgen05.mma (M = N = 128) per (row
//     tile, column block) into one of four 128-column TMEM accumulators;
//   - 8 epilogue warps read each accumulator (tcgen05.ld; warp (g, h) lanes 32 g.. and
//     columns 64 h..), take 2^x on MUFU and keep the tile sums in shared memory, then build
//     the combination's row CDF (row totals, row log weights, their exact 2^40 fixed-point
//     prefix sums) before releasing its draws, and add the increment of Eq. (Lab) to log L.
// So the exponentials of one combination overlap the draws and the operand build of two
// others, and the period of a combination is the larger of the two.
// The arithmetic is the split path's, function for function (the column and row terms of
// merge_parts.cuh, the operand packing and epilogue sums of tc_ops.cuh, draw_pair), and the
// column mean is reduced in the same block-size-independent order, so the pairs, maps and
// log L equal the split path's bit for bit.
//
// Every wait is bounded and abort-aware: a role whose wait runs out records
// DSMC_ERR_TIMEOUT and raises the CTA's abort flag; the other roles stop at their next wait,
// the core warps wait (bounded) for their bulk copies in flight, the control thread for its
// last committed MMA, and the CTA frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "merge_parts.cuh"
#include "tc_ops.cuh"

namespace dsmc {

namespace {

using namespace parts;
using namespace tc;

constexpr int kFNmax = 512;                 // largest N of the fused level
#ifndef DSMC_FUSED_EPI_WARPS
#define DSMC_FUSED_EPI_WARPS 8
#endif
constexpr int kFEpiWarps = DSMC_FUSED_EPI_WARPS;  // lane quarter warp % 4, kFEpiCols columns each
static_assert(kFEpiWarps == 4 || kFEpiWarps == 8, "4 or 8 epilogue warps");
constexpr int kFEpiCols = 4 * 128 / kFEpiWarps;   // columns of a block per epilogue warp (64 or 128)
// operand build and draws: the rest of 20 warps (at most 5 per scheduler: 96 registers)
constexpr int kFCoreWarps = 19 - kFEpiWarps;
constexpr int kFCtrlWarp = kFEpiWarps + kFCoreWarps;  // TMEM and MMA issue
constexpr int kFThreads = (kFCtrlWarp + 1) * 32;
constexpr int kFCoreThreads = kFCoreWarps * 32;
constexpr int kFCore0 = kFEpiWarps * 32;
constexpr int kFAcc = 4;                    // TMEM accumulators of 128 columns
constexpr uint32_t kFTmemCols = kFAcc * kMmaN;
constexpr int kBarCore = 1;                 // named barrier of the core warps
constexpr int kBarEpi = 2;                  // named barrier of the epilogue warps
constexpr int kFTileBytes = kMmaM * 32;     // one 128-row tile of one 32-byte K plane
constexpr int kFTiles = kFNmax / 32;        // tiles of 32 columns per row (tile width 32)
// Row stride (floats) of the stage's tile sums: 18, not 16, so that the rows of a warp fall
// on different banks (the epilogue stores 32 consecutive rows, the draws read random rows).
constexpr int kFTs = kFTiles + 2;

__host__ __device__ constexpr size_t rnd(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte offsets inside one stage (one combination's data, N <= 512):
//   opU, opV  the MMA row and column operands, [512][32 B] each, canonical K-major layout
//   fV, fB    v_j [N][D] and beta_j, padded after every 32 columns (FP32)
//   fU        u_i [N][D];  fAl alpha_i;  fDl delta_i;  fG the row offsets g_i (row_offset)
//   T         tile weights [N][kFTs] (16 tiles and a 2-float pad per row)
//   cum       exact prefix sums of the row weights (u64);  fL the row log weights
template <int D>
struct Stage {
  static constexpr size_t opU = 0;
  static constexpr size_t opV = opU + (size_t)kFNmax * 32;
  static constexpr size_t fV = opV + (size_t)kFNmax * 32;
  static constexpr size_t fB = fV + rnd((size_t)(kFNmax * D + (kFNmax / 32) * kVPad<D>) * 4, 16);
  static constexpr size_t fU = fB + rnd((size_t)(kFNmax + kFNmax / 32) * 4, 16);
  static constexpr size_t fAl = fU + (size_t)kFNmax * D * 4;
  static constexpr size_t fDl = fAl + (size_t)kFNmax * 4;
  static constexpr size_t fG = fDl + (size_t)kFNmax * 4;
  static constexpr size_t T = fG + (size_t)kFNmax * 4;
  static constexpr size_t cum = T + (size_t)kFNmax * kFTs * 4;
  static constexpr size_t fL = cum + (size_t)kFNmax * 8;
  static constexpr size_t bytes = rnd(fL + (size_t)kFNmax * 4, 1024);
};

// The inputs of the next operand build (its two particle slices and the leaf weights or
// index maps beside them), brought in by bulk copies while the previous combination draws.
struct Inputs {
  static constexpr size_t xc = 0;                          // X_c      [N][d] FP32
  static constexpr size_t xl = xc + (size_t)kFNmax * 4 * 4;  // X_{c-1}  [N][d] FP32
  static constexpr size_t r0 = xl + (size_t)kFNmax * 4 * 4;  // log w_c or first map [N]
  static constexpr size_t l0 = r0 + (size_t)kFNmax * 4;      // log w_{c-1} or last map [N]
  static constexpr size_t bytes = l0 + (size_t)kFNmax * 4;
};

template <int D>
__host__ __device__ constexpr size_t fused_tc_smem() {
  return 2 * Stage<D>::bytes + Inputs::bytes + 1024;  // two stages, the inputs, alignment slack
}

__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier over n threads that also ANDs a predicate across them.
__device__ __forceinline__ bool bar_and(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// n 32-bit words from global to shared memory by a group of nt threads (vector loads when
// both ends are 16-byte aligned).
template <typename T>
__device__ __forceinline__ void stage_group(T* dst, const T* src, int n, int tid, int nt) {
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const int n4 = n >> 2;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (int t = tid; t < n4; t += nt) d4[t] = __ldg(s4 + t);
    for (int t = 4 * n4 + tid; t < n; t += nt) dst[t] = __ldg(src + t);
  } else {
    for (int t = tid; t < n; t += nt) dst[t] = __ldg(src + t);
  }
}

// Shared scratch of the core warps.
struct CoreScratch {
  float gsum[kMaxColumnGroups * 4];
  float red[kFCoreWarps];
  float mu[4];
  float bstar;
  // the descriptor of a build's combination and its observation and proposal rows, read one
  // build ahead (double-buffered by the parity of the build: build m reads slot m & 1 while
  // the next one's is written)
  Comb nx_cb[2];
  float nx_yc[2][4], nx_qm[2][4], nx_qs[2][4];
  int in_bulk;    // the next build's inputs come by bulk copy (1) or are staged by it (0)
  int in_pend;    // bulk copies issued and not yet waited for
  int in_phase;   // completed phases of the inputs barrier
};

// Global sources of combination s's build inputs.
struct InputSrc {
  const float *xc, *xl;
  const void *r0, *l0;
  uint32_t bx, bw;  // bytes of a slice, of a weight / map row
};

__device__ __forceinline__ InputSrc input_src(const MergeArgs& a, const Comb& cb) {
  const int N = a.N, d = a.d, c = cb.c, sR = cb.b - cb.c + 1;
  InputSrc r;
  r.xc = cb.X + (size_t)c * N * d;
  r.xl = cb.X + (size_t)(c - 1) * N * d;
  r.r0 = sR == 1 ? static_cast<const void*>(cb.logw + (size_t)c * N)
                 : static_cast<const void*>(cb.first + ((size_t)(ceil_log2(sR) & 1) * cb.K + c) * N);
  r.l0 = cb.level == 0 ? static_cast<const void*>(cb.logw + (size_t)(c - 1) * N)
                       : static_cast<const void*>(cb.last + ((size_t)(cb.level & 1) * cb.K + cb.at) * N);
  r.bx = (uint32_t)(N * d * 4);
  r.bw = (uint32_t)(N * 4);
  return r;
}

// One thread: the bulk copies of combination cb's inputs into `inb`, completing on `bar`,
// when every source and size is 16-byte aligned (true when N is a multiple of 4 and d
// divides evenly); otherwise nothing is issued and the build stages them itself.
__device__ __forceinline__ bool issue_inputs(const MergeArgs& a, const Comb& cb, unsigned char* inb, uint32_t bar) {
  const InputSrc r = input_src(a, cb);
  const uintptr_t al = reinterpret_cast<uintptr_t>(r.xc) | reinterpret_cast<uintptr_t>(r.xl) |
                       reinterpret_cast<uintptr_t>(r.r0) | reinterpret_cast<uintptr_t>(r.l0) | r.bx | r.bw;
  if ((al & 15) != 0) return false;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * r.bx + 2 * r.bw)
               : "memory");
  const void* src[4] = {r.xc, r.xl, r.r0, r.l0};
  const size_t off[4] = {Inputs::xc, Inputs::xl, Inputs::r0, Inputs::l0};
  const uint32_t len[4] = {r.bx, r.bx, r.bw, r.bw};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(inb + off[q])),
                 "l"(src[q]), "r"(len[q]), "r"(bar)
                 : "memory");
  return true;
}

// The observation row and proposal row of the descriptor in scratch slot q (one thread).
template <int D>
__device__ __forceinline__ void read_rows(const MergeArgs& a, const ModelParams<D>& mp, CoreScratch& sc, int q) {
  const Comb& cb = sc.nx_cb[q];
  float qm[D], qs[D];
  proposal_at<D>(mp, cb.y, cb.prop_mean, cb.prop_std, cb.c, qm, qs);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    sc.nx_yc[q][kk] = kk < D && kk < a.d ? cb.y[(size_t)cb.c * a.d + kk] : 0.f;
    sc.nx_qm[q][kk] = kk < D ? qm[kk] : 0.f;
    sc.nx_qs[q][kk] = kk < D ? qs[kk] : 1.f;
  }
}

// Operand build of combination s into stage st (the core warps): the two particle slices and
// index maps staged with vector loads, the column pass (states, b'_j, mu, B*, v_j, beta_j),
// the row pass (u_i, alpha_i, the row shift), FP32 copies for the draws and the MMA rows.
template <int D, int KIND>
__device__ __forceinline__ void core_load(const MergeArgs& a, const ModelParams<D>& mp, unsigned char* st, int s,
                                          unsigned char* inb, int ct, int cw, int lane, int RT, CoreScratch& sc,
                                          Comb* cb_stage, double* cbase_stage, int par, int s_next) {
  using L = Stage<D>;
  const int N = a.N, d = a.d;
  unsigned char* opU = st + L::opU;
  unsigned char* opV = st + L::opV;
  float* fV = reinterpret_cast<float*>(st + L::fV);
  float* fB = reinterpret_cast<float*>(st + L::fB);
  float* fU = reinterpret_cast<float*>(st + L::fU);
  float* fAl = reinterpret_cast<float*>(st + L::fAl);
  float* fDl = reinterpret_cast<float*>(st + L::fDl);
  float* fG = reinterpret_cast<float*>(st + L::fG);
  const Comb cb = sc.nx_cb[par];  // read one build ahead
  if (ct == 0) *cb_stage = cb;  // for the draws of this stage
  const int at = cb.at, c = cb.c, b = cb.b, K = cb.K;
  const bool left_leaf = (cb.level == 0);
  const int sR = b - c + 1;
  const bool right_leaf = (sR == 1);
  const int bufL = cb.level & 1, bufR = ceil_log2(sR) & 1;
  // the inputs: bulk-copied beforehand, or staged here with vector loads
  float* sXc = reinterpret_cast<float*>(inb + Inputs::xc);
  float* sXl = reinterpret_cast<float*>(inb + Inputs::xl);
  float* sR0 = reinterpret_cast<float*>(inb + Inputs::r0);
  float* sL0 = reinterpret_cast<float*>(inb + Inputs::l0);
  if (!sc.in_bulk) {
    stage_group(sXc, cb.X + (size_t)c * N * d, N * d, ct, kFCoreThreads);
    stage_group(sXl, cb.X + (size_t)(c - 1) * N * d, N * d, ct, kFCoreThreads);
    if (right_leaf)
      stage_group(sR0, cb.logw + (size_t)c * N, N, ct, kFCoreThreads);
    else
      stage_group(reinterpret_cast<int32_t*>(sR0), cb.first + ((size_t)bufR * K + c) * N, N, ct, kFCoreThreads);
    if (left_leaf)
      stage_group(sL0, cb.logw + (size_t)(c - 1) * N, N, ct, kFCoreThreads);
    else
      stage_group(reinterpret_cast<int32_t*>(sL0), cb.last + ((size_t)bufL * K + at) * N, N, ct, kFCoreThreads);
  }
  const int32_t* firstR = right_leaf ? nullptr : reinterpret_cast<const int32_t*>(sR0);
  const float* lwc = right_leaf ? sR0 : nullptr;
  const int32_t* lastL = left_leaf ? nullptr : reinterpret_cast<const int32_t*>(sL0);
  const float* lwl = left_leaf ? sL0 : nullptr;
  float yc[D], qm[D], qs[D], qinv[D];
#pragma unroll
  for (int kk = 0; kk < D; ++kk) {
    yc[kk] = sc.nx_yc[par][kk];
    qm[kk] = sc.nx_qm[par][kk];
    qs[kk] = sc.nx_qs[par][kk];
  }
  const float qnorm = proposal_consts<D>(d, qs, qinv);
  if (!sc.in_bulk) bar_sync(kBarCore, kFCoreThreads);  // the inputs it staged (bulk ones were waited for)
  // The last core warp has one group of the column pass and one row of the row pass, the
  // others up to two: in those idle second rounds one of its threads reads the next build's
  // descriptor, then its observation and proposal rows (dependent global round trips, off
  // the critical path), into the other scratch slot.
  const bool prefetcher = s_next >= 0 && cw == kFCoreWarps - 1 && lane == 0;

  // column pass: b'_j, states, the column mean mu (groups of 32 Q columns, each summed by
  // one warp lane-sequentially then by a butterfly, group sums in group order: the same
  // order as every other column pass) and B* = max_j b'_j
  bool bad = false, corrupt = false;
  float mu[D], bstar;
  {
    const int Qg = (N + 1023) / 1024, Wd = 32 * Qg;
    const int G = (N + Wd - 1) / Wd;
    float bmax = -INFINITY;
    for (int gg = cw; gg < G; gg += kFCoreWarps) {
      float accs[D];
#pragma unroll
      for (int kk = 0; kk < D; ++kk) accs[kk] = 0.f;
      for (int cc = 0; cc < Qg; ++cc) {
        const int j = Wd * gg + 32 * cc + lane;
        if (j < N) {
          float x[D];
          const float bp = column_bprime<D>(mp, N, d, a.logN, yc, qm, qinv, qnorm, sXc, firstR, lwc, j, x, corrupt);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) fV[vidx<D, true>(j) + kk] = x[kk];
          fB[bidx<true>(j)] = bp;
          bad |= isnan(bp);
          bmax = fmaxf(bmax, bp);
#pragma unroll
          for (int kk = 0; kk < D; ++kk) accs[kk] += x[kk];
        }
      }
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        const float t = warp_sum(accs[kk]);
        if (lane == 0) sc.gsum[gg * D + kk] = t;
      }
    }
    if (prefetcher) sc.nx_cb[par ^ 1] = comb_of(a, s_next);
    bmax = warp_max(bmax);
    if (lane == 0) sc.red[cw] = bmax;
    bar_sync(kBarCore, kFCoreThreads);
    if (ct < D) {  // G <= kFNmax / 32 groups: the loads first, then the sum in group order
      float gs[kFNmax / 32];
#pragma unroll
      for (int gg = 0; gg < kFNmax / 32; ++gg) gs[gg] = gg < G ? sc.gsum[gg * D + ct] : 0.f;
      float t = 0.f;
#pragma unroll
      for (int gg = 0; gg < kFNmax / 32; ++gg)
        if (gg < G) t += gs[gg];
      sc.mu[ct] = t / (float)N;
    }
    if (ct == 0) {
      float t = sc.red[0];
      for (int w = 1; w < kFCoreWarps; ++w) t = fmaxf(t, sc.red[w]);
      sc.bstar = t;
    }
    bar_sync(kBarCore, kFCoreThreads);
#pragma unroll
    for (int kk = 0; kk < D; ++kk) mu[kk] = sc.mu[kk];
    bstar = sc.bstar;
  }
  // columns: v_j = x_j - mu, beta_j, the MMA column rows [v, 1, 1, beta_hi, beta_lo]
  for (int j = ct; j < N; j += kFCoreThreads) {
    float v[D];
#pragma unroll
    for (int kk = 0; kk < D; ++kk) v[kk] = fV[vidx<D, true>(j) + kk];
    const float bj = column_beta<D>(mp, v, mu, fB[bidx<true>(j)], bstar);
#pragma unroll
    for (int kk = 0; kk < D; ++kk) fV[vidx<D, true>(j) + kk] = v[kk];
    fB[bidx<true>(j)] = bj;
    float ext[4];
    ext[0] = 1.f;
    ext[1] = 1.f;
    split_mma(bj, KIND, &ext[2], &ext[3]);
    store_mma_row_t<D, KIND>(opV, kFNmax, j, v, ext);
    if (a.inspect) {
#pragma unroll
      for (int kk = 0; kk < D; ++kk) a.ws.V[((size_t)s * N + j) * D + kk] = v[kk];
      a.ws.beta[(size_t)s * N + j] = bj;
    }
  }
  {  // rows and columns past N within the last tile are zero
    const float zero[D] = {};
    const float zext[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j = N + ct; j < RT * kMmaM; j += kFCoreThreads) {
      store_mma_row_t<D, KIND>(opV, kFNmax, j, zero, zext);
      store_mma_row_t<D, KIND>(opU, kFNmax, j, zero, zext);
    }
  }
  bar_sync(kBarCore, kFCoreThreads);  // the rows read a sample of the columns
  // rows: u_i, alpha_i (less the row shift delta_i, which moves into shift_i), and the MMA
  // row [u, alpha_hi, alpha_lo, 1, 1]
  if (ct == 0) *cbase_stage = comb_base(left_leaf, a.logN, mp.log_f_max, bstar);
  for (int i = ct; i < N; i += kFCoreThreads) {
    float ul[D], ai;
    const float al0 = row_terms<D>(mp, N, d, a.logN, sXl, lastL, lwl, i, mu, ul, ai, corrupt);
    const float dl = row_shift<D, true>(ul, al0, fV, fB, N);
    const float al = __fsub_rn(al0, dl);
    bad |= isnan(ai);
#pragma unroll
    for (int kk = 0; kk < D; ++kk) fU[(size_t)i * D + kk] = ul[kk];
    fAl[i] = al;
    fDl[i] = 0.f;
    fG[i] = row_offset(left_leaf, ai, dl);
    float ext[4];
    split_mma(al, KIND, &ext[0], &ext[1]);
    ext[2] = 1.f;
    ext[3] = 1.f;
    store_mma_row_t<D, KIND>(opU, kFNmax, i, ul, ext);
    if (a.inspect) {
#pragma unroll
      for (int kk = 0; kk < D; ++kk) a.ws.U[((size_t)s * N + i) * D + kk] = ul[kk];
      a.ws.alpha[(size_t)s * N + i] = al;
      a.ws.shift[(size_t)s * N + i] =
          row_shift_total(shift_base(lwl != nullptr ? ai : -a.logN, mp.log_f_max, bstar), dl);
    }
  }
  if (prefetcher) read_rows<D>(a, mp, sc, par ^ 1);
  if (corrupt) record_status(a.ws.status, DSMC_ERR_INVALID_ARG);
  if (bad) record_status(a.ws.status, DSMC_ERR_NONFINITE);
  fence_proxy_async();  // the operand rows, written by these threads, feed the tensor core
  bar_sync(kBarCore, kFCoreThreads);
}

// Shared scratch of the epilogue warps' row CDF.
struct EpiScratch {
  float red[kFEpiWarps];
  unsigned long long rowtot[kFNmax / 32];
  unsigned long long S;  // the row weights' exact fixed-point total
  float M;               // their base-2 maximum
  int n_under, nonfinite, degenerate;
};

// Row CDF of combination s in stage st, by the epilogue warps once its tile sums are
// complete (et = thread among them, ew = warp): the row totals (row_total's definition, from
// the two halves the epilogue accumulated), the row log weights, a row whose total
// underflows recomputed with its exact maximum, the row weights r_i = 2^(l_i - M) as exact
// 2^40 fixed-point images and their inclusive prefix sums (16 rows of 32, one shuffle scan
// per row, the rows' totals carried), then the increment of Eq. (Lab) and log L.
template <int D>
__device__ __forceinline__ void epi_row_cdf(const MergeArgs& a, unsigned char* st, int s, int et, int ew, int lane,
                                            EpiScratch& se) {
  using L = Stage<D>;
  constexpr int NT = kFEpiWarps * 32;
  const int N = a.N, nT = a.nT, nTp = a.nTp;  // nTp: the workspace's row stride (inspection)
  float* fV = reinterpret_cast<float*>(st + L::fV);
  float* fB = reinterpret_cast<float*>(st + L::fB);
  float* fU = reinterpret_cast<float*>(st + L::fU);
  float* fAl = reinterpret_cast<float*>(st + L::fAl);
  float* fDl = reinterpret_cast<float*>(st + L::fDl);
  const float* fG = reinterpret_cast<const float*>(st + L::fG);
  float* Tq = reinterpret_cast<float*>(st + L::T);
  unsigned long long* cum = reinterpret_cast<unsigned long long*>(st + L::cum);
  float* fL = reinterpret_cast<float*>(st + L::fL);
  int* under = reinterpret_cast<int*>(cum);  // rows that underflowed (before cum is built)
  // (se.n_under and se.nonfinite are zero here: cleared before the first row CDF and at the
  // end of every one)
  float mloc = -INFINITY;
  const float* tot_o = reinterpret_cast<const float*>(cum) + kFNmax;
  for (int i = et; i < N; i += NT) {
    float t = __fadd_rn(fL[i], tot_o[i]);  // row_total: the halves the epilogue accumulated
    if (isnan(t)) {
      se.nonfinite = 1;
      t = 0.f;
    }
    if (t < 0x1p-64f) {
      under[atomicAdd(&se.n_under, 1)] = i;
    } else {
      if (a.inspect) a.ws.rowsum[(size_t)s * N + i] = t;
      const float v = row_log2_weight(fG[i], fDl[i], t);
      fL[i] = v;
      mloc = fmaxf(mloc, v);
    }
  }
  mloc = warp_max(mloc);
  if (lane == 0) se.red[ew] = mloc;
  bar_sync(kBarEpi, NT);
  if (se.n_under > 0) {  // rare: exact-max recomputation, then the maximum again
    for (int uq = ew; uq < se.n_under; uq += kFEpiWarps) {
      const int i = under[uq];
      float si, dl;
      recompute_row<D, true>(fU + (size_t)i * D, fAl[i], fV, fB, N, a.B, nT, Tq + (size_t)i * kFTs, &si, &dl);
      __syncwarp();
      if (lane == 0) {
        si = row_total_small(Tq + (size_t)i * kFTs, nT);
        si = isnan(si) ? 0.f : si;
        if (a.inspect) a.ws.rowsum[(size_t)s * N + i] = si;
        fDl[i] = dl;
        fL[i] = row_log2_weight(fG[i], dl, si);
      }
    }
    bar_sync(kBarEpi, NT);
    mloc = -INFINITY;
    for (int i = et; i < N; i += NT) mloc = fmaxf(mloc, fL[i]);
    mloc = warp_max(mloc);
    if (lane == 0) se.red[ew] = mloc;
    bar_sync(kBarEpi, NT);
  }
  float M = se.red[0];
  for (int w = 1; w < kFEpiWarps; ++w) M = fmaxf(M, se.red[w]);
  const bool degenerate = !(M > -INFINITY) || isnan(M);
  for (int i = et; i < N; i += NT) {
    const float r = row_weight(fL[i], M, degenerate);
    if (a.inspect) a.ws.rw[(size_t)s * N + i] = r;
    cum[i] = (unsigned long long)__float2ull_rz(r * 0x1p40f);
  }
  bar_sync(kBarEpi, NT);
  // prefix sums (integer: exact in any order): each warp scans its rows of 32, then every
  // element takes the totals of the rows before its own
  const int C = (N + 31) / 32;
  for (int c = ew; c < C; c += kFEpiWarps) {
    const int i = 32 * c + lane;
    unsigned long long v = i < N ? cum[i] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (i < N) cum[i] = v;
    if (lane == 31) se.rowtot[c] = v;
  }
  bar_sync(kBarEpi, NT);
  // the rows' totals (C <= 32) scanned by every warp at once, lane q holding row q's
  unsigned long long tl = lane < C ? se.rowtot[lane] : 0ull;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, tl, o);
    if (lane >= o) tl += t;
  }
  for (int c = ew; c < C; c += kFEpiWarps) {
    const unsigned long long carry = __shfl_sync(0xffffffffu, tl, c > 0 ? c - 1 : 0);
    const int i = 32 * c + lane;
    if (i < N && c > 0) cum[i] += carry;
  }
  const unsigned long long S_all = __shfl_sync(0xffffffffu, tl, C - 1);
  if (et == 0) {
    const unsigned long long S = S_all;
    se.S = S;
    se.M = M;
    se.degenerate = degenerate ? 1 : 0;
  }
  bar_sync(kBarEpi, NT);
  if (a.inspect) {
    for (int i = et; i < N; i += NT) {
      a.ws.cum[(size_t)s * N + i] = cum[i];
      a.ws.delta[(size_t)s * N + i] = fDl[i];
      for (int kt = 0; kt < nT; ++kt) a.ws.T[((size_t)s * N + i) * nTp + kt] = Tq[(size_t)i * kFTs + kt];
    }
  }
}

// The increment of Eq. (Lab) and log L of the new block (one thread, after the tile sums'
// barrier has released the draws: its global read-modify-write is off their path), from the
// combination base cbase its build computed; then the row CDF's flags are cleared for the
// next combination.
__device__ __forceinline__ void epi_increment(const MergeArgs& a, int s, double cbase, EpiScratch& se) {
  const Comb cb = comb_of(a, s);
  const unsigned long long S = se.S;
  const bool degenerate = se.degenerate != 0;
  const double inc = degenerate ? (double)NAN : lab_increment(cbase, se.M, log_fixed_total(S));
  cb.logL[cb.at] = cb.logL[cb.at] + cb.logL[cb.c] + inc;
  if (degenerate || S == 0ull) record_status(a.ws.status, DSMC_ERR_DEGENERATE);
  if (se.nonfinite) record_status(a.ws.status, DSMC_ERR_NONFINITE);
  se.n_under = 0;
  se.nonfinite = 0;
}

// The pairs of combination s from stage st (the core warps), each in three exact inverse-CDF
// stages over the row CDF the epilogue warps built, and the new block's index maps.
template <int D>
__device__ __forceinline__ void core_draw(const MergeArgs& a, unsigned char* st, const Comb& cb, int ct) {
  using L = Stage<D>;
  const int N = a.N;
  // the output pointers are recomputed from the stage's descriptor at each store rather than
  // held through the draws (fewer live registers: no spills); thread 0 also writes slot 0
  // of a conditional combination
  if (ct == 0) (void)slot_out(a, cb, true);
  DrawIn in;
  in.sys = (a.resampler == DSMC_SYSTEMATIC && !cb.conditional) ? 1 : 0;
  in.cum = reinterpret_cast<unsigned long long*>(st + L::cum);
  in.T = reinterpret_cast<float*>(st + L::T);
  in.U = reinterpret_cast<float*>(st + L::fU);
  in.alpha = reinterpret_cast<float*>(st + L::fAl);
  in.delta = reinterpret_cast<float*>(st + L::fDl);
  in.V = reinterpret_cast<float*>(st + L::fV);
  in.beta = reinterpret_cast<float*>(st + L::fB);
  in.N = N;
  in.B = a.B;
  in.nT = a.nT;
  in.nTp = kFTs;
  const int n_lo = cb.conditional ? 1 : 0;
  const int n_hi = N + ((cb.conditional && cb.root) ? 1 : 0);
  // each slot's map loads are issued when it is drawn and its stores made after the next
  // slot of the thread, so the loads of a merged block's maps overlap that draw
  int pn = -1, pi = 0, pj = 0;
  int32_t pf = 0, pq = 0;
  for (int n = n_lo + ct; n < n_hi; n += kFCoreThreads) {
    int i, j;
    draw_pair<D, true, true, true>(in, cb.seed, cb.base, cb.gid, n, i, j);
    int32_t fi, lj;
    const SlotOut o = slot_out(a, cb, false);
    o.maps(i, j, fi, lj);
    if (pn >= 0) o.store(pn, pi, pj, pf, pq);
    pn = n;
    pi = i;
    pj = j;
    pf = fi;
    pq = lj;
  }
  if (pn >= 0) slot_out(a, cb, false).store(pn, pi, pj, pf, pq);
  // (no barrier here: the next build starts with one, before it writes this stage)
}

template <int D, int KIND>
__global__ void __launch_bounds__(kFThreads, 1) merge_tc_fused_kernel(MergeArgs a, ModelParams<D> mp) {
  using L = Stage<D>;
  extern __shared__ __align__(1024) unsigned char fsm_raw[];
  unsigned char* fsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(fsm_raw) + 1023) & ~(uintptr_t)1023);
  // ops_full: a stage's operands are built; tiles_full: its tile sums are complete;
  // acc_full / acc_free: a TMEM accumulator holds a block / has been read out
  __shared__ __align__(8) uint64_t ops_full[2], tiles_full[2], acc_full[kFAcc], acc_free[kFAcc], in_full;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;
  __shared__ CoreScratch sc;
  __shared__ EpiScratch se;
  __shared__ Comb cbs[2];  // the combination of each stage (written by its build)
  __shared__ double cbase_s[2];  // and its combination base C (comb_base)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N = a.N;
  const int RT = (N + kMmaM - 1) / kMmaM;
  const int ncomb = a.mc > (int)blockIdx.x ? (a.mc - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const volatile int* abort_v = &abort_s;
  auto raise_abort = [&]() {
    if (atomicExch(&abort_s, 1) == 0) record_status(a.ws.status, DSMC_ERR_TIMEOUT);
  };

  if (threadIdx.x == 0) {
    abort_s = 0;
    se.n_under = 0;
    se.nonfinite = 0;
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&ops_full[q]), 1);
      mbar_init(smem_u32(&tiles_full[q]), kFEpiWarps);
    }
    for (int q = 0; q < kFAcc; ++q) {
      mbar_init(smem_u32(&acc_full[q]), 1);
      mbar_init(smem_u32(&acc_free[q]), kFEpiWarps);
    }
    mbar_init(smem_u32(&in_full), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == kFCtrlWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kFTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tb = tmem_base;

  if (warp < kFEpiWarps) {
    // ------------------------------------------------------------------ epilogue
    // warp (g, h) reads TMEM lanes 32 g .. 32 g + 31 (its rows) and columns kFEpiCols h ..
    // of each block, 64 at a time: two 32-column tile weights per row and 64 columns
    const int g = warp & 3, h = warp >> 2;
    int blk = 0;
    bool stop = false;
    for (int k = 0; k < ncomb && !stop; ++k) {
      float* Tq = reinterpret_cast<float*>(fsm + (size_t)(k & 1) * L::bytes + L::T);
      // the row total's two halves (row_total's definition): the even and the odd tile pairs,
      // each accumulated in ascending order as the blocks come (warp h holds pairs of
      // parity h), kept in fL and in the upper half of cum until the row CDF
      float* tot_e = reinterpret_cast<float*>(fsm + (size_t)(k & 1) * L::bytes + L::fL);
      float* tot_o = reinterpret_cast<float*>(fsm + (size_t)(k & 1) * L::bytes + L::cum) + kFNmax;
      for (int rt = 0; rt < RT && !stop; ++rt) {
        const int row = rt * kMmaM + 32 * g + lane;
        float h_even = 0.f, h_odd = 0.f;
        for (int cb = 0; cb < RT; ++cb, ++blk) {
          const int acc = blk & (kFAcc - 1);
          const bool ok = __all_sync(0xffffffffu, mbar_wait_or_abort(smem_u32(&acc_full[acc]),
                                                                    (uint32_t)(blk / kFAcc) & 1, abort_v));
          if (!ok) {
            if (lane == 0) raise_abort();
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int part = 0; part < kFEpiCols / 64; ++part) {
            const int col0 = cb * kMmaN + kFEpiCols * h + 64 * part;
            uint32_t acc0[32], acc1[32];
            const uint32_t taddr =
                tb + ((uint32_t)(32 * g) << 16) + (uint32_t)acc * kMmaN + (uint32_t)(kFEpiCols * h + 64 * part);
            tmem_ld32(taddr, acc0);
            tmem_ld32(taddr + 32, acc1);
            tmem_wait();
            if (part == kFEpiCols / 64 - 1) {
              asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&acc_free[acc]));
            }
            float t0, t1;
            if (col0 + 64 <= N) {
              t0 = exp_sum32<false>(acc0, 32);
              t1 = exp_sum32<false>(acc1, 32);
            } else {
              t0 = exp_sum32<true>(acc0, N - col0);
              t1 = exp_sum32<true>(acc1, N - col0 - 32);
            }
            if (row < N) {
              if (col0 + 32 < N)
                *reinterpret_cast<float2*>(Tq + (size_t)row * kFTs + col0 / 32) = make_float2(t0, t1);
              else if (col0 < N)
                Tq[(size_t)row * kFTs + col0 / 32] = t0;
            }
            const float q = __fadd_rn(t0, t1);  // 0 past the last tile
            if ((col0 / 64) & 1)
              h_odd = __fadd_rn(h_odd, q);
            else
              h_even = __fadd_rn(h_even, q);
          }
        }
        if (row < N) {
          if (kFEpiWarps == 4 || h == 0) tot_e[row] = h_even;
          if (kFEpiWarps == 4 || h == 1) tot_o[row] = h_odd;
        }
      }
      // every epilogue warp reaches this barrier (a stopped one straight from its wait), so
      // they agree whether to go on; then the row CDF of this combination
      if (!bar_and(kBarEpi, kFEpiWarps * 32, !stop)) break;
      epi_row_cdf<D>(a, fsm + (size_t)(k & 1) * L::bytes, blockIdx.x + k * gridDim.x, threadIdx.x, warp, lane, se);
      // the combination base is read before the draws are released: the build that follows
      // them rewrites it
      const double cbase_k = threadIdx.x == 0 ? cbase_s[k & 1] : 0.0;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tiles_full[k & 1]));
      if (threadIdx.x == 0) epi_increment(a, blockIdx.x + k * gridDim.x, cbase_k, se);
    }
  } else if (warp < kFCtrlWarp) {
    // ------------------------------------------------------------------ core warps
    // loads of combinations 0 and 1, then for every k: the draws of k (once its tile sums
    // are complete) and the load of k + 2 into the stage k has just released
    const int ct = threadIdx.x - kFCore0, cw = ct >> 5;
    unsigned char* inb = fsm + 2 * L::bytes;
    const uint32_t in_bar = smem_u32(&in_full);
    auto comb = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
    // Build m (of combination m) reads its descriptor from scratch slot m & 1 and prefetches
    // the next build's into the other slot.  After build m has read the inputs buffer (its
    // closing fence orders those reads before the bulk copies), one thread starts the next
    // build's inputs from that descriptor.
    auto bulk_next = [&](int m) {
      if (ct == 0) sc.in_bulk = sc.in_pend = issue_inputs(a, sc.nx_cb[(m + 1) & 1], inb, in_bar) ? 1 : 0;
    };
    // every core thread waits for bulk-copied inputs; false on an abort or a timeout
    // (sync_first: a barrier first, where no other one has passed since sc.in_bulk was written)
    auto inputs_ready = [&](bool sync_first) -> bool {
      if (sync_first) bar_sync(kBarCore, kFCoreThreads);
      bool ok = true;
      if (sc.in_bulk) ok = mbar_wait_or_abort(in_bar, (uint32_t)sc.in_phase & 1, abort_v);
      ok = bar_and(kBarCore, kFCoreThreads, ok);
      if (ct == 0 && sc.in_bulk && ok) {
        ++sc.in_phase;
        sc.in_pend = 0;
      }
      return ok;
    };
    bool ok = true;
    if (ct == 0) {
      sc.in_phase = sc.in_pend = sc.in_bulk = 0;
      if (ncomb > 0) {  // the first build's descriptor and inputs
        sc.nx_cb[0] = comb_of(a, comb(0));
        read_rows<D>(a, mp, sc, 0);
        sc.in_bulk = sc.in_pend = issue_inputs(a, sc.nx_cb[0], inb, in_bar) ? 1 : 0;
      }
    }
    for (int k = 0; k < ncomb && k < 2 && ok; ++k) {
      ok = inputs_ready(true);
      if (!ok) break;
      core_load<D, KIND>(a, mp, fsm + (size_t)k * L::bytes, comb(k), inb, ct, cw, lane, RT, sc, &cbs[k],
                         &cbase_s[k], k & 1, k + 1 < ncomb ? comb(k + 1) : -1);
      if (k + 1 < ncomb) bulk_next(k);
      if (ct == 0) mbar_arrive(smem_u32(&ops_full[k]));
    }
    for (int k = 0; k < ncomb && ok; ++k) {
      const int q = k & 1;
      const bool tiles_ok =
          ct != 0 || mbar_wait_or_abort(smem_u32(&tiles_full[q]), (uint32_t)(k >> 1) & 1, abort_v);
      if (!bar_and(kBarCore, kFCoreThreads, tiles_ok)) {
        ok = false;
        break;
      }
      core_draw<D>(a, fsm + (size_t)q * L::bytes, cbs[q], ct);
      if (k + 2 < ncomb) {
        ok = inputs_ready(false);  // the draws' end and the build's start: its barrier
        if (!ok) break;
        core_load<D, KIND>(a, mp, fsm + (size_t)q * L::bytes, comb(k + 2), inb, ct, cw, lane, RT, sc, &cbs[q],
                           &cbase_s[q], k & 1, k + 3 < ncomb ? comb(k + 3) : -1);
        if (k + 3 < ncomb) bulk_next(k + 2);
        if (ct == 0) mbar_arrive(smem_u32(&ops_full[q]));
      }
    }
    if (!ok) {
      bar_sync(kBarCore, kFCoreThreads);
      if (ct == 0) {
        raise_abort();
        // bulk copies still in flight land before the CTA leaves (bounded)
        if (sc.in_pend) mbar_wait(in_bar, (uint32_t)sc.in_phase & 1);
      }
    }
  } else if (lane == 0) {
    // ------------------------------------------------------------------ control: MMA issue
    // one MMA per (row tile, column block) of each combination once its operands are built,
    // into the accumulator the epilogue has released (four accumulators in flight)
    int blk = 0, issued = 0;
    bool ok = true;
    for (int k = 0; k < ncomb && ok; ++k) {
      const int q = k & 1;
      ok = mbar_wait_or_abort(smem_u32(&ops_full[q]), (uint32_t)(k >> 1) & 1, abort_v);
      if (!ok) break;
      const uint32_t sU = smem_u32(fsm + (size_t)q * L::bytes + L::opU);
      const uint32_t sV = smem_u32(fsm + (size_t)q * L::bytes + L::opV);
      for (int rt = 0; rt < RT && ok; ++rt) {
        for (int cb = 0; cb < RT; ++cb, ++blk) {
          const int acc = blk & (kFAcc - 1);
          if (blk >= kFAcc) {
            ok = mbar_wait_or_abort(smem_u32(&acc_free[acc]), (uint32_t)(blk / kFAcc - 1) & 1, abort_v);
            if (!ok) break;
          }
          if (a.stall) continue;  // test switch: nothing is issued, no accumulator completes
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          mma<KIND>(tb + (uint32_t)acc * kMmaN, smem_desc(sU + (uint32_t)(rt * kFTileBytes)),
                    smem_desc(sV + (uint32_t)(cb * kFTileBytes)), 0u);
          mma_commit(smem_u32(&acc_full[acc]));
          ++issued;
        }
      }
    }
    if (!ok) raise_abort();
    if (issued > 0 && !a.stall) {  // the last committed MMA completes before TMEM is freed
      const int last = blk - 1;
      mbar_wait(smem_u32(&acc_full[last & (kFAcc - 1)]), (uint32_t)(last / kFAcc) & 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kFCtrlWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(kFTmemCols));
  }
}

template <int D, int KIND>
cudaError_t fused_tc_t(const MergeArgs& a, const void* mp, cudaStream_t st) {
  constexpr size_t smem = fused_tc_smem<D>();
  static_assert(smem <= 227 * 1024, "two stages must fit one SM's shared memory");
  cudaError_t e = cudaFuncSetAttribute(merge_tc_fused_kernel<D, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int sms = a.sms > 0 ? a.sms : 1;
  const int grid = a.mc < sms ? a.mc : sms;
  merge_tc_fused_kernel<D, KIND><<<grid, kFThreads, smem, st>>>(a, *static_cast<const ModelParams<D>*>(mp));
  return cudaGetLastError();
}

}  // namespace

// Whether a level of this shape can run as the fused tensor-core kernel: N <= 512 (tile
// width 32), padded dimension D <= 4 with one 32-byte K plane, BF16 or TF32.
bool fused_tc_supported(int D, int N, int compute, int planes) {
  return (compute == DSMC_BF16 || compute == DSMC_TF32) && planes == 1 && N >= 1 && N <= kFNmax && D <= 4;
}

cudaError_t launch_merge_tc_fused(int D, const MergeArgs& a, const void* mp, cudaStream_t s) {
  if (a.B != 32 || a.nTp > kFTiles) return cudaErrorInvalidValue;
  if (a.compute == DSMC_BF16) {
    switch (D) {
      case 1: return fused_tc_t<1, DSMC_BF16>(a, mp, s);
      case 2: return fused_tc_t<2, DSMC_BF16>(a, mp, s);
      case 4: return fused_tc_t<4, DSMC_BF16>(a, mp, s);
    }
  } else if (a.compute == DSMC_TF32) {
    switch (D) {
      case 1: return fused_tc_t<1, DSMC_TF32>(a, mp, s);
      case 2: return fused_tc_t<2, DSMC_TF32>(a, mp, s);
      case 4: return fused_tc_t<4, DSMC_TF32>(a, mp, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace dsmc
