// kernels.cuh -- argument blocks and launch wrappers shared by the kernels and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace dsmc {

// Pointers into the caller's workspace (layout fixed by Plan in api.cu).
struct WsPtrs {
  int* status;       // first device error (0 = none)
  float* U;          // [Mc][N][D]   log2(e) Q^{-1} (A x_L + c - mu)
  float* alpha;      // [Mc][N]      row term of the base-2 exponent
  float* V;          // [Mc][N][D]   x_R - mu
  float* beta;       // [Mc][N]      column term of the base-2 exponent
  double* shift;     // [Mc][N]      per-row shift (natural log): a_i + log f_max + B* + dl_i ln 2
  float* g;          // [Mc][N]      dense samplers: the same shift less the combination base,
                     //              in base 2 (shift_i = cbase + g_i ln 2)
  double* cbase;     // [Mc]         dense samplers: the combination base (natural log)
  double* logbar;    // [Mc]         log omega-bar, bound of the whole N x N matrix
  float* T;          // [Mc][N][nTp] tile weights, relative to the row shift
  float* rw;         // [Mc][N]      row weights of the row stage
  float* rowsum;     // [Mc][N]      row totals (sums of the tile weights)
  unsigned long long* cum;  // [Mc][N] exact 2^40 fixed-point prefix sums of the row weights
  float* delta;      // [Mc][N]      extra base-2 shift of rows recomputed after underflow
  int32_t* first;    // [2][K][N]    first-time particle index of each block (double-buffered)
  int32_t* last;     // [2][K][N]    last-time particle index of each block
  int32_t* star;     // [2]          root pair of the next reference (conditional mode)
  double* inc;       // [Mc]         log normalising-constant increments
  // tensor-core operands (compute = DSMC_TF32 / DSMC_BF16): [u, alpha_hi, alpha_lo, 1, 1]
  // and [v, 1, 1, beta_hi, beta_lo] rounded to the MMA type, in 32-byte K planes, each
  // plane in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices, row
  // group g at g*256 B, chunk c at c*128 B), rows padded to a multiple of 128.
  unsigned char* Ub; // [Mc][planes][Nr][32 B]
  unsigned char* Vb; // [Mc][planes][Nr][32 B]
  // rejection sampling with factorised proposals (DSMC_RS_FACTORED)
  float* alpha0;     // [Mc][N]      alpha_i before the row shift: -log2(e) 1/2 w_i' Q^-1 w_i
  float* kappa;      // [Mc][N]      log2(e) (dist_j^2 Q^-1 / 2 - 1/2 v_j' Q^-1 v_j): with alpha0_i
                     //              and u_i . v_j, the base-2 log acceptance of pair (i, j)
  float* pa;         // [Mc][N]      row proposal: log a_i from the prologue, then e^(a_i - max a)
  float* pc;         // [Mc][N]      column proposal: b'_j - dist_j^2 Q^-1 / 2, then relative weight
  unsigned long long* cumA;  // [Mc][N] exact 2^40 fixed-point prefix sums of the row proposal
  unsigned long long* cumC;  // [Mc][N] the same of the column proposal
  unsigned long long* attempts_total;  // attempts of the rejection samplers since the last
                                      // init (inspection: acceptance rate)
};

// One sequence of a batched launch (device memory; built by the host per batch).
struct SeqDesc {
  int K, L;                  // steps, levels
  float* X;                  // [K][N][d]
  float* logw;               // [K][N]
  const float* y;            // [K][d]
  double* logL;              // [K]
  int32_t* pairs;            // [K-1][2][N]
  int32_t* first;            // [2][K][N] map buffers of this sequence
  int32_t* last;             // [2][K][N]
  int32_t* star;             // [2]
  const float* prop_mean;    // [K][d] (DSMC_PROP_GAUSS) or null
  const float* prop_std;     // [K][d]
  uint64_t seed;
  uint32_t base;
  int conditional;
  const float* x_ref;        // [K][d] reference of a conditional sweep, or null
  double* mean;              // [K][d] outputs of the resolve
  double* m2;                // [K][d] or null
  float* x_star;             // [K][d] next reference (conditional), or null
  double* logL_out;          // one double, or null
};

// Block b of a launch over every time step of a batch: sequence s with
// kstart[s] <= b < kstart[s + 1], time t = b - kstart[s] (thread 0 searches, all read).
__device__ __forceinline__ void batch_time(const int* kstart, int n_seq, int b, int& seq, int& t) {
  __shared__ int s_seq;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n_seq - 1;  // last s with kstart[s] <= b
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (kstart[mid] <= b) lo = mid; else hi = mid - 1;
    }
    s_seq = lo;
  }
  __syncthreads();
  seq = s_seq;
  t = b - kstart[seq];
}

// One combination of a batched launch: sequence, combination index within its level, its
// row in the sequence's pairs array, and the level (one launch may mix levels).
struct CombItem {
  int seq, m, gid, level;
};

struct MergeArgs {
  int K, N, d, level;
  int m0;            // first combination (within the level) of this launch chunk
  int mc;            // combinations in this chunk
  int gid0;          // global (level-major) id of combination m0
  int B, nT, nTp;    // tile width, tiles per row, padded tiles per row
  int CH, CW;        // column chunks and chunk width of the row-sum kernel
  int rows_per_cta;  // row-sum kernel rows per CTA
  int conditional;   // Algorithm 5 when non-zero
  int root;          // this level holds the root combination
  int resampler;
  int compute;       // DSMC_FP32, DSMC_TF32 or DSMC_BF16
  int Nr;            // N rounded up to 128 (tensor-core operand rows)
  int mma_planes;    // 32-byte K planes of the tensor-core operands
  int sms;           // SMs of the device (persistent grids)
  int inspect;       // fused kernels also store their intermediate weights in the workspace
                     // (dsmc_debug_keep_weights), for the inspection entry points
  int stall;         // test switch: the tensor-core control warp issues no MMA, so every
                     // wait on an accumulator runs out (dsmc_debug_stall_tensor_cores)
  uint64_t seed;
  uint32_t base;
  uint32_t rs_max;
  float logN;
  const float* X;    // [K][N][d]
  const float* logw; // [K][N]
  const float* y;    // [K][d]
  double* logL;      // [K]
  int32_t* pairs;    // [K-1][2][N]
  const float* prop_mean;  // [K][d] (DSMC_PROP_GAUSS) or null
  const float* prop_std;
  const SeqDesc* seqs;     // batched launches: the sequences (device), else null
  const CombItem* items;   // batched launches: combination m0 + s is items[m0 + s]
  WsPtrs ws;
};

// Block geometry of combination m (0-based within level l): left [a, c-1], right [c, b].
__host__ __device__ __forceinline__ void merge_geom(int K, int level, int m, int& a, int& c,
                                                    int& b) {
  const int size = 1 << level;
  a = 2 * m * size;
  c = a + size;
  b = min(a + 2 * size, K) - 1;
}

// Everything combination s of a launch needs from its sequence.
struct Comb {
  int K, level, m, gid, at, c, b;
  bool root;
  int conditional;
  const float* X;
  const float* logw;
  const float* y;
  double* logL;
  int32_t* pairs;
  int32_t* first;
  int32_t* last;
  int32_t* star;
  const float* prop_mean;
  const float* prop_std;
  uint64_t seed;
  uint32_t base;
};

__device__ __forceinline__ Comb comb_of(const MergeArgs& a, int s) {
  Comb cb;
  if (a.items == nullptr) {
    cb.K = a.K;
    cb.level = a.level;
    cb.m = a.m0 + s;
    cb.gid = a.gid0 + s;
    cb.root = a.root != 0;
    cb.conditional = a.conditional;
    cb.X = a.X;
    cb.logw = a.logw;
    cb.y = a.y;
    cb.logL = a.logL;
    cb.pairs = a.pairs;
    cb.first = a.ws.first;
    cb.last = a.ws.last;
    cb.star = a.ws.star;
    cb.prop_mean = a.prop_mean;
    cb.prop_std = a.prop_std;
    cb.seed = a.seed;
    cb.base = a.base;
  } else {
    const CombItem it = a.items[a.m0 + s];
    const SeqDesc& q = a.seqs[it.seq];
    cb.K = q.K;
    cb.level = it.level;
    cb.m = it.m;
    cb.gid = it.gid;
    cb.root = (it.level == q.L - 1);
    cb.conditional = q.conditional;
    cb.X = q.X;
    cb.logw = q.logw;
    cb.y = q.y;
    cb.logL = q.logL;
    cb.pairs = q.pairs;
    cb.first = q.first;
    cb.last = q.last;
    cb.star = q.star;
    cb.prop_mean = q.prop_mean;
    cb.prop_std = q.prop_std;
    cb.seed = q.seed;
    cb.base = q.base;
  }
  merge_geom(cb.K, cb.level, cb.m, cb.at, cb.c, cb.b);
  return cb;
}

struct InitArgs {
  int K, N, d;
  float logN;        // (float) log N, from FP64
  const SeqDesc* seqs;   // batched launch over every (sequence, t): the sequences, else null
  const int* kstart;     // [n_seq + 1] first block of each sequence
  int n_seq;
  uint64_t seed;
  uint32_t base;
  const float* y;
  const float* x_ref;
  float* X;
  float* logw;
  double* logL;
  int* status;
};

struct GatherArgs {
  int K, N, d, L;
  const SeqDesc* seqs;   // batched launch over every (sequence, t), else null
  const int* kstart;     // [n_seq + 1]
  int n_seq;
  const int32_t* S;  // [K][N+1] leaf index of every output trajectory (and the root draw) per t
  int level_off[33];
  const float* X;
  const float* logw;
  const int32_t* pairs;
  const int32_t* star;
  float* traj;
  double* mean;
  double* m2;
  float* x_star;
  int* status;
};

// The linearised Gaussian smoother of Section 4.1 (Algorithm 4): the model in FP64 (device
// pointers into its workspace, set by launch_pit), observations [K][d].
struct PitArgs {
  int K, d, kind;
  const float* y;
  const double *F, *Q, *R, *P0, *c, *m0;   // [d][d] x 4, [d] x 2
  const double *Ft, *ct;                    // per-step transitions [K][d][d], [K][d], or null
  double mu;                                // SV, COX: the stationary mean (first linearisation)
  double tau0, tau1, tau2;                  // THETA_LOGISTIC
};
size_t pit_workspace_bytes(int K, int d);
cudaError_t launch_pit(PitArgs pa, const double* model, int iterations, const float* init_mean, float* mean_out,
                       float* std_out, void* ws, cudaStream_t st, int* n_launches);

// Launchers (defined in the .cu files, dispatched on the padded dimension D).
cudaError_t launch_init(int D, const InitArgs& a, const void* mp, cudaStream_t s);
cudaError_t launch_prologue(int D, const MergeArgs& a, const void* mp, cudaStream_t s);
cudaError_t launch_rowsum(int D, const MergeArgs& a, cudaStream_t s);
cudaError_t launch_rowsum_tc(const MergeArgs& a, cudaStream_t s);
cudaError_t launch_sample_dense(int D, const MergeArgs& a, cudaStream_t s);
cudaError_t launch_sample_rs(int D, const MergeArgs& a, cudaStream_t s);
cudaError_t launch_rsf_cdf(const MergeArgs& a, cudaStream_t s);
cudaError_t launch_debug_lazy(int D, const MergeArgs& a, int s_local, float* pa, float* pc, float* acc,
                              cudaStream_t s);
cudaError_t launch_epilogue(const MergeArgs& a, cudaStream_t s);
bool fused_tc_supported(int D, int N, int compute, int planes);
cudaError_t launch_merge_tc_fused(int D, const MergeArgs& a, const void* mp, cudaStream_t s);
cudaError_t launch_gather(int D, const GatherArgs& a, cudaStream_t s);
cudaError_t launch_resolve_level(const MergeArgs& a, cudaStream_t s);
cudaError_t launch_debug_weights(int D, const MergeArgs& a, int s_local, float* logW, float* r,
                                 float* rowsum, float* tiles, float* e, float* ratio,
                                 cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                          cudaStream_t s);

}  // namespace dsmc
