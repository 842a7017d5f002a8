/*
 * dsmc.h -- C ABI of the GB300 (sm_103a) implementation of dSMC, the de-Sequentialized
 * Monte Carlo particle smoother of Corenflos, Chopin and Sarkka (arXiv 2202.02264).
 *
 * The data-parallel hot path is the divide-and-conquer combination of Section 2 applied
 * over ceil(log2 K) tree levels:
 *   - Algorithm 2: independent proposals q_t and leaf weights for every (t, n);
 *   - Appendix A, Algorithm 6: left-aligned blocks of 2^l steps, block pairs (2m, 2m+1)
 *     combined at level l, an unpaired last block passed through unchanged;
 *   - Algorithm 1 (Combine): the N x N product-form log-weights of Eq. (normalized-weights)
 *     with the stitching weight omega_c = p_c h_c / nu_c of Proposition 2, N pair draws,
 *     and the concatenated trajectories;
 *   - Algorithm 8: rejection-sampling lazy resampling, which never forms the N x N matrix;
 *   - Algorithm 5 (ConditionalCombine) and the star trajectory of Section 3.1, for the
 *     parallel-in-time particle Gibbs sampler of Section 3.2.
 *
 * Conventions shared by every entry point:
 *   - Time steps are t = 0..K-1 (the paper's t = 0..T with K = T + 1).  N particles, state
 *     dimension dx in 1..32; observations have dimension dx (identity observation map).
 *   - "device" pointers are CUDA global-memory pointers on the current device; "host"
 *     pointers are ordinary CPU memory.  The library allocates no device memory: the
 *     caller passes every buffer, sized by dsmc_state_sizes() and dsmc_workspace_size().
 *     The library never frees caller memory.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL is the
 *     legacy default stream).  Argument errors are returned synchronously and nothing is
 *     launched.  Errors found on the device (non-finite or degenerate weights, the
 *     rejection-sampling attempt cap) are recorded in a status word inside the workspace
 *     and read with dsmc_stream_status(), which synchronises the stream.
 *   - Random numbers are Philox4x32-10 keyed by `seed`, with the counter
 *     (slot, time-or-combination id, purpose | counter_base << 4, j); results are
 *     deterministic for a given (seed, counter_base) and do not depend on the launch
 *     configuration.
 *   - The library never aborts or traps.
 */
#ifndef DSMC_H
#define DSMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DSMC_OK = 0,
  DSMC_ERR_INVALID_ARG = 1,  /* a pointer, size or parameter is invalid; nothing launched */
  DSMC_ERR_UNSUPPORTED = 2,  /* a valid request outside the supported range (e.g. N, dx) */
  DSMC_ERR_WORKSPACE = 3,    /* ws_bytes smaller than dsmc_workspace_size() */
  DSMC_ERR_CUDA = 5,         /* a CUDA launch or copy failed; see dsmc_last_error() */
  DSMC_ERR_NONFINITE = 6,    /* device: a log-weight was NaN */
  DSMC_ERR_DEGENERATE = 7,   /* device: every weight of a combination was zero */
  DSMC_ERR_RS_LIMIT = 8,     /* device: a rejection-sampling slot hit rs_max_attempts */
  DSMC_ERR_TIMEOUT = 9,      /* device: a bounded wait gave up */
  DSMC_ERR_BOUND = 10        /* device: a lazy sampler met a pair above its bound by more
                                than FP32 rounding (ratio > 1 + 2^-10): a broken bound */
} dsmc_status_t;

enum { DSMC_MODEL_LGSSM = 0, DSMC_MODEL_SV = 1, DSMC_MODEL_COX = 2, DSMC_MODEL_THETA_LOGISTIC = 3,
       DSMC_MODEL_CRW = 4 };
enum { DSMC_PROP_OBS = 0, DSMC_PROP_GAUSS = 1, DSMC_PROP_UNIFORM = 2 };
enum { DSMC_NU_EQ_Q = 0, DSMC_NU_PROP_H = 1 };
enum { DSMC_FP32 = 0, DSMC_TF32 = 1, DSMC_BF16 = 2 };
enum { DSMC_MULTINOMIAL = 0, DSMC_RS = 1, DSMC_MH = 2, DSMC_SYSTEMATIC = 3, DSMC_RS_FACTORED = 4 };

/* The state-space model of Eq. (ssm) (Section 1).  All arrays are HOST, row-major, FP64,
 * read during the call only.  Every transition is Gaussian, N(m(x_{t-1}), Q).
 *   LGSSM: x_0 ~ N(m0, P0), x_t = A x_{t-1} + N(0, Q), y_t = x_t + N(0, R).
 *   SV (dx = 1): x_0 ~ N(mu, sigma^2/(1-phi^2)), x_t = mu + phi (x_{t-1} - mu) + sigma e,
 *                y_t = exp(x_t / 2) v, e, v ~ N(0, 1).
 *   COX (dx = 1, the photon-count model of Section 5.1): x_0 ~ N(mu, sigma^2/(1-phi^2)),
 *                x_t = mu + phi (lam x_{t-1} - mu) + sigma e, y_t ~ Poisson(exp(x_t)).
 *   THETA_LOGISTIC (dx = 1, the population model of Section 5.2): x_0 ~ N(0, 1),
 *                x_t = x_{t-1} + tau0 - tau1 exp(tau2 x_{t-1}) + sigma e,
 *                y_t = x_t + obs_sd v.
 *   CRW (dx = 1, the constrained random walk of Section 5.3): x_0 ~ N(0, 1),
 *                x_t = x_{t-1} + sigma e, potential h_t(x) = 1 if |x| <= bound else 0 (y is
 *                not read; pass any [K][1] array).
 * Fields a kind does not use are ignored (A, Q, R, m0, P0 by every kind but LGSSM). */
typedef struct {
  int kind;              /* DSMC_MODEL_* */
  int dx;                /* 1..32 (1 for every kind but LGSSM) */
  const double* A;       /* [dx][dx] */
  const double* Q;       /* [dx][dx], symmetric positive definite */
  const double* R;       /* [dx][dx], symmetric positive definite */
  const double* m0;      /* [dx] */
  const double* P0;      /* [dx][dx], symmetric positive definite */
  double mu, phi, sigma; /* SV and COX: |phi| < 1, sigma > 0; THETA_LOGISTIC, CRW: sigma > 0 */
  double lam;            /* COX: the factor of x_{t-1} inside the autoregression */
  double tau0, tau1, tau2; /* THETA_LOGISTIC: the growth terms */
  double obs_sd;         /* THETA_LOGISTIC: observation noise standard deviation > 0 */
  double bound;          /* CRW: the constraint half-width > 0 */
} dsmc_model_t;

/* The proposals q_t of Algorithm 2 and the auxiliary laws nu_t of Definition 1.
 *   DSMC_PROP_OBS:     q_t = N(y_t, scale^2 I).
 *   DSMC_PROP_GAUSS:   q_t = N(mean[t], diag(std[t]^2)); mean, std are DEVICE [K][dx] FP32.
 *   DSMC_PROP_UNIFORM: q_t = U([-scale, scale]^dx) (the constrained random walk's proposal).
 *   nu = DSMC_NU_EQ_Q:   nu_t = q_t for t >= 1 (the paper's experiments).
 *   nu = DSMC_NU_PROP_H: nu_t proportional to h_t(y_t | .), so that the combination weight
 *                        is log p_t(x_t | x_{t-1}) up to a constant (LGSSM, SV,
 *                        THETA_LOGISTIC and CRW; the COX potential has no finite normaliser
 *                        when y_t = 0). */
typedef struct {
  int kind;
  double scale;
  const float* mean;
  const float* std;
  int nu;
} dsmc_proposal_t;

typedef struct {
  int K;                      /* time steps, >= 1 */
  int N;                      /* particles, >= 1 (>= 2 when conditional); <= 16384 dense */
  int compute;                /* cross-term precision: DSMC_FP32 (CUDA cores, default),
                                 DSMC_TF32 (dx <= 16) or DSMC_BF16 (any dx) on the tensor
                                 cores: the whole base-2 exponent alpha_i + beta_j + u_i.v_j
                                 is one MMA, alpha and beta entering as two-term splits in
                                 the MMA type; FP32 accumulate, exp and sums; dense N <= 4096.
                                 Ignored by the lazy samplers (DSMC_RS, DSMC_RS_FACTORED,
                                 DSMC_MH), which evaluate their proposed pairs in FP32 */
  int resampler;              /* how a combination draws its N pairs:
                                 DSMC_MULTINOMIAL (Algorithm 1): N independent draws from the
                                 normalised N x N weights, by the exact three-stage
                                 fixed-point inverse CDF (row, tile, column);
                                 DSMC_SYSTEMATIC (Algorithm 1's systematic option): the same
                                 stages at the positions (k + U) / N of the flattened CDF, one
                                 uniform U per combination (conditional combinations stay
                                 multinomial, Algorithm 5);
                                 DSMC_RS (Algorithm 8): uniform pair proposals accepted with
                                 probability omega_ij / omega-bar, omega-bar = f_max
                                 e^{max_i a_i} max_j e^{b'_j} (for dx = 1 the factor of column
                                 j is tightened to e^{b'_j - dist_j^2 / 2Q}, dist_j the distance
                                 from x_j to the hull of the transition means A x_i + c of the
                                 time-(c-1) particles);
                                 DSMC_RS_FACTORED (rejection with factorised proposals, the
                                 future-work item of the paper's discussion): row i proposed
                                 with probability proportional to e^{a_i}, column j to
                                 e^{b'_j} (times e^{-dist_j^2 / 2Q} for dx = 1), accepted
                                 with probability f(x_j | x_i) / f_max (times
                                 e^{dist_j^2 / 2Q}): the same target, with the expected
                                 attempts divided by the spread of the leaf and observation
                                 weights;
                                 DSMC_MH (Algorithm 7): per slot, B Metropolis-Hastings steps
                                 from (n mod N, n mod N) with uniform pair proposals, accepted
                                 iff u r(I,J) < r(I*,J*) in FP32, r the pair's ratio
                                 omega / omega-bar; biased for finite B.
                                 The two rejection samplers retire accepted slots and refill
                                 their lanes (warp-compacted retry); a slot that reaches
                                 rs_max_attempts keeps the pair (-1, -1) and records
                                 DSMC_ERR_RS_LIMIT; a ratio above 1 + 2^-10 records
                                 DSMC_ERR_BOUND */
  uint64_t seed;              /* Philox key */
  uint32_t counter_base;      /* < 2^28; e.g. the particle-Gibbs sweep index */
  uint32_t rs_max_attempts;   /* DSMC_RS, DSMC_RS_FACTORED: cap of attempts per slot (0 means
                                 2^26, which the uniform proposals of the stochastic-
                                 volatility workload at N = 16384 need for their worst
                                 combinations; the factorised proposals need far fewer);
                                 DSMC_MH: the steps B of each slot's chain (0 means 64) */
  int max_merges_per_launch;  /* 0 = default; bounds the workspace */
  int fused_max_merges;       /* dense sampler: levels with at most this many combinations run
                                 as one fused launch (a thread-block cluster per combination,
                                 FP32 cross term); 0 = default (32; none with a
                                 tensor-core precision and dx > 8), < 0 = never */
  int tc_fused;               /* dense sampler with a tensor-core precision, N <= 512, dx <= 4:
                                 > 0 = every level chunk not run as a fused small level runs
                                 as one persistent warp-specialised kernel (operand rows,
                                 tcgen05 cross term, exponentials, row CDF and draws of each
                                 combination on one SM; nothing but pairs, maps and log L
                                 written); 0 (default) or < 0 = the split kernels (terms,
                                 tile sums, draws).  Same results.  Needs tile_cols 32. */
  int tile_cols;              /* dense sampler: columns per tile of the row tile sums, the
                                 tiles the sampler's tile stage picks from before its column
                                 stage recomputes the chosen tile's columns: 32 or 64, with
                                 at most 64 tiles per row; 0 = default (32 up to N = 2048,
                                 then the smallest multiple of 32 giving <= 64 tiles).  Another
                                 tile width draws from the same law with the same uniforms
                                 split differently across the stages, so the pairs differ;
                                 the weights do not. */
} dsmc_config_t;

/* Caller-owned DEVICE state of one smoothing (sizes from dsmc_state_sizes()).
 *   X      [K][N][dx] FP32  Algorithm 2 particles; merges never modify them
 *   logw   [K][N]     FP32  normalised leaf log-weights
 *   logL   [K]        FP64  log normalising constant of the block starting at t
 *   pairs  [K-1][2][N] int32 (l_n, r_n) of every combination, level-major order: all
 *                      combinations of level 0 by ascending start time, then level 1, ...
 */
typedef struct {
  float* X;
  float* logw;
  double* logL;
  int32_t* pairs;
} dsmc_state_t;

/* Human-readable text of a status code (static storage). */
const char* dsmc_status_string(dsmc_status_t s);

/* Text of the last error raised in this thread (thread-local, valid until the next call). */
const char* dsmc_last_error(void);

/* Bytes of the four state arrays, in the order X, logw, logL, pairs.  Host call. */
dsmc_status_t dsmc_state_sizes(const dsmc_config_t* cfg, const dsmc_model_t* model,
                               size_t bytes_out[4]);

/* Bytes of device workspace every call below needs for this (cfg, model).  Host call. */
dsmc_status_t dsmc_workspace_size(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                  size_t* bytes);

/* Algorithm 2 (and its conditional form, Section 3.2: slot 0 of every time step is
 * x_ref[t], weighted like the others).  y: DEVICE [K][dx] FP32.  x_ref: DEVICE [K][dx]
 * FP32 or NULL.  Writes state->X, state->logw, state->logL.  Resets the status word. */
dsmc_status_t dsmc_init_particles(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                  const dsmc_proposal_t* prop, const float* y,
                                  const float* x_ref, dsmc_state_t* state, void* ws,
                                  size_t ws_bytes, void* stream);

/* One level l of Algorithm 6: every combination of adjacent 2^l-blocks (Algorithm 1, or
 * Algorithm 5 when `conditional`).  Must be called for l = 0, 1, ..., ceil(log2 K) - 1 in
 * order after dsmc_init_particles with the same state and workspace.  Writes the pairs of
 * the level's combinations and updates state->logL. */
dsmc_status_t dsmc_merge_level(const dsmc_config_t* cfg, const dsmc_model_t* model,
                               const dsmc_proposal_t* prop, const float* y, int level,
                               int conditional, dsmc_state_t* state, void* ws,
                               size_t ws_bytes, void* stream);

/* Resolves the output trajectories from the stored pairs (composition of the resampling
 * arrays of the Remark in Section 3.1) and gathers them.  traj_out: DEVICE [K][N][dx] FP32
 * or NULL; mean_out: DEVICE [K][dx] FP64 (smoothing means); m2_out: DEVICE [K][dx] FP64 or
 * NULL (second moments); x_star_out: DEVICE [K][dx] FP32 or NULL (conditional mode: the
 * trajectory chosen by the extra root draw). */
dsmc_status_t dsmc_resolve(const dsmc_config_t* cfg, const dsmc_model_t* model,
                           const dsmc_state_t* state, float* traj_out, double* mean_out,
                           double* m2_out, float* x_star_out, void* ws, size_t ws_bytes,
                           void* stream);

/* The whole smoother: init, every level, resolve.  logL_out: DEVICE FP64 scalar, the log
 * normalising-constant estimate of Eq. (rec-loglik) (NaN with DSMC_RS or DSMC_MH, which never form
 * the N x N sums). */
dsmc_status_t dsmc_smooth(const dsmc_config_t* cfg, const dsmc_model_t* model,
                          const dsmc_proposal_t* prop, const float* y, dsmc_state_t* state,
                          float* traj_out, double* mean_out, double* m2_out, double* logL_out,
                          void* ws, size_t ws_bytes, void* stream);

/* One conditional dSMC sweep (Section 3.2): slot 0 carries x_ref_in through every
 * combination; x_ref_out (DEVICE [K][dx] FP32, may alias x_ref_in) receives the next
 * reference trajectory, drawn from the root's weights (Section 3.1).  N >= 2. */
dsmc_status_t dsmc_conditional_smooth(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                      const dsmc_proposal_t* prop, const float* y,
                                      const float* x_ref_in, float* x_ref_out,
                                      dsmc_state_t* state, float* traj_out, double* mean_out,
                                      double* logL_out, void* ws, size_t ws_bytes,
                                      void* stream);

/* Size of the library's static device scratch used by dsmc_smooth_noalloc (32 MiB). */
#define DSMC_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/* dsmc_smooth without a caller-supplied workspace, for callers that cannot allocate device
 * memory: code that runs inside another allocator's pool or a memory budget it does not
 * own, plugins and runtimes that forbid cudaMalloc after start-up, and hosts whose own
 * allocator must stay the only one.  (The paper has no counterpart: this is an interface
 * convenience of this library.)
 *   - The workspace is a fixed DSMC_NOALLOC_SCRATCH_BYTES array inside the library, held on
 *     every device that loads the library until the process exits.  A problem whose
 *     workspace (dsmc_workspace_size) is larger returns DSMC_ERR_WORKSPACE and launches
 *     nothing.  The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 *     routine.
 *   - The first call on a device looks up the array's device address (once per device,
 *     with that device current); make that first call before any stream capture.  The
 *     address is kept for the life of the process: it does not survive a reset of the
 *     device (cudaDeviceReset, or a release of its primary context), which unloads the
 *     array; do not call this entry point on a device after resetting it.
 *   - Every call shares the one array and leaves its contents behind; the smoother clears
 *     what must start at zero (its status word) at the start of each call.  Calls whose
 *     work overlaps on the GPU (other streams, other host threads) race on the array:
 *     serialise them.
 *   - The state, y and outputs are the caller's, as for dsmc_smooth.  device_status: HOST
 *     pointer or NULL; if given, the call synchronises `stream` and stores the first device
 *     error of this smoothing (the workspace is not reachable otherwise). */
dsmc_status_t dsmc_smooth_noalloc(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                  const dsmc_proposal_t* prop, const float* y, dsmc_state_t* state,
                                  float* traj_out, double* mean_out, double* m2_out,
                                  double* logL_out, dsmc_status_t* device_status, void* stream);

/* ---- Parallel-in-time Gaussian proposals (Section 4.1, Algorithm 4).  The model is
 * linearised around Gaussian marginals q_t = N(m_t, P_t) and smoothed exactly by the
 * temporally parallel Kalman filter and RTS smoother (prefix scans of an associative
 * operator over the K steps, ceil(log2 K) levels each, FP64 on the device); the smoothed
 * marginals become the next q_t.  For the linear-Gaussian model the linearisation is the
 * model itself and one pass is exact (the Kalman/RTS marginals).  For the stochastic-
 * volatility model, whose observation noise is not additive, each pass expands
 * log h_t(y_t | x) to second order around m_t (a Gaussian pseudo-observation with variance
 * 1 / lambda_t, lambda_t = y_t^2 e^{-m_t} / 2; none where lambda_t vanishes), starting from
 * init_mean or the stationary mean; the iterations move to the posterior mode and its
 * curvature.  The Poisson-count model (Section 5.1) is expanded the same way around m_t
 * (lambda_t = e^{m_t}, pseudo-observation m_t + (y_t - lambda_t) / lambda_t).  The
 * theta-logistic model (Section 5.2) has a linear-Gaussian observation; its transition mean
 * x + tau0 - tau1 e^{tau2 x} is linearised around the previous pass's mean of step t - 1
 * (F_t = 1 - tau1 tau2 e^{tau2 m}, the iterated extended Kalman smoother), the first pass
 * around init_mean or else the observations.  The constrained random walk (Section 5.3) has
 * no Gaussian expansion: DSMC_ERR_UNSUPPORTED.  The outputs are the means and the marginal
 * standard deviations, ready for DSMC_PROP_GAUSS with nu = DSMC_NU_EQ_Q (q_t = nu_t, as the
 * paper uses them).
 *   y:          DEVICE [K][dx] FP32 observations
 *   iterations: passes of the non-linear models (>= 1; the linear-Gaussian model takes one;
 *               the paper runs 25 for a first approximation, then one per parameter update
 *               started from the previous means)
 *   init_mean:  DEVICE [K][dx] FP32 linearisation point of the first pass, or NULL
 *   mean_out, std_out: DEVICE [K][dx] FP32
 *   ws:         DEVICE workspace of dsmc_gaussian_proposals_workspace_size bytes; its first
 *               word is a status word (dsmc_stream_status) recording DSMC_ERR_NONFINITE. */
dsmc_status_t dsmc_gaussian_proposals_workspace_size(const dsmc_model_t* model, int K, size_t* bytes);
dsmc_status_t dsmc_gaussian_proposals(const dsmc_model_t* model, int K, const float* y, int iterations,
                                      const float* init_mean, float* mean_out, float* std_out, void* ws,
                                      size_t ws_bytes, void* stream);

/* Synchronises `stream` and returns in *device_status the first error any kernel recorded
 * in this workspace since the last dsmc_init_particles (DSMC_OK if none). */
dsmc_status_t dsmc_stream_status(void* ws, void* stream, dsmc_status_t* device_status);

/* ---- Batched smoothing: many independent sequences of one model, particle count and
 * precision (one dsmc_config_t; its K and seed are ignored) in one call.  Every sequence has
 * its own length, observations, seed, state and outputs; the combinations of level l of
 * all sequences (Algorithm 6) are launched together, so a level's kernels see the whole
 * batch's work.  Each sequence's result is the one dsmc_smooth (or, with x_ref_in,
 * dsmc_conditional_smooth) gives for it alone with the same seed and counter_base: the
 * draws depend only on (seed, counter_base, combination id within the sequence, slot).
 * The workspace (dsmc_batch_workspace_size) holds the merge workspace, the per-sequence
 * index maps and the batch's descriptor tables. */
typedef struct {
  int K;                   /* steps of this sequence, >= 1 */
  const float* y;          /* DEVICE [K][dx] FP32 */
  const float* prop_mean;  /* DEVICE [K][dx] when the proposal kind is DSMC_PROP_GAUSS, else NULL */
  const float* prop_std;   /* DEVICE [K][dx] */
  dsmc_state_t state;      /* DEVICE buffers sized by dsmc_state_sizes for this K */
  double* mean_out;        /* DEVICE [K][dx] FP64 smoothing means */
  double* m2_out;          /* DEVICE [K][dx] FP64 second moments, or NULL */
  double* logL_out;        /* DEVICE FP64 scalar, or NULL */
  const float* x_ref_in;   /* DEVICE [K][dx]: a conditional (particle-Gibbs) sweep, or NULL */
  float* x_ref_out;        /* DEVICE [K][dx]: the next reference (conditional only; may alias) */
  uint64_t seed;
  uint32_t counter_base;   /* < 2^28 */
  void* maps;              /* DEVICE scratch of dsmc_seq_maps_bytes(K, N) bytes for the sequence's
                              index maps and root draw, or NULL (batched call: kept in its workspace;
                              required by dsmc_serve_tick, where it lives across ticks) */
} dsmc_seq_t;

/* Bytes of a sequence's own index-map scratch (dsmc_seq_t.maps).  Host call. */
size_t dsmc_seq_maps_bytes(int K, int N);

/* Workspace bytes of a batch with sequence lengths K[0..n_seq) (HOST array).  Host call. */
dsmc_status_t dsmc_batch_workspace_size(const dsmc_config_t* cfg, const dsmc_model_t* model, int n_seq,
                                        const int* K, size_t* bytes);

/* Writes the batch's descriptor tables (sequence pointers, seeds, the level-major list of
 * combinations) into the workspace: host-to-device copies on `stream`, then synchronises
 * it.  seqs: HOST array of n_seq. */
dsmc_status_t dsmc_batch_prepare(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                 const dsmc_proposal_t* prop, int n_seq, const dsmc_seq_t* seqs, void* ws,
                                 size_t ws_bytes, void* stream);

/* Launches the whole batched smoothing (init, every level, resolve) on `stream` after
 * dsmc_batch_prepare with the same arguments; asynchronous, no host-device copies or
 * synchronisation, so it can be captured in a CUDA graph and replayed. */
dsmc_status_t dsmc_batch_run(const dsmc_config_t* cfg, const dsmc_model_t* model, const dsmc_proposal_t* prop,
                             int n_seq, const dsmc_seq_t* seqs, void* ws, size_t ws_bytes, void* stream);

/* dsmc_batch_prepare followed by dsmc_batch_run. */
dsmc_status_t dsmc_smooth_batch(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                const dsmc_proposal_t* prop, int n_seq, const dsmc_seq_t* seqs, void* ws,
                                size_t ws_bytes, void* stream);

/* ---- Continuous batching (serving).  A request is a sequence that advances one stage per
 * tick: stage -1 = Algorithm 2, stages 0 .. L-1 = level l of Algorithm 6 (L = ceil(log2 K)),
 * stage L = resolve (outputs written).  dsmc_serve_tick runs, for every sequence of the call,
 * its stage[i] (HOST array), the combinations of all sequences launched together (levels may
 * differ between sequences); sequences may join and leave between ticks.  Every sequence
 * needs its own maps scratch.  A sequence's results equal those of dsmc_smooth (or
 * dsmc_conditional_smooth) for it alone: the draws depend only on its own seed, counter base
 * and combination ids, and whether a level runs fused depends only on that sequence.  The
 * tick uploads its tables (host-to-device copies on `stream`, then synchronises it) and
 * returns with the launches queued.  The status word (dsmc_stream_status on ws) is reset at
 * the start of each tick. */
dsmc_status_t dsmc_serve_workspace_size(const dsmc_config_t* cfg, const dsmc_model_t* model, int max_seq,
                                        int max_combinations, size_t* bytes);

dsmc_status_t dsmc_serve_tick(const dsmc_config_t* cfg, const dsmc_model_t* model, const dsmc_proposal_t* prop,
                              int n_seq, const dsmc_seq_t* seqs, const int* stage, void* ws, size_t ws_bytes,
                              void* stream);

/* ---- Measurement: CUDA-event timing of the fused exp / tile-sum kernel (the N x N part of
 * Algorithm 1), recorded on the stream that kernel runs on. */

/* enable = 1 starts timing the calls made from this host thread (counters reset);
 * enable = 0 stops.  Host call; no device work. */
dsmc_status_t dsmc_profile_enable(int enable);

/* Synchronises the events recorded since dsmc_profile_enable(1) and returns, all HOST:
 *   rowsum_ms        summed device time of the exp / tile-sum launches (ms)
 *   rowsum_launches  their number
 *   rowsum_pairs     pair exponentials they evaluated (sum over launches of merges * N^2)
 *   all_launches     kernel launches of every kind made by the library. */
dsmc_status_t dsmc_profile_read(double* rowsum_ms, int64_t* rowsum_launches, double* rowsum_pairs,
                                int64_t* all_launches);

/* Per-kernel-kind breakdown: when enabled, CUDA events on the launching stream around every
 * launch (of this host thread) of each kind; read returns the summed milliseconds and launch
 * counts per kind, index DSMC_KIND_*, and synchronises those events.  Enabling resets. */
enum {
  DSMC_KIND_INIT = 0,       /* Algorithm 2 */
  DSMC_KIND_PROLOGUE = 1,   /* column / row terms of the split path */
  DSMC_KIND_TILE_SUMS = 2,  /* the N x N exponentials and tile sums (CUDA or tensor cores) */
  DSMC_KIND_DRAWS = 3,      /* row CDF, pair draws and index maps (dense or rejection) */
  DSMC_KIND_FUSED = 4,      /* fused single-launch levels */
  DSMC_KIND_RESOLVE = 5,    /* top-down composition of the pairs */
  DSMC_KIND_GATHER = 6,     /* gather of the trajectories and moments */
  DSMC_KIND_FUSED_TC = 7,   /* fused tensor-core levels (terms, exponentials and draws) */
  DSMC_KINDS = 8
};
dsmc_status_t dsmc_profile_breakdown_enable(int enable);
dsmc_status_t dsmc_profile_breakdown_read(double* ms /* [DSMC_KINDS] */, int64_t* launches /* [DSMC_KINDS] */);

/* Arithmetic unit rates of the current device, for the roofline of the exponential kernels
 * (which are bound by these units, not by HBM): results per second of MUFU ex2.approx,
 * FP32 FFMA, packed FFMA2 (one per instruction lane), FADD and FP64 DFMA (the lazy samplers'
 * row shifts and the per-combination increments are FP64), each the best of three timed
 * launches (CUDA events on `stream`, after one warm-up launch) of eight independent
 * dependency chains per thread, four 256-thread CTAs per SM.  The paper has no counterpart:
 * this is a measurement aid.  sink: DEVICE, one float the kernels may write (they do not for
 * their fixed inputs).  ops_per_s: HOST [5].  Synchronises `stream`. */
dsmc_status_t dsmc_profile_unit_rates(float* sink, double ops_per_s[5], void* stream);

/* ---- Inspection entry points used by the parity tests (same arithmetic as the path). */

/* Test switch for the bounded waits: while enabled, the tensor-core tile-sum launches
 * issue no MMA, so their waits on the accumulators run out after their iteration limit
 * (about a second); the kernel then records DSMC_ERR_TIMEOUT, frees its tensor memory and
 * returns, and the context stays usable.  Off by default; host state of this process. */
dsmc_status_t dsmc_debug_stall_tensor_cores(int enable);

/* Test switch for the inspection entry points: while enabled, the fused tensor-core levels
 * (tc_fused) also store the intermediate weights they otherwise keep in shared memory (row
 * and column terms, tile sums, row weights, prefix sums) in the workspace, where
 * dsmc_debug_merge_weights and dsmc_debug_row_shift read them.  It adds stores only; every
 * result is the same.  Off by default; host state of this process. */
dsmc_status_t dsmc_debug_keep_weights(int enable);

/* Philox4x32-10 of n counters: ctr DEVICE [n][4] uint32, out DEVICE [n][4] uint32. */
dsmc_status_t dsmc_debug_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                                void* stream);

/* After dsmc_merge_level(level), the device's own weights of combination `m` of that
 * level (it must belong to the last launch chunk of the level):
 *   logW   DEVICE [N][N] FP32 or NULL: log-weights log omega + logw_L + logw_R as the
 *          device evaluates them (per-row shift + ln2 * the base-2 exponent);
 *   r      DEVICE [N] FP32 or NULL: row weights of the row stage;
 *   rowsum DEVICE [N] FP32 or NULL: row totals (the sums of each row's tile weights);
 *   tiles  DEVICE [N][n_tiles] FP32 or NULL: tile weights of the tile stage;
 *   e      DEVICE [N][N] FP32 or NULL: element weights of the column stage;
 *   ratio  DEVICE [N][N] FP32 or NULL: rejection acceptance ratios omega / omega-bar;
 *   info   HOST int[4] or NULL: {tile width B, n_tiles, combination id, left block leaf}. */
dsmc_status_t dsmc_debug_merge_weights(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                       int level, int m, float* logW, float* r, float* rowsum,
                                       float* tiles, float* e, float* ratio, int info[4],
                                       void* ws, size_t ws_bytes, void* stream);

/* After dsmc_merge_level(level) with a dense resampler, the per-row scale of the tile and
 * element weights of combination `m` (in the last launch chunk of the level): every weight
 * w of row i stands for exp(shift_i + delta_i ln 2) w, so log of a tile's sum of pair
 * weights (Eq. normalized-weights, unnormalised) is shift_i + delta_i ln 2 + ln t_ik.
 *   shift DEVICE [N] FP64 or NULL; delta DEVICE [N] FP32 or NULL (the extra base-2 shift of
 *   a row recomputed after underflow, else 0). */
dsmc_status_t dsmc_debug_row_shift(const dsmc_config_t* cfg, const dsmc_model_t* model, int level, int m,
                                   double* shift, float* delta, void* ws, size_t ws_bytes, void* stream);

/* After dsmc_merge_level(level) with resampler DSMC_RS_FACTORED, the factorised proposals
 * and acceptance ratios of combination `m` of that level (it must belong to the last launch
 * chunk of the level), as the device evaluated them:
 *   pa   DEVICE [N] FP32 or NULL: row proposal weights e^{a_i - max_i a_i} in [0, 1];
 *   pc   DEVICE [N] FP32 or NULL: column proposal weights e^{c_j - max_j c_j} in [0, 1],
 *        c_j = b'_j (less dist_j^2 / 2Q for dx = 1);
 *   acc  DEVICE [N][N] FP32 or NULL: acceptance ratios f(x_j | x_i) / f_max (times
 *        e^{dist_j^2 / 2Q} for dx = 1);
 *   info HOST int[4] or NULL: {N, 0, combination id, left block leaf}.
 * The proposal draws take trunc(pa 2^40) and trunc(pc 2^40) as exact fixed-point weights. */
dsmc_status_t dsmc_debug_lazy_weights(const dsmc_config_t* cfg, const dsmc_model_t* model, int level, int m,
                                      float* pa, float* pc, float* acc, int info[4], void* ws, size_t ws_bytes,
                                      void* stream);

/* Attempts the rejection samplers (DSMC_RS, DSMC_RS_FACTORED) made in this workspace since
 * the last dsmc_init_particles (or batched / served call): the acceptance rate of a
 * smoothing is the number of drawn slots over this count.  attempts: HOST.  Synchronises
 * `stream`. */
dsmc_status_t dsmc_lazy_attempts(const dsmc_config_t* cfg, const dsmc_model_t* model, void* ws, size_t ws_bytes,
                                 void* stream, uint64_t* attempts);

#ifdef __cplusplus
}
#endif

#endif /* DSMC_H */
