/*
 * dsmc_oracle.c -- plain FP64 CPU oracle of dSMC (de-Sequentialized Monte Carlo,
 * Corenflos, Chopin and Sarkka, arXiv 2202.02264).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs use it.  It shares no code, header or constant table with the CUDA library.
 *
 * What it follows, step by step and in the paper's order:
 *   - Algorithm 2 (smoother initialisation): independent proposals q_t, leaf weights
 *     h_0 P_0 / q_0 at t = 0 and nu_t / q_t for t >= 1, normalisation, L_t = mean weight.
 *   - Appendix A, Algorithm 6 (ParallelReshapeCombination): left-aligned blocks of size
 *     2^l; at level l, block pair (2m, 2m+1) is combined when the right block exists,
 *     otherwise the left block is passed through unchanged.
 *   - Algorithm 1 (Combine) with the product-form weights of Eq. (normalized-weights)
 *     and the stitching weight omega_c = p_c h_c / nu_c of Proposition 2; the
 *     trajectories are copied explicitly, as the two ParFor loops of Algorithm 1 do.
 *   - The normalising-constant increment of Eq. (Lab), weighted form.
 *   - Algorithm 5 (ConditionalCombine) and the star-trajectory draw of Section 3.1.
 *   - Algorithm 8 (rejection-sampling lazy resampling), with (I, J, u) redrawn at every
 *     attempt (standard rejection sampling) and an attempt cap.
 *
 * Readings of the paper this file takes (they are listed with reasons in the design
 * notes): time runs t = 0..K-1; pair index m/i is the left block (time c-1) and n/j the
 * right block (time c); multinomial resampling by inverse CDF on the row-major flattened
 * N x N matrix with one uniform per output slot; conditional slot 0 is the reference
 * trajectory; the next reference comes from one extra pair draw at the root.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11), key = 64-bit seed, counter = (slot, id, purpose | base<<4,
 * j).  The conversions to uniforms are:
 *   u23(w)     = ((w >> 9) + 0.5) * 2^-23        (exact in FP32 and FP64, inside (0, 1))
 *   u53(w0,w1) = (((w0 << 21) | (w1 >> 11)) + 0.5) * 2^-53
 * Normals are Box-Muller pairs from (u23(w0), u23(w1)) and (u23(w2), u23(w3)).
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off -fopenmp (no -ffast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PURPOSE_INIT 1u
#define ORC_PURPOSE_DENSE 2u
#define ORC_PURPOSE_RS 3u
#define ORC_PURPOSE_MH 4u
#define ORC_PURPOSE_SYS 5u
#define ORC_PURPOSE_RSF 6u
#define ORC_PURPOSE_RSU 7u

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_OOM 3
#define ORC_ERR_DEGENERATE 7
#define ORC_ERR_RS_LIMIT 8

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10                                                                          */
/* ------------------------------------------------------------------------------------ */

/* One Philox4x32 round: two 32x32->64 multiplications by the round constants, the high
 * halves xor-ed with the other two words and the round key, the words permuted. */
static void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k0;
  uint32_t n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

/* Ten rounds; the key is bumped by the Weyl constants before every round but the first. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c, k0, k1);
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

/* Many counters at once (for the CPU/GPU stream comparison). ctrs: [n][4], out: [n][4]. */
void orc_philox_many(int64_t n, const uint32_t* ctrs, const uint32_t key[2], uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

static void draw(uint32_t seed_lo, uint32_t seed_hi, uint32_t slot, uint32_t id,
                 uint32_t purpose, uint32_t base, uint32_t j, uint32_t w[4]) {
  uint32_t ctr[4] = {slot, id, purpose | (base << 4), j};
  uint32_t key[2] = {seed_lo, seed_hi};
  orc_philox4x32_10(ctr, key, w);
}

static double u23(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }
static double u53(uint32_t w0, uint32_t w1) {
  uint64_t m = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
  return ((double)m + 0.5) * 0x1p-53;
}

/* ------------------------------------------------------------------------------------ */
/* Model: state-space model of Eq. (ssm) / Feynman-Kac form of Eq. (fk)                   */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int kind; /* 0: linear-Gaussian x_t = A x_{t-1} + N(0,Q), y_t = x_t + N(0,R), x_0 ~ N(m0,P0)
               1: stochastic volatility x_t = mu + phi (x_{t-1} - mu) + sigma e,
                  y_t = exp(x_t / 2) v, x_0 ~ N(mu, sigma^2 / (1 - phi^2)), d = 1
               2: Poisson counts (Section 5.1) x_t = mu + phi (lam x_{t-1} - mu) + sigma e,
                  y_t ~ Poisson(exp(x_t)), x_0 ~ N(mu, sigma^2 / (1 - phi^2)), d = 1
               3: theta-logistic (Section 5.2) x_t = x_{t-1} + tau0 - tau1 exp(tau2 x_{t-1})
                  + sigma e, y_t = x_t + obs_sd v, x_0 ~ N(0, 1), d = 1
               4: constrained random walk (Section 5.3) x_t = x_{t-1} + sigma e, potential
                  1{|x_t| <= bound}, x_0 ~ N(0, 1), d = 1 */
  int d;
  const double *A, *Q, *R, *m0, *P0; /* row-major d x d / d */
  double mu, phi, sigma;
  int prop_kind;     /* 0: q_t = N(y_t, s^2 I);  1: q_t = N(mean_t, diag(std_t^2));
                        2: q_t = U([-s, s]^d) */
  double prop_scale; /* s */
  const double *prop_mean, *prop_std; /* [K][d] when prop_kind == 1 */
  int nu;            /* 0: nu_t = q_t;  1: nu_t proportional to h_t(y_t | .) */
  double lam, tau0, tau1, tau2, obs_sd, bound;
} orc_model;

typedef struct {
  int K, N;
  uint32_t seed_lo, seed_hi, counter_base;
  int resampler; /* 0: multinomial inverse CDF on the full N x N matrix; 1: rejection
                    (Algorithm 8); 2: Metropolis-Hastings (Algorithm 7); 3: systematic
                    inverse CDF on the full matrix (multinomial when conditional);
                    4: rejection with factorised pair proposals */
  uint32_t rs_max_attempts;
  int conditional;
} orc_config;

static const double LOG_2PI = 1.8378770664093454835606594728112;

/* Cholesky factor L (lower) of a d x d SPD matrix; returns 0 on success. */
static int cholesky(int d, const double* S, double* L) {
  memset(L, 0, sizeof(double) * d * d);
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = S[i * d + j];
      for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
      if (i == j) {
        if (!(s > 0.0)) return -1;
        L[i * d + i] = sqrt(s);
      } else {
        L[i * d + j] = s / L[j * d + j];
      }
    }
  }
  return 0;
}

/* log N(x; m, L L^T) by forward substitution. */
static double gauss_logpdf_chol(int d, const double* x, const double* m, const double* L) {
  double z[64];
  double quad = 0.0, logdet = 0.0;
  for (int i = 0; i < d; ++i) {
    double s = x[i] - m[i];
    for (int k = 0; k < i; ++k) s -= L[i * d + k] * z[k];
    z[i] = s / L[i * d + i];
    quad += z[i] * z[i];
    logdet += log(L[i * d + i]);
  }
  return -0.5 * quad - logdet - 0.5 * d * LOG_2PI;
}

static double normal_logpdf(double x, double m, double s) {
  double z = (x - m) / s;
  return -0.5 * z * z - log(s) - 0.5 * LOG_2PI;
}

typedef struct {
  const orc_model* m;
  int K;
  const double* y; /* [K][d] */
  double LQ[32 * 32], LR[32 * 32], LP0[32 * 32];
} model_ctx;

static int ctx_init(model_ctx* c, const orc_model* m, int K, const double* y) {
  c->m = m;
  c->K = K;
  c->y = y;
  if (m->d < 1 || m->d > 32) return ORC_ERR_INVALID;
  if (m->kind == 0) {
    if (cholesky(m->d, m->Q, c->LQ) || cholesky(m->d, m->R, c->LR) || cholesky(m->d, m->P0, c->LP0))
      return ORC_ERR_INVALID;
  } else if (m->kind == 1 || m->kind == 2) {
    if (m->d != 1 || !(m->sigma > 0.0) || !(fabs(m->phi) < 1.0)) return ORC_ERR_INVALID;
  } else if (m->kind == 3) {
    if (m->d != 1 || !(m->sigma > 0.0) || !(m->obs_sd > 0.0)) return ORC_ERR_INVALID;
  } else if (m->kind == 4) {
    if (m->d != 1 || !(m->sigma > 0.0) || !(m->bound > 0.0)) return ORC_ERR_INVALID;
  } else {
    return ORC_ERR_INVALID;
  }
  return ORC_OK;
}

/* The transition mean m(x) of a one-dimensional model kind (1..4). */
static double trans_mean_1d(const orc_model* m, double x) {
  switch (m->kind) {
    case 1: return m->mu + m->phi * (x - m->mu);
    case 2: return m->mu + m->phi * (m->lam * x - m->mu);
    case 3: return x + m->tau0 - m->tau1 * exp(m->tau2 * x);
    default: return x;
  }
}

/* log p_t(x' | x): transition density P_t of Eq. (ssm). */
static double log_f(const model_ctx* c, const double* x, const double* xn) {
  const orc_model* m = c->m;
  if (m->kind == 0) {
    double mean[32];
    for (int i = 0; i < m->d; ++i) {
      double s = 0.0;
      for (int k = 0; k < m->d; ++k) s += m->A[i * m->d + k] * x[k];
      mean[i] = s;
    }
    return gauss_logpdf_chol(m->d, xn, mean, c->LQ);
  }
  return normal_logpdf(xn[0], trans_mean_1d(m, x[0]), m->sigma);
}

/* sup over (x, x') of log p_t(x' | x): the Gaussian density at its mode. */
static double log_f_max(const model_ctx* c) {
  const orc_model* m = c->m;
  if (m->kind == 0) {
    double logdet = 0.0;
    for (int i = 0; i < m->d; ++i) logdet += log(c->LQ[i * m->d + i]);
    return -logdet - 0.5 * m->d * LOG_2PI;
  }
  return -log(m->sigma) - 0.5 * LOG_2PI;
}

/* log h_t(y_t | x): observation density. */
static double log_h(const model_ctx* c, int t, const double* x) {
  const orc_model* m = c->m;
  const double* yt = c->y + (size_t)t * m->d;
  if (m->kind == 0) return gauss_logpdf_chol(m->d, yt, x, c->LR);
  if (m->kind == 2) return yt[0] * x[0] - exp(x[0]) - lgamma(yt[0] + 1.0);  /* Poisson(exp(x)) */
  if (m->kind == 3) return normal_logpdf(yt[0], x[0], m->obs_sd);
  if (m->kind == 4) return fabs(x[0]) <= m->bound ? 0.0 : -INFINITY;
  /* y | x ~ N(0, exp(x)) */
  return -0.5 * LOG_2PI - 0.5 * x[0] - 0.5 * yt[0] * yt[0] * exp(-x[0]);
}

/* log P_0(x): prior of x_0. */
static double log_p0(const model_ctx* c, const double* x) {
  const orc_model* m = c->m;
  if (m->kind == 0) return gauss_logpdf_chol(m->d, x, m->m0, c->LP0);
  if (m->kind == 3 || m->kind == 4) return normal_logpdf(x[0], 0.0, 1.0);
  double s0 = m->sigma / sqrt(1.0 - m->phi * m->phi);
  return normal_logpdf(x[0], m->mu, s0);
}

static void prop_params(const model_ctx* c, int t, int i, double* mean, double* sd) {
  const orc_model* m = c->m;
  if (m->prop_kind == 0) {
    *mean = c->y[(size_t)t * m->d + i];
    *sd = m->prop_scale;
  } else {
    *mean = m->prop_mean[(size_t)t * m->d + i];
    *sd = m->prop_std[(size_t)t * m->d + i];
  }
}

/* log q_t(x): independent diagonal-Gaussian proposal, or the uniform one on [-s, s]^d. */
static double log_q(const model_ctx* c, int t, const double* x) {
  if (c->m->prop_kind == 2) {
    for (int i = 0; i < c->m->d; ++i)
      if (fabs(x[i]) > c->m->prop_scale) return -INFINITY;
    return -c->m->d * log(2.0 * c->m->prop_scale);
  }
  double s = 0.0;
  for (int i = 0; i < c->m->d; ++i) {
    double mu, sd;
    prop_params(c, t, i, &mu, &sd);
    s += normal_logpdf(x[i], mu, sd);
  }
  return s;
}

/* log nu_t(x) for t >= 1 (Definition 1): either q_t itself, or h_t(y_t | .) normalised
 * over x.  For the linear-Gaussian model with identity observation matrix the latter is
 * N(x; y_t, R); for the stochastic-volatility model the integral of h_t over x is 1/|y_t|. */
static double log_nu(const model_ctx* c, int t, const double* x) {
  const orc_model* m = c->m;
  if (m->nu == 0) return log_q(c, t, x);
  if (m->kind == 0 || m->kind == 3) return log_h(c, t, x);
  if (m->kind == 4) return log_h(c, t, x) - log(2.0 * m->bound);
  return log_h(c, t, x) + log(fabs(c->y[t]));
}

/* log omega_c(x_{c-1}, x_c) = log p_c(x_c | x_{c-1}) + log h_c(x_c) - log nu_c(x_c)
 * (Proposition 2, Eq. weights-formula). */
static double log_omega(const model_ctx* c, int tc, const double* xprev, const double* xcur) {
  return log_f(c, xprev, xcur) + log_h(c, tc, xcur) - log_nu(c, tc, xcur);
}

/* Box-Muller normals for particle (t, n): dims 4j..4j+3 come from the counter j. */
static void draw_particle(const orc_config* cf, int d, int t, int n, double* z) {
  for (int j = 0; 4 * j < d; ++j) {
    uint32_t w[4];
    draw(cf->seed_lo, cf->seed_hi, (uint32_t)n, (uint32_t)t, ORC_PURPOSE_INIT, cf->counter_base,
         (uint32_t)j, w);
    for (int p = 0; p < 2; ++p) {
      double u1 = u23(w[2 * p]), u2 = u23(w[2 * p + 1]);
      double r = sqrt(-2.0 * log(u1));
      double th = 6.283185307179586476925286766559 * u2;
      int k0 = 4 * j + 2 * p;
      if (k0 < d) z[k0] = r * cos(th);
      if (k0 + 1 < d) z[k0 + 1] = r * sin(th);
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 2: smoother initialisation                                                  */
/* ------------------------------------------------------------------------------------ */

/* X: [K][N][d]; logw: [K][N] normalised log-weights; logL: [K] log L_t.
 * x_ref (conditional mode, Section 3.2): slot 0 at every t is x_ref[t], weighted like the
 * others.  Returns ORC_OK or an error code. */
int orc_init(const orc_model* m, const orc_config* cf, const double* y, const double* x_ref,
             double* X, double* logw, double* logL) {
  model_ctx c;
  int st = ctx_init(&c, m, cf->K, y);
  if (st) return st;
  const int K = cf->K, N = cf->N, d = m->d;
#pragma omp parallel for schedule(static)
  for (int t = 0; t < K; ++t) {
    double* lw = logw + (size_t)t * N;
    for (int n = 0; n < N; ++n) {
      double* x = X + ((size_t)t * N + n) * d;
      if (cf->conditional && n == 0) {
        for (int i = 0; i < d; ++i) x[i] = x_ref[(size_t)t * d + i];
      } else if (m->prop_kind == 2) {  /* U([-s, s]^d): x = s (2 u - 1), u23 of the words */
        for (int j = 0; 4 * j < d; ++j) {
          uint32_t w[4];
          draw(cf->seed_lo, cf->seed_hi, (uint32_t)n, (uint32_t)t, ORC_PURPOSE_INIT, cf->counter_base, (uint32_t)j,
               w);
          for (int p = 0; p < 4 && 4 * j + p < d; ++p) x[4 * j + p] = m->prop_scale * (2.0 * u23(w[p]) - 1.0);
        }
      } else {
        double z[32];
        draw_particle(cf, d, t, n, z);
        for (int i = 0; i < d; ++i) {
          double mu, sd;
          prop_params(&c, t, i, &mu, &sd);
          x[i] = mu + sd * z[i];
        }
      }
      if (t == 0)
        lw[n] = log_h(&c, 0, x) + log_p0(&c, x) - log_q(&c, 0, x);
      else
        lw[n] = log_nu(&c, t, x) - log_q(&c, t, x);
    }
    double mx = -INFINITY;
    for (int n = 0; n < N; ++n) mx = lw[n] > mx ? lw[n] : mx;
    double s = 0.0;
    for (int n = 0; n < N; ++n) s += exp(lw[n] - mx);
    double lse = mx + log(s);
    for (int n = 0; n < N; ++n) lw[n] -= lse;
    logL[t] = lse - log((double)N);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 6 schedule                                                                   */
/* ------------------------------------------------------------------------------------ */

int orc_num_levels(int K) {
  int L = 0;
  while ((1 << L) < K) ++L;
  return L;
}

/* Number of combinations at level l: block pairs (2m, 2m+1) of size 2^l whose right block
 * starts before K. */
int orc_merges_at_level(int K, int l) {
  int64_t size = (int64_t)1 << l;
  if (size >= K) return 0;
  return (int)((K - size + 2 * size - 1) / (2 * size));
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1 / 5 / 8                                                                    */
/* ------------------------------------------------------------------------------------ */

/* Draw one pair from the N x N weights by inverse CDF on the row-major flattened matrix:
 * the first flat index whose inclusive cumulative sum exceeds u * S. */
static int64_t inverse_cdf(const double* C, const double* E, int64_t n, double u) {
  double target = u * C[n - 1];
  int64_t lo = 0, hi = n; /* first index with C > target */
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (C[mid] > target) hi = mid; else lo = mid + 1;
  }
  if (lo >= n) { /* rounding pushed the target past the total: last positive entry */
    lo = n - 1;
    while (lo > 0 && !(E[lo] > 0.0)) --lo;
  }
  return lo;
}

/* Multinomial pair draws for slots [n0, n1): one u53 uniform per slot from the counter
 * (n, gid, DENSE | base<<4, 0), inverse CDF over the row-major flattened matrix.
 * E: [N*N] nonnegative weights, C: their inclusive cumulative sums. */
static void dense_draws(int N, const double* E, const double* C, uint32_t seed_lo,
                        uint32_t seed_hi, uint32_t base, uint32_t gid, int n0, int n1,
                        int32_t* li, int32_t* ri) {
  int64_t NN = (int64_t)N * N;
  for (int n = n0; n < n1; ++n) {
    uint32_t w[4];
    draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_DENSE, base, 0u, w);
    int64_t f = inverse_cdf(C, E, NN, u53(w[0], w[1]));
    li[n - n0] = (int32_t)(f / N);
    ri[n - n0] = (int32_t)(f % N);
  }
}

/* Systematic pair draws for slots [n0, n1) (Algorithm 1 names systematic resampling beside
 * multinomial): one uniform U per combination, u53 of the counter (0, gid, SYS | base<<4, 0),
 * and slot k takes the positions (k + U) / N of the row-major flattened matrix's CDF. */
static void systematic_draws(int N, const double* E, const double* C, uint32_t seed_lo,
                             uint32_t seed_hi, uint32_t base, uint32_t gid, int n0, int n1,
                             int32_t* li, int32_t* ri) {
  int64_t NN = (int64_t)N * N;
  uint32_t w[4];
  draw(seed_lo, seed_hi, 0u, gid, ORC_PURPOSE_SYS, base, 0u, w);
  const double U = u53(w[0], w[1]);
  for (int n = n0; n < n1; ++n) {
    int64_t f = inverse_cdf(C, E, NN, ((double)n + U) / (double)N);
    li[n - n0] = (int32_t)(f / N);
    ri[n - n0] = (int32_t)(f % N);
  }
}

/* Rejection draws (Algorithm 8) for slots [n0, n1) given the log-weights logW[i][j] and a
 * bound logbar >= max logW: per attempt (I, J, u) = (w0 N >> 32, w1 N >> 32, u23(w2)) from
 * the counter (n, gid, RS | base<<4, attempt); accept when u < exp(logW_IJ - logbar).
 * logW is evaluated through the callback so that the N x N matrix need not exist. */
typedef double (*pair_logw_fn)(const void* ctx, int i, int j);
static int rs_draws(int N, pair_logw_fn fn, const void* ctx, double logbar, uint32_t seed_lo,
                    uint32_t seed_hi, uint32_t base, uint32_t gid, int n0, int n1,
                    uint32_t max_attempts, int32_t* li, int32_t* ri, uint64_t* attempts) {
  int status = ORC_OK;
  for (int n = n0; n < n1; ++n) {
    uint32_t att;
    int I = 0, J = 0, ok = 0;
    for (att = 0; att < max_attempts; ++att) {
      uint32_t w[4];
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RS, base, att, w);
      I = (int)(((uint64_t)w[0] * (uint64_t)N) >> 32);
      J = (int)(((uint64_t)w[1] * (uint64_t)N) >> 32);
      double u = u23(w[2]);
      if (u < exp(fn(ctx, I, J) - logbar)) { ok = 1; ++att; break; }
    }
    if (!ok) status = ORC_ERR_RS_LIMIT;
    if (attempts) *attempts += att;
    li[n - n0] = I;
    ri[n - n0] = J;
  }
  return status;
}

/* Rejection draws with factorised pair proposals (the future-work item of the paper's
 * discussion: propose pairs by their a-priori weights).  The target log-weight of a pair is
 * la[i] + lc[j] + lacc(i, j) with lacc <= 0; the proposal draws I with probability
 * proportional to exp(la[i]) and J proportional to exp(lc[j]), independently, by inverse CDF
 * on u53 uniforms of the counter (n, gid, RSF | base<<4, attempt) (words 0-1 for I, 2-3 for
 * J), and accepts when u < exp(lacc(I, J)), u = u23 of word 0 of the counter
 * (n, gid, RSU | base<<4, attempt).  Accepted pairs follow the target exactly; the expected
 * number of attempts is sum_i e^la_i sum_j e^lc_j / sum_ij e^(la_i + lc_j + lacc_ij). */
static int rsf_draws(int N, const double* la, const double* lc, pair_logw_fn lacc, const void* ctx,
                     uint32_t seed_lo, uint32_t seed_hi, uint32_t base, uint32_t gid, int n0, int n1,
                     uint32_t max_attempts, int32_t* li, int32_t* ri, uint64_t* attempts) {
  double *EA = (double*)malloc(sizeof(double) * N), *CA = (double*)malloc(sizeof(double) * N);
  double *EC = (double*)malloc(sizeof(double) * N), *CC = (double*)malloc(sizeof(double) * N);
  if (!EA || !CA || !EC || !CC) { free(EA); free(CA); free(EC); free(CC); return ORC_ERR_OOM; }
  double ma = -INFINITY, mc = -INFINITY, sa = 0.0, sc = 0.0;
  for (int i = 0; i < N; ++i) ma = la[i] > ma ? la[i] : ma;
  for (int j = 0; j < N; ++j) mc = lc[j] > mc ? lc[j] : mc;
  for (int i = 0; i < N; ++i) { EA[i] = exp(la[i] - ma); sa += EA[i]; CA[i] = sa; }
  for (int j = 0; j < N; ++j) { EC[j] = exp(lc[j] - mc); sc += EC[j]; CC[j] = sc; }
  int status = ORC_OK;
  for (int n = n0; n < n1; ++n) {
    uint32_t att;
    int I = 0, J = 0, ok = 0;
    for (att = 0; att < max_attempts; ++att) {
      uint32_t w[4], v[4];
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RSF, base, att, w);
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RSU, base, att, v);
      I = (int)inverse_cdf(CA, EA, N, u53(w[0], w[1]));
      J = (int)inverse_cdf(CC, EC, N, u53(w[2], w[3]));
      if (u23(v[0]) < exp(lacc(ctx, I, J))) { ok = 1; ++att; break; }
    }
    if (!ok) status = ORC_ERR_RS_LIMIT;
    if (attempts) *attempts += att;
    li[n - n0] = I;
    ri[n - n0] = J;
  }
  free(EA); free(CA); free(EC); free(CC);
  return status;
}

typedef struct {
  const model_ctx* mc;
  const double *Zl, *Zr, *wl, *bcol;
  int d;
} rs_ctx;

static double rs_model_logw(const void* p, int i, int j) {
  const rs_ctx* r = (const rs_ctx*)p;
  return log_f(r->mc, r->Zl + (size_t)i * r->d, r->Zr + (size_t)j * r->d) + r->wl[i] + r->bcol[j];
}

typedef struct {
  const double* W;
  int N;
} mat_ctx;

static double mat_logw(const void* p, int i, int j) {
  const mat_ctx* m = (const mat_ctx*)p;
  return m->W[(size_t)i * m->N + j];
}

/* The factorised sampler's log acceptance for the model: log p_c(xr_J | xl_I) - log f_max,
 * plus dist_J^2 / 2Q for one-dimensional states (the column factor took the hull term out). */
typedef struct {
  const model_ctx* mc;
  const double *Zl, *Zr, *dist;
  double lfmax, halfQi;
  int d;
} rsf_ctx;

static double rsf_model_lacc(const void* p, int i, int j) {
  const rsf_ctx* r = (const rsf_ctx*)p;
  double v = log_f(r->mc, r->Zl + (size_t)i * r->d, r->Zr + (size_t)j * r->d) - r->lfmax;
  if (r->dist) v += r->halfQi * r->dist[j] * r->dist[j];
  return v;
}

/* Exported for the sampler tests: factorised-proposal rejection draws for slots [n0, n1)
 * from row and column log-weights la, lc [N] and log acceptances lacc [N][N] (<= 0). */
int orc_rsf_pairs(int N, const double* la, const double* lc, const double* lacc, uint32_t seed_lo,
                  uint32_t seed_hi, uint32_t base, uint32_t gid, int n0, int n1, uint32_t max_attempts,
                  int32_t* li, int32_t* ri, uint64_t* attempts) {
  mat_ctx m = {lacc, N};
  return rsf_draws(N, la, lc, mat_logw, &m, seed_lo, seed_hi, base, gid, n0, n1, max_attempts, li, ri,
                   attempts);
}

/* Exported for the sampler tests: systematic draws from a given FP64 log-weight matrix. */
int orc_sys_pairs(int N, const double* logW, uint32_t seed_lo, uint32_t seed_hi, uint32_t base,
                  uint32_t gid, int n0, int n1, int32_t* li, int32_t* ri) {
  int64_t NN = (int64_t)N * N;
  double* E = (double*)malloc(sizeof(double) * NN);
  double* C = (double*)malloc(sizeof(double) * NN);
  if (!E || !C) { free(E); free(C); return ORC_ERR_OOM; }
  double M = -INFINITY;
  for (int64_t f = 0; f < NN; ++f) M = logW[f] > M ? logW[f] : M;
  double S = 0.0;
  for (int64_t f = 0; f < NN; ++f) { E[f] = exp(logW[f] - M); S += E[f]; C[f] = S; }
  systematic_draws(N, E, C, seed_lo, seed_hi, base, gid, n0, n1, li, ri);
  free(E);
  free(C);
  return ORC_OK;
}

/* Exported for the sampler tests: dense multinomial draws from a given FP64 log-weight
 * matrix (the same code path Combine uses). */
int orc_dense_pairs(int N, const double* logW, uint32_t seed_lo, uint32_t seed_hi, uint32_t base,
                    uint32_t gid, int n0, int n1, int32_t* li, int32_t* ri) {
  int64_t NN = (int64_t)N * N;
  double* E = (double*)malloc(sizeof(double) * NN);
  double* C = (double*)malloc(sizeof(double) * NN);
  if (!E || !C) { free(E); free(C); return ORC_ERR_OOM; }
  double M = -INFINITY;
  for (int64_t f = 0; f < NN; ++f) M = logW[f] > M ? logW[f] : M;
  double S = 0.0;
  for (int64_t f = 0; f < NN; ++f) { E[f] = exp(logW[f] - M); S += E[f]; C[f] = S; }
  dense_draws(N, E, C, seed_lo, seed_hi, base, gid, n0, n1, li, ri);
  free(E);
  free(C);
  return ORC_OK;
}

/* Exported for the sampler tests: rejection draws from a given FP64 log-weight matrix. */
int orc_rs_pairs(int N, const double* logW, double logbar, uint32_t seed_lo, uint32_t seed_hi,
                 uint32_t base, uint32_t gid, int n0, int n1, uint32_t max_attempts, int32_t* li,
                 int32_t* ri, uint64_t* attempts) {
  mat_ctx m = {logW, N};
  return rs_draws(N, mat_logw, &m, logbar, seed_lo, seed_hi, base, gid, n0, n1, max_attempts, li,
                  ri, attempts);
}

/* Algorithm 7 (Metropolis-Hastings lazy resampling), FP64, on a pair log-weight
 * evaluator: slot n starts at (n mod N, n mod N); at step b it draws (slot n, combination
 * gid, purpose MH, counter base, b): I* = floor(w0 N / 2^32), J* = floor(w1 N / 2^32),
 * u = u23(w2), and moves to (I*, J*) when u < omega(I*, J*) / omega(I, J), here
 * exp(logW* - logW) (a current weight of zero accepts any proposal of positive weight).
 * The target includes both leaf weights (the log-weights of Eq. normalized-weights).  After
 * B steps the pair is the slot's draw. */
static void mh_draws(int N, pair_logw_fn fn, const void* ctx, uint32_t seed_lo, uint32_t seed_hi,
                     uint32_t base, uint32_t gid, int n0, int n1, uint32_t B, int32_t* li,
                     int32_t* ri) {
  for (int n = n0; n < n1; ++n) {
    int I = n % N, J = n % N;
    double cur = fn(ctx, I, J);
    for (uint32_t b = 0; b < B; ++b) {
      uint32_t w[4];
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_MH, base, b, w);
      const int Is = (int)(((uint64_t)w[0] * (uint64_t)N) >> 32);
      const int Js = (int)(((uint64_t)w[1] * (uint64_t)N) >> 32);
      const double prop = fn(ctx, Is, Js);
      const double u = u23(w[2]);
      const int accept = (cur == -INFINITY) ? (prop > -INFINITY) : (u < exp(prop - cur));
      if (accept) {
        I = Is;
        J = Js;
        cur = prop;
      }
    }
    li[n - n0] = I;
    ri[n - n0] = J;
  }
}

/* Algorithm 7 on a given log-weight matrix [N][N]. */
int orc_mh_pairs(int N, const double* logW, uint32_t seed_lo, uint32_t seed_hi, uint32_t base,
                 uint32_t gid, int n0, int n1, uint32_t B, int32_t* li, int32_t* ri) {
  mat_ctx m = {logW, N};
  mh_draws(N, mat_logw, &m, seed_lo, seed_hi, base, gid, n0, n1, B, li, ri);
  return ORC_OK;
}

/* The same chain on the device's own FP32 weight ratios r = omega / omega-bar [N][N]: the
 * move is taken iff u r(I, J) < r(I*, J*) in FP32 (one rounding of the product), the form
 * the device evaluates. */
int orc_kp_mh_pairs(int N, const float* ratio, uint32_t seed_lo, uint32_t seed_hi, uint32_t base,
                    uint32_t gid, int n0, int n1, uint32_t B, int32_t* li, int32_t* ri) {
  for (int n = n0; n < n1; ++n) {
    int I = n % N, J = n % N;
    float cur = ratio[(size_t)I * N + J];
    for (uint32_t b = 0; b < B; ++b) {
      uint32_t w[4];
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_MH, base, b, w);
      const int Is = (int)(((uint64_t)w[0] * (uint64_t)N) >> 32);
      const int Js = (int)(((uint64_t)w[1] * (uint64_t)N) >> 32);
      const float prop = ratio[(size_t)Is * N + Js];
      const float u = (float)u23(w[2]);
      const float lhs = u * cur;
      if (lhs < prop) {
        I = Is;
        J = Js;
        cur = prop;
      }
    }
    li[n - n0] = I;
    ri[n - n0] = J;
  }
  return ORC_OK;
}

typedef struct {
  double* Z;       /* [K][N][d]: value at time t of trajectory n of the block holding t */
  double* logw;    /* [K][N]: block weights, stored at the block's start time */
  double* logL;    /* [K]: block log normalising constant, at the block's start time */
} blocks;

/* Combine left block [a, c-1] with right block [c, b] (Algorithm 1, or Algorithm 5 when
 * conditional).  pairs: [2][N] output (l_n, r_n).  star: if non-NULL ([K][d]), one extra
 * draw (I*, J*) from the same W, at slot N, gives the next reference trajectory
 * [left trajectory I*, right trajectory J*] (Section 3.1), read before the copy. */
static int combine(const model_ctx* mc, const orc_config* cf, blocks* B, int a, int c, int b,
                   int gid, int32_t* pairs, double* star, uint64_t* attempts) {
  const int N = cf->N, d = mc->m->d;
  const double* wl = B->logw + (size_t)a * N;
  const double* wr = B->logw + (size_t)c * N;
  int status = ORC_OK;
  int n0 = cf->conditional ? 1 : 0;
  int nslots = N + (star ? 1 : 0);
  int32_t* li = (int32_t*)malloc(sizeof(int32_t) * nslots);
  int32_t* ri = (int32_t*)malloc(sizeof(int32_t) * nslots);
  double inc;
  if (!li || !ri) { free(li); free(ri); return ORC_ERR_OOM; }

  if (cf->resampler == 0 || cf->resampler == 3) {
    int64_t NN = (int64_t)N * N;
    double* W = (double*)malloc(sizeof(double) * NN);
    double* C = (double*)malloc(sizeof(double) * NN);
    if (!W || !C) { free(W); free(C); free(li); free(ri); return ORC_ERR_OOM; }
    double M = -INFINITY;
    for (int i = 0; i < N; ++i) {
      const double* xl = B->Z + ((size_t)(c - 1) * N + i) * d;
      for (int j = 0; j < N; ++j) {
        const double* xr = B->Z + ((size_t)c * N + j) * d;
        double v = log_omega(mc, c, xl, xr) + wl[i] + wr[j];
        W[(int64_t)i * N + j] = v;
        if (v > M) M = v;
      }
    }
    if (!(M > -INFINITY) || isnan(M)) {
      free(W); free(C); free(li); free(ri);
      return ORC_ERR_DEGENERATE;
    }
    double S = 0.0;
    for (int64_t f = 0; f < NN; ++f) {
      W[f] = exp(W[f] - M);
      S += W[f];
      C[f] = S;
    }
    inc = M + log(S);
    if (cf->resampler == 3 && !cf->conditional)  /* conditional combinations stay multinomial */
      systematic_draws(N, W, C, cf->seed_lo, cf->seed_hi, cf->counter_base, (uint32_t)gid, n0, nslots,
                       li + n0, ri + n0);
    else
      dense_draws(N, W, C, cf->seed_lo, cf->seed_hi, cf->counter_base, (uint32_t)gid, n0, nslots,
                  li + n0, ri + n0);
    free(W);
    free(C);
  } else {
    /* the lazy samplers: only the proposed pairs' weights are evaluated.  Algorithm 8 with
     * the finite-set bound log wbar = log f_max + max_i a_i + max_j b'_j, or Algorithm 7
     * (B = rs_max_attempts Metropolis-Hastings steps; 0 means 64);
     * b'_j = logw_R[j] + log h_c - log nu_c. */
    double amax = -INFINITY, bmax = -INFINITY;
    double* bcol = (double*)malloc(sizeof(double) * N);
    if (!bcol) { free(li); free(ri); return ORC_ERR_OOM; }
    for (int i = 0; i < N; ++i) amax = wl[i] > amax ? wl[i] : amax;
    for (int j = 0; j < N; ++j) {
      const double* xr = B->Z + ((size_t)c * N + j) * d;
      bcol[j] = wr[j] + log_h(mc, c, xr) - log_nu(mc, c, xr);
      bmax = bcol[j] > bmax ? bcol[j] : bmax;
    }
    double logbar = log_f_max(mc) + amax + bmax;
    rs_ctx rc = {mc, B->Z + (size_t)(c - 1) * N * d, B->Z + (size_t)c * N * d, wl, bcol, d};
    if (cf->resampler == 4) {
      /* factorised proposals: rows by the left weights, columns by b'_j (for d = 1 less
       * dist_j^2 / 2Q, dist_j the distance from xr_j to the hull of the transition means of
       * the left block's end states), acceptance f / f_max (times e^{dist_j^2 / 2Q}) */
      double* lc = (double*)malloc(sizeof(double) * N);
      double* dist = d == 1 ? (double*)malloc(sizeof(double) * N) : NULL;
      if (!lc || (d == 1 && !dist)) { free(lc); free(dist); free(bcol); free(li); free(ri); return ORC_ERR_OOM; }
      double halfQi = 0.0;
      if (d == 1) {
        const orc_model* m = mc->m;
        const double Q = m->kind == 0 ? m->Q[0] : m->sigma * m->sigma;
        halfQi = 0.5 / Q;
        double lo = INFINITY, hi = -INFINITY;
        for (int i = 0; i < N; ++i) {
          const double xi = B->Z[(size_t)(c - 1) * N + i];
          const double mi = m->kind == 0 ? m->A[0] * xi : trans_mean_1d(m, xi);
          lo = mi < lo ? mi : lo;
          hi = mi > hi ? mi : hi;
        }
        for (int j = 0; j < N; ++j) {
          const double x = B->Z[(size_t)c * N + j];
          dist[j] = x > hi ? x - hi : (x < lo ? lo - x : 0.0);
        }
      }
      for (int j = 0; j < N; ++j) lc[j] = bcol[j] - (d == 1 ? halfQi * dist[j] * dist[j] : 0.0);
      rsf_ctx fc = {mc, B->Z + (size_t)(c - 1) * N * d, B->Z + (size_t)c * N * d, dist, log_f_max(mc), halfQi, d};
      status = rsf_draws(N, wl, lc, rsf_model_lacc, &fc, cf->seed_lo, cf->seed_hi, cf->counter_base,
                         (uint32_t)gid, n0, nslots, cf->rs_max_attempts, li + n0, ri + n0, attempts);
      free(lc);
      free(dist);
    } else if (cf->resampler == 2)
      mh_draws(N, rs_model_logw, &rc, cf->seed_lo, cf->seed_hi, cf->counter_base, (uint32_t)gid, n0,
               nslots, cf->rs_max_attempts ? cf->rs_max_attempts : 64u, li + n0, ri + n0);
    else
      status = rs_draws(N, rs_model_logw, &rc, logbar, cf->seed_lo, cf->seed_hi, cf->counter_base,
                        (uint32_t)gid, n0, nslots, cf->rs_max_attempts, li + n0, ri + n0, attempts);
    free(bcol);
    /* the increment still needs the full weighted sum (Eq. Lab) */
    double M = -INFINITY;
    double* row = (double*)malloc(sizeof(double) * N);
    if (!row) { free(li); free(ri); return ORC_ERR_OOM; }
    double S = 0.0;
    for (int i = 0; i < N; ++i) {
      const double* xl = B->Z + ((size_t)(c - 1) * N + i) * d;
      for (int j = 0; j < N; ++j) {
        const double* xr = B->Z + ((size_t)c * N + j) * d;
        row[j] = log_omega(mc, c, xl, xr) + wl[i] + wr[j];
      }
      for (int j = 0; j < N; ++j) {
        if (row[j] > M) { S *= exp(M - row[j]); M = row[j]; }
        S += exp(row[j] - M);
      }
    }
    free(row);
    inc = M + log(S);
  }
  if (cf->conditional) {
    li[0] = 0;
    ri[0] = 0;
  }
  for (int n = 0; n < N; ++n) {
    pairs[n] = li[n];
    pairs[N + n] = ri[n];
  }
  if (star) {
    for (int t = a; t <= b; ++t) {
      int src = t < c ? li[N] : ri[N];
      for (int k = 0; k < d; ++k) star[(size_t)t * d + k] = B->Z[((size_t)t * N + src) * d + k];
    }
  }

  /* the two copy loops of Algorithm 1 */
  double* tmp = (double*)malloc(sizeof(double) * (size_t)N * d);
  if (!tmp) { free(li); free(ri); return ORC_ERR_OOM; }
  for (int t = a; t <= b; ++t) {
    const int32_t* src = t < c ? li : ri;
    double* Zt = B->Z + (size_t)t * N * d;
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < d; ++k) tmp[(size_t)n * d + k] = Zt[(size_t)src[n] * d + k];
    memcpy(Zt, tmp, sizeof(double) * (size_t)N * d);
  }
  free(tmp);
  double* lwa = B->logw + (size_t)a * N;
  for (int n = 0; n < N; ++n) lwa[n] = -log((double)N);
  B->logL[a] = B->logL[a] + B->logL[c] + inc;
  free(li);
  free(ri);
  return status;
}

/* Full dSMC smoother (Algorithm 2 followed by Algorithm 6 with Combine / ConditionalCombine).
 *   y        [K][d]
 *   x_ref    [K][d] or NULL (required when cf->conditional)
 *   X_leaf   [K][N][d] or NULL: the Algorithm 2 particles
 *   pairs    [K-1][2][N] or NULL: (l_n, r_n) of every combination, level-major order
 *   traj     [K][N][d] or NULL: the N output trajectories
 *   mean     [K][d]: smoothing means (weighted by the root weights)
 *   m2       [K][d] or NULL: smoothing second moments
 *   logL     scalar: log of the normalising-constant estimate
 *   x_star   [K][d] or NULL: conditional mode, the next reference trajectory
 *   rs_attempts: total rejection-sampling attempts (may be NULL) */
int orc_smooth(const orc_model* m, const orc_config* cf, const double* y, const double* x_ref,
               double* X_leaf, int32_t* pairs, double* traj, double* mean, double* m2,
               double* logL, double* x_star, uint64_t* rs_attempts) {
  model_ctx mc;
  int st = ctx_init(&mc, m, cf->K, y);
  if (st) return st;
  const int K = cf->K, N = cf->N, d = m->d;
  if (K < 1 || N < 1 || (cf->conditional && (!x_ref || N < 2))) return ORC_ERR_INVALID;
  blocks B;
  B.Z = (double*)malloc(sizeof(double) * (size_t)K * N * d);
  B.logw = (double*)malloc(sizeof(double) * (size_t)K * N);
  B.logL = (double*)malloc(sizeof(double) * (size_t)K);
  if (!B.Z || !B.logw || !B.logL) { free(B.Z); free(B.logw); free(B.logL); return ORC_ERR_OOM; }
  st = orc_init(m, cf, y, x_ref, B.Z, B.logw, B.logL);
  if (st) goto done;
  if (X_leaf) memcpy(X_leaf, B.Z, sizeof(double) * (size_t)K * N * d);

  int L = orc_num_levels(K);
  int gid = 0;
  uint64_t attempts = 0;
  int status = ORC_OK;
  int32_t* pbuf = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)N * (K > 1 ? K - 1 : 1));
  if (!pbuf) { st = ORC_ERR_OOM; goto done; }
  for (int l = 0; l < L; ++l) {
    int size = 1 << l;
    int M = orc_merges_at_level(K, l);
    int root = (l == L - 1);
    int lvl_status = ORC_OK;
    uint64_t lvl_att = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : lvl_att) reduction(max : lvl_status)
    for (int mm = 0; mm < M; ++mm) {
      int a = 2 * mm * size, c = a + size;
      int b = (a + 2 * size < K ? a + 2 * size : K) - 1;
      uint64_t att = 0;
      int s = combine(&mc, cf, &B, a, c, b, gid + mm, pbuf + (size_t)(gid + mm) * 2 * N,
                      (root && cf->conditional) ? x_star : NULL, &att);
      lvl_att += att;
      if (s > lvl_status) lvl_status = s;
    }
    attempts += lvl_att;
    if (lvl_status == ORC_ERR_DEGENERATE || lvl_status == ORC_ERR_OOM) { st = lvl_status; free(pbuf); goto done; }
    if (lvl_status) status = lvl_status;
    gid += M;
  }
  if (pairs && K > 1) memcpy(pairs, pbuf, sizeof(int32_t) * 2 * (size_t)N * (K - 1));
  free(pbuf);
  if (rs_attempts) *rs_attempts = attempts;

  /* Output: the root block.  For K >= 2 it is uniformly weighted (every Combine returns
   * 1/N weights); for K == 1 it is the Algorithm 2 leaf with its own weights. */
  for (int t = 0; t < K; ++t) {
    for (int k = 0; k < d; ++k) {
      double s1 = 0.0, s2 = 0.0;
      for (int n = 0; n < N; ++n) {
        double w = exp(B.logw[n]); /* root weights live at start time 0 */
        double x = B.Z[((size_t)t * N + n) * d + k];
        s1 += w * x;
        s2 += w * x * x;
      }
      mean[(size_t)t * d + k] = s1;
      if (m2) m2[(size_t)t * d + k] = s2;
    }
  }
  if (traj) memcpy(traj, B.Z, sizeof(double) * (size_t)K * N * d);
  *logL = B.logL[0];

  if (cf->conditional && x_star && K == 1) {
    /* no combination: draw the next reference from the weighted leaf at t = 0 */
    double* E = (double*)malloc(sizeof(double) * N);
    double* C = (double*)malloc(sizeof(double) * N);
    if (!E || !C) { free(E); free(C); st = ORC_ERR_OOM; goto done; }
    double S = 0.0;
    for (int n = 0; n < N; ++n) { E[n] = exp(B.logw[n]); S += E[n]; C[n] = S; }
    uint32_t w[4];
    draw(cf->seed_lo, cf->seed_hi, (uint32_t)N, 0u, ORC_PURPOSE_DENSE, cf->counter_base, 0u, w);
    int64_t f = inverse_cdf(C, E, N, u53(w[0], w[1]));
    for (int k = 0; k < d; ++k) x_star[k] = B.Z[(size_t)f * d + k];
    free(E);
    free(C);
  }
  st = status;
done:
  free(B.Z);
  free(B.logw);
  free(B.logL);
  return st;
}

/* ------------------------------------------------------------------------------------ */
/* log omega matrix for given particles (parity of the merge log-weights)                */
/* ------------------------------------------------------------------------------------ */

/* out[i][j] = log omega_c(xl_i, xr_j) + wl[i] + wr[j]  (FP64; Eq. normalized-weights),
 * for Nl left states and Nr right states. */
int orc_logw_matrix(const orc_model* m, int K, const double* y, int c, int Nl, int Nr,
                    const double* xl, const double* xr, const double* wl, const double* wr,
                    double* out) {
  model_ctx mc;
  int st = ctx_init(&mc, m, K, y);
  if (st) return st;
  const int d = m->d;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Nl; ++i)
    for (int j = 0; j < Nr; ++j)
      out[(size_t)i * Nr + j] =
          log_omega(&mc, c, xl + (size_t)i * d, xr + (size_t)j * d) + wl[i] + wr[j];
  return ORC_OK;
}

/* The bounds of Algorithm 8 for one combination (reading of the paper): out[0] is the
 * finite-set bound log f_max + max_i a_i + max_j b'_j with b'_j = wr_j + log h_c(xr_j) -
 * log nu_c(xr_j); for one-dimensional states out[1] is the hull bound log f_max + max_i a_i
 * + max_j (b'_j - dist_j^2 / 2Q), dist_j the distance from xr_j to [min_i m_i, max_i m_i],
 * m_i the transition mean of xl_i (out[1] = out[0] when d > 1). */
int orc_rs_bounds(const orc_model* m, int K, const double* y, int c, int Nl, int Nr,
                  const double* xl, const double* xr, const double* wl, const double* wr,
                  double out[2]) {
  model_ctx mc;
  int st = ctx_init(&mc, m, K, y);
  if (st) return st;
  const int d = m->d;
  double amax = -INFINITY, bmax = -INFINITY, hmax = -INFINITY;
  for (int i = 0; i < Nl; ++i) amax = wl[i] > amax ? wl[i] : amax;
  double lo = INFINITY, hi = -INFINITY, Q = 0.0;
  if (d == 1) {
    Q = m->kind == 0 ? m->Q[0] : m->sigma * m->sigma;
    for (int i = 0; i < Nl; ++i) {
      const double mi = m->kind == 0 ? m->A[0] * xl[i] : trans_mean_1d(m, xl[i]);
      lo = mi < lo ? mi : lo;
      hi = mi > hi ? mi : hi;
    }
  }
  for (int j = 0; j < Nr; ++j) {
    const double* x = xr + (size_t)j * d;
    const double b = wr[j] + log_h(&mc, c, x) - log_nu(&mc, c, x);
    bmax = b > bmax ? b : bmax;
    if (d == 1) {
      double dist = x[0] > hi ? x[0] - hi : (x[0] < lo ? lo - x[0] : 0.0);
      const double h = b - dist * dist / (2.0 * Q);
      hmax = h > hmax ? h : hmax;
    }
  }
  out[0] = log_f_max(&mc) + amax + bmax;
  out[1] = d == 1 ? log_f_max(&mc) + amax + hmax : out[0];
  return ORC_OK;
}

/* log f_max, log h, log nu for tests of the model densities. */
int orc_model_logdens(const orc_model* m, int K, const double* y, int t, const double* xprev,
                      const double* x, double out[5]) {
  model_ctx mc;
  int st = ctx_init(&mc, m, K, y);
  if (st) return st;
  out[0] = log_f(&mc, xprev, x);
  out[1] = log_h(&mc, t, x);
  out[2] = log_nu(&mc, t, x);
  out[3] = log_q(&mc, t, x);
  out[4] = log_f_max(&mc);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Pair samplers in the device's precision (the bit-exact index contract)                */
/* ------------------------------------------------------------------------------------ */

/* Three-stage inverse CDF: row, then 32..512-wide column tile, then column.
 * Inputs are the device's own FP32 weights, all relative to one shift per row:
 *   r[i]        row weight (relative to the largest row), in [0, 1]
 *   t[i][k]     tile weight of row i, tile k (columns kB .. kB+B-1)
 *   e[i][j]     element weight (same per-row shift as t)
 * Every decision is an exact integer computation on fixed-point images of these weights,
 * so it does not depend on any summation order:
 *   row:    Rq_i = trunc(r_i 2^40); T = floor(U S / 2^64), U = (w0 << 32) | w1, S = sum Rq;
 *           row = #{i : Rq_0 + ... + Rq_i <= T}
 *   tile:   q_k = q24(t_ik; max_k t_ik), T = floor(w2 Q / 2^32), Q = sum q;
 *           tile = #{k : prefix <= T}
 *   column: q_j = q24(e_ij; t_ik) over the tile's columns, the same with w3
 * where q24(x; ref) = floor(x 2^k) with k = min(24 - E, 127), 2^(E-2) <= ref < 2^(E-1) (one
 * binade of headroom), saturated at 2^32 - 1, computed on the bit patterns as the
 * significand shifted by the exponent difference; negative and NaN x give 0.  A weight equal to its
 * reference keeps 23 significant bits, as many as its FP32 value.  A zero weight is never
 * chosen; a tile whose column weights are all zero yields its first column.
 * Slots n in [n0, n1) use the counter (n, gid, DENSE | base<<4, 0). */
static uint64_t mulhi64(uint64_t a, uint64_t b) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  return (uint64_t)(p >> 64);
}

static uint64_t row_quant(float r) {
  if (!(r > 0.0f)) return 0;
  if (r > 1.0f) r = 1.0f;
  return (uint64_t)(r * 0x1p40f);
}

static uint32_t float_bits(float x) {
  uint32_t b;
  memcpy(&b, &x, sizeof b);
  return b;
}

/* biased exponent of the reference plus one binade of headroom */
static int ref_exponent(float ref) {
  uint32_t b = float_bits(ref);
  int be = (int)((b >> 23) & 0xFFu);
  return be + 1;
}

static uint64_t q24(float x, int ref_be) {
  uint32_t b = float_bits(x);
  if (b >> 31) return 0;                      /* negative (and -0) */
  int be = (int)((b >> 23) & 0xFFu);
  if (be == 0xFF) return (b & 0x7FFFFFu) ? 0 : 0xFFFFFFFFu;   /* NaN, +inf */
  /* x = M 2^ex exactly: normal M = 1.f * 2^23, ex = be - 150; subnormal M = f, ex = -149 */
  uint64_t M = be ? (uint64_t)((b & 0x7FFFFFu) | 0x800000u) : (uint64_t)(b & 0x7FFFFFu);
  int ex = be ? be - 150 : -149;
  int k = 150 - ref_be;                       /* the scale 2^(24 - E) */
  if (k > 127) k = 127;
  int sh = ex + k;                            /* image = floor(M 2^sh) */
  if (sh <= -64) return 0;
  if (sh <= 0) return M >> (-sh);
  if (sh >= 9) return 0xFFFFFFFFu;            /* M < 2^24: at least 2^33 */
  uint64_t v = M << sh;
  return v > 0xFFFFFFFFu ? 0xFFFFFFFFu : v;
}

/* index of the first prefix sum of q[0..n) exceeding floor(w Q / 2^32); 0 if all are zero */
static int fixed_pick(const uint64_t* q, int n, uint32_t w) {
  uint64_t Q = 0;
  for (int k = 0; k < n; ++k) Q += q[k];
  if (Q == 0) return 0;
  uint64_t T = mulhi64((uint64_t)w << 32, Q);
  uint64_t c = 0;
  int idx = 0;
  for (int k = 0; k < n; ++k) {
    c += q[k];
    if (c <= T) idx = k + 1;
  }
  return idx < n ? idx : n - 1;
}

int orc_kp_dense_pairs(int N, int B, const float* r, const float* t, const float* e,
                       uint32_t seed_lo, uint32_t seed_hi, uint32_t base,
                       uint32_t gid, int n0, int n1, int32_t* li, int32_t* ri) {
  int nT = (N + B - 1) / B;
  uint64_t* cum = (uint64_t*)malloc(sizeof(uint64_t) * N);
  uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * (nT > B ? nT : B));
  if (!cum || !q) { free(cum); free(q); return ORC_ERR_OOM; }
  uint64_t S = 0;
  for (int i = 0; i < N; ++i) {
    S += row_quant(r[i]);
    cum[i] = S;
  }
  if (S == 0) { free(cum); free(q); return ORC_ERR_DEGENERATE; }
  for (int n = n0; n < n1; ++n) {
    uint32_t w[4];
    draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_DENSE, base, 0u, w);
    uint64_t U = ((uint64_t)w[0] << 32) | (uint64_t)w[1];
    uint64_t T = mulhi64(U, S);
    int i = 0;
    while (i < N - 1 && cum[i] <= T) ++i;
    const float* ti = t + (size_t)i * nT;
    float tmax = 0.0f;
    for (int k = 0; k < nT; ++k) tmax = ti[k] > tmax ? ti[k] : tmax;
    int rbe = ref_exponent(tmax);
    for (int k = 0; k < nT; ++k) q[k] = q24(ti[k], rbe);
    int k = fixed_pick(q, nT, w[2]);
    int j0 = k * B;
    int width = (j0 + B <= N) ? B : N - j0;
    int tbe = ref_exponent(ti[k]);
    for (int j = 0; j < width; ++j) q[j] = q24(e[(size_t)i * N + j0 + j], tbe);
    li[n - n0] = i;
    ri[n - n0] = j0 + fixed_pick(q, width, w[3]);
  }
  free(cum);
  free(q);
  return ORC_OK;
}

/* Algorithm 8 in the device's precision: ratio[I][J] = exp(logW_IJ - log wbar) as the
 * device computed it (FP32); per attempt (I, J, u) = (w0 N >> 32, w1 N >> 32, u23(w2)),
 * counter (n, gid, RS | base<<4, attempt); accept when u < ratio, u = u23(w2). */
int orc_kp_rs_pairs(int N, const float* ratio, uint32_t seed_lo, uint32_t seed_hi, uint32_t base,
                    uint32_t gid, int n0, int n1, uint32_t max_attempts, int32_t* li, int32_t* ri,
                    uint32_t* attempts) {
  int status = ORC_OK;
  for (int n = n0; n < n1; ++n) {
    uint32_t a;
    int I = 0, J = 0, ok = 0;
    for (a = 0; a < max_attempts; ++a) {
      uint32_t w[4];
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RS, base, a, w);
      I = (int)(((uint64_t)w[0] * (uint64_t)N) >> 32);
      J = (int)(((uint64_t)w[1] * (uint64_t)N) >> 32);
      float u = (float)u23(w[2]);
      if (u < ratio[(size_t)I * N + J]) { ok = 1; ++a; break; }
    }
    if (!ok) status = ORC_ERR_RS_LIMIT;
    li[n - n0] = ok ? I : -1;  /* a slot that hit the cap keeps no index */
    ri[n - n0] = ok ? J : -1;
    attempts[n - n0] = a;
  }
  return status;
}

/* Systematic variant of the three-stage sampler (same inputs and images as
 * orc_kp_dense_pairs).  One 64-bit uniform U per combination (words 0-1 of the counter
 * (0, gid, SYS | base<<4, 0)) gives V = floor(U S / 2^64); slot k takes the row target
 * T_k = floor((k S + V) / N) = k q + floor((k r + V) / N), S = q N + r (exact integers);
 * the remainder of T_k inside its row, as a fraction of the row's fixed-point weight, is the
 * uniform word of the tile stage, w2 = trunc((T_k - cum_{i-1}) / Rq_i 2^32) (FP64 quotient,
 * correctly rounded), and the remainder of the tile target inside its tile, as a fraction
 * of the tile's image, the word of the column stage.  Each slot's position in the flattened
 * fixed-point CDF moves by S / N from slot to slot. */
static int fixed_pick_rem(const uint64_t* q, int n, uint32_t w, uint32_t* wnext) {
  uint64_t Q = 0;
  for (int k = 0; k < n; ++k) Q += q[k];
  if (Q == 0) { *wnext = w; return 0; }
  uint64_t T = mulhi64((uint64_t)w << 32, Q);
  uint64_t c = 0, before = 0;
  int idx = 0;
  for (int k = 0; k < n; ++k) {
    c += q[k];
    if (c <= T) { idx = k + 1; before = c; }
  }
  if (idx > n - 1) idx = n - 1;
  *wnext = q[idx] ? (uint32_t)(((double)(T - before) / (double)q[idx]) * 4294967296.0) : 0u;
  return idx;
}

int orc_kp_sys_pairs(int N, int B, const float* r, const float* t, const float* e,
                     uint32_t seed_lo, uint32_t seed_hi, uint32_t base,
                     uint32_t gid, int n0, int n1, int32_t* li, int32_t* ri) {
  int nT = (N + B - 1) / B;
  uint64_t* cum = (uint64_t*)malloc(sizeof(uint64_t) * N);
  uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * (nT > B ? nT : B));
  if (!cum || !q) { free(cum); free(q); return ORC_ERR_OOM; }
  uint64_t S = 0;
  for (int i = 0; i < N; ++i) {
    S += row_quant(r[i]);
    cum[i] = S;
  }
  if (S == 0) { free(cum); free(q); return ORC_ERR_DEGENERATE; }
  uint32_t w0[4];
  draw(seed_lo, seed_hi, 0u, gid, ORC_PURPOSE_SYS, base, 0u, w0);
  const uint64_t V = mulhi64(((uint64_t)w0[0] << 32) | (uint64_t)w0[1], S);
  const uint64_t qq = S / (uint64_t)N, rr = S % (uint64_t)N;
  for (int n = n0; n < n1; ++n) {
    const uint64_t k = (uint64_t)n;
    const uint64_t T = k * qq + (k * rr + V) / (uint64_t)N;
    int i = 0;
    while (i < N - 1 && cum[i] <= T) ++i;
    const uint64_t prev = i ? cum[i - 1] : 0;
    const uint32_t w2 = (uint32_t)(((double)(T - prev) / (double)(cum[i] - prev)) * 4294967296.0);
    const float* ti = t + (size_t)i * nT;
    float tmax = 0.0f;
    for (int kk = 0; kk < nT; ++kk) tmax = ti[kk] > tmax ? ti[kk] : tmax;
    int rbe = ref_exponent(tmax);
    for (int kk = 0; kk < nT; ++kk) q[kk] = q24(ti[kk], rbe);
    uint32_t w3;
    int kt = fixed_pick_rem(q, nT, w2, &w3);
    int j0 = kt * B;
    int width = (j0 + B <= N) ? B : N - j0;
    int tbe = ref_exponent(ti[kt]);
    for (int j = 0; j < width; ++j) q[j] = q24(e[(size_t)i * N + j0 + j], tbe);
    li[n - n0] = i;
    ri[n - n0] = j0 + fixed_pick(q, width, w3);
  }
  free(cum);
  free(q);
  return ORC_OK;
}

/* Factorised-proposal rejection sampler in the device's precision: ra [N] and rc [N] are the
 * device's FP32 row and column proposal weights (relative to their maxima, in [0, 1]), acc
 * [N][N] its FP32 acceptance ratios.  Proposal images Rq = trunc(ra 2^40), Cq = trunc(rc
 * 2^40) with exact prefix sums; per attempt I = #{cumA <= floor(U1 SA / 2^64)} with U1 =
 * words 0-1 of the counter (n, gid, RSF | base<<4, attempt), J likewise from words 2-3 and
 * SC, and the pair is accepted when u < acc[I][J] in FP32, u = u23 of word 0 of the counter
 * (n, gid, RSU | base<<4, attempt).  A slot that reaches max_attempts keeps the index -1. */
int orc_kp_rsf_pairs(int N, const float* ra, const float* rc, const float* acc, uint32_t seed_lo,
                     uint32_t seed_hi, uint32_t base, uint32_t gid, int n0, int n1,
                     uint32_t max_attempts, int32_t* li, int32_t* ri, uint32_t* attempts) {
  uint64_t* cA = (uint64_t*)malloc(sizeof(uint64_t) * N);
  uint64_t* cC = (uint64_t*)malloc(sizeof(uint64_t) * N);
  if (!cA || !cC) { free(cA); free(cC); return ORC_ERR_OOM; }
  uint64_t SA = 0, SC = 0;
  for (int i = 0; i < N; ++i) { SA += row_quant(ra[i]); cA[i] = SA; }
  for (int j = 0; j < N; ++j) { SC += row_quant(rc[j]); cC[j] = SC; }
  if (SA == 0 || SC == 0) { free(cA); free(cC); return ORC_ERR_DEGENERATE; }
  int status = ORC_OK;
  for (int n = n0; n < n1; ++n) {
    uint32_t a;
    int I = 0, J = 0, ok = 0;
    for (a = 0; a < max_attempts; ++a) {
      uint32_t w[4], v[4];
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RSF, base, a, w);
      draw(seed_lo, seed_hi, (uint32_t)n, gid, ORC_PURPOSE_RSU, base, a, v);
      const uint64_t TA = mulhi64(((uint64_t)w[0] << 32) | (uint64_t)w[1], SA);
      const uint64_t TC = mulhi64(((uint64_t)w[2] << 32) | (uint64_t)w[3], SC);
      I = 0;
      while (I < N - 1 && cA[I] <= TA) ++I;
      J = 0;
      while (J < N - 1 && cC[J] <= TC) ++J;
      const float u = (float)u23(v[0]);
      if (u < acc[(size_t)I * N + J]) { ok = 1; ++a; break; }
    }
    if (!ok) status = ORC_ERR_RS_LIMIT;
    li[n - n0] = ok ? I : -1;
    ri[n - n0] = ok ? J : -1;
    attempts[n - n0] = a;
  }
  free(cA);
  free(cC);
  return status;
}
