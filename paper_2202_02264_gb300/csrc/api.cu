// api.cu -- the C ABI of include/dsmc.h: argument checks, the FP64 model pre-computation,
// the workspace layout, and the level loop of Algorithm 6 (Appendix A).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace dsmc {
int rowsum_rows_per_thread(int D);
cudaError_t launch_level_fused(int D, const MergeArgs& a, const void* mp, int C, cudaStream_t s);
cudaError_t level_fused_max_clusters(int D, const MergeArgs& a, int C, int* n);
size_t fused_level_smem(int D, int N, int C);
cudaError_t launch_k1_star(const float* logw, int N, uint64_t seed, uint32_t base, int32_t* star,
                           cudaStream_t s);
}  // namespace dsmc

using namespace dsmc;

namespace {

thread_local std::string g_last_error;

// Per-thread measurement state: events around every exp / tile-sum launch, launch counts.
struct Profile {
  bool on = false;
  std::vector<cudaEvent_t> start, stop;
  size_t used = 0;
  int64_t launches = 0;
  double pairs = 0.0;
};
thread_local Profile g_prof;

// An event recorded on a capturing stream joins the graph as an event-record node only with
// cudaEventRecordExternal; without it the record is internal to the capture and the event
// cannot be read after a replay.
cudaError_t record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  return cudaEventRecord(e, s);
}

cudaError_t prof_begin(cudaStream_t s) {
  if (!g_prof.on) return cudaSuccess;
  if (g_prof.used == g_prof.start.size()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    g_prof.start.push_back(a);
    g_prof.stop.push_back(b);
  }
  return record(g_prof.start[g_prof.used], s);
}

cudaError_t prof_end(cudaStream_t s, double pairs) {
  if (!g_prof.on) return cudaSuccess;
  g_prof.pairs += pairs;
  return record(g_prof.stop[g_prof.used++], s);
}

void prof_count(int n) {
  if (g_prof.on) g_prof.launches += n;
}

// Per-kernel-kind breakdown: events around every launch of a kind (dsmc_profile_breakdown_*).
struct Breakdown {
  bool on = false;
  std::vector<cudaEvent_t> a, b;
  std::vector<int> kind;
  size_t used = 0;
};
thread_local Breakdown g_bd;

// Test switch of dsmc_debug_stall_tensor_cores: tile-sum launches issue no MMA.
bool g_stall_tc = false;
// Test switch of dsmc_debug_keep_weights: fused levels store their intermediate weights.
bool g_keep_weights = false;

cudaError_t bd_begin(cudaStream_t s, int kind) {
  if (!g_bd.on) return cudaSuccess;
  if (g_bd.used == g_bd.a.size()) {
    cudaEvent_t x, y;
    cudaError_t e = cudaEventCreate(&x);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&y);
    if (e != cudaSuccess) return e;
    g_bd.a.push_back(x);
    g_bd.b.push_back(y);
    g_bd.kind.push_back(0);
  }
  g_bd.kind[g_bd.used] = kind;
  return record(g_bd.a[g_bd.used], s);
}

cudaError_t bd_end(cudaStream_t s) {
  if (!g_bd.on) return cudaSuccess;
  return record(g_bd.b[g_bd.used++], s);
}

dsmc_status_t fail(dsmc_status_t st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

dsmc_status_t cuda_fail(cudaError_t e, const char* what) {
  return fail(DSMC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int kMaxDim = 32;
constexpr int kMaxDenseN = 16384;
constexpr int kDefaultMergeCap = 1024;
constexpr uint32_t kDefaultMhSteps = 64;   // Algorithm 7's B when rs_max_attempts is 0
constexpr uint32_t kDefaultRsCap = 1u << 26;  // rejection samplers' attempt cap when it is 0
constexpr int kRowsumCtasPerSm = 8;  // FP32 tile-sum kernel: several CTAs per SM

// The current device's SM count (queried once per device; sizes grids and chunks).
cudaError_t device_sms(int* n) {
  static std::mutex mu;
  static int cache[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  if (dev < 0 || dev >= 64) return cudaDeviceGetAttribute(n, cudaDevAttrMultiProcessorCount, dev);
  if (cache[dev] == 0) {
    e = cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  *n = cache[dev];
  return cudaSuccess;
}

int pad_dim(int d) {
  int D = 1;
  while (D < d) D <<= 1;
  return D;
}

int merges_at_level(int K, int l) {
  const long size = 1L << l;
  if (size >= K) return 0;
  return (int)((K - size + 2 * size - 1) / (2 * size));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
  int K, N, d, D, L;
  int compute, Nr, planes;
  int B, nT, nTp;
  int Mc;
  int R, rows_per_cta;
  bool dense;
  int level_off[33];
  size_t o_status, o_U, o_alpha, o_V, o_beta, o_shift, o_g, o_cbase, o_logbar, o_inc, o_T, o_rw, o_rowsum, o_cum,
      o_delta, o_first, o_last, o_star, o_Ub, o_Vb, o_attempts, o_alpha0, o_kappa, o_pa, o_pc, o_cumA, o_cumC,
      total;
};

void chunking(const Plan& p, int mc, int sms, int& CH, int& CW) {
  if (p.compute != DSMC_FP32) {
    // tensor-core path: 128-row CTAs, two per SM, chunks of whole 128-column blocks
    const int RT = (p.N + 127) / 128;
    const int nblk = (p.N + 127) / 128;
    int want = (sms * 2 * 2 + mc * RT - 1) / (mc * RT);
    want = std::max(1, std::min(want, nblk));
    const int bpc = (nblk + want - 1) / want;
    CW = bpc * 128;
    CH = (nblk + bpc - 1) / bpc;
    return;
  }
  const int RT = (p.N + p.rows_per_cta - 1) / p.rows_per_cta;
  int want = (sms * kRowsumCtasPerSm + mc * RT - 1) / (mc * RT);
  want = std::max(1, std::min(want, p.nT));
  const int tpc = (p.nT + want - 1) / want;
  CW = tpc * p.B;
  CH = (p.nT + tpc - 1) / tpc;
}

// Workspace plan of one smoothing; a batched call passes the level-0 combination count of
// the whole batch (M0) and keeps the per-sequence index maps outside (no_maps).
void make_plan(const dsmc_config_t* cfg, const dsmc_model_t* model, Plan& p, int M0_batch = -1,
               bool no_maps = false) {
  p.K = cfg->K;
  p.N = cfg->N;
  p.d = model->dx;
  p.D = pad_dim(model->dx);
  p.L = 0;
  while ((1 << p.L) < p.K) ++p.L;
  p.dense = cfg->resampler == DSMC_MULTINOMIAL || cfg->resampler == DSMC_SYSTEMATIC;
  const bool factored = cfg->resampler == DSMC_RS_FACTORED;
  // the cross-term precision only matters to the dense N x N pass; the lazy sampler
  // evaluates its proposed pairs in FP32 and needs no tensor-core operands
  p.compute = p.dense ? cfg->compute : DSMC_FP32;
  p.Nr = (p.N + 127) / 128 * 128;
  {
    const int kp = p.compute == DSMC_BF16 ? 16 : 8;
    p.planes = (p.D + 4 + kp - 1) / kp;
  }
  const int nT0 = std::min((p.N + 31) / 32, 64);
  const int per = (p.N + nT0 - 1) / nT0;
  p.B = cfg->tile_cols > 0 ? cfg->tile_cols : 32 * ((per + 31) / 32);
  p.nT = (p.N + p.B - 1) / p.B;
  p.nTp = (p.nT + 3) / 4 * 4;
  const int M0 = std::max(1, M0_batch >= 0 ? M0_batch : merges_at_level(p.K, 0));
  const int cap = cfg->max_merges_per_launch > 0 ? cfg->max_merges_per_launch : kDefaultMergeCap;
  p.Mc = std::max(1, std::min(M0, cap));
  p.R = rowsum_rows_per_thread(p.D);
  const int NT = std::min(128, std::max(32, ((p.N + p.R - 1) / p.R + 31) / 32 * 32));
  p.rows_per_cta = p.R * NT;
  int off = 0;
  for (int l = 0; l < p.L; ++l) {
    p.level_off[l] = off;
    off += merges_at_level(p.K, l);
  }
  p.level_off[p.L] = off;
  const size_t MN = (size_t)p.Mc * p.N;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  p.o_status = take(sizeof(int));
  p.o_attempts = take(sizeof(unsigned long long));
  p.o_U = take(MN * p.D * sizeof(float));
  p.o_alpha = take(MN * sizeof(float));
  p.o_V = take(MN * p.D * sizeof(float));
  p.o_beta = take(MN * sizeof(float));
  p.o_shift = take(MN * sizeof(double));
  p.o_g = take(p.dense ? MN * sizeof(float) : 0);
  p.o_cbase = take(p.dense ? (size_t)p.Mc * sizeof(double) : 0);
  p.o_logbar = take((size_t)p.Mc * sizeof(double));
  p.o_inc = take((size_t)p.Mc * sizeof(double));
  p.o_T = take(p.dense ? MN * p.nTp * sizeof(float) : 0);
  p.o_rw = take(MN * sizeof(float));
  p.o_rowsum = take(p.dense ? MN * sizeof(float) : 0);
  p.o_cum = take(p.dense ? MN * sizeof(unsigned long long) : 0);
  p.o_delta = take(MN * sizeof(float));
  p.o_first = take(no_maps ? 0 : 2 * (size_t)p.K * p.N * sizeof(int32_t));
  p.o_last = take(no_maps ? 0 : 2 * (size_t)p.K * p.N * sizeof(int32_t));
  p.o_star = take(2 * sizeof(int32_t));
  const bool tc = p.compute != DSMC_FP32;
  p.o_Ub = take(tc ? (size_t)p.Mc * p.planes * p.Nr * 32 : 0);
  p.o_Vb = take(tc ? (size_t)p.Mc * p.planes * p.Nr * 32 : 0);
  p.o_alpha0 = take(factored ? MN * sizeof(float) : 0);
  p.o_kappa = take(factored ? MN * sizeof(float) : 0);
  p.o_pa = take(factored ? MN * sizeof(float) : 0);
  p.o_pc = take(factored ? MN * sizeof(float) : 0);
  p.o_cumA = take(factored ? MN * sizeof(unsigned long long) : 0);
  p.o_cumC = take(factored ? MN * sizeof(unsigned long long) : 0);
  p.total = o;
}

WsPtrs ws_ptrs(const Plan& p, void* ws) {
  char* b = static_cast<char*>(ws);
  WsPtrs w;
  w.status = reinterpret_cast<int*>(b + p.o_status);
  w.U = reinterpret_cast<float*>(b + p.o_U);
  w.alpha = reinterpret_cast<float*>(b + p.o_alpha);
  w.V = reinterpret_cast<float*>(b + p.o_V);
  w.beta = reinterpret_cast<float*>(b + p.o_beta);
  w.shift = reinterpret_cast<double*>(b + p.o_shift);
  w.g = reinterpret_cast<float*>(b + p.o_g);
  w.cbase = reinterpret_cast<double*>(b + p.o_cbase);
  w.logbar = reinterpret_cast<double*>(b + p.o_logbar);
  w.inc = reinterpret_cast<double*>(b + p.o_inc);
  w.T = reinterpret_cast<float*>(b + p.o_T);
  w.rw = reinterpret_cast<float*>(b + p.o_rw);
  w.rowsum = reinterpret_cast<float*>(b + p.o_rowsum);
  w.cum = reinterpret_cast<unsigned long long*>(b + p.o_cum);
  w.delta = reinterpret_cast<float*>(b + p.o_delta);
  w.first = reinterpret_cast<int32_t*>(b + p.o_first);
  w.last = reinterpret_cast<int32_t*>(b + p.o_last);
  w.star = reinterpret_cast<int32_t*>(b + p.o_star);
  w.Ub = reinterpret_cast<unsigned char*>(b + p.o_Ub);
  w.Vb = reinterpret_cast<unsigned char*>(b + p.o_Vb);
  w.attempts_total = reinterpret_cast<unsigned long long*>(b + p.o_attempts);
  w.alpha0 = reinterpret_cast<float*>(b + p.o_alpha0);
  w.kappa = reinterpret_cast<float*>(b + p.o_kappa);
  w.pa = reinterpret_cast<float*>(b + p.o_pa);
  w.pc = reinterpret_cast<float*>(b + p.o_pc);
  w.cumA = reinterpret_cast<unsigned long long*>(b + p.o_cumA);
  w.cumC = reinterpret_cast<unsigned long long*>(b + p.o_cumC);
  return w;
}

// ---- FP64 host linear algebra for the parameter pre-computation
bool cholesky(int d, const double* S, double* L) {
  std::memset(L, 0, sizeof(double) * d * d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = S[i * d + j];
      for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
      if (i == j) {
        if (!(s > 0.0) || !std::isfinite(s)) return false;
        L[i * d + i] = std::sqrt(s);
      } else {
        L[i * d + j] = s / L[j * d + j];
      }
    }
  return true;
}

// inverse and log-determinant of an SPD matrix through its Cholesky factor
bool spd_inverse(int d, const double* S, double* Si, double* logdet) {
  double L[kMaxDim * kMaxDim], Li[kMaxDim * kMaxDim];
  if (!cholesky(d, S, L)) return false;
  std::memset(Li, 0, sizeof(Li));
  for (int i = 0; i < d; ++i) {
    Li[i * d + i] = 1.0 / L[i * d + i];
    for (int j = 0; j < i; ++j) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s -= L[i * d + k] * Li[k * d + j];
      Li[i * d + j] = s / L[i * d + i];
    }
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = std::max(i, j); k < d; ++k) s += Li[k * d + i] * Li[k * d + j];
      Si[i * d + j] = s;
    }
  double ld = 0.0;
  for (int i = 0; i < d; ++i) ld += 2.0 * std::log(L[i * d + i]);
  *logdet = ld;
  return true;
}

constexpr double kLog2Pi = 1.8378770664093454836;

struct alignas(16) ParamBuf {
  unsigned char bytes[sizeof(ModelParams<kMaxDim>)];
  const float* prop_mean;  // the proposal arrays of a single-sequence call (or null)
  const float* prop_std;
};

template <int D>
dsmc_status_t fill_params(const dsmc_model_t* m, const dsmc_proposal_t* pr, ParamBuf& buf) {
  ModelParams<D>* mp = reinterpret_cast<ModelParams<D>*>(buf.bytes);
  std::memset(mp, 0, sizeof(ModelParams<D>));
  const int d = m->dx;
  mp->kind = m->kind;
  mp->d = d;
  mp->prop_kind = pr->kind;
  mp->nu = pr->nu;
  mp->prop_scale = (float)pr->scale;
  mp->log_prop_scale = (float)std::log(pr->scale > 0 ? pr->scale : 1.0);
  mp->prop_mean = pr->mean;
  mp->prop_std = pr->std;
  if (m->kind != DSMC_MODEL_LGSSM) {  // the one-dimensional kinds
    const double s2 = m->sigma * m->sigma;
    double A = 1.0, c = 0.0, m0 = 0.0, v0 = 1.0;
    if (m->kind == DSMC_MODEL_SV || m->kind == DSMC_MODEL_COX) {
      A = m->kind == DSMC_MODEL_COX ? m->phi * m->lam : m->phi;
      c = m->mu * (1.0 - m->phi);
      m0 = m->mu;
      v0 = s2 / (1.0 - m->phi * m->phi);
    }
    mp->A[0] = (float)A;
    mp->c[0] = (float)c;
    mp->Qi[0] = (float)(1.0 / s2);
    mp->P0i[0] = (float)(1.0 / v0);
    mp->m0[0] = (float)m0;
    mp->log_f_max = (float)(-0.5 * (kLog2Pi + std::log(s2)));
    mp->log_p0_norm = (float)(-0.5 * (kLog2Pi + std::log(v0)));
    mp->log_h_norm = (float)(-0.5 * kLog2Pi);
    mp->tau0 = (float)m->tau0;
    mp->tau1 = (float)m->tau1;
    mp->tau2 = (float)m->tau2;
    mp->bound = (float)m->bound;
    if (m->kind == DSMC_MODEL_THETA_LOGISTIC) {  // y_t = x_t + N(0, obs_sd^2)
      const double r2 = m->obs_sd * m->obs_sd;
      mp->Ri[0] = (float)(1.0 / r2);
      mp->log_h_norm = (float)(-0.5 * (kLog2Pi + std::log(r2)));
    }
    return DSMC_OK;
  }
  double Qi[kMaxDim * kMaxDim], Ri[kMaxDim * kMaxDim], P0i[kMaxDim * kMaxDim];
  double ldQ, ldR, ldP;
  if (!spd_inverse(d, m->Q, Qi, &ldQ)) return fail(DSMC_ERR_INVALID_ARG, "Q is not positive definite");
  if (!spd_inverse(d, m->R, Ri, &ldR)) return fail(DSMC_ERR_INVALID_ARG, "R is not positive definite");
  if (!spd_inverse(d, m->P0, P0i, &ldP)) return fail(DSMC_ERR_INVALID_ARG, "P0 is not positive definite");
  for (int i = 0; i < d; ++i) {
    mp->m0[i] = (float)m->m0[i];
    for (int j = 0; j < d; ++j) {
      mp->A[i * D + j] = (float)m->A[i * d + j];
      mp->Qi[i * D + j] = (float)Qi[i * d + j];
      mp->Ri[i * D + j] = (float)Ri[i * d + j];
      mp->P0i[i * D + j] = (float)P0i[i * d + j];
    }
  }
  mp->log_f_max = (float)(-0.5 * (d * kLog2Pi + ldQ));
  mp->log_h_norm = (float)(-0.5 * (d * kLog2Pi + ldR));
  mp->log_p0_norm = (float)(-0.5 * (d * kLog2Pi + ldP));
  return DSMC_OK;
}

dsmc_status_t make_params(int D, const dsmc_model_t* m, const dsmc_proposal_t* pr, ParamBuf& buf) {
  buf.prop_mean = pr->mean;
  buf.prop_std = pr->std;
  switch (D) {
    case 1: return fill_params<1>(m, pr, buf);
    case 2: return fill_params<2>(m, pr, buf);
    case 4: return fill_params<4>(m, pr, buf);
    case 8: return fill_params<8>(m, pr, buf);
    case 16: return fill_params<16>(m, pr, buf);
    case 32: return fill_params<32>(m, pr, buf);
  }
  return fail(DSMC_ERR_UNSUPPORTED, "state dimension");
}

dsmc_status_t check_config(const dsmc_config_t* cfg, const dsmc_model_t* model) {
  if (!cfg || !model) return fail(DSMC_ERR_INVALID_ARG, "null config or model");
  if (cfg->K < 1) return fail(DSMC_ERR_INVALID_ARG, "K must be >= 1");
  if (cfg->N < 1) return fail(DSMC_ERR_INVALID_ARG, "N must be >= 1");
  if (cfg->K > (1 << 24) || cfg->N > (1 << 24)) return fail(DSMC_ERR_UNSUPPORTED, "K or N too large");
  if (cfg->resampler != DSMC_MULTINOMIAL && cfg->resampler != DSMC_RS && cfg->resampler != DSMC_MH &&
      cfg->resampler != DSMC_SYSTEMATIC && cfg->resampler != DSMC_RS_FACTORED)
    return fail(DSMC_ERR_INVALID_ARG, "unknown resampler");
  const bool dense = cfg->resampler == DSMC_MULTINOMIAL || cfg->resampler == DSMC_SYSTEMATIC;
  if (dense && cfg->N > kMaxDenseN)
    return fail(DSMC_ERR_UNSUPPORTED, "dense resampling supports N <= 16384; use DSMC_RS or DSMC_RS_FACTORED");
  if (cfg->compute != DSMC_FP32 && cfg->compute != DSMC_TF32 && cfg->compute != DSMC_BF16)
    return fail(DSMC_ERR_INVALID_ARG, "unknown compute precision");
  if (cfg->compute == DSMC_TF32 && model->dx > 16)
    return fail(DSMC_ERR_UNSUPPORTED, "the TF32 tensor-core cross term supports dx <= 16");
  if (cfg->compute != DSMC_FP32 && dense && cfg->N > 4096)
    return fail(DSMC_ERR_UNSUPPORTED, "the tensor-core cross term supports N <= 4096");
  if (cfg->counter_base >= (1u << 28)) return fail(DSMC_ERR_INVALID_ARG, "counter_base must be < 2^28");
  if (cfg->tile_cols != 0) {
    if (cfg->tile_cols != 32 && cfg->tile_cols != 64) return fail(DSMC_ERR_INVALID_ARG, "tile_cols must be 0, 32 or 64");
    if ((cfg->N + cfg->tile_cols - 1) / cfg->tile_cols > 64)
      return fail(DSMC_ERR_UNSUPPORTED, "tile_cols gives more than 64 tiles per row at this N");
  }
  if (model->dx < 1 || model->dx > kMaxDim) return fail(DSMC_ERR_UNSUPPORTED, "dx must be in 1..32");
  if (model->kind == DSMC_MODEL_SV || model->kind == DSMC_MODEL_COX) {
    if (model->dx != 1) return fail(DSMC_ERR_INVALID_ARG, "the SV and COX models have dx = 1");
    if (!(model->sigma > 0.0) || !(std::fabs(model->phi) < 1.0))
      return fail(DSMC_ERR_INVALID_ARG, "SV and COX need sigma > 0 and |phi| < 1");
    if (model->kind == DSMC_MODEL_COX && !std::isfinite(model->lam))
      return fail(DSMC_ERR_INVALID_ARG, "COX needs a finite lam");
  } else if (model->kind == DSMC_MODEL_THETA_LOGISTIC) {
    if (model->dx != 1) return fail(DSMC_ERR_INVALID_ARG, "the theta-logistic model has dx = 1");
    if (!(model->sigma > 0.0) || !(model->obs_sd > 0.0) || !std::isfinite(model->tau0) ||
        !std::isfinite(model->tau1) || !std::isfinite(model->tau2))
      return fail(DSMC_ERR_INVALID_ARG, "theta-logistic needs sigma, obs_sd > 0 and finite tau");
  } else if (model->kind == DSMC_MODEL_CRW) {
    if (model->dx != 1) return fail(DSMC_ERR_INVALID_ARG, "the constrained random walk has dx = 1");
    if (!(model->sigma > 0.0) || !(model->bound > 0.0))
      return fail(DSMC_ERR_INVALID_ARG, "the constrained random walk needs sigma, bound > 0");
  } else if (model->kind == DSMC_MODEL_LGSSM) {
    if (!model->A || !model->Q || !model->R || !model->m0 || !model->P0)
      return fail(DSMC_ERR_INVALID_ARG, "LGSSM needs A, Q, R, m0, P0");
  } else {
    return fail(DSMC_ERR_INVALID_ARG, "unknown model kind");
  }
  return DSMC_OK;
}

dsmc_status_t check_prop(const dsmc_config_t* cfg, const dsmc_model_t* model,
                         const dsmc_proposal_t* prop) {
  (void)cfg;
  if (!prop) return fail(DSMC_ERR_INVALID_ARG, "null proposal");
  if (prop->kind == DSMC_PROP_OBS) {
    if (!(prop->scale > 0.0)) return fail(DSMC_ERR_INVALID_ARG, "proposal scale must be > 0");
  } else if (prop->kind == DSMC_PROP_GAUSS) {
    if (!prop->mean || !prop->std) return fail(DSMC_ERR_INVALID_ARG, "proposal mean/std arrays");
  } else if (prop->kind == DSMC_PROP_UNIFORM) {
    if (!(prop->scale > 0.0)) return fail(DSMC_ERR_INVALID_ARG, "uniform proposal needs scale > 0");
  } else {
    return fail(DSMC_ERR_INVALID_ARG, "unknown proposal kind");
  }
  if (prop->nu != DSMC_NU_EQ_Q && prop->nu != DSMC_NU_PROP_H)
    return fail(DSMC_ERR_INVALID_ARG, "unknown nu choice");
  if (prop->nu == DSMC_NU_PROP_H && model->kind == DSMC_MODEL_COX)
    return fail(DSMC_ERR_UNSUPPORTED, "the COX potential has no normalised nu (y_t = 0)");
  return DSMC_OK;
}

dsmc_status_t check_ws(const Plan& p, void* ws, size_t ws_bytes) {
  if (!ws) return fail(DSMC_ERR_INVALID_ARG, "null workspace");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(DSMC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < p.total) return fail(DSMC_ERR_WORKSPACE, "workspace too small");
  return DSMC_OK;
}

dsmc_status_t check_state(const dsmc_state_t* st, int K) {
  if (!st || !st->X || !st->logw || !st->logL || (K > 1 && !st->pairs))
    return fail(DSMC_ERR_INVALID_ARG, "state buffers");
  return DSMC_OK;
}

#define DSMC_TRY(x)                      \
  do {                                   \
    dsmc_status_t _st = (x);             \
    if (_st != DSMC_OK) return _st;      \
  } while (0)

#define DSMC_CUDA(x, what)               \
  do {                                   \
    cudaError_t _e = (x);                \
    if (_e != cudaSuccess) return cuda_fail(_e, what); \
  } while (0)

MergeArgs merge_args(const Plan& p, const dsmc_config_t* cfg, const float* y, int level,
                     int conditional, const dsmc_state_t* st, const WsPtrs& w) {
  MergeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.K = p.K;
  a.N = p.N;
  a.d = p.d;
  a.level = level;
  a.B = p.B;
  a.nT = p.nT;
  a.nTp = p.nTp;
  a.rows_per_cta = p.rows_per_cta;
  a.conditional = conditional;
  a.root = (level == p.L - 1);
  a.resampler = cfg->resampler;
  a.compute = p.compute;
  a.stall = g_stall_tc ? 1 : 0;
  a.inspect = g_keep_weights ? 1 : 0;
  a.Nr = p.Nr;
  a.mma_planes = p.planes;
  a.seed = cfg->seed;
  a.base = cfg->counter_base;
  // DSMC_RS: attempts per slot before DSMC_ERR_RS_LIMIT; DSMC_MH: the chain's steps B
  a.rs_max = cfg->rs_max_attempts ? cfg->rs_max_attempts
                                  : (cfg->resampler == DSMC_MH ? kDefaultMhSteps : kDefaultRsCap);
  a.logN = (float)std::log((double)p.N);
  a.prop_mean = nullptr;
  a.prop_std = nullptr;
  a.seqs = nullptr;
  a.items = nullptr;
  a.X = st->X;
  a.logw = st->logw;
  a.y = y;
  a.logL = st->logL;
  a.pairs = st->pairs;
  a.ws = w;
  return a;
}

dsmc_status_t do_init(const Plan& p, const dsmc_config_t* cfg, const ParamBuf& mp,
                      const float* y, const float* x_ref, dsmc_state_t* st, const WsPtrs& w,
                      cudaStream_t s) {
  DSMC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), s), "reset status");
  DSMC_CUDA(cudaMemsetAsync(w.attempts_total, 0, sizeof(unsigned long long), s), "reset attempts");
  DSMC_CUDA(cudaMemsetAsync(w.star, 0, 2 * sizeof(int32_t), s), "reset star");
  InitArgs a;
  std::memset(&a, 0, sizeof(a));
  a.K = p.K;
  a.N = p.N;
  a.logN = (float)std::log((double)p.N);
  a.d = p.d;
  a.seed = cfg->seed;
  a.base = cfg->counter_base;
  a.y = y;
  a.x_ref = x_ref;
  a.X = st->X;
  a.logw = st->logw;
  a.logL = st->logL;
  a.status = w.status;
  DSMC_CUDA(bd_begin(s, DSMC_KIND_INIT), "profile event");
  DSMC_CUDA(launch_init(p.D, a, mp.bytes, s), "init kernel");
  DSMC_CUDA(bd_end(s), "profile event");
  prof_count(1);
  return DSMC_OK;
}

// The fused single-launch level (dense sampler only): cluster size C for a level of M
// combinations, or 0 for the split path.  C doubles while the level still fills at most
// one wave of the SMs and every CTA keeps at least 32 rows; the shared-memory footprint
// (all N column terms per CTA) must fit one SM.
constexpr int kDefaultFusedMaxMerges = 32;
constexpr size_t kFusedSmemLimit = 220 * 1024;

// Smallest cluster size whose per-CTA shared memory fits (0: the fused level never fits).
int fused_min_cluster(const Plan& p) {
  for (int C = 1; C <= 16; C *= 2)
    if (fused_level_smem(p.D, p.N, C) <= kFusedSmemLimit) return C;
  return 0;
}

int fused_policy(const Plan& p, const dsmc_config_t* cfg, int M) {
  if (!p.dense) return 0;
  // default: fused levels evaluate the cross term in FP32 on the CUDA cores, (d + 2) FMAs a
  // pair; with a tensor-core precision and d > 8 the split path's MMA is the cheaper one
  if (cfg->fused_max_merges == 0 && p.compute != DSMC_FP32 && p.D > 8) return 0;
  const int cap = cfg->fused_max_merges == 0 ? kDefaultFusedMaxMerges : cfg->fused_max_merges;
  if (cap < 0 || M > cap) return 0;
  return fused_min_cluster(p);
}

// Largest cluster size <= C that the device can schedule for this shape (queried once).
int fused_schedulable(const Plan& p, const MergeArgs& a, int C) {
  static std::mutex mu;
  static std::vector<std::pair<long long, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const long long key = ((((long long)dev * 64 + p.D) * 32768 + p.N) * 64 + a.B) * 32 + C;
  {
    std::lock_guard<std::mutex> g(mu);
    for (auto& kv : cache)
      if (kv.first == key) return kv.second;
  }
  int ok = 0;
  for (int c = C; c >= 1 && !ok; c /= 2) {
    int n = 0;
    if (level_fused_max_clusters(p.D, a, c, &n) == cudaSuccess && n > 0) ok = c;
  }
  cudaGetLastError();
  std::lock_guard<std::mutex> g(mu);
  cache.emplace_back(key, ok);
  return ok;
}

// Whether a sequence's level with M combinations runs as the fused single-launch level.
// The rule depends only on the sequence's own level (never on what else is launched with
// it), so a sequence's result is the same alone, in a batch or in a serving mix.
bool fused_eligible(const Plan& p, const dsmc_config_t* cfg, int M) { return fused_policy(p, cfg, M) > 0; }

// Cluster size for a fused launch of M combinations: C doubles while the launch still
// fills at most one wave of the SMs and every CTA keeps at least 32 rows.
int fused_cluster(const Plan& p, int M, int sms) {
  int C = 1;
  while (C < 16 && (size_t)M * C * 2 <= (size_t)sms && p.N / (2 * C) >= 32) C *= 2;
  return std::max(C, fused_min_cluster(p));
}

// The launches of M combinations: of the single sequence in `st` at `level` (items null),
// or the list items[0..M) over the sequences `seqs` (levels per item), in chunks of Mc,
// either as fused levels or through the split kernels.
dsmc_status_t launch_combs(const Plan& p, const dsmc_config_t* cfg, const ParamBuf& mp, const float* y,
                           int level, int conditional, dsmc_state_t* st, const WsPtrs& w, cudaStream_t s,
                           int M, const CombItem* items, const SeqDesc* seqs, bool fused) {
  int sms = 0;
  DSMC_CUDA(device_sms(&sms), "SM count");
  const int Cf = fused ? fused_cluster(p, M, sms) : 0;
  for (int m0 = 0; m0 < M; m0 += p.Mc) {
    MergeArgs a = merge_args(p, cfg, y, level, conditional, st, w);
    a.prop_mean = mp.prop_mean;
    a.prop_std = mp.prop_std;
    a.items = items;
    a.seqs = seqs;
    a.m0 = m0;
    a.mc = std::min(p.Mc, M - m0);
    a.gid0 = items ? 0 : p.level_off[level] + m0;
    a.sms = sms;
    chunking(p, a.mc, sms, a.CH, a.CW);
    if (Cf > 0) {
      const int C = fused_schedulable(p, a, Cf);
      if (C > 0) {
        DSMC_CUDA(bd_begin(s, DSMC_KIND_FUSED), "profile event");
        DSMC_CUDA(launch_level_fused(p.D, a, mp.bytes, C, s), "fused level kernel");
        DSMC_CUDA(bd_end(s), "profile event");
        prof_count(1);
        continue;
      }
    }
    if (p.dense && cfg->tc_fused > 0 && p.B == 32 && fused_tc_supported(p.D, p.N, p.compute, p.planes)) {
      DSMC_CUDA(prof_begin(s), "profile event");
      DSMC_CUDA(bd_begin(s, DSMC_KIND_FUSED_TC), "profile event");
      DSMC_CUDA(launch_merge_tc_fused(p.D, a, mp.bytes, s), "fused tensor-core level kernel");
      DSMC_CUDA(bd_end(s), "profile event");
      DSMC_CUDA(prof_end(s, (double)a.mc * p.N * p.N), "profile event");
      prof_count(1);
      continue;
    }
    DSMC_CUDA(bd_begin(s, DSMC_KIND_PROLOGUE), "profile event");
    DSMC_CUDA(launch_prologue(p.D, a, mp.bytes, s), "prologue kernel");
    DSMC_CUDA(bd_end(s), "profile event");
    if (p.dense) {
      DSMC_CUDA(prof_begin(s), "profile event");
      DSMC_CUDA(bd_begin(s, DSMC_KIND_TILE_SUMS), "profile event");
      if (p.compute == DSMC_FP32)
        DSMC_CUDA(launch_rowsum(p.D, a, s), "tile-sum kernel");
      else
        DSMC_CUDA(launch_rowsum_tc(a, s), "tensor-core tile-sum kernel");
      DSMC_CUDA(bd_end(s), "profile event");
      DSMC_CUDA(prof_end(s, (double)a.mc * p.N * p.N), "profile event");
      DSMC_CUDA(bd_begin(s, DSMC_KIND_DRAWS), "profile event");
      DSMC_CUDA(launch_sample_dense(p.D, a, s), "dense sampler kernel");
      DSMC_CUDA(bd_end(s), "profile event");
      prof_count(3);
    } else {
      DSMC_CUDA(bd_begin(s, DSMC_KIND_DRAWS), "profile event");
      if (cfg->resampler == DSMC_RS_FACTORED) {
        DSMC_CUDA(launch_rsf_cdf(a, s), "proposal CDF kernel");
        prof_count(1);
      }
      DSMC_CUDA(launch_sample_rs(p.D, a, s), "lazy sampler kernel");
      DSMC_CUDA(launch_epilogue(a, s), "epilogue kernel");
      DSMC_CUDA(bd_end(s), "profile event");
      prof_count(3);
    }
  }
  return DSMC_OK;
}

dsmc_status_t do_level(const Plan& p, const dsmc_config_t* cfg, const ParamBuf& mp,
                       const float* y, int level, int conditional, dsmc_state_t* st,
                       const WsPtrs& w, cudaStream_t s) {
  const int M = merges_at_level(p.K, level);
  return launch_combs(p, cfg, mp, y, level, conditional, st, w, s, M, nullptr, nullptr,
                      fused_eligible(p, cfg, M));
}

// The gather of one sequence from its composed maps S (w.first, [K][N+1]).
dsmc_status_t do_gather(const Plan& p, const dsmc_state_t* st, float* traj, double* mean, double* m2,
                        float* x_star, const WsPtrs& w, cudaStream_t s) {
  GatherArgs g;
  std::memset(&g, 0, sizeof(g));
  g.K = p.K;
  g.N = p.N;
  g.d = p.d;
  g.L = p.L;
  for (int l = 0; l <= p.L; ++l) g.level_off[l] = p.level_off[l];
  g.S = w.first;
  g.X = st->X;
  g.logw = st->logw;
  g.pairs = st->pairs;
  g.star = w.star;
  g.traj = traj;
  g.mean = mean;
  g.m2 = m2;
  g.x_star = x_star;
  g.status = w.status;
  DSMC_CUDA(bd_begin(s, DSMC_KIND_GATHER), "profile event");
  DSMC_CUDA(launch_gather(p.D, g, s), "gather kernel");
  DSMC_CUDA(bd_end(s), "profile event");
  prof_count(1);
  return DSMC_OK;
}

// Resolution of one sequence: the top-down composition of its pairs (one launch per level,
// root first), then the gather.  w.first must hold [K][N+1] int32 (the map buffers do).
dsmc_status_t do_resolve(const Plan& p, const dsmc_state_t* st, float* traj, double* mean,
                         double* m2, float* x_star, const WsPtrs& w, cudaStream_t s) {
  dsmc_config_t c;
  std::memset(&c, 0, sizeof(c));
  c.K = p.K;
  c.N = p.N;
  for (int l = p.L - 1; l >= 0; --l) {
    MergeArgs a = merge_args(p, &c, nullptr, l, 0, const_cast<dsmc_state_t*>(st), w);
    a.m0 = 0;
    a.mc = merges_at_level(p.K, l);
    a.gid0 = p.level_off[l];
    DSMC_CUDA(bd_begin(s, DSMC_KIND_RESOLVE), "profile event");
    DSMC_CUDA(launch_resolve_level(a, s), "resolve kernel");
    DSMC_CUDA(bd_end(s), "profile event");
    prof_count(1);
  }
  return do_gather(p, st, traj, mean, m2, x_star, w, s);
}

struct Prepared {
  Plan p;
  ParamBuf mp;
  WsPtrs w;
};

dsmc_status_t prepare(const dsmc_config_t* cfg, const dsmc_model_t* model,
                      const dsmc_proposal_t* prop, void* ws, size_t ws_bytes, Prepared& pr) {
  DSMC_TRY(check_config(cfg, model));
  if (prop) DSMC_TRY(check_prop(cfg, model, prop));
  make_plan(cfg, model, pr.p);
  DSMC_TRY(check_ws(pr.p, ws, ws_bytes));
  pr.mp.prop_mean = nullptr;
  pr.mp.prop_std = nullptr;
  if (prop) DSMC_TRY(make_params(pr.p.D, model, prop, pr.mp));
  pr.w = ws_ptrs(pr.p, ws);
  return DSMC_OK;
}

dsmc_status_t run_smooth(const dsmc_config_t* cfg, const dsmc_model_t* model,
                         const dsmc_proposal_t* prop, const float* y, const float* x_ref_in,
                         float* x_ref_out, dsmc_state_t* st, float* traj, double* mean,
                         double* m2, double* logL_out, void* ws, size_t ws_bytes, void* stream) {
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, prop, ws, ws_bytes, pr));
  DSMC_TRY(check_state(st, cfg->K));
  if (!y || !mean) return fail(DSMC_ERR_INVALID_ARG, "y and mean_out are required");
  const bool cond = x_ref_in != nullptr;
  if (cond && cfg->N < 2) return fail(DSMC_ERR_INVALID_ARG, "conditional dSMC needs N >= 2");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DSMC_TRY(do_init(pr.p, cfg, pr.mp, y, x_ref_in, st, pr.w, s));
  for (int l = 0; l < pr.p.L; ++l) DSMC_TRY(do_level(pr.p, cfg, pr.mp, y, l, cond ? 1 : 0, st, pr.w, s));
  if (cond && pr.p.K == 1)
  {
    DSMC_CUDA(launch_k1_star(st->logw, pr.p.N, cfg->seed, cfg->counter_base, pr.w.star, s), "star kernel");
    prof_count(1);
  }
  DSMC_TRY(do_resolve(pr.p, st, traj, mean, m2, cond ? x_ref_out : nullptr, pr.w, s));
  if (logL_out)
    DSMC_CUDA(cudaMemcpyAsync(logL_out, st->logL, sizeof(double), cudaMemcpyDeviceToDevice, s), "logL copy");
  return DSMC_OK;
}

// ---- Scratch for callers that cannot allocate device memory (dsmc_smooth_noalloc).
// A fixed-size device array owned by the library: every device that loads this library
// holds it until the process exits.  Its device address is looked up once per device.
constexpr size_t kNoAllocScratchBytes = DSMC_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};

dsmc_status_t noalloc_scratch(void** ptr) {
  int dev = 0;
  DSMC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(DSMC_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    // the host-side name of the array is not a device address: ask the runtime for it
    void* p = nullptr;
    DSMC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return DSMC_OK;
}

// ---- Batched smoothing: many sequences of one (model, N, precision), their combinations
// of each level launched together (one item list per level, chunks of Mc).
template <int D>
void set_prop_t(ParamBuf& b, const float* mean, const float* sd) {
  ModelParams<D>* mp = reinterpret_cast<ModelParams<D>*>(b.bytes);
  mp->prop_mean = mean;
  mp->prop_std = sd;
  b.prop_mean = mean;
  b.prop_std = sd;
}

void set_prop(int D, ParamBuf& b, const float* mean, const float* sd) {
  switch (D) {
    case 1: set_prop_t<1>(b, mean, sd); break;
    case 2: set_prop_t<2>(b, mean, sd); break;
    case 4: set_prop_t<4>(b, mean, sd); break;
    case 8: set_prop_t<8>(b, mean, sd); break;
    case 16: set_prop_t<16>(b, mean, sd); break;
    default: set_prop_t<32>(b, mean, sd); break;
  }
}

int levels_of(int K) {
  int L = 0;
  while ((1 << L) < K) ++L;
  return L;
}

struct BatchLayout {
  Plan p;                        // merge workspace for Mc combinations (K = the longest sequence)
  int n_seq = 0, Lmax = 0;
  std::vector<int> level_start;  // [Lmax + 1] offsets of each level's items
  std::vector<int> level_fused;  // [Lmax] end of the level's fused items (they come first)
  std::vector<size_t> map_off;   // per sequence: byte offset of its first / last maps
  size_t n_items = 0;
  size_t o_desc = 0, o_kstart = 0, o_items = 0, o_maps = 0, o_star = 0, total = 0;
  long long sumK = 0;
};

dsmc_status_t batch_layout(const dsmc_config_t* cfg, const dsmc_model_t* model, int n_seq, const int* K,
                           BatchLayout& bl) {
  if (n_seq < 1 || !K) return fail(DSMC_ERR_INVALID_ARG, "a batch needs n_seq >= 1 sequence lengths");
  int Kmax = 0;
  long long m0 = 0, items = 0;
  for (int i = 0; i < n_seq; ++i) {
    if (K[i] < 1) return fail(DSMC_ERR_INVALID_ARG, "every sequence needs K >= 1");
    Kmax = std::max(Kmax, K[i]);
    m0 += merges_at_level(K[i], 0);
    items += K[i] - 1;
  }
  if (items > (1LL << 30)) return fail(DSMC_ERR_INVALID_ARG, "too many combinations in one batch");
  dsmc_config_t c = *cfg;
  c.K = Kmax;
  DSMC_TRY(check_config(&c, model));
  make_plan(&c, model, bl.p, (int)std::min<long long>(m0, 1 << 30), true);
  bl.n_seq = n_seq;
  bl.Lmax = levels_of(Kmax);
  bl.level_start.assign(bl.Lmax + 1, 0);
  bl.level_fused.assign(bl.Lmax, 0);
  for (int l = 0; l < bl.Lmax; ++l) {
    long long cnt = 0, cf = 0;
    for (int i = 0; i < n_seq; ++i) {
      const int M = merges_at_level(K[i], l);
      cnt += M;
      if (M > 0 && fused_eligible(bl.p, cfg, M)) cf += M;
    }
    bl.level_start[l + 1] = bl.level_start[l] + (int)cnt;
    bl.level_fused[l] = bl.level_start[l] + (int)cf;
  }
  bl.n_items = (size_t)items;
  bl.sumK = 0;
  for (int i = 0; i < n_seq; ++i) bl.sumK += K[i];
  if (bl.sumK > (1LL << 31) - 1) return fail(DSMC_ERR_INVALID_ARG, "too many time steps in one batch");
  size_t o = bl.p.total;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  bl.o_desc = take((size_t)n_seq * sizeof(SeqDesc));
  bl.o_kstart = take((size_t)(n_seq + 1) * sizeof(int));
  bl.o_items = take(bl.n_items * sizeof(CombItem));
  bl.o_star = take((size_t)n_seq * 2 * sizeof(int32_t));
  bl.map_off.resize(n_seq);
  bl.o_maps = o;
  for (int i = 0; i < n_seq; ++i) bl.map_off[i] = take(2 * 2 * (size_t)K[i] * cfg->N * sizeof(int32_t));
  bl.total = o;
  return DSMC_OK;
}

// Host copies of the descriptors and the level-major item list of a batch.
dsmc_status_t batch_tables(const dsmc_config_t* cfg, const BatchLayout& bl, const dsmc_seq_t* seqs,
                           char* ws, std::vector<SeqDesc>& desc, std::vector<CombItem>& items,
                           std::vector<int>& kstart) {
  const int N = cfg->N;
  desc.resize(bl.n_seq);
  for (int i = 0; i < bl.n_seq; ++i) {
    const dsmc_seq_t& q = seqs[i];
    SeqDesc& d = desc[i];
    d.K = q.K;
    d.L = levels_of(q.K);
    d.X = q.state.X;
    d.logw = q.state.logw;
    d.y = q.y;
    d.logL = q.state.logL;
    d.pairs = q.state.pairs;
    if (q.maps) {
      d.first = static_cast<int32_t*>(q.maps);
      d.last = d.first + 2 * (size_t)q.K * N;
      d.star = d.last + 2 * (size_t)q.K * N;
    } else {
      d.first = reinterpret_cast<int32_t*>(ws + bl.map_off[i]);
      d.last = d.first + 2 * (size_t)q.K * N;
      d.star = reinterpret_cast<int32_t*>(ws + bl.o_star) + 2 * (size_t)i;
    }
    d.prop_mean = q.prop_mean;
    d.prop_std = q.prop_std;
    d.seed = q.seed;
    d.base = q.counter_base;
    d.conditional = q.x_ref_in != nullptr ? 1 : 0;
    d.x_ref = q.x_ref_in;
    d.mean = q.mean_out;
    d.m2 = q.m2_out;
    d.x_star = q.x_ref_out;
    d.logL_out = q.logL_out;
  }
  kstart.assign(bl.n_seq + 1, 0);
  for (int i = 0; i < bl.n_seq; ++i) kstart[i + 1] = kstart[i] + seqs[i].K;
  items.resize(bl.n_items);
  std::vector<int> off(bl.n_seq, 0);  // per sequence: combinations of the levels so far
  for (int l = 0; l < bl.Lmax; ++l) {
    size_t at_f = bl.level_start[l], at_s = bl.level_fused[l];
    for (int i = 0; i < bl.n_seq; ++i) {
      const int M = merges_at_level(seqs[i].K, l);
      const bool fz = M > 0 && fused_eligible(bl.p, cfg, M);
      for (int m = 0; m < M; ++m) items[fz ? at_f++ : at_s++] = CombItem{i, m, off[i] + m, l};
      off[i] += M;
    }
  }
  return DSMC_OK;
}

dsmc_status_t check_batch(const dsmc_config_t* cfg, const dsmc_model_t* model, const dsmc_proposal_t* prop,
                          int n_seq, const dsmc_seq_t* seqs) {
  if (!prop) return fail(DSMC_ERR_INVALID_ARG, "null proposal");
  if (n_seq < 1 || !seqs) return fail(DSMC_ERR_INVALID_ARG, "a batch needs n_seq >= 1 sequences");
  for (int i = 0; i < n_seq; ++i) {
    const dsmc_seq_t& q = seqs[i];
    if (q.K < 1 || !q.y || !q.mean_out) return fail(DSMC_ERR_INVALID_ARG, "sequence: K, y and mean_out");
    DSMC_TRY(check_state(&q.state, q.K));
    if (prop->kind == DSMC_PROP_GAUSS && (!q.prop_mean || !q.prop_std))
      return fail(DSMC_ERR_INVALID_ARG, "sequence: proposal mean/std arrays");
    if (q.x_ref_in && cfg->N < 2) return fail(DSMC_ERR_INVALID_ARG, "conditional dSMC needs N >= 2");
    if (q.counter_base >= (1u << 28)) return fail(DSMC_ERR_INVALID_ARG, "counter_base must be < 2^28");
  }
  dsmc_config_t c = *cfg;
  c.K = seqs[0].K;
  DSMC_TRY(check_config(&c, model));
  dsmc_proposal_t pp = *prop;
  pp.mean = seqs[0].prop_mean;
  pp.std = seqs[0].prop_std;
  DSMC_TRY(check_prop(&c, model, &pp));
  return DSMC_OK;
}

std::vector<int> batch_lengths(int n_seq, const dsmc_seq_t* seqs) {
  std::vector<int> K(n_seq);
  for (int i = 0; i < n_seq; ++i) K[i] = seqs[i].K;
  return K;
}

// The root-draw pair of sequence i: in its own maps scratch, or slot i of `stars`.
int32_t* seq_star(const dsmc_seq_t& q, int N, char* stars, int i) {
  if (q.maps) return static_cast<int32_t*>(q.maps) + 4 * (size_t)q.K * N;
  return reinterpret_cast<int32_t*>(stars) + 2 * (size_t)i;
}

// Everything of a batched call that the launches need.
struct BatchRun {
  BatchLayout bl;
  ParamBuf mp;
  WsPtrs w;
};

dsmc_status_t batch_setup(const dsmc_config_t* cfg, const dsmc_model_t* model, const dsmc_proposal_t* prop,
                          int n_seq, const dsmc_seq_t* seqs, void* ws, size_t ws_bytes, BatchRun& br) {
  DSMC_TRY(check_batch(cfg, model, prop, n_seq, seqs));
  const std::vector<int> K = batch_lengths(n_seq, seqs);
  DSMC_TRY(batch_layout(cfg, model, n_seq, K.data(), br.bl));
  if (!ws) return fail(DSMC_ERR_INVALID_ARG, "null workspace");
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return fail(DSMC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (ws_bytes < br.bl.total) return fail(DSMC_ERR_WORKSPACE, "workspace too small for the batch");
  br.mp.prop_mean = nullptr;
  br.mp.prop_std = nullptr;
  dsmc_proposal_t pp = *prop;
  pp.mean = nullptr;
  pp.std = nullptr;
  DSMC_TRY(make_params(br.bl.p.D, model, &pp, br.mp));
  br.w = ws_ptrs(br.bl.p, ws);
  return DSMC_OK;
}

dsmc_status_t batch_upload(const dsmc_config_t* cfg, const BatchRun& br, const dsmc_seq_t* seqs, void* ws,
                           cudaStream_t s) {
  std::vector<SeqDesc> desc;
  std::vector<CombItem> items;
  std::vector<int> kstart;
  char* b = static_cast<char*>(ws);
  DSMC_TRY(batch_tables(cfg, br.bl, seqs, b, desc, items, kstart));
  DSMC_CUDA(cudaMemcpyAsync(b + br.bl.o_desc, desc.data(), desc.size() * sizeof(SeqDesc),
                            cudaMemcpyHostToDevice, s), "descriptor upload");
  DSMC_CUDA(cudaMemcpyAsync(b + br.bl.o_kstart, kstart.data(), kstart.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s), "time-step table upload");
  if (!items.empty())
    DSMC_CUDA(cudaMemcpyAsync(b + br.bl.o_items, items.data(), items.size() * sizeof(CombItem),
                              cudaMemcpyHostToDevice, s), "item upload");
  // pageable sources: the copies are staged before the calls return; wait for them so the
  // host tables may go out of scope whatever the runtime does
  DSMC_CUDA(cudaStreamSynchronize(s), "upload synchronize");
  return DSMC_OK;
}

dsmc_status_t batch_launch(const dsmc_config_t* cfg, const dsmc_model_t* model, const BatchRun& br,
                           const dsmc_seq_t* seqs, void* ws, cudaStream_t s) {
  const BatchLayout& bl = br.bl;
  const Plan& p = bl.p;
  char* b = static_cast<char*>(ws);
  DSMC_CUDA(cudaMemsetAsync(br.w.status, 0, sizeof(int), s), "reset status");
  DSMC_CUDA(cudaMemsetAsync(br.w.attempts_total, 0, sizeof(unsigned long long), s), "reset attempts");
  DSMC_CUDA(cudaMemsetAsync(b + bl.o_star, 0, (size_t)bl.n_seq * 2 * sizeof(int32_t), s), "reset stars");
  for (int i = 0; i < bl.n_seq; ++i)
    if (seqs[i].maps)
      DSMC_CUDA(cudaMemsetAsync(seq_star(seqs[i], p.N, nullptr, i), 0, 2 * sizeof(int32_t), s), "reset star");
  // Algorithm 2: one launch over every time step of every sequence
  const SeqDesc* descs = reinterpret_cast<const SeqDesc*>(b + bl.o_desc);
  const int* kstart = reinterpret_cast<const int*>(b + bl.o_kstart);
  {
    InitArgs ia;
    std::memset(&ia, 0, sizeof(ia));
    ia.K = (int)bl.sumK;
    ia.N = p.N;
    ia.d = p.d;
    ia.logN = (float)std::log((double)p.N);
    ia.seqs = descs;
    ia.kstart = kstart;
    ia.n_seq = bl.n_seq;
    ia.status = br.w.status;
    DSMC_CUDA(bd_begin(s, DSMC_KIND_INIT), "profile event");
    DSMC_CUDA(launch_init(p.D, ia, br.mp.bytes, s), "init kernel");
    DSMC_CUDA(bd_end(s), "profile event");
    prof_count(1);
  }
  // the levels of Algorithm 6, every sequence's combinations of a level together
  const CombItem* items = reinterpret_cast<const CombItem*>(b + bl.o_items);
  dsmc_state_t none = {nullptr, nullptr, nullptr, nullptr};
  for (int l = 0; l < bl.Lmax; ++l) {
    const int Mf = bl.level_fused[l] - bl.level_start[l];
    const int Ms = bl.level_start[l + 1] - bl.level_fused[l];
    if (Mf > 0)
      DSMC_TRY(launch_combs(p, cfg, br.mp, nullptr, l, 0, &none, br.w, s, Mf, items + bl.level_start[l], descs,
                            true));
    if (Ms > 0)
      DSMC_TRY(launch_combs(p, cfg, br.mp, nullptr, l, 0, &none, br.w, s, Ms, items + bl.level_fused[l], descs,
                            false));
  }
  // resolution: the top-down composition, every sequence's combinations of a level together
  // (root levels first)
  for (int l = bl.Lmax - 1; l >= 0; --l) {
    const int M = bl.level_start[l + 1] - bl.level_start[l];
    if (M == 0) continue;
    MergeArgs a = merge_args(p, cfg, nullptr, l, 0, &none, br.w);
    a.items = items + bl.level_start[l];
    a.seqs = descs;
    a.m0 = 0;
    a.mc = M;
    DSMC_CUDA(bd_begin(s, DSMC_KIND_RESOLVE), "profile event");
    DSMC_CUDA(launch_resolve_level(a, s), "resolve kernel");
    DSMC_CUDA(bd_end(s), "profile event");
    prof_count(1);
  }
  // the root draw of conditional sequences of length 1 (from the weighted leaf)
  for (int i = 0; i < bl.n_seq; ++i) {
    const dsmc_seq_t& q = seqs[i];
    if (q.x_ref_in != nullptr && q.K == 1) {
      DSMC_CUDA(launch_k1_star(q.state.logw, p.N, q.seed, q.counter_base, seq_star(q, p.N, b + bl.o_star, i), s),
                "star kernel");
      prof_count(1);
    }
  }
  // the gather: one launch over every time step of every sequence (means, second moments,
  // next references, log L of the root)
  {
    GatherArgs g;
    std::memset(&g, 0, sizeof(g));
    g.K = (int)bl.sumK;
    g.N = p.N;
    g.d = p.d;
    g.seqs = descs;
    g.kstart = kstart;
    g.n_seq = bl.n_seq;
    g.status = br.w.status;
    DSMC_CUDA(bd_begin(s, DSMC_KIND_GATHER), "profile event");
  DSMC_CUDA(launch_gather(p.D, g, s), "gather kernel");
  DSMC_CUDA(bd_end(s), "profile event");
    prof_count(1);
  }
  (void)model;
  return DSMC_OK;
}

// ---- Continuous batching: one tick = one stage of every sequence of the call.
// Workspace: the merge workspace for Mc combinations (Mc = the launch cap), then the tick's
// descriptor table and its combination list.
dsmc_status_t serve_plan(const dsmc_config_t* cfg, const dsmc_model_t* model, Plan& p) {
  dsmc_config_t c = *cfg;
  c.K = 2;
  DSMC_TRY(check_config(&c, model));
  const int cap = cfg->max_merges_per_launch > 0 ? cfg->max_merges_per_launch : kDefaultMergeCap;
  make_plan(&c, model, p, cap, true);
  return DSMC_OK;
}

int level_offset(int K, int level) {
  int off = 0;
  for (int l = 0; l < level; ++l) off += merges_at_level(K, l);
  return off;
}

dsmc_status_t serve_tick(const dsmc_config_t* cfg, const dsmc_model_t* model, const dsmc_proposal_t* prop,
                         int n_seq, const dsmc_seq_t* seqs, const int* stage, void* ws, size_t ws_bytes,
                         cudaStream_t s) {
  DSMC_TRY(check_batch(cfg, model, prop, n_seq, seqs));
  if (!stage) return fail(DSMC_ERR_INVALID_ARG, "null stage array");
  for (int i = 0; i < n_seq; ++i) {
    if (!seqs[i].maps) return fail(DSMC_ERR_INVALID_ARG, "serving needs every sequence's maps scratch");
    if (stage[i] < -1 || stage[i] > levels_of(seqs[i].K)) return fail(DSMC_ERR_INVALID_ARG, "stage out of range");
  }
  Plan p;
  DSMC_TRY(serve_plan(cfg, model, p));
  if (!ws) return fail(DSMC_ERR_INVALID_ARG, "null workspace");
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return fail(DSMC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  ParamBuf mp;
  mp.prop_mean = nullptr;
  mp.prop_std = nullptr;
  dsmc_proposal_t pp = *prop;
  pp.mean = nullptr;
  pp.std = nullptr;
  DSMC_TRY(make_params(p.D, model, &pp, mp));
  const WsPtrs w = ws_ptrs(p, ws);
  char* b = static_cast<char*>(ws);
  const int N = p.N;
  // tables: descriptors, then the combinations (fused-eligible first)
  std::vector<SeqDesc> desc(n_seq);
  std::vector<CombItem> fz, sp;
  for (int i = 0; i < n_seq; ++i) {
    const dsmc_seq_t& q = seqs[i];
    SeqDesc& d = desc[i];
    d.K = q.K;
    d.L = levels_of(q.K);
    d.X = q.state.X;
    d.logw = q.state.logw;
    d.y = q.y;
    d.logL = q.state.logL;
    d.pairs = q.state.pairs;
    d.first = static_cast<int32_t*>(q.maps);
    d.last = d.first + 2 * (size_t)q.K * N;
    d.star = d.last + 2 * (size_t)q.K * N;
    d.prop_mean = q.prop_mean;
    d.prop_std = q.prop_std;
    d.seed = q.seed;
    d.base = q.counter_base;
    d.conditional = q.x_ref_in != nullptr ? 1 : 0;
    d.x_ref = q.x_ref_in;
    d.mean = q.mean_out;
    d.m2 = q.m2_out;
    d.x_star = q.x_ref_out;
    d.logL_out = q.logL_out;
    const int l = stage[i];
    if (l >= 0 && l < d.L) {
      const int M = merges_at_level(q.K, l);
      const int off = level_offset(q.K, l);
      std::vector<CombItem>& dst = fused_eligible(p, cfg, M) ? fz : sp;
      for (int m = 0; m < M; ++m) dst.push_back(CombItem{i, m, off + m, l});
    }
  }
  const size_t o_desc = align256(p.total);
  const size_t o_items = align256(o_desc + (size_t)n_seq * sizeof(SeqDesc));
  const size_t need = o_items + (fz.size() + sp.size()) * sizeof(CombItem);
  if (ws_bytes < need) return fail(DSMC_ERR_WORKSPACE, "workspace too small for this tick");
  std::vector<CombItem> items(fz);
  items.insert(items.end(), sp.begin(), sp.end());
  DSMC_CUDA(cudaMemcpyAsync(b + o_desc, desc.data(), desc.size() * sizeof(SeqDesc), cudaMemcpyHostToDevice, s),
            "descriptor upload");
  if (!items.empty())
    DSMC_CUDA(cudaMemcpyAsync(b + o_items, items.data(), items.size() * sizeof(CombItem), cudaMemcpyHostToDevice,
                              s), "item upload");
  DSMC_CUDA(cudaStreamSynchronize(s), "upload synchronize");
  DSMC_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), s), "reset status");
  DSMC_CUDA(cudaMemsetAsync(w.attempts_total, 0, sizeof(unsigned long long), s), "reset attempts");
  // stage -1: Algorithm 2
  for (int i = 0; i < n_seq; ++i) {
    if (stage[i] != -1) continue;
    const dsmc_seq_t& q = seqs[i];
    DSMC_CUDA(cudaMemsetAsync(desc[i].star, 0, 2 * sizeof(int32_t), s), "reset star");
    ParamBuf mpi = mp;
    set_prop(p.D, mpi, q.prop_mean, q.prop_std);
    InitArgs ia;
    std::memset(&ia, 0, sizeof(ia));
    ia.K = q.K;
    ia.N = N;
    ia.logN = (float)std::log((double)N);
    ia.d = p.d;
    ia.seed = q.seed;
    ia.base = q.counter_base;
    ia.y = q.y;
    ia.x_ref = q.x_ref_in;
    ia.X = q.state.X;
    ia.logw = q.state.logw;
    ia.logL = q.state.logL;
    ia.status = w.status;
    DSMC_CUDA(bd_begin(s, DSMC_KIND_INIT), "profile event");
    DSMC_CUDA(launch_init(p.D, ia, mpi.bytes, s), "init kernel");
    DSMC_CUDA(bd_end(s), "profile event");
    prof_count(1);
  }
  // merge stages: every sequence's level, together
  const SeqDesc* descs = reinterpret_cast<const SeqDesc*>(b + o_desc);
  const CombItem* dev_items = reinterpret_cast<const CombItem*>(b + o_items);
  dsmc_state_t none = {nullptr, nullptr, nullptr, nullptr};
  if (!fz.empty())
    DSMC_TRY(launch_combs(p, cfg, mp, nullptr, 0, 0, &none, w, s, (int)fz.size(), dev_items, descs, true));
  if (!sp.empty())
    DSMC_TRY(launch_combs(p, cfg, mp, nullptr, 0, 0, &none, w, s, (int)sp.size(), dev_items + fz.size(), descs,
                          false));
  // stage L: resolve
  for (int i = 0; i < n_seq; ++i) {
    const dsmc_seq_t& q = seqs[i];
    if (stage[i] != desc[i].L) continue;
    dsmc_config_t c = *cfg;
    c.K = q.K;
    Plan pi;
    make_plan(&c, model, pi, 1, true);
    WsPtrs wi = w;
    wi.star = desc[i].star;
    wi.first = desc[i].first;
    const bool cond = q.x_ref_in != nullptr;
    if (cond && q.K == 1) {
      DSMC_CUDA(launch_k1_star(q.state.logw, N, q.seed, q.counter_base, wi.star, s), "star kernel");
      prof_count(1);
    }
    dsmc_state_t st = q.state;
    DSMC_TRY(do_resolve(pi, &st, nullptr, q.mean_out, q.m2_out, cond ? q.x_ref_out : nullptr, wi, s));
    if (q.logL_out)
      DSMC_CUDA(cudaMemcpyAsync(q.logL_out, q.state.logL, sizeof(double), cudaMemcpyDeviceToDevice, s),
                "logL copy");
  }
  return DSMC_OK;
}

}  // namespace

extern "C" {

const char* dsmc_status_string(dsmc_status_t s) {
  switch (s) {
    case DSMC_OK: return "ok";
    case DSMC_ERR_INVALID_ARG: return "invalid argument";
    case DSMC_ERR_UNSUPPORTED: return "unsupported";
    case DSMC_ERR_WORKSPACE: return "workspace too small";
    case DSMC_ERR_CUDA: return "CUDA error";
    case DSMC_ERR_NONFINITE: return "non-finite log-weight";
    case DSMC_ERR_DEGENERATE: return "all weights of a combination are zero";
    case DSMC_ERR_RS_LIMIT: return "rejection sampling reached its attempt cap";
    case DSMC_ERR_TIMEOUT: return "bounded wait timed out";
    case DSMC_ERR_BOUND: return "a lazy sampler's pair exceeded its bound";
  }
  return "unknown status";
}

const char* dsmc_last_error(void) { return g_last_error.c_str(); }

dsmc_status_t dsmc_state_sizes(const dsmc_config_t* cfg, const dsmc_model_t* model,
                               size_t bytes_out[4]) {
  DSMC_TRY(check_config(cfg, model));
  if (!bytes_out) return fail(DSMC_ERR_INVALID_ARG, "null output");
  const size_t K = cfg->K, N = cfg->N, d = model->dx;
  bytes_out[0] = K * N * d * sizeof(float);
  bytes_out[1] = K * N * sizeof(float);
  bytes_out[2] = K * sizeof(double);
  bytes_out[3] = (K > 1 ? K - 1 : 0) * 2 * N * sizeof(int32_t);
  return DSMC_OK;
}

dsmc_status_t dsmc_workspace_size(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                  size_t* bytes) {
  DSMC_TRY(check_config(cfg, model));
  if (!bytes) return fail(DSMC_ERR_INVALID_ARG, "null output");
  Plan p;
  make_plan(cfg, model, p);
  *bytes = p.total;
  return DSMC_OK;
}

dsmc_status_t dsmc_init_particles(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                  const dsmc_proposal_t* prop, const float* y,
                                  const float* x_ref, dsmc_state_t* state, void* ws,
                                  size_t ws_bytes, void* stream) {
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, prop, ws, ws_bytes, pr));
  DSMC_TRY(check_state(state, cfg->K));
  if (!y) return fail(DSMC_ERR_INVALID_ARG, "y is required");
  return do_init(pr.p, cfg, pr.mp, y, x_ref, state, pr.w, static_cast<cudaStream_t>(stream));
}

dsmc_status_t dsmc_merge_level(const dsmc_config_t* cfg, const dsmc_model_t* model,
                               const dsmc_proposal_t* prop, const float* y, int level,
                               int conditional, dsmc_state_t* state, void* ws,
                               size_t ws_bytes, void* stream) {
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, prop, ws, ws_bytes, pr));
  DSMC_TRY(check_state(state, cfg->K));
  if (!y) return fail(DSMC_ERR_INVALID_ARG, "y is required");
  if (level < 0 || level >= pr.p.L) return fail(DSMC_ERR_INVALID_ARG, "level out of range");
  if (conditional && cfg->N < 2) return fail(DSMC_ERR_INVALID_ARG, "conditional dSMC needs N >= 2");
  return do_level(pr.p, cfg, pr.mp, y, level, conditional ? 1 : 0, state, pr.w,
                  static_cast<cudaStream_t>(stream));
}

dsmc_status_t dsmc_resolve(const dsmc_config_t* cfg, const dsmc_model_t* model,
                           const dsmc_state_t* state, float* traj_out, double* mean_out,
                           double* m2_out, float* x_star_out, void* ws, size_t ws_bytes,
                           void* stream) {
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, nullptr, ws, ws_bytes, pr));
  DSMC_TRY(check_state(state, cfg->K));
  if (!mean_out) return fail(DSMC_ERR_INVALID_ARG, "mean_out is required");
  return do_resolve(pr.p, state, traj_out, mean_out, m2_out, x_star_out, pr.w,
                    static_cast<cudaStream_t>(stream));
}

dsmc_status_t dsmc_smooth(const dsmc_config_t* cfg, const dsmc_model_t* model,
                          const dsmc_proposal_t* prop, const float* y, dsmc_state_t* state,
                          float* traj_out, double* mean_out, double* m2_out, double* logL_out,
                          void* ws, size_t ws_bytes, void* stream) {
  return run_smooth(cfg, model, prop, y, nullptr, nullptr, state, traj_out, mean_out, m2_out,
                    logL_out, ws, ws_bytes, stream);
}

dsmc_status_t dsmc_conditional_smooth(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                      const dsmc_proposal_t* prop, const float* y,
                                      const float* x_ref_in, float* x_ref_out,
                                      dsmc_state_t* state, float* traj_out, double* mean_out,
                                      double* logL_out, void* ws, size_t ws_bytes,
                                      void* stream) {
  if (!x_ref_in || !x_ref_out) return fail(DSMC_ERR_INVALID_ARG, "x_ref_in and x_ref_out are required");
  return run_smooth(cfg, model, prop, y, x_ref_in, x_ref_out, state, traj_out, mean_out, nullptr,
                    logL_out, ws, ws_bytes, stream);
}

dsmc_status_t dsmc_smooth_noalloc(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                  const dsmc_proposal_t* prop, const float* y, dsmc_state_t* state,
                                  float* traj_out, double* mean_out, double* m2_out,
                                  double* logL_out, dsmc_status_t* device_status, void* stream) {
  DSMC_TRY(check_config(cfg, model));
  Plan p;
  make_plan(cfg, model, p);
  if (p.total > kNoAllocScratchBytes)
    return fail(DSMC_ERR_WORKSPACE,
                "this problem needs " + std::to_string(p.total) + " bytes of workspace, more than the " +
                    std::to_string(kNoAllocScratchBytes) +
                    "-byte static scratch of dsmc_smooth_noalloc; use dsmc_smooth with a caller buffer");
  void* ws = nullptr;
  DSMC_TRY(noalloc_scratch(&ws));
  DSMC_TRY(run_smooth(cfg, model, prop, y, nullptr, nullptr, state, traj_out, mean_out, m2_out,
                      logL_out, ws, kNoAllocScratchBytes, stream));
  if (device_status) {
    int h = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DSMC_CUDA(cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, s), "status copy");
    DSMC_CUDA(cudaStreamSynchronize(s), "stream synchronize");
    *device_status = static_cast<dsmc_status_t>(h);
  }
  return DSMC_OK;
}

dsmc_status_t dsmc_gaussian_proposals_workspace_size(const dsmc_model_t* model, int K, size_t* bytes) {
  if (!model || !bytes) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  dsmc_config_t c;
  std::memset(&c, 0, sizeof(c));
  c.K = K;
  c.N = 1;
  DSMC_TRY(check_config(&c, model));
  *bytes = pit_workspace_bytes(K, model->dx);
  return DSMC_OK;
}

dsmc_status_t dsmc_gaussian_proposals(const dsmc_model_t* model, int K, const float* y, int iterations,
                                      const float* init_mean, float* mean_out, float* std_out, void* ws,
                                      size_t ws_bytes, void* stream) {
  if (!model || !y || !mean_out || !std_out) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  dsmc_config_t c;
  std::memset(&c, 0, sizeof(c));
  c.K = K;
  c.N = 1;
  DSMC_TRY(check_config(&c, model));
  if (iterations < 1) return fail(DSMC_ERR_INVALID_ARG, "iterations must be >= 1");
  if (!ws) return fail(DSMC_ERR_INVALID_ARG, "null workspace");
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return fail(DSMC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  const int d = model->dx;
  if (ws_bytes < pit_workspace_bytes(K, d)) return fail(DSMC_ERR_WORKSPACE, "workspace too small");
  // the model in FP64: F, Q, R, P0 [d][d], c, m0 [d]
  std::vector<double> mdl(4 * (size_t)d * d + 2 * (size_t)d, 0.0);
  double* F = mdl.data();
  double* Q = F + d * d;
  double* R = Q + d * d;
  double* P0 = R + d * d;
  double* cc = P0 + d * d;
  double* m0 = cc + d;
  PitArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.K = K;
  pa.d = d;
  pa.kind = model->kind;
  pa.y = y;
  if (model->kind != DSMC_MODEL_LGSSM) {
    if (model->kind == DSMC_MODEL_CRW)
      return fail(DSMC_ERR_UNSUPPORTED, "the constrained random walk has no Gaussian linearisation");
    const double s2 = model->sigma * model->sigma;
    Q[0] = s2;
    if (model->kind == DSMC_MODEL_THETA_LOGISTIC) {
      F[0] = 1.0;  // replaced by the per-step linearisation
      R[0] = model->obs_sd * model->obs_sd;
      P0[0] = 1.0;
      m0[0] = 0.0;
      pa.tau0 = model->tau0;
      pa.tau1 = model->tau1;
      pa.tau2 = model->tau2;
    } else {  // SV, COX: pseudo-observations carry their own variances
      F[0] = model->kind == DSMC_MODEL_COX ? model->phi * model->lam : model->phi;
      R[0] = 0.0;
      P0[0] = s2 / (1.0 - model->phi * model->phi);
      cc[0] = model->mu * (1.0 - model->phi);
      m0[0] = model->mu;
      pa.mu = model->mu;
    }
  } else {
    double L[kMaxDim * kMaxDim];
    if (!cholesky(d, model->Q, L) || !cholesky(d, model->R, L) || !cholesky(d, model->P0, L))
      return fail(DSMC_ERR_INVALID_ARG, "Q, R and P0 must be positive definite");
    for (int i = 0; i < d * d; ++i) {
      F[i] = model->A[i];
      Q[i] = model->Q[i];
      R[i] = model->R[i];
      P0[i] = model->P0[i];
    }
    for (int i = 0; i < d; ++i) m0[i] = model->m0[i];
  }
  int launches = 0;
  DSMC_CUDA(launch_pit(pa, mdl.data(), iterations, init_mean, mean_out, std_out, ws,
                       static_cast<cudaStream_t>(stream), &launches),
            "linearised smoother kernels");
  prof_count(launches);
  return DSMC_OK;
}

dsmc_status_t dsmc_stream_status(void* ws, void* stream, dsmc_status_t* device_status) {
  if (!ws || !device_status) return fail(DSMC_ERR_INVALID_ARG, "null workspace or output");
  int h = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the status word is the first field of every workspace layout
  DSMC_CUDA(cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, s), "status copy");
  DSMC_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  *device_status = static_cast<dsmc_status_t>(h);
  return DSMC_OK;
}

dsmc_status_t dsmc_profile_enable(int enable) {
  g_prof.on = enable != 0;
  g_prof.used = 0;
  g_prof.launches = 0;
  g_prof.pairs = 0.0;
  return DSMC_OK;
}

dsmc_status_t dsmc_profile_read(double* rowsum_ms, int64_t* rowsum_launches, double* rowsum_pairs,
                                int64_t* all_launches) {
  double ms = 0.0;
  for (size_t i = 0; i < g_prof.used; ++i) {
    DSMC_CUDA(cudaEventSynchronize(g_prof.stop[i]), "profile synchronize");
    float t = 0.f;
    DSMC_CUDA(cudaEventElapsedTime(&t, g_prof.start[i], g_prof.stop[i]), "profile elapsed");
    ms += t;
  }
  if (rowsum_ms) *rowsum_ms = ms;
  if (rowsum_launches) *rowsum_launches = (int64_t)g_prof.used;
  if (rowsum_pairs) *rowsum_pairs = g_prof.pairs;
  if (all_launches) *all_launches = g_prof.launches;
  return DSMC_OK;
}

dsmc_status_t dsmc_profile_breakdown_enable(int enable) {
  g_bd.on = enable != 0;
  g_bd.used = 0;
  return DSMC_OK;
}

dsmc_status_t dsmc_profile_breakdown_read(double* ms, int64_t* launches) {
  if (!ms || !launches) return fail(DSMC_ERR_INVALID_ARG, "null output");
  for (int k = 0; k < DSMC_KINDS; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i < g_bd.used; ++i) {
    DSMC_CUDA(cudaEventSynchronize(g_bd.b[i]), "profile synchronize");
    float t = 0.f;
    DSMC_CUDA(cudaEventElapsedTime(&t, g_bd.a[i], g_bd.b[i]), "profile elapsed");
    const int k = g_bd.kind[i];
    ms[k] += t;
    launches[k] += 1;
  }
  return DSMC_OK;
}

dsmc_status_t dsmc_debug_stall_tensor_cores(int enable) {
  g_stall_tc = enable != 0;
  return DSMC_OK;
}

dsmc_status_t dsmc_debug_keep_weights(int enable) {
  g_keep_weights = enable != 0;
  return DSMC_OK;
}

dsmc_status_t dsmc_debug_philox(const uint32_t* ctr, int64_t n, uint64_t seed, uint32_t* out,
                                void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return fail(DSMC_ERR_INVALID_ARG, "philox buffers");
  DSMC_CUDA(launch_philox(ctr, n, seed, out, static_cast<cudaStream_t>(stream)), "philox kernel");
  return DSMC_OK;
}

dsmc_status_t dsmc_debug_merge_weights(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                       int level, int m, float* logW, float* r, float* rowsum,
                                       float* tiles, float* e, float* ratio, int info[4],
                                       void* ws, size_t ws_bytes, void* stream) {
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, nullptr, ws, ws_bytes, pr));
  const Plan& p = pr.p;
  if (level < 0 || level >= p.L) return fail(DSMC_ERR_INVALID_ARG, "level out of range");
  const int M = merges_at_level(p.K, level);
  if (m < 0 || m >= M) return fail(DSMC_ERR_INVALID_ARG, "combination out of range");
  const int last_chunk = ((M - 1) / p.Mc) * p.Mc;
  if (m < last_chunk) return fail(DSMC_ERR_INVALID_ARG, "combination not in the last launch chunk");
  if (!p.dense && (r || rowsum || tiles))
    return fail(DSMC_ERR_INVALID_ARG, "row/tile weights exist only with dense resampling");
  dsmc_state_t dummy = {nullptr, nullptr, nullptr, nullptr};
  MergeArgs a = merge_args(p, cfg, nullptr, level, 0, &dummy, pr.w);
  a.m0 = last_chunk;
  a.mc = std::min(p.Mc, M - last_chunk);
  a.gid0 = p.level_off[level] + last_chunk;
  if (info) {
    info[0] = p.B;
    info[1] = p.nT;
    info[2] = p.level_off[level] + m;
    info[3] = level == 0 ? 1 : 0;
  }
  DSMC_CUDA(launch_debug_weights(p.D, a, m - last_chunk, logW, r, rowsum, tiles, e, ratio,
                                 static_cast<cudaStream_t>(stream)), "inspection kernel");
  return DSMC_OK;
}

dsmc_status_t dsmc_debug_lazy_weights(const dsmc_config_t* cfg, const dsmc_model_t* model, int level, int m,
                                      float* pa, float* pc, float* acc, int info[4], void* ws, size_t ws_bytes,
                                      void* stream) {
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, nullptr, ws, ws_bytes, pr));
  const Plan& p = pr.p;
  if (cfg->resampler != DSMC_RS_FACTORED)
    return fail(DSMC_ERR_INVALID_ARG, "factorised proposals exist only with DSMC_RS_FACTORED");
  if (level < 0 || level >= p.L) return fail(DSMC_ERR_INVALID_ARG, "level out of range");
  const int M = merges_at_level(p.K, level);
  if (m < 0 || m >= M) return fail(DSMC_ERR_INVALID_ARG, "combination out of range");
  const int last_chunk = ((M - 1) / p.Mc) * p.Mc;
  if (m < last_chunk) return fail(DSMC_ERR_INVALID_ARG, "combination not in the last launch chunk");
  dsmc_state_t dummy = {nullptr, nullptr, nullptr, nullptr};
  MergeArgs a = merge_args(p, cfg, nullptr, level, 0, &dummy, pr.w);
  a.m0 = last_chunk;
  a.mc = std::min(p.Mc, M - last_chunk);
  a.gid0 = p.level_off[level] + last_chunk;
  if (info) {
    info[0] = p.N;
    info[1] = 0;
    info[2] = p.level_off[level] + m;
    info[3] = level == 0 ? 1 : 0;
  }
  DSMC_CUDA(launch_debug_lazy(p.D, a, m - last_chunk, pa, pc, acc, static_cast<cudaStream_t>(stream)),
            "inspection kernel");
  return DSMC_OK;
}

dsmc_status_t dsmc_debug_row_shift(const dsmc_config_t* cfg, const dsmc_model_t* model, int level, int m,
                                   double* shift, float* delta, void* ws, size_t ws_bytes, void* stream) {
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, nullptr, ws, ws_bytes, pr));
  const Plan& p = pr.p;
  if (!p.dense) return fail(DSMC_ERR_INVALID_ARG, "row shifts exist only with a dense resampler");
  if (level < 0 || level >= p.L) return fail(DSMC_ERR_INVALID_ARG, "level out of range");
  const int M = merges_at_level(p.K, level);
  if (m < 0 || m >= M) return fail(DSMC_ERR_INVALID_ARG, "combination out of range");
  const int last_chunk = ((M - 1) / p.Mc) * p.Mc;
  if (m < last_chunk) return fail(DSMC_ERR_INVALID_ARG, "combination not in the last launch chunk");
  const size_t off = (size_t)(m - last_chunk) * p.N;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (shift)
    DSMC_CUDA(cudaMemcpyAsync(shift, pr.w.shift + off, sizeof(double) * p.N, cudaMemcpyDeviceToDevice, s),
              "shift copy");
  if (delta)
    DSMC_CUDA(cudaMemcpyAsync(delta, pr.w.delta + off, sizeof(float) * p.N, cudaMemcpyDeviceToDevice, s),
              "delta copy");
  return DSMC_OK;
}

dsmc_status_t dsmc_lazy_attempts(const dsmc_config_t* cfg, const dsmc_model_t* model, void* ws, size_t ws_bytes,
                                 void* stream, uint64_t* attempts) {
  if (!attempts) return fail(DSMC_ERR_INVALID_ARG, "null output");
  Prepared pr;
  DSMC_TRY(prepare(cfg, model, nullptr, ws, ws_bytes, pr));
  unsigned long long h = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DSMC_CUDA(cudaMemcpyAsync(&h, pr.w.attempts_total, sizeof(h), cudaMemcpyDeviceToHost, s), "attempts copy");
  DSMC_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  *attempts = h;
  return DSMC_OK;
}

dsmc_status_t dsmc_batch_workspace_size(const dsmc_config_t* cfg, const dsmc_model_t* model, int n_seq,
                                        const int* K, size_t* bytes) {
  if (!cfg || !model || !bytes) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  BatchLayout bl;
  DSMC_TRY(batch_layout(cfg, model, n_seq, K, bl));
  *bytes = bl.total;
  return DSMC_OK;
}

dsmc_status_t dsmc_batch_prepare(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                 const dsmc_proposal_t* prop, int n_seq, const dsmc_seq_t* seqs, void* ws,
                                 size_t ws_bytes, void* stream) {
  if (!cfg || !model) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  BatchRun br;
  DSMC_TRY(batch_setup(cfg, model, prop, n_seq, seqs, ws, ws_bytes, br));
  return batch_upload(cfg, br, seqs, ws, static_cast<cudaStream_t>(stream));
}

dsmc_status_t dsmc_batch_run(const dsmc_config_t* cfg, const dsmc_model_t* model, const dsmc_proposal_t* prop,
                             int n_seq, const dsmc_seq_t* seqs, void* ws, size_t ws_bytes, void* stream) {
  if (!cfg || !model) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  BatchRun br;
  DSMC_TRY(batch_setup(cfg, model, prop, n_seq, seqs, ws, ws_bytes, br));
  return batch_launch(cfg, model, br, seqs, ws, static_cast<cudaStream_t>(stream));
}

dsmc_status_t dsmc_smooth_batch(const dsmc_config_t* cfg, const dsmc_model_t* model,
                                const dsmc_proposal_t* prop, int n_seq, const dsmc_seq_t* seqs, void* ws,
                                size_t ws_bytes, void* stream) {
  if (!cfg || !model) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  BatchRun br;
  DSMC_TRY(batch_setup(cfg, model, prop, n_seq, seqs, ws, ws_bytes, br));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DSMC_TRY(batch_upload(cfg, br, seqs, ws, s));
  return batch_launch(cfg, model, br, seqs, ws, s);
}

size_t dsmc_seq_maps_bytes(int K, int N) {
  if (K < 1 || N < 1) return 0;
  return (size_t)4 * K * N * sizeof(int32_t) + 2 * sizeof(int32_t);
}

dsmc_status_t dsmc_serve_workspace_size(const dsmc_config_t* cfg, const dsmc_model_t* model, int max_seq,
                                        int max_combinations, size_t* bytes) {
  if (!cfg || !model || !bytes) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  if (max_seq < 1 || max_combinations < 0) return fail(DSMC_ERR_INVALID_ARG, "max_seq >= 1, max_combinations >= 0");
  Plan p;
  DSMC_TRY(serve_plan(cfg, model, p));
  const size_t o_desc = align256(p.total);
  const size_t o_items = align256(o_desc + (size_t)max_seq * sizeof(SeqDesc));
  *bytes = align256(o_items + (size_t)max_combinations * sizeof(CombItem));
  return DSMC_OK;
}

dsmc_status_t dsmc_serve_tick(const dsmc_config_t* cfg, const dsmc_model_t* model, const dsmc_proposal_t* prop,
                              int n_seq, const dsmc_seq_t* seqs, const int* stage, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!cfg || !model) return fail(DSMC_ERR_INVALID_ARG, "null argument");
  return serve_tick(cfg, model, prop, n_seq, seqs, stage, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
