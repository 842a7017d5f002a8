// pit.cu -- the parallel-in-time linearised Gaussian smoother of Section 4.1 (Algorithm 4),
// whose marginals N(m_t, P_t) become the proposals q_t = nu_t of Algorithm 2.
//
// The model is linearised around the current marginals and smoothed exactly by the
// temporally parallel Kalman filter and Rauch-Tung-Striebel smoother (Sarkka and
// Garcia-Fernandez, "Temporal parallelization of Bayesian smoothers", 2021): both passes are
// prefix scans of an associative operator over per-step elements, so a pass over K steps has
// ceil(log2 K) levels.  For the linear-Gaussian model the linearisation is the model itself
// (one iteration is exact).  For the stochastic-volatility and Poisson-count models, whose
// observations are not additive Gaussian, log h_t(y_t | x) is expanded to second order
// around the current mean m_t, which is a Gaussian pseudo-observation z_t = m_t + g_t /
// lambda_t with variance 1 / lambda_t (g_t, lambda_t the first and negated second
// derivatives; no observation where lambda_t vanishes); iterating moves the marginals to the
// posterior mode and its curvature.  For the theta-logistic model the observation is
// linear-Gaussian and the transition mean is linearised around the previous pass's mean of
// step t - 1 (per-step F_t, c_t: the iterated extended smoother).
//
// Every quantity is FP64 (the work is O(K d^3 log K), small next to the smoother itself).
// Filtering element of step t (observation matrix I, transition x_t = F x_{t-1} + c + N(0, Q),
// observation y_t with noise covariance R_t, gain K_t = S_t^-1 in the row form below):
//   t = 0:  S = P0 + R_0, G = P0 S^-1; A = 0, b = m0 + G (y_0 - m0), C = P0 - G P0, eta = 0, J = 0
//   t > 0:  S = Q + R_t, G = Q S^-1; A = (I - G) F, b = (I - G) c + G y_t, C = (I - G) Q,
//           eta = F' S^-1 (y_t - c), J = F' S^-1 F
// combined (i before j) with M = I + C_i J_j and X = M^-1 [A_i | b_i + C_i eta_j | C_i]:
//   A = A_j X_A, b = A_j X_b + b_j, C = A_j X_C A_j' + C_j,
//   eta = X_A' (eta_j - J_j b_i) + eta_i, J = X_A' J_j A_i + J_i;
// the prefix of step t holds the filtered mean b and covariance C.  Smoothing element of
// step t < K - 1: E = P_t F' (F P_t F' + Q)^-1, g = m_t - E (F m_t + c), L = P_t - E F P_t
// (t = K - 1: E = 0, g = m_t, L = P_t), combined (i before j) as (E_i E_j, E_i g_j + g_i,
// E_i L_j E_i' + L_i); the suffix of step t holds the smoothed mean g and covariance L.
#include <cmath>

#include "kernels.cuh"

namespace dsmc {

namespace {

constexpr int kPitThreads = 128;

// The per-step elements in the workspace (FP64, d x d row-major matrices).
struct PitWs {
  double *A, *b, *C, *eta, *J;   // filtering elements, [K][d][d] / [K][d]
  double *A2, *b2, *C2, *eta2, *J2;
  double *E, *g, *L;             // smoothing elements
  double *E2, *g2, *L2;
  double *z, *r;                 // SV pseudo-observations and their variances [K] (r < 0: none)
  double* mlin;                  // linearisation points [K] (the previous smoothed means)
  double *Ft, *ct;               // per-step linearised transitions [K][d][d], [K][d]
};

// ---- small dense linear algebra in shared memory, all threads of the CTA
__device__ void mat_mul(double* out, const double* A, bool tA, const double* B, bool tB, int n, int k, int m) {
  // out[n][m] = op(A)[n][k] op(B)[k][m]
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
    const int r = e / m, cc = e - r * m;
    double s = 0.0;
    for (int q = 0; q < k; ++q) {
      const double a = tA ? A[q * n + r] : A[r * k + q];
      const double bb = tB ? B[cc * k + q] : B[q * m + cc];
      s = fma(a, bb, s);
    }
    out[e] = s;
  }
  __syncthreads();
}

// Solves M X = Rhs in place (Rhs [d][nc] <- X) by Gauss-Jordan elimination with partial
// pivoting; M [d][d] is destroyed.  piv_s: one shared int.
__device__ void gj_solve(double* M, double* Rhs, int d, int nc, int* piv_s) {
  for (int k = 0; k < d; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(M[k * d + k]);
      for (int r = k + 1; r < d; ++r)
        if (fabs(M[r * d + k]) > best) {
          best = fabs(M[r * d + k]);
          p = r;
        }
      *piv_s = p;
    }
    __syncthreads();
    const int p = *piv_s;
    if (p != k) {
      for (int cc = threadIdx.x; cc < d + nc; cc += blockDim.x) {
        double* x = cc < d ? &M[k * d + cc] : &Rhs[k * nc + cc - d];
        double* y = cc < d ? &M[p * d + cc] : &Rhs[p * nc + cc - d];
        const double t = *x;
        *x = *y;
        *y = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / M[k * d + k];
    __syncthreads();
    for (int cc = threadIdx.x; cc < d + nc; cc += blockDim.x) {
      if (cc < d) M[k * d + cc] *= inv;
      else Rhs[k * nc + cc - d] *= inv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < d * (d + nc); e += blockDim.x) {
      const int r = e / (d + nc), cc = e - r * (d + nc);
      if (r == k) continue;
      const double f = M[r * d + k];
      if (cc < d) {
        if (cc != k) M[r * d + cc] -= f * M[k * d + cc];
      } else {
        Rhs[r * nc + cc - d] -= f * Rhs[k * nc + cc - d];
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < d; r += blockDim.x)
      if (r != k) M[r * d + k] = 0.0;
    __syncthreads();
  }
}

// ---- filtering elements (one CTA per step)
__global__ void __launch_bounds__(kPitThreads) pit_filter_elements(PitArgs p, PitWs w) {
  extern __shared__ double sm[];
  const int t = blockIdx.x, d = p.d, dd = d * d;
  // the transition into step t: per-step linearisation (theta-logistic) or the model's
  const double* Fm = (p.Ft != nullptr && t > 0) ? p.Ft + (size_t)t * dd : p.F;
  const double* cv = (p.ct != nullptr && t > 0) ? p.ct + (size_t)t * d : p.c;
  double* S = sm;            // [d][d]
  double* G = S + dd;        // [d][d]: scratch of the first solve, then the gain
  double* T1 = G + dd;       // [d][d]
  double* yv = T1 + dd;      // [d]
  double* R2 = yv + d;       // [d][d + 1]
  __shared__ int piv;
  __shared__ int has_obs;
  // the observation (or SV pseudo-observation) and its noise covariance
  if (threadIdx.x == 0) has_obs = 1;
  __syncthreads();
  if (p.kind == DSMC_MODEL_SV || p.kind == DSMC_MODEL_COX) {  // pseudo-observations
    if (threadIdx.x == 0) {
      const double rr = w.r[t];
      has_obs = rr > 0.0;
      yv[0] = w.z[t];
      S[0] = (t == 0 ? p.P0[0] : p.Q[0]) + (rr > 0.0 ? rr : 0.0);
    }
  } else {
    for (int e = threadIdx.x; e < dd; e += blockDim.x) S[e] = (t == 0 ? p.P0[e] : p.Q[e]) + p.R[e];
    for (int k = threadIdx.x; k < d; k += blockDim.x) yv[k] = (double)p.y[(size_t)t * d + k];
  }
  __syncthreads();
  double* A = w.A + (size_t)t * dd;
  double* b = w.b + (size_t)t * d;
  double* C = w.C + (size_t)t * dd;
  double* eta = w.eta + (size_t)t * d;
  double* J = w.J + (size_t)t * dd;
  const double* P = t == 0 ? p.P0 : p.Q;
  if (!has_obs) {  // no information at this step: the prior / transition as is
    for (int e = threadIdx.x; e < dd; e += blockDim.x) {
      A[e] = t == 0 ? 0.0 : Fm[e];
      C[e] = P[e];
      J[e] = 0.0;
    }
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
      b[k] = t == 0 ? p.m0[k] : cv[k];
      eta[k] = 0.0;
    }
    return;
  }
  // G = P S^-1: solve S X = P (S, P symmetric), G = X'
  for (int e = threadIdx.x; e < dd; e += blockDim.x) T1[e] = P[e];
  __syncthreads();
  {
    double* Sc = G;  // scratch copy of S for the solve
    for (int e = threadIdx.x; e < dd; e += blockDim.x) Sc[e] = S[e];
    __syncthreads();
    gj_solve(Sc, T1, d, d, &piv);  // T1 = S^-1 P
  }
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    G[e] = T1[cc * d + r];
  }
  __syncthreads();
  if (t == 0) {
    for (int e = threadIdx.x; e < dd; e += blockDim.x) {
      const int r = e / d, cc = e - r * d;
      double s = 0.0;
      for (int q = 0; q < d; ++q) s = fma(G[r * d + q], P[q * d + cc], s);
      T1[e] = P[e] - s;  // C = P0 - G P0
    }
    __syncthreads();
    for (int e = threadIdx.x; e < dd; e += blockDim.x) {
      const int r = e / d, cc = e - r * d;
      A[e] = 0.0;
      C[e] = 0.5 * (T1[r * d + cc] + T1[cc * d + r]);
      J[e] = 0.0;
    }
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < d; ++q) s = fma(G[k * d + q], yv[q] - p.m0[q], s);
      b[k] = p.m0[k] + s;
      eta[k] = 0.0;
    }
    return;
  }
  // t > 0: I - G into T1
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    T1[e] = (r == cc ? 1.0 : 0.0) - G[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double sa = 0.0, sc = 0.0;
    for (int q = 0; q < d; ++q) {
      sa = fma(T1[r * d + q], Fm[q * d + cc], sa);
      sc = fma(T1[r * d + q], p.Q[q * d + cc], sc);
    }
    A[e] = sa;
    C[e] = sc;  // symmetrised below
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) s = fma(G[k * d + q], yv[q], fma(T1[k * d + q], cv[q], s));
    b[k] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    if (r < cc) {
      const double v = 0.5 * (C[r * d + cc] + C[cc * d + r]);
      C[r * d + cc] = v;
      C[cc * d + r] = v;
    }
  }
  // eta = F' S^-1 (y - c), J = F' S^-1 F: solve S X = [F | y - c] (S solved in place)
  for (int e = threadIdx.x; e < d * (d + 1); e += blockDim.x) {
    const int r = e / (d + 1), cc = e - r * (d + 1);
    R2[e] = cc < d ? Fm[r * d + cc] : yv[r] - cv[r];
  }
  __syncthreads();
  gj_solve(S, R2, d, d + 1, &piv);  // R2 = S^-1 [F | y - c]
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double s = 0.0;
    for (int q = 0; q < d; ++q) s = fma(Fm[q * d + r], R2[q * (d + 1) + cc], s);
    J[e] = s;
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) s = fma(Fm[q * d + k], R2[q * (d + 1) + d], s);
    eta[k] = s;
  }
}

// ---- one level of the filtering prefix scan: step t >= off takes (t - off) (x) t
__global__ void __launch_bounds__(kPitThreads) pit_filter_combine(int K, int d, int off, PitWs in, PitWs out) {
  extern __shared__ double sm[];
  const int t = blockIdx.x;
  const int dd = d * d;
  double* Ao = out.A + (size_t)t * dd;
  double* bo = out.b + (size_t)t * d;
  double* Co = out.C + (size_t)t * dd;
  double* eo = out.eta + (size_t)t * d;
  double* Jo = out.J + (size_t)t * dd;
  const double* Aj = in.A + (size_t)t * dd;
  const double* bj = in.b + (size_t)t * d;
  const double* Cj = in.C + (size_t)t * dd;
  const double* ej = in.eta + (size_t)t * d;
  const double* Jj = in.J + (size_t)t * dd;
  if (t < off) {  // already a full prefix: copied through
    for (int e = threadIdx.x; e < dd; e += blockDim.x) {
      Ao[e] = Aj[e];
      Co[e] = Cj[e];
      Jo[e] = Jj[e];
    }
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
      bo[k] = bj[k];
      eo[k] = ej[k];
    }
    return;
  }
  const int i = t - off;
  const double* Ai = in.A + (size_t)i * dd;
  const double* bi = in.b + (size_t)i * d;
  const double* Ci = in.C + (size_t)i * dd;
  const double* ei = in.eta + (size_t)i * d;
  const double* Ji = in.J + (size_t)i * dd;
  const int nc = 2 * d + 1;
  double* M = sm;              // [d][d]
  double* X = M + dd;          // [d][2d + 1]: [A_i | b_i + C_i eta_j | C_i], then solved
  double* T = X + d * nc;      // [d][d]
  double* v = T + dd;          // [d]
  __shared__ int piv;
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double s = 0.0;
    for (int q = 0; q < d; ++q) s = fma(Ci[r * d + q], Jj[q * d + cc], s);
    M[e] = (r == cc ? 1.0 : 0.0) + s;
  }
  for (int e = threadIdx.x; e < d * nc; e += blockDim.x) {
    const int r = e / nc, cc = e - r * nc;
    double val;
    if (cc < d) {
      val = Ai[r * d + cc];
    } else if (cc == d) {
      double s = bi[r];
      for (int q = 0; q < d; ++q) s = fma(Ci[r * d + q], ej[q], s);
      val = s;
    } else {
      val = Ci[r * d + cc - d - 1];
    }
    X[e] = val;
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {  // v = eta_j - J_j b_i
    double s = ej[k];
    for (int q = 0; q < d; ++q) s = fma(-Jj[k * d + q], bi[q], s);
    v[k] = s;
  }
  __syncthreads();
  gj_solve(M, X, d, nc, &piv);
  // A = A_j X_A, b = A_j X_b + b_j, T = A_j X_C
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double sa = 0.0, st = 0.0;
    for (int q = 0; q < d; ++q) {
      sa = fma(Aj[r * d + q], X[q * nc + cc], sa);
      st = fma(Aj[r * d + q], X[q * nc + d + 1 + cc], st);
    }
    Ao[e] = sa;
    T[e] = st;
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = bj[k];
    for (int q = 0; q < d; ++q) s = fma(Aj[k * d + q], X[q * nc + d], s);
    bo[k] = s;
  }
  __syncthreads();
  // C = T A_j' + C_j (symmetrised), J = X_A' J_j A_i + J_i, eta = X_A' v + eta_i
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double sc = 0.0, sc2 = 0.0;
    for (int q = 0; q < d; ++q) {
      sc = fma(T[r * d + q], Aj[cc * d + q], sc);
      sc2 = fma(T[cc * d + q], Aj[r * d + q], sc2);
    }
    Co[e] = 0.5 * (sc + sc2) + 0.5 * (Cj[r * d + cc] + Cj[cc * d + r]);
    double sj = 0.0;
    for (int q = 0; q < d; ++q) {
      double jq = 0.0;  // (J_j A_i)[q][cc]
      for (int u = 0; u < d; ++u) jq = fma(Jj[q * d + u], Ai[u * d + cc], jq);
      sj = fma(X[q * nc + r], jq, sj);
    }
    Jo[e] = sj + Ji[e];
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = ei[k];
    for (int q = 0; q < d; ++q) s = fma(X[q * nc + k], v[q], s);
    eo[k] = s;
  }
}

// ---- smoothing elements from the filtered moments (b, C of the filtering prefix)
__global__ void __launch_bounds__(kPitThreads) pit_smooth_elements(PitArgs p, PitWs f, PitWs w) {
  extern __shared__ double sm[];
  const int t = blockIdx.x, d = p.d, dd = d * d;
  const double* m = f.b + (size_t)t * d;
  const double* P = f.C + (size_t)t * dd;
  double* E = w.E + (size_t)t * dd;
  double* g = w.g + (size_t)t * d;
  double* L = w.L + (size_t)t * dd;
  if (t == p.K - 1) {
    for (int e = threadIdx.x; e < dd; e += blockDim.x) {
      E[e] = 0.0;
      L[e] = P[e];
    }
    for (int k = threadIdx.x; k < d; k += blockDim.x) g[k] = m[k];
    return;
  }
  double* Pp = sm;          // F P F' + Q
  double* FP = Pp + dd;     // F P, then solved: Pp^-1 F P = E'
  double* T = FP + dd;
  double* fm = T + dd;      // F m + c
  __shared__ int piv;
  // the transition from step t to t + 1
  const double* Fm = p.Ft != nullptr ? p.Ft + (size_t)(t + 1) * dd : p.F;
  const double* cv = p.ct != nullptr ? p.ct + (size_t)(t + 1) * d : p.c;
  mat_mul(FP, Fm, false, P, false, d, d, d);
  mat_mul(T, FP, false, Fm, true, d, d, d);
  for (int e = threadIdx.x; e < dd; e += blockDim.x) Pp[e] = T[e] + p.Q[e];
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = cv[k];
    for (int q = 0; q < d; ++q) s = fma(Fm[k * d + q], m[q], s);
    fm[k] = s;
  }
  __syncthreads();
  gj_solve(Pp, FP, d, d, &piv);  // FP = Pp^-1 F P = E'
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    E[e] = FP[cc * d + r];
  }
  // L = P - E F P = P - FP' (F P); g = m - E fm
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double s = 0.0;
    for (int q = 0; q < d; ++q) {
      double fpq = 0.0;  // (F P)[q][cc]
      for (int u = 0; u < d; ++u) fpq = fma(Fm[q * d + u], P[u * d + cc], fpq);
      s = fma(FP[q * d + r], fpq, s);
    }
    T[e] = P[e] - s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    L[e] = 0.5 * (T[r * d + cc] + T[cc * d + r]);
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = m[k];
    for (int q = 0; q < d; ++q) s = fma(-FP[q * d + k], fm[q], s);
    g[k] = s;
  }
}

// ---- one level of the smoothing suffix scan: step t + off < K gives t (x) (t + off)
__global__ void __launch_bounds__(kPitThreads) pit_smooth_combine(int K, int d, int off, PitWs in, PitWs out) {
  extern __shared__ double sm[];
  const int t = blockIdx.x, dd = d * d;
  const double* Ei = in.E + (size_t)t * dd;
  const double* gi = in.g + (size_t)t * d;
  const double* Li = in.L + (size_t)t * dd;
  double* Eo = out.E + (size_t)t * dd;
  double* go = out.g + (size_t)t * d;
  double* Lo = out.L + (size_t)t * dd;
  if (t + off >= K) {
    for (int e = threadIdx.x; e < dd; e += blockDim.x) {
      Eo[e] = Ei[e];
      Lo[e] = Li[e];
    }
    for (int k = threadIdx.x; k < d; k += blockDim.x) go[k] = gi[k];
    return;
  }
  const int j = t + off;
  const double* Ej = in.E + (size_t)j * dd;
  const double* gj = in.g + (size_t)j * d;
  const double* Lj = in.L + (size_t)j * dd;
  double* T = sm;  // E_i L_j
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double se = 0.0, st = 0.0;
    for (int q = 0; q < d; ++q) {
      se = fma(Ei[r * d + q], Ej[q * d + cc], se);
      st = fma(Ei[r * d + q], Lj[q * d + cc], st);
    }
    Eo[e] = se;
    T[e] = st;
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double s = gi[k];
    for (int q = 0; q < d; ++q) s = fma(Ei[k * d + q], gj[q], s);
    go[k] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int r = e / d, cc = e - r * d;
    double s = 0.0, s2 = 0.0;
    for (int q = 0; q < d; ++q) {
      s = fma(T[r * d + q], Ei[cc * d + q], s);
      s2 = fma(T[cc * d + q], Ei[r * d + q], s2);
    }
    Lo[e] = 0.5 * (s + s2) + 0.5 * (Li[r * d + cc] + Li[cc * d + r]);
  }
}

// ---- the SV linearisation around the current means, and the outputs
// lambda = y^2 e^{-m} / 2 (negated second derivative of log h at m), gradient
// g = -1/2 + lambda; pseudo-observation z = m + g / lambda with variance 1 / lambda.
__global__ void pit_sv_linearise(int K, const float* y, const double* m, double mu, double* z, double* r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K) return;
  const double mt = m ? m[t] : mu;
  const double yt = (double)y[t];
  const double lam = 0.5 * yt * yt * exp(-mt);
  if (lam > 1e-300 && isfinite(lam)) {
    z[t] = mt + (lam - 0.5) / lam;
    r[t] = 1.0 / lam;
  } else {
    z[t] = 0.0;
    r[t] = -1.0;
  }
}

// COX: log h = y x - e^x, so lambda = e^{m} and the gradient is y - e^{m}: the
// pseudo-observation z = m + (y - e^m) / e^m with variance e^{-m}.
__global__ void pit_cox_linearise(int K, const float* y, const double* m, double mu, double* z, double* r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K) return;
  const double mt = m ? m[t] : mu;
  const double lam = exp(mt);
  z[t] = mt + ((double)y[t] - lam) / lam;
  r[t] = 1.0 / lam;
}

// THETA_LOGISTIC: the transition into step t linearised around the previous mean m_{t-1}:
// F_t = 1 - tau1 tau2 e^{tau2 m}, c_t = m + tau0 - tau1 e^{tau2 m} - F_t m.
__global__ void pit_theta_linearise(int K, const double* m, double tau0, double tau1, double tau2, double* Ft,
                                    double* ct) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K) return;
  if (t == 0) {
    Ft[0] = 1.0;
    ct[0] = 0.0;
    return;
  }
  const double mp = m[t - 1];
  const double e = exp(tau2 * mp);
  const double F = 1.0 - tau1 * tau2 * e;
  Ft[t] = F;
  ct[t] = mp + tau0 - tau1 * e - F * mp;
}

__global__ void pit_sv_from_float(int K, const float* m_in, double* m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < K) m[t] = (double)m_in[t];
}

__global__ void pit_outputs(int K, int d, const double* g, const double* L, float* mean_out, float* std_out,
                            double* mean64, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K * d) return;
  const int t = e / d, k = e - t * d;
  const double m = g[e];
  const double v = L[(size_t)t * d * d + k * d + k];
  if (!isfinite(m) || !(v > 0.0) || !isfinite(v)) record_status(status, DSMC_ERR_NONFINITE);
  mean_out[e] = (float)m;
  std_out[e] = (float)sqrt(v > 0.0 ? v : 0.0);
  if (mean64) mean64[e] = m;
}

size_t pit_smem(int d) {
  // the largest shared footprint: the filtering elements (S, G, T1, y, [F | y - c]) and the
  // filtering combination (M, X, T, v) both take 4 d^2 + 2 d doubles
  return sizeof(double) * (4 * (size_t)d * d + 2 * (size_t)d);
}

}  // namespace

// Workspace of the linearised smoother for K steps of dimension d: the status word, the
// model matrices (F, Q, R, P0 [d][d], c, m0 [d]) and the per-step elements, 256-byte aligned.
size_t pit_workspace_bytes(int K, int d) {
  const size_t dd = (size_t)d * d, Kd = (size_t)K * d, Kdd = (size_t)K * dd;
  auto r256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t o = 256 + r256((4 * dd + 2 * d) * sizeof(double));
  const size_t parts[] = {Kdd, Kd, Kdd, Kd, Kdd, Kdd, Kd, Kdd, Kd, Kdd,
                          Kdd, Kd, Kdd, Kdd, Kd, Kdd, (size_t)K, (size_t)K, (size_t)K, Kdd, Kd};
  for (size_t n : parts) o += r256(n * sizeof(double));
  return o;
}

namespace {

PitWs carve(void* ws, int K, int d, int** status, double** params) {
  char* p = static_cast<char*>(ws);
  const size_t dd = (size_t)d * d, Kd = (size_t)K * d, Kdd = (size_t)K * dd;
  *status = reinterpret_cast<int*>(p);
  *params = reinterpret_cast<double*>(p + 256);
  size_t o = 256 + (((4 * dd + 2 * d) * sizeof(double) + 255) & ~(size_t)255);
  auto take = [&](size_t n) {
    double* r = reinterpret_cast<double*>(p + o);
    o = (o + n * sizeof(double) + 255) & ~(size_t)255;
    return r;
  };
  PitWs w;
  w.A = take(Kdd); w.b = take(Kd); w.C = take(Kdd); w.eta = take(Kd); w.J = take(Kdd);
  w.A2 = take(Kdd); w.b2 = take(Kd); w.C2 = take(Kdd); w.eta2 = take(Kd); w.J2 = take(Kdd);
  w.E = take(Kdd); w.g = take(Kd); w.L = take(Kdd);
  w.E2 = take(Kdd); w.g2 = take(Kd); w.L2 = take(Kdd);
  w.z = take(K); w.r = take(K); w.mlin = take(K);
  w.Ft = take(Kdd); w.ct = take(Kd);
  return w;
}

PitWs swap_filter(const PitWs& w) {
  PitWs s = w;
  s.A = w.A2; s.b = w.b2; s.C = w.C2; s.eta = w.eta2; s.J = w.J2;
  s.A2 = w.A; s.b2 = w.b; s.C2 = w.C; s.eta2 = w.eta; s.J2 = w.J;
  return s;
}

PitWs swap_smooth(const PitWs& w) {
  PitWs s = w;
  s.E = w.E2; s.g = w.g2; s.L = w.L2;
  s.E2 = w.E; s.g2 = w.g; s.L2 = w.L;
  return s;
}

}  // namespace

// The iterations of Algorithm 4 (see the top of this file); every launch on `st`.  `model`:
// HOST [4 d^2 + 2 d] FP64 = F, Q, R, P0 ([d][d]), c, m0 ([d]), copied into the workspace.
cudaError_t launch_pit(PitArgs pa, const double* model, int iterations, const float* init_mean, float* mean_out,
                       float* std_out, void* ws, cudaStream_t st, int* n_launches) {
  const int K = pa.K, d = pa.d;
  const size_t dd = (size_t)d * d;
  int* status = nullptr;
  double* params = nullptr;
  PitWs w = carve(ws, K, d, &status, &params);
  cudaError_t e = cudaMemcpyAsync(params, model, (4 * dd + 2 * d) * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  pa.F = params;
  pa.Q = params + dd;
  pa.R = params + 2 * dd;
  pa.P0 = params + 3 * dd;
  pa.c = params + 4 * dd;
  pa.m0 = params + 4 * dd + d;
  const size_t smem = pit_smem(d);
  for (auto fn : {(const void*)pit_filter_elements, (const void*)pit_filter_combine, (const void*)pit_smooth_elements,
                  (const void*)pit_smooth_combine}) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  int launches = 0;
  const bool pseudo = pa.kind == DSMC_MODEL_SV || pa.kind == DSMC_MODEL_COX;  // observation linearised
  const bool theta = pa.kind == DSMC_MODEL_THETA_LOGISTIC;                    // transition linearised
  const bool iter = pseudo || theta;
  const int it_n = iter ? (iterations > 0 ? iterations : 1) : 1;
  bool have_m = false;  // linearise around mlin (else around the stationary mean, or y_t)
  if (iter && (init_mean || theta)) {
    pit_sv_from_float<<<(K + 127) / 128, 128, 0, st>>>(K, init_mean ? init_mean : pa.y, w.mlin);
    ++launches;
    have_m = true;
  }
  pa.Ft = theta ? w.Ft : nullptr;
  pa.ct = theta ? w.ct : nullptr;
  for (int it = 0; it < it_n; ++it) {
    if (pa.kind == DSMC_MODEL_SV) {
      pit_sv_linearise<<<(K + 127) / 128, 128, 0, st>>>(K, pa.y, have_m ? w.mlin : nullptr, pa.mu, w.z, w.r);
      ++launches;
    } else if (pa.kind == DSMC_MODEL_COX) {
      pit_cox_linearise<<<(K + 127) / 128, 128, 0, st>>>(K, pa.y, have_m ? w.mlin : nullptr, pa.mu, w.z, w.r);
      ++launches;
    } else if (theta) {
      pit_theta_linearise<<<(K + 127) / 128, 128, 0, st>>>(K, w.mlin, pa.tau0, pa.tau1, pa.tau2, w.Ft, w.ct);
      ++launches;
    }
    PitWs f = w;
    pit_filter_elements<<<K, kPitThreads, smem, st>>>(pa, f);
    ++launches;
    for (int off = 1; off < K; off <<= 1) {
      const PitWs out = swap_filter(f);
      pit_filter_combine<<<K, kPitThreads, smem, st>>>(K, d, off, f, out);
      ++launches;
      f = out;
    }
    PitWs s = f;  // the filtered moments are f's (b, C); s names the smoothing buffers
    pit_smooth_elements<<<K, kPitThreads, smem, st>>>(pa, f, s);
    ++launches;
    for (int off = 1; off < K; off <<= 1) {
      const PitWs out = swap_smooth(s);
      pit_smooth_combine<<<K, kPitThreads, smem, st>>>(K, d, off, s, out);
      ++launches;
      s = out;
    }
    pit_outputs<<<(K * d + 127) / 128, 128, 0, st>>>(K, d, s.g, s.L, mean_out, std_out, nullptr, status);
    ++launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (iter && it + 1 < it_n) {  // the next linearisation point: this iteration's means
      e = cudaMemcpyAsync(w.mlin, s.g, sizeof(double) * (size_t)K, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
      have_m = true;
    }
  }
  *n_launches = launches;
  return cudaGetLastError();
}

}  // namespace dsmc
