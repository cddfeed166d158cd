/*
 * oracle.c -- plain, slow, FP64 CPU restatement of the BSDE method of
 * Labart & Lelong.  TEST INFRASTRUCTURE ONLY: it is loaded by tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline leg, never by the
 * product path.  Compiled with -O2 -ffp-contract=off so that every
 * expression is rounded as written.
 *
 * Each function cites the passage it follows.  Nothing here is blocked,
 * fused or reordered beyond what the definition states.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11, Section 3): ten rounds of
 *   (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0))
 * with the key bumped by the Weyl constants between rounds.  The paper's
 * DCMT generator (Section 4.4) is replaced by this counter-based generator,
 * which gives independent streams without any creation step.
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform on (0,1): (w + 1/2) 2^-32, never 0 nor 1 */
double orc_uniform(uint32_t w) { return ((double)w + 0.5) / 4294967296.0; }

/* Box and Muller (1958): two independent N(0,1) from two uniforms */
void orc_box_muller(uint32_t w0, uint32_t w1, double* z0, double* z1) {
  const double two_pi = 6.283185307179586476925286766559;
  double u0 = orc_uniform(w0), u1 = orc_uniform(w1);
  double radius = sqrt(-2.0 * log(u0));
  *z0 = radius * cos(two_pi * u1);
  *z1 = radius * sin(two_pi * u1);
}

/* Cholesky-Banachiewicz, C = L L^T (Section 6.2: the correlation matrix
 * C = (rho 1_{i!=j} + 1_{i=j}) is factored as L L^*).  Returns 0 on success,
 * -1 if C is not positive definite. */
int orc_cholesky(int d, const double* C, double* L) {
  for (int i = 0; i < d * d; ++i) L[i] = 0.0;
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = C[i * d + j];
      for (int q = 0; q < j; ++q) s -= L[i * d + q] * L[j * d + q];
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

/* Algorithm 2, first step of iteration k: n points drawn uniformly on the
 * box [lo_0,hi_0] x prod_j [lo_j,hi_j] (the time interval times D). */
void orc_points(const orc_model* m, uint32_t k, int n, double* t, double* x) {
  const int dp = m->d + 1;
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < dp; ++c) {
      uint32_t ctr[4] = {(uint32_t)(c / 4), (uint32_t)i, 0u, (ORC_TAG_PTS << 24) | k};
      uint32_t out[4];
      orc_philox4x32_10(ctr, m->key, out);
      double u = orc_uniform(out[c % 4]);
      double y = m->lo[c] + (m->hi[c] - m->lo[c]) * u;
      if (c == 0)
        t[i] = y;
      else
        x[(size_t)(c - 1) * n + i] = y;
    }
  }
}

/* the q-th standard normal of path (k,i,path): Box-Muller on lanes (0,1) and
 * (2,3) of Philox block q/4 */
static double normal_from_block(const uint32_t out[4], int lane) {
  double z0, z1;
  if (lane < 2) {
    orc_box_muller(out[0], out[1], &z0, &z1);
  } else {
    orc_box_muller(out[2], out[3], &z0, &z1);
  }
  return (lane % 2 == 0) ? z0 : z1;
}

void orc_normals_path(const orc_model* m, uint32_t k, uint32_t i, uint32_t path, int count,
                      double* z) {
  for (int q = 0; q < count; ++q) {
    uint32_t ctr[4] = {(uint32_t)(q / 4), path, i, (ORC_TAG_Z << 24) | k};
    uint32_t out[4];
    orc_philox4x32_10(ctr, m->key, out);
    z[q] = normal_from_block(out, q % 4);
  }
}

void orc_bridge_normals(const orc_model* m, uint32_t k, uint32_t i, uint32_t path, double* z) {
  for (int j = 0; j < m->d; ++j) {
    uint32_t ctr[4] = {(uint32_t)(j / 4), path, i, (ORC_TAG_B << 24) | k};
    uint32_t out[4];
    orc_philox4x32_10(ctr, m->key, out);
    z[j] = normal_from_block(out, j % 4);
  }
}

/* local volatility of asset j (0-based) at time t and log-price x_j */
double orc_sigma(const orc_model* m, int j, double t, double xj) {
  switch (m->vol_kind) {
    case ORC_VOL_CONST:
      return m->va[j];
    case ORC_VOL_ABS_TANH:
      return m->va[j] + m->vb * exp(-t) * fabs(tanh(xj - m->kappa[j]));
    case ORC_VOL_SIN_TANH:
      /* assets are numbered from 1 (Section 5.1) */
      return m->va[j] + m->vb * sin((double)(j + 1) + t) * tanh(xj - m->kappa[j]);
    case ORC_VOL_DUPIRE: {
      /* eq. vol_locale (Section 6.3), written on the price S = e^x */
      double S = exp(xj);
      double dev = S * exp(m->r * t) - m->s_dupire;
      return 0.6 * (1.2 - exp(-0.1 * t) * exp(-0.001 * dev * dev)) * exp(-0.05 * sqrt(t));
    }
    default:
      return 0.0;
  }
}

/* basket payoff, eq. put_payoff / call_payoff (Section 6.2.1) on x = log S */
double orc_payoff(const orc_model* m, const double* x) {
  double basket = 0.0;
  for (int j = 0; j < m->d; ++j) basket += m->w[j] * exp(x[j]);
  double v = (m->payoff == ORC_PAYOFF_PUT) ? (m->K - basket) : (basket - m->K);
  return v > 0.0 ? v : 0.0;
}

/* the obstacle inside the penalty: Phi(x) (eq. bsde-penal-2), or the raw
 * intrinsic value without its positive part */
static double obstacle(const orc_model* m, const double* x) {
  if (m->obstacle == 0) return orc_payoff(m, x);
  double basket = 0.0;
  for (int j = 0; j < m->d; ++j) basket += m->w[j] * exp(x[j]);
  return (m->payoff == ORC_PAYOFF_PUT) ? (m->K - basket) : (basket - m->K);
}

/* Chebyshev polynomials T_e on [-1,1] by the three-term recurrence
 * T_{e+1} = 2 x T_e - T_{e-1}, with its first and second derivatives. */
static void chebyshev(int eta, double x, double* T, double* dT, double* d2T) {
  T[0] = 1.0; dT[0] = 0.0; d2T[0] = 0.0;
  if (eta >= 1) { T[1] = x; dT[1] = 1.0; d2T[1] = 0.0; }
  for (int e = 1; e < eta; ++e) {
    T[e + 1] = 2.0 * x * T[e] - T[e - 1];
    dT[e + 1] = 2.0 * T[e] + 2.0 * x * dT[e] - dT[e - 1];
    d2T[e + 1] = 4.0 * dT[e] + 2.0 * x * d2T[e] - d2T[e - 1];
  }
}

/* u^k(t,x) = sum_l alpha_l B_l(t,x) and its derivatives; Section 3.2.2
 * takes the derivatives of u^k as those of the fitted polynomial.  B_l = prod_v T_{nu_lv}(xi_v) with the variates
 * reduced to [-1,1]^{d'} (Section 3.2.2, domain reduction):
 * xi_v = (2 y_v - lo_v - hi_v) / (hi_v - lo_v). */
void orc_basis_eval(const orc_model* m, const orc_basis* b, const double* alpha, double t,
                    const double* x, double* u, double* ut, double* ux, double* uxx) {
  const int dp = b->dp, d = dp - 1, eta = b->eta;
  double xi[ORC_MAXD + 1], sc[ORC_MAXD + 1];
  double T[ORC_MAXD + 1][16], dT[ORC_MAXD + 1][16], d2T[ORC_MAXD + 1][16];
  for (int v = 0; v < dp; ++v) {
    double y = (v == 0) ? t : x[v - 1];
    xi[v] = (2.0 * y - m->lo[v] - m->hi[v]) / (m->hi[v] - m->lo[v]);
    sc[v] = 2.0 / (m->hi[v] - m->lo[v]);
    chebyshev(eta, xi[v], T[v], dT[v], d2T[v]);
  }
  double U = 0.0, Ut = 0.0;
  for (int j = 0; j < d; ++j) {
    ux[j] = 0.0;
    for (int q = 0; q < d; ++q) uxx[j * d + q] = 0.0;
  }
  for (int l = 0; l < b->p; ++l) {
    const int* nu = b->nu + (size_t)l * dp;
    int act[ORC_MAXD + 1], na = 0;
    for (int v = 0; v < dp; ++v)
      if (nu[v] > 0) act[na++] = v;
    /* value */
    double val = 1.0;
    for (int a = 0; a < na; ++a) val *= T[act[a]][nu[act[a]]];
    U += alpha[l] * val;
    /* first derivatives: differentiate one factor */
    for (int a = 0; a < na; ++a) {
      int v = act[a];
      double g = dT[v][nu[v]];
      for (int c = 0; c < na; ++c)
        if (c != a) g *= T[act[c]][nu[act[c]]];
      if (v == 0)
        Ut += alpha[l] * sc[0] * g;
      else
        ux[v - 1] += alpha[l] * sc[v] * g;
    }
    /* second derivatives in the space variates */
    for (int a = 0; a < na; ++a) {
      int v = act[a];
      if (v == 0) continue;
      for (int c = 0; c < na; ++c) {
        int w = act[c];
        if (w == 0) continue;
        double h;
        if (a == c) {
          h = d2T[v][nu[v]];
          for (int e = 0; e < na; ++e)
            if (e != a) h *= T[act[e]][nu[act[e]]];
        } else {
          h = dT[v][nu[v]] * dT[w][nu[w]];
          for (int e = 0; e < na; ++e)
            if (e != a && e != c) h *= T[act[e]][nu[act[e]]];
        }
        uxx[(v - 1) * d + (w - 1)] += alpha[l] * sc[v] * sc[w] * h;
      }
    }
  }
  *u = U;
  *ut = Ut;
}

/* One Monte Carlo sample of Algorithm 2:
 *   a_m = psi^N(t_i, x_i, f_{u^k} + (d_t + L^N) u^k, Phi - u^k, W, U)
 *       = (T - t_i) g1(tau, X^N_tau) + g2(X^N_T),  tau = t_i + (T - t_i) U
 * (eq. psiN, Section 3.1), with
 *   g1 = f(tau, X_tau, u^k) + d_t u^k + L^N u^k,  g2 = Phi - u^k(T, .),
 *   L^N u(s, X_s) = 1/2 sum A_jl(phi(s), X_phi(s)) d2_jl u(s, X_s)
 *                  + sum b_j(phi(s), X_phi(s)) d_j u(s, X_s)
 * (Section 3.1), the penalised driver f(t,x,y) = -r y + lambda (Phi(x) - y)^+
 * of eq. bsde-penal-2 ((Y - Phi)^- = (Phi - Y)^+), and the log-price Euler
 * scheme eqs3 with the model eq. eq4: b_j = r - delta_j - sigma_j^2/2,
 * A = diag(sigma) C diag(sigma), W increments sqrt(h) L G (Section 6.2).
 * The N Euler steps run on the regular grid of [t_i, T].  U is one 32-bit
 * word w: U = (s* + theta)/N with s* = floor(w N / 2^32) and theta the
 * remaining fraction; X^N_tau is the Euler interpolation eqs3 inside step
 * s*, sampled exactly through a Brownian bridge on that step. */
double orc_path_a(const orc_model* m, const orc_basis* b, const double* alpha, double ti,
                  const double* xi, uint32_t k, uint32_t i, uint32_t path, orc_path_info* info) {
  const int d = m->d, N = m->N;
  const double T = m->T;
  const double h = (T - ti) / (double)N;
  const double sqh = sqrt(h);

  /* the uniform time U */
  uint32_t ctr[4] = {0u, path, i, (ORC_TAG_U << 24) | k}, out[4];
  orc_philox4x32_10(ctr, m->key, out);
  uint64_t wN = (uint64_t)out[0] * (uint64_t)N;
  int sstar = (int)(wN >> 32);
  double theta = ((double)(uint32_t)(wN & 0xffffffffu) + 0.5) / 4294967296.0;
  double tau = ti + ((double)sstar + theta) * h;

  /* Euler scheme eqs3 on the regular grid t_s = t_i + s h, s = 0..N */
  double* Z = (double*)malloc(sizeof(double) * (size_t)N * d);
  double* X = (double*)malloc(sizeof(double) * (size_t)(N + 1) * d);
  orc_normals_path(m, k, i, path, N * d, Z);
  for (int j = 0; j < d; ++j) X[j] = xi[j];
  for (int s = 0; s < N; ++s) {
    double ts = ti + (double)s * h;
    const double* Xs = X + (size_t)s * d;
    double* Xn = X + (size_t)(s + 1) * d;
    const double* Zs = Z + (size_t)s * d;
    for (int j = 0; j < d; ++j) {
      double sig = orc_sigma(m, j, ts, Xs[j]);
      double drift = m->r - m->div[j] - 0.5 * sig * sig;
      double dW = 0.0;
      for (int q = 0; q <= j; ++q) dW += m->L[j * d + q] * Zs[q];
      dW *= sqh;
      Xn[j] = Xs[j] + drift * h + sig * dW;
    }
  }

  /* X^N at tau: coefficients frozen at t_{s*}; the increment of W from
   * t_{s*} to tau given the step's increment sqrt(h) Z_{s*} is
   * theta sqrt(h) Z_{s*} + sqrt(theta (1-theta) h) Z_b. */
  double Zb[ORC_MAXD], Wb[ORC_MAXD], sig_s[ORC_MAXD], drift_s[ORC_MAXD], Xtau[ORC_MAXD];
  orc_bridge_normals(m, k, i, path, Zb);
  const double ts_star = ti + (double)sstar * h;
  const double* Xstar = X + (size_t)sstar * d;
  const double* Zstar = Z + (size_t)sstar * d;
  for (int j = 0; j < d; ++j)
    Wb[j] = theta * sqh * Zstar[j] + sqrt(theta * (1.0 - theta) * h) * Zb[j];
  for (int j = 0; j < d; ++j) {
    sig_s[j] = orc_sigma(m, j, ts_star, Xstar[j]);
    drift_s[j] = m->r - m->div[j] - 0.5 * sig_s[j] * sig_s[j];
    double lw = 0.0;
    for (int q = 0; q <= j; ++q) lw += m->L[j * d + q] * Wb[q];
    Xtau[j] = Xstar[j] + drift_s[j] * theta * h + sig_s[j] * lw;
  }

  /* g1 at (tau, X_tau) */
  double u, ut, ux[ORC_MAXD], uxx[ORC_MAXD * ORC_MAXD];
  orc_basis_eval(m, b, alpha, tau, Xtau, &u, &ut, ux, uxx);
  double Lu = 0.0;
  for (int j = 0; j < d; ++j) Lu += drift_s[j] * ux[j];
  double diff = 0.0;
  for (int j = 0; j < d; ++j)
    for (int q = 0; q < d; ++q) diff += sig_s[j] * sig_s[q] * m->C[j * d + q] * uxx[j * d + q];
  Lu += 0.5 * diff;
  double phitau = obstacle(m, Xtau);
  double pen = phitau - u;
  double f = -m->r * u + m->lambda * (pen > 0.0 ? pen : 0.0);
  double g1 = f + ut + Lu;

  /* g2 at X_T */
  const double* XT = X + (size_t)N * d;
  double uT, uTt, uTx[ORC_MAXD], uTxx[ORC_MAXD * ORC_MAXD];
  orc_basis_eval(m, b, alpha, T, XT, &uT, &uTt, uTx, uTxx);
  double phiT = orc_payoff(m, XT);
  double g2 = phiT - uT;
  double a = (T - ti) * g1 + g2;

  if (info) {
    info->sstar = sstar; info->theta = theta; info->tau = tau;
    info->u = u; info->ut = ut; info->Lu = Lu; info->f = f; info->g1 = g1;
    info->uT = uT; info->phiT = phiT; info->phitau = phitau; info->a = a;
    for (int j = 0; j < d; ++j) {
      info->XT[j] = XT[j]; info->Xtau[j] = Xtau[j]; info->Xs[j] = Xstar[j];
    }
  }
  free(Z);
  free(X);
  return a;
}

/* eq. chat of Algorithm 2: c_i = (1/M) sum_m a_m, summed in m order */
typedef struct {
  const orc_model* m;
  const orc_basis* b;
  const double* alpha;
  int npts;
  const uint32_t* idx;
  const double *t, *x;
  uint32_t k;
  double* c;
  int first, stride;
} corr_job;

static void* corr_worker(void* arg) {
  corr_job* J = (corr_job*)arg;
  const int d = J->m->d;
  double xi[ORC_MAXD];
  for (int q = J->first; q < J->npts; q += J->stride) {
    for (int j = 0; j < d; ++j) xi[j] = J->x[(size_t)j * J->npts + q];
    double sum = 0.0;
    for (int path = 0; path < J->m->M; ++path)
      sum += orc_path_a(J->m, J->b, J->alpha, J->t[q], xi, J->k, J->idx[q], (uint32_t)path, NULL);
    J->c[q] = sum / (double)J->m->M;
  }
  return NULL;
}

void orc_correction(const orc_model* m, const orc_basis* b, const double* alpha, int npts,
                    const uint32_t* idx, const double* t, const double* x, uint32_t k, int nthreads,
                    double* c) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  corr_job jobs[256];
  for (int w = 0; w < nthreads; ++w) {
    corr_job J = {m, b, alpha, npts, idx, t, x, k, c, w, nthreads};
    jobs[w] = J;
  }
  if (nthreads == 1) {
    corr_worker(&jobs[0]);
    return;
  }
  for (int w = 0; w < nthreads; ++w) pthread_create(&th[w], NULL, corr_worker, &jobs[w]);
  for (int w = 0; w < nthreads; ++w) pthread_join(th[w], NULL);
}

/* the M individual samples a_m of one point, for the pin tests (their
 * sample variance gives the Monte Carlo standard error of c_i) */
void orc_samples(const orc_model* m, const orc_basis* b, const double* alpha, double ti,
                 const double* xi, uint32_t k, uint32_t i, int npaths, double* a) {
  for (int p = 0; p < npaths; ++p) a[p] = orc_path_a(m, b, alpha, ti, xi, k, i, (uint32_t)p, NULL);
}

/* Paths only (no evaluation), for the pin tests of the Euler scheme and
 * of the Brownian bridge: X_T, X_tau and tau of npaths paths. */
void orc_simulate_XT(const orc_model* m, uint32_t k, uint32_t i, double ti, const double* xi,
                     int npaths, double* XT, double* Xtau, double* tau) {
  const int d = m->d;
  /* zero polynomial: only the paths matter */
  int nu0[ORC_MAXD + 1] = {0};
  orc_basis b0 = {1, d + 1, 1, nu0};
  double alpha0 = 0.0;
  orc_path_info info;
  for (int p = 0; p < npaths; ++p) {
    orc_path_a(m, &b0, &alpha0, ti, xi, k, i, (uint32_t)p, &info);
    for (int j = 0; j < d; ++j) {
      XT[(size_t)p * d + j] = info.XT[j];
      Xtau[(size_t)p * d + j] = info.Xtau[j];
    }
    tau[p] = info.tau;
  }
}
