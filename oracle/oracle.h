/*
 * oracle.h -- plain FP64 CPU restatement of the Picard-iteration /
 * adaptive-control-variate BSDE solver of Labart & Lelong ("A Parallel
 * Algorithm for solving BSDEs", Algorithm 2 of Section 4.1 and the pricing
 * model of Section 5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this code.  It shares no code with
 * the CUDA library: Philox4x32-10, Box-Muller, the Euler scheme, the basis
 * and the driver are written here independently from their published
 * definitions.
 *
 * Counter layout shared (as a specification, not as code) with the CUDA
 * path; key = (seed & 0xffffffff, seed >> 32):
 *   points  : ctr = (blk, i, 0, TAG_PTS<<24 | k), coordinate c = 4*blk+lane
 *   U draw  : ctr = (0,   m, i, TAG_U  <<24 | k), lane 0
 *   normals : ctr = (q>>2, m, i, TAG_Z <<24 | k), lane q&3, q = s*d + j
 *   bridge  : ctr = (j>>2, m, i, TAG_B <<24 | k), lane j&3, j < d
 */
#ifndef BSDE_ORACLE_H
#define BSDE_ORACLE_H
#include <stdint.h>

#define ORC_MAXD 16

#define ORC_TAG_PTS 1u
#define ORC_TAG_U 2u
#define ORC_TAG_Z 3u
#define ORC_TAG_B 4u

/* volatility families (Section 5.1 eq. eq4 with sigma_ij = sigma_i L_ij) */
#define ORC_VOL_CONST 0    /* sigma_j = a_j                                   */
#define ORC_VOL_ABS_TANH 1 /* a_j + b e^{-t} |tanh(x_j - kappa_j)|            */
#define ORC_VOL_SIN_TANH 2 /* a_j + b sin(j + t) tanh(x_j - kappa_j), j=1..d  */
#define ORC_VOL_DUPIRE 3   /* eq. vol_locale of Section 6.3                   */

#define ORC_PAYOFF_PUT 0
#define ORC_PAYOFF_CALL 1

typedef struct {
  int d;          /* number of assets                                 */
  int N;          /* Euler time steps per path (from t_i to T)        */
  int M;          /* Monte Carlo paths per point                      */
  int payoff;     /* ORC_PAYOFF_*                                     */
  int obstacle;   /* 0: lambda (Phi(x)-y)^+ ; 1: lambda (raw-y)^+     */
  int vol_kind;   /* ORC_VOL_*                                        */
  double T, r, lambda, K;
  double w[ORC_MAXD];      /* basket weights                         */
  double va[ORC_MAXD];     /* a_j                                    */
  double vb;               /* b                                      */
  double kappa[ORC_MAXD];  /* kappa_j (log-strike of the smile)      */
  double s_dupire;         /* s of eq. vol_locale                    */
  double div[ORC_MAXD];    /* dividend rates delta_j                 */
  double C[ORC_MAXD * ORC_MAXD]; /* correlation, row-major d x d     */
  double L[ORC_MAXD * ORC_MAXD]; /* lower Cholesky factor, C = L L^T */
  double lo[ORC_MAXD + 1], hi[ORC_MAXD + 1]; /* box of (t, x)        */
  uint32_t key[2];
} orc_model;

typedef struct {
  int p;          /* number of basis functions                       */
  int dp;         /* d' = d + 1 variates                              */
  int eta;        /* maximal partial degree present                   */
  const int* nu;  /* p x dp multi-indices, row-major                  */
} orc_basis;

/* diagnostics of one path, used by the pin tests */
typedef struct {
  int sstar;
  double theta, tau, u, ut, Lu, f, g1, uT, phiT, phitau, a;
  double XT[ORC_MAXD], Xtau[ORC_MAXD], Xs[ORC_MAXD];
} orc_path_info;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t w);
void orc_box_muller(uint32_t w0, uint32_t w1, double* z0, double* z1);
int orc_cholesky(int d, const double* C, double* L);
void orc_points(const orc_model* m, uint32_t k, int n, double* t, double* x /* [j][i] */);
void orc_normals_path(const orc_model* m, uint32_t k, uint32_t i, uint32_t path, int count, double* z);
void orc_bridge_normals(const orc_model* m, uint32_t k, uint32_t i, uint32_t path, double* z);
double orc_sigma(const orc_model* m, int j, double t, double xj);
double orc_payoff(const orc_model* m, const double* x);
void orc_basis_eval(const orc_model* m, const orc_basis* b, const double* alpha, double t,
                    const double* x, double* u, double* ut, double* ux, double* uxx);
double orc_path_a(const orc_model* m, const orc_basis* b, const double* alpha, double ti,
                  const double* xi, uint32_t k, uint32_t i, uint32_t path, orc_path_info* info);
void orc_correction(const orc_model* m, const orc_basis* b, const double* alpha, int npts,
                    const uint32_t* idx, const double* t, const double* x /* [j][npts] */,
                    uint32_t k, int nthreads, double* c);
void orc_samples(const orc_model* m, const orc_basis* b, const double* alpha, double ti,
                 const double* xi, uint32_t k, uint32_t i, int npaths, double* a);
void orc_simulate_XT(const orc_model* m, uint32_t k, uint32_t i, double ti, const double* xi,
                     int npaths, double* XT /* [path][d] */, double* Xtau, double* tau);

#endif
