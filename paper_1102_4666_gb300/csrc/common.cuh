// common.cuh -- shared device helpers and the internal launch interfaces of
// the BSDE kernels (Labart & Lelong, Algorithm 2).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#define BSDE_DMAX 16
#define BSDE_NNZ_MAX 8  // active variates per basis function
#define BSDE_RANKS_MAX 64  // ranks of a point-sharded solve (BSDE_MAX_RANKS of the C ABI)

// device addresses, as this device sees them, of every rank's correction
// buffer and arrival-counter array (peer exchange of a sharded solve)
struct PeerPtrs {
  double* c[BSDE_RANKS_MAX];
  uint32_t* flag[BSDE_RANKS_MAX];
};

// Philox4x32-10 counter tags (top byte of the fourth counter word)
#define TAG_PTS 1u
#define TAG_U 2u
#define TAG_Z 3u
#define TAG_B 4u

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by the Philox constants, swaps and xors the high
// halves with words 1/3 and the round key.  Key schedule: Weyl increments.
// ---------------------------------------------------------------------------
struct Philox {
  uint32_t k0, k1;
  __device__ __forceinline__ uint4 operator()(uint32_t c0, uint32_t c1, uint32_t c2,
                                              uint32_t c3) const {
    uint32_t a = k0, b = k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      // one 32x32 -> 64-bit multiply each (wide integer multiply-add)
      const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u;
      const uint64_t p1 = (uint64_t)c2 * 0xCD9E8D57u;
      const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
      const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
      const uint32_t n0 = hi1 ^ c1 ^ a;
      const uint32_t n2 = hi0 ^ c3 ^ b;
      c0 = n0;
      c1 = lo1;
      c2 = n2;
      c3 = lo0;
      a += 0x9E3779B9u;
      b += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
  }
};

// ---------------------------------------------------------------------------
// Precision traits (Box-Muller returns scale * (z0, z1)): the FP32 path uses the fast hardware approximations
// (MUFU) where their error is far below the Monte Carlo noise; the FP64 path
// uses CUDA's double-precision math library.
// ---------------------------------------------------------------------------
template <typename R>
struct Math;

template <>
struct Math<float> {
  // Box-Muller pair from two 32-bit words, u = (w + 1/2) 2^-32 in (0,1],
  // returning scale * (z0, z1).  k = bm_factor(scale) = -2 ln(2) scale^2
  // folds the scale and the change of logarithm base into one product:
  // (scale r)^2 = -2 ln(u0) scale^2 = log2(u0) k.
  __device__ __forceinline__ static float bm_factor(float scale) {
    return -1.3862943611198906f * scale * scale;
  }
  __device__ __forceinline__ static void box_muller(uint32_t w0, uint32_t w1, float& z0,
                                                    float& z1, float k) {
    // u0 = (w0 + 1/2) 2^-32 and the angle 2 pi u1 - pi in (-pi, pi] (straight
    // from w1; cos/sin flip sign) in one packed FP32x2 multiply-add
    const float2 ua = __ffma2_rn(make_float2(__uint2float_rn(w0), __uint2float_rn(w1)),
                                 make_float2(2.3283064365386963e-10f, 1.4629180792671596e-09f),
                                 make_float2(1.1641532182693481e-10f, -3.1415926528f));
    float lg;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(ua.x));
    // radius: r2 = lg * k >= 0 (lg <= 0, k < 0), one approximate square
    // root (sqrt(0) = 0 at u0 = 1: no clamp needed)
    const float r2 = lg * k;
    float rad, s, c;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rad) : "f"(r2));
    // The .ftz forms: no operand here is subnormal (u0 >= 2^-33; r2 is 0 or
    // above 1e-20 for any step h >= 1e-10; |angle| is 0 or above 1e-9), so
    // flushing changes no result and saves the subnormal handling of the
    // non-ftz forms.
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(ua.y));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(ua.y));
    const float2 zz = __fmul2_rn(make_float2(-rad, -rad), make_float2(c, s));
    z0 = zz.x;
    z1 = zz.y;
  }
  // e^x = 2^(x log2 e); results below the normal range flush to 0
  __device__ __forceinline__ static float exp(float x) {
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x * 1.4426950408889634f));
    return e;
  }
  __device__ __forceinline__ static float sqrt(float x) { return sqrtf(x); }
  __device__ __forceinline__ static float sin(float x) { return sinf(x); }
  __device__ __forceinline__ static float exp_acc(float x) { return expf(x); }
  __device__ __forceinline__ static float fabs(float x) { return fabsf(x); }
  __device__ __forceinline__ static float fmax(float a, float b) { return fmaxf(a, b); }
};

template <>
struct Math<double> {
  // the FP64 path applies the scale after the square root
  __device__ __forceinline__ static double bm_factor(double scale) { return scale; }
  __device__ __forceinline__ static void box_muller(uint32_t w0, uint32_t w1, double& z0,
                                                    double& z1, double scale) {
    const double u0 = ((double)w0 + 0.5) * 2.3283064365386962890625e-10;
    const double u1 = ((double)w1 + 0.5) * 2.3283064365386962890625e-10;
    const double rad = ::sqrt(-2.0 * ::log(u0)) * scale;
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
  }
  __device__ __forceinline__ static double exp(double x) { return ::exp(x); }
  __device__ __forceinline__ static double sqrt(double x) { return ::sqrt(x); }
  __device__ __forceinline__ static double sin(double x) { return ::sin(x); }
  __device__ __forceinline__ static double exp_acc(double x) { return ::exp(x); }
  __device__ __forceinline__ static double fabs(double x) { return ::fabs(x); }
  __device__ __forceinline__ static double fmax(double a, double b) { return ::fmax(a, b); }
};

// ---------------------------------------------------------------------------
// Host-side description of one solve, shared by the launchers.
// ---------------------------------------------------------------------------
struct ModelHost {
  int d = 0;
  int vol_kind = 0;
  int payoff = 0;
  int obstacle = 0;
  double T = 1.0, r = 0.0, lambda = 0.0, K = 0.0;
  double a[BSDE_DMAX] = {0}, kappa[BSDE_DMAX] = {0}, div[BSDE_DMAX] = {0};
  double w[BSDE_DMAX] = {0}, S0[BSDE_DMAX] = {0};
  double b = 0.0, s_dupire = 0.0;
  double C[BSDE_DMAX * BSDE_DMAX] = {0};
  double L[BSDE_DMAX * BSDE_DMAX] = {0};
};

struct GridHost {
  int n = 0;
  int resample = 1;
  double lo[BSDE_DMAX + 1] = {0}, hi[BSDE_DMAX + 1] = {0};
};

// Device pointers of one resident problem (one context or one served request)
struct ProblemDev {
  int n = 0, n_pad = 0, p = 0, p_pad = 0, eta = 0, chunks = 0;
  int gram_splits = 0;        // K splits of the tensor-core Gram (mixed)
  // point sharding: the path kernel and the per-point reduction cover the
  // points [shard_i0, shard_i0 + shard_n) only (shard_n = 0: all n points)
  int shard_i0 = 0, shard_n = 0;
  double* t = nullptr;        // [n]
  double* x = nullptr;        // [d][n]
  double* B = nullptr;        // [p][n_pad] FP64 basis matrix, point index fastest
  float* Bhi = nullptr;       // [p_pad][n_pad] tf32-rounded high part (mixed)
  float* Blo = nullptr;       // [p_pad][n_pad] tf32-rounded remainder (mixed)
  double* partial = nullptr;  // [n][chunks] per-chunk sums of a_m
  double* c = nullptr;        // [n] corrections
  double* A = nullptr;        // [nfact][p][p] Gram matrices, then their Cholesky factors
  float* gram_part = nullptr; // split-K partial tiles of the tensor-core Gram
  double* rhs = nullptr;      // [p]
  double* delta = nullptr;    // [p] solution of the normal equations
  double* res = nullptr;      // [p] refinement residual
  double* v = nullptr;        // [max(n, p)] B delta
  double* dinv = nullptr;     // [nfact][p] reciprocal diagonals of the Cholesky factors
  double* diag0 = nullptr;    // [nfact][p] original diagonals (relative pivot test)
  double* Ainv = nullptr;     // [nfact][p][p] inverses of the Gram matrices
  double* alpha = nullptr;    // [p] coefficients (FP64 master)
  float* alpha32 = nullptr;   // [p] FP32 copy for the mixed path kernel
  uint2* pairs = nullptr;     // [p] packed (variate, degree) bytes
  uint8_t* nnz = nullptr;     // [p] active variates per basis function
  uint32_t* key = nullptr;    // [2] Philox key (device copy, read by the points kernel)
  uint32_t seed_key[2] = {0, 0};  // the same key on the host, a parameter of the path kernel
  int* status = nullptr;      // [1] device status bits
  double* out = nullptr;      // report block (see OUT_* offsets)
  // dense evaluation (basis of total degree <= 3, or <= 4 for d <= 5):
  // monomial coefficients
  bool dense = false;
  bool dense4 = false;        // monomials up to degree 4 (graded order)
  int tree = 0;               // > 0: monomials up to this degree in prefix-tree order
  int pm = 0;                 // number of monomials, C(d + 4, 3) or C(d + 5, 4)
  double* beta = nullptr;     // [pm]
  float* beta32 = nullptr;    // [pm]
  int* conv_row = nullptr;    // [pm + 1] CSR rows of the Chebyshev -> monomial map
  int* conv_l = nullptr;      // basis-function index of each entry
  double* conv_c = nullptr;   // coefficient of each entry
  // pivoted-QR refit workspace (ls_mode 1)
  double* qr_W = nullptr;     // [p][n_pad] design matrix, then R and the reflectors
  double* qr_y = nullptr;     // [n] right-hand side, then Q^T c
  double* qr_nrm = nullptr;   // [p] squared norms of the remaining columns
  double* qr_tau = nullptr;   // [p] reflector coefficients
  int* qr_perm = nullptr;     // [p] column permutation
  int* qr_rank = nullptr;     // [1] numerical rank
};

// offsets in ProblemDev::out
#define OUT_PRICE 0
#define OUT_DUDX 1                        // d values
#define OUT_PRICE_IT (1 + BSDE_DMAX)      // BSDE_MAX_IT values
#define OUT_RES2 (OUT_PRICE_IT + 64)
#define OUT_RESI (OUT_RES2 + 64)
#define OUT_SIZE (OUT_RESI + 64)

// device status bits
#define ST_NOT_PD 1
#define ST_TIMEOUT 2
#define ST_BADARG 4

// launchers (one translation unit each)
void launch_points(const ModelHost& m, const GridHost& g, const ProblemDev& P, uint32_t k,
                   cudaStream_t st);
void launch_basis(const ModelHost& m, const GridHost& g, const ProblemDev& P, bool mixed,
                  cudaStream_t st);
// path kernel: returns cudaSuccess or the launch error
cudaError_t launch_paths(const ModelHost& m, const GridHost& g, const ProblemDev& P, int M, int N,
                         uint32_t k, bool mixed, int tpb, int ppt, cudaStream_t st);
void launch_reduce_c(const ProblemDev& P, int M, cudaStream_t st);
void launch_gram_f64(const ProblemDev& P, cudaStream_t st);
cudaError_t launch_gram_tc(const ProblemDev& P, cudaStream_t st);
// K splits of the tensor-core Gram (want > 0: that many, capped by the
// K-blocks; 0: one wave of the device's SMs) and the bytes of its partial tiles
int gram_tc_splits(int p_pad, int n_pad, int want);
size_t gram_tc_part_bytes(int p_pad, int n_pad, int splits);
// multiprocessor count of the current device (cached per device)
int device_sm_count();
void launch_rhs(const ProblemDev& P, cudaStream_t st);
// batched over nb Gram matrices (P.A, P.dinv, P.diag0, P.Ainv hold nb of them)
void launch_cholesky(const ProblemDev& P, int nb, cudaStream_t st);
void launch_refine_residual(const ProblemDev& P, cudaStream_t st);
void launch_update(const ProblemDev& P, int k, cudaStream_t st);
void launch_eval_x0(const ModelHost& m, const GridHost& g, const ProblemDev& P, int k,
                    cudaStream_t st);
void launch_eval_points(const ModelHost& m, const GridHost& g, const ProblemDev& P, int q,
                        const double* t, const double* x, double* price, double* dudx,
                        cudaStream_t st);
size_t paths_smem_bytes(int d, int p, int eta, int N, int tpb, bool mixed, bool dense);
void launch_cheb2mono(const ProblemDev& P, cudaStream_t st);
void launch_qr_solve(const ProblemDev& P, cudaStream_t st);
void launch_inverse(const ProblemDev& P, int nb, cudaStream_t st);
void launch_inv_gemv(const ProblemDev& P, const double* b, double* x, int accumulate, cudaStream_t st);
int paths_supported_d(int d);
// peer exchange of a sharded solve: push this rank's block [i0, i0 + count)
// of `mine` into every other rank's buffer (at region_off) and raise their
// counters to `epoch`; then wait, at most wait_ms, for the others' counters
// in `flags` (ST_TIMEOUT in status when the bound passes)
cudaError_t launch_exchange_peers(const double* mine, int i0, int count, int rank, int nranks,
                                  const PeerPtrs& pp, size_t region_off, uint32_t epoch,
                                  cudaStream_t st);
cudaError_t launch_exchange_wait(const uint32_t* flags, int rank, int nranks, uint32_t epoch,
                                 double wait_ms, int* status, cudaStream_t st);
