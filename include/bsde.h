/*
 * bsde.h -- C ABI of the GB300 (sm_103a) solver for the Picard-iteration /
 * adaptive-control-variate BSDE method of Labart & Lelong, "A Parallel
 * Algorithm for solving BSDEs -- Application to the pricing and hedging of
 * American options" (arXiv:1102.4666).
 *
 * The library prices and hedges European and American (penalised) basket
 * options in a d-dimensional local-volatility model (Section 5) by solving
 * the BSDE  -dY = f(t,X,Y,Z) dt - Z dW,  Y_T = Phi(X_T)  (eq. eqs1) with the
 * driver f(t,x,y) = -r y + lambda (Phi(x) - y)^+ (eq. bsde-penal-2).  Every
 * step of Algorithm 2 runs in CUDA kernels: the random points, the Monte
 * Carlo correction c^k at every point (Euler paths, u^k, grad u^k and
 * (d_t + L^N) u^k along each path, per-point reduction), the Gram matrix
 * and right-hand side of the least-squares refit (eq. alphasys), its FP64
 * Cholesky solve, the coefficient update and the price/delta read-out.
 *
 * Conventions shared by every entry point:
 *   - All functions return an int status: BSDE_OK (0) or a negative
 *     BSDE_ERR_* code; bsde_last_error() then holds a message.  No entry
 *     point aborts the process or traps the GPU.
 *   - Host pointers (const double*, double*) are plain host memory owned by
 *     the caller; the library copies what it needs before returning.
 *   - Device memory is owned by the context and released by bsde_destroy();
 *     it comes from the caller's allocation hooks when given (for example
 *     PyTorch's caching allocator), else from a stream-ordered memory pool
 *     of the library (allocated and freed on the context's stream).
 *   - Calls on one context must not overlap (one host thread at a time).
 *   - Requires an sm_103a GPU; without one bsde_create() returns
 *     BSDE_ERR_CUDA.
 */
#ifndef BSDE_GB300_H
#define BSDE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* exported symbols of the shared library */
#if defined(__GNUC__)
#define BSDE_API __attribute__((visibility("default")))
#else
#define BSDE_API
#endif

#define BSDE_MAX_D 16  /* maximal number of assets d                      */
#define BSDE_MAX_IT 64 /* maximal number of Picard iterations per solve   */

/* status codes */
#define BSDE_OK 0
#define BSDE_ERR_INVALID_ARG -1 /* an argument is out of range            */
#define BSDE_ERR_STATE -2       /* a call came before its prerequisites   */
#define BSDE_ERR_ILLPOSED -3    /* basis larger than half the points      */
#define BSDE_ERR_NOMEM -4       /* allocation failed or budget exceeded   */
#define BSDE_ERR_NOT_PD -5      /* Gram matrix not positive definite      */
#define BSDE_ERR_TIMEOUT -6     /* a bounded device wait gave up          */
#define BSDE_ERR_CUDA -7        /* CUDA runtime error                     */
#define BSDE_ERR_EXCHANGE -8    /* the exchange hook of a sharded solve failed */

/* arithmetic of the path simulation and evaluation */
#define BSDE_PREC_FP64 0  /* everything in FP64 ("plain" comparator)      */
#define BSDE_PREC_MIXED 1 /* FP32 paths/basis/driver, FP64 per-point sums,
                             3xTF32 tensor-core Gram, FP64 Cholesky       */

/* volatility families sigma_j(t, x) of the model eq. eq4, Section 5.1, with
 * sigma_ij = sigma_j(t, x) L_ij and L the Cholesky factor of the correlation */
#define BSDE_VOL_CONST 0    /* sigma_j = a_j                                 */
#define BSDE_VOL_ABS_TANH 1 /* a_j + b e^{-t} |tanh(x_j - kappa_j)|          */
#define BSDE_VOL_SIN_TANH 2 /* a_j + b sin(j + t) tanh(x_j - kappa_j), j=1..d */
#define BSDE_VOL_DUPIRE 3   /* eq. vol_locale of Section 6.3 on S_j = e^{x_j} */

#define BSDE_PAYOFF_PUT 0  /* (K - sum_j w_j S_j)^+, eq. put_payoff            */
#define BSDE_PAYOFF_CALL 1 /* (sum_j w_j S_j - K)^+, eq. call_payoff           */

#define BSDE_OBSTACLE_PAYOFF 0 /* penalty lambda (Phi(x) - y)^+ (eq. bsde-penal-2) */
#define BSDE_OBSTACLE_RAW 1    /* penalty lambda (raw intrinsic - y)^+             */

typedef struct bsde_ctx bsde_ctx;

/* Allocation hooks: alloc(bytes, stream, user) returns device memory (or
 * NULL on failure); free(ptr, stream, user) releases it. */
typedef void* (*bsde_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*bsde_free_fn)(void* ptr, void* stream, void* user);

typedef struct {
  int device;           /* CUDA device ordinal                                */
  void* stream;         /* cudaStream_t to work on; NULL: the library creates
                           its own non-blocking stream                        */
  bsde_alloc_fn alloc;  /* optional device allocator (NULL: a stream-ordered
                           memory pool of the library, cudaMallocFromPoolAsync) */
  bsde_free_fn free;    /* its release function (required with alloc)          */
  void* alloc_user;     /* passed back to alloc/free                           */
  size_t mem_budget;    /* bytes of device memory the context may hold; 0 = no
                           limit; exceeding it gives BSDE_ERR_NOMEM            */
  int precision;        /* BSDE_PREC_*                                        */
} bsde_create_opts;

/* Create a context.  *out is written only on success. */
BSDE_API int bsde_create(bsde_ctx** out, const bsde_create_opts* opts);

/* Release the context and all device memory it holds.  NULL is allowed. */
BSDE_API void bsde_destroy(bsde_ctx* ctx);

/* Message of the last failing call on ctx (never NULL; "" when none).  With
 * ctx == NULL, the message of the last failing bsde_create in this thread. */
BSDE_API const char* bsde_last_error(const bsde_ctx* ctx);

/* Volatility and correlation of the model eq. eq4 (Section 5.1) with the
 * correlated Brownian motion of Section 6.2 (C = L L^*). */
typedef struct {
  int d;               /* number of assets, 1..BSDE_MAX_D; the path kernels  */
                       /* are compiled for d = 1..10 (bsde_solve and        */
                       /* bsde_iterate return BSDE_ERR_INVALID_ARG above)    */
  int kind;            /* BSDE_VOL_*                                          */
  const double* a;     /* d values a_j (NULL: a_scalar for every asset)      */
  double a_scalar;
  double b;            /* amplitude b of the local part                      */
  const double* kappa; /* d values kappa_j (NULL: kappa_scalar)              */
  double kappa_scalar;
  double s_dupire;     /* s of eq. vol_locale (BSDE_VOL_DUPIRE)              */
  double rho;          /* constant correlation, used when corr == NULL       */
  const double* corr;  /* optional d x d correlation matrix, row-major       */
  const double* div;   /* optional d dividend rates delta_j (NULL: 0)        */
} bsde_sigma;

/* Payoff Phi of the option (Section 6.2.1) on S = e^x. */
typedef struct {
  int kind;               /* BSDE_PAYOFF_*                                   */
  double K;               /* strike                                          */
  double T;               /* maturity                                        */
  const double* S0;       /* d spot prices (the read-out point x0 = log S0)  */
  const double* weights;  /* d basket weights (NULL: 1/d each)               */
} bsde_payoff;

/* Penalisation of eq. bsde-penal-2: lambda = 0 gives the European option
 * (Section 5.5), lambda > 0 the penalised approximation of the American
 * option (Section 5.4). */
typedef struct {
  double lambda;
  int obstacle; /* BSDE_OBSTACLE_* */
} bsde_penalty;

/* Set the model: volatility, interest rate r, payoff and penalty.  All
 * inputs are copied.  Fails with BSDE_ERR_INVALID_ARG when d is out of range,
 * the correlation is not positive definite, or a parameter is not finite. */
BSDE_API int bsde_set_model(bsde_ctx* ctx, const bsde_sigma* sigma, double r, const bsde_payoff* payoff,
                   const bsde_penalty* penalty);

/* Set the approximation grid of Algorithm 2: n random points per iteration,
 * uniform on the box [lo_0, hi_0] x prod_j [lo_j, hi_j] of (t, x = log S)
 * (d+1 values each; the time box is normally [0, T]).  The polynomial
 * variates are reduced to [-1,1]^{d+1} on this machine (Section 3.2.2).
 * resample_each_iter = 1 draws fresh points every iteration (Algorithm 2);
 * 0 keeps the points of iteration 0. */
BSDE_API int bsde_set_grid(bsde_ctx* ctx, int n, const double* lo, const double* hi,
                  int resample_each_iter);

typedef struct {
  int M;            /* Monte Carlo paths per point                        */
  int N_steps;      /* Euler steps per path, on [t_i, T]; the path kernel
                       keeps per-step volatility coefficients and Philox
                       words in shared memory (about 12 d bytes per step
                       with FP32 paths, 20 d with FP64), so very long
                       paths give BSDE_ERR_INVALID_ARG                  */
  int eta;          /* maximal total degree of the basis                  */
  double q;         /* hyperbolic index of eq. hyper_set (1 = total degree) */
  int K_it;         /* Picard iterations, 1..BSDE_MAX_IT                  */
  uint64_t seed;    /* Philox4x32-10 key                                  */
  int k_start;      /* first iteration index (0; >0 resumes from the
                       coefficients set by bsde_set_coeffs)               */
  int refine_steps; /* iterative-refinement steps of the normal equations
                       with an FP64 residual (MIXED: default 2 when < 0)  */
  int use_graph;    /* 1: replay the solve as one captured CUDA graph      */
  int timing;       /* 1: record per-kernel CUDA-event timings in the report */
  int allow_underdetermined; /* 1: skip the p <= n/2 check (a basis larger
                                than the point set makes the Gram matrix
                                singular: the solve then ends with
                                BSDE_ERR_NOT_PD)                       */
  int eval_mode;    /* evaluation of u^k along the paths: 0 automatic, 1
                       per-thread Chebyshev tables (any degree), 2 dense
                       monomial form (constant correlation; total degree
                       <= 3, or <= 4 for d <= 5; with BSDE_PREC_MIXED
                       also <= 4 for d <= 10 and <= 6 for d <= 5)      */
  int paths_tpb;    /* threads per CTA of the path kernel (0: automatic;
                       32..256, a multiple of 32)                       */
  int paths_ppt;    /* paths per thread of the path kernel (0: automatic;
                       1..16)                                           */
  int ls_mode;      /* least-squares refit (eq. alpha): 0 normal equations,
                       tensor-core/FP64 Gram + FP64 Cholesky + refinement;
                       1 FP64 Householder QR with column pivoting and rank
                       truncation at 1e-13 |R_00| on the design matrix (the
                       role of LAPACK dgelsy in Section 3.2.2; slower, for
                       ill-conditioned or rank-deficient bases)        */
  int gram_splits;  /* slices of the point dimension of the tensor-core Gram
                       matrix (BSDE_PREC_MIXED; each slice accumulates in
                       FP32, the slices are summed in FP64): 0 automatic
                       (one wave of the device's multiprocessors), else
                       that many, at most one per 32 points; 0..4096    */
} bsde_solve_params;

typedef struct {
  int status;                  /* BSDE_OK or the error of the solve         */
  int d, p, K_it;              /* problem sizes                             */
  double price;                /* u^{K_it}(0, log S0)                        */
  double delta[BSDE_MAX_D];    /* dV/dS_j = (du/dx_j)(0, log S0) / S0_j      */
  double dudx[BSDE_MAX_D];     /* du/dx_j (0, log S0)                        */
  double price_iter[BSDE_MAX_IT];  /* price after each iteration           */
  double resid_l2[BSDE_MAX_IT];    /* ||alpha^{k+1} - alpha^k||_2           */
  double resid_linf[BSDE_MAX_IT];  /* ||alpha^{k+1} - alpha^k||_inf         */
  double ms_total;             /* device time of the whole solve (events)   */
  double ms_paths;             /* device time of the path kernels (timing=1) */
  double ms_gram;              /* device time of the Gram matrices, their
                                  Cholesky factors and inverses, built for a
                                  group of iterations ahead of their path
                                  kernels (timing=1)                         */
  double ms_solve;             /* device time of the refit after the paths
                                  (RHS, inverse products, refinement; the
                                  whole pivoted-QR refit with ls_mode 1)     */
  double path_steps;           /* K_it * n * M * N                          */
  double path_steps_per_s;     /* path_steps / ms_total                     */
  int path_launches;           /* path-kernel launches in the solve          */
  int kernel_launches;         /* all kernel launches in the solve           */
  int rank;                    /* numerical rank of the last refit (ls_mode 1;
                                  p with ls_mode 0)                           */
} bsde_report;

/* Run Algorithm 2 for K_it iterations from alpha = 0 (or from the
 * coefficients of bsde_set_coeffs when k_start > 0).  Synchronous: the
 * report is complete on return.  Errors: BSDE_ERR_STATE without model/grid,
 * BSDE_ERR_ILLPOSED when the basis size p exceeds n/2, BSDE_ERR_NOMEM,
 * BSDE_ERR_NOT_PD when the Cholesky factorisation of the Gram matrix meets a
 * non-positive pivot, BSDE_ERR_CUDA. */
BSDE_API int bsde_solve(bsde_ctx* ctx, const bsde_solve_params* params, bsde_report* report);

/* One iteration k -> k+1 of Algorithm 2 from the coefficients alpha_in
 * (p values; NULL keeps the current ones).  Optional outputs (NULL to skip):
 * t_out (n), x_out (d x n, row j holds x_j of every point), c_out (n, the
 * Monte Carlo corrections c^k_i of eq. chat), alpha_out (p, alpha^{k+1}).
 * The context's coefficients become alpha^{k+1}. */
BSDE_API int bsde_iterate(bsde_ctx* ctx, const bsde_solve_params* params, int k, const double* alpha_in,
                 double* t_out, double* x_out, double* c_out, double* alpha_out);

/* The Gram matrix A = sum_i B(t_i, x_i) B(t_i, x_i)^T of the normal
 * equations (eq. alphasys, Section 3.2.2) at the n points of iteration k,
 * B_l the basis functions in the order of bsde_basis_indices: A_out
 * receives p x p FP64 values, row-major (cap: its capacity in values,
 * at least p * p).  It is the matrix that the refit of iteration k in a
 * solve with the same parameters factorises: with BSDE_PREC_MIXED the 3xTF32
 * tensor-core product (each basis value split into two TF32 parts, FP32
 * accumulation within each of gram_splits slices of the points, the slices
 * summed in FP64), with BSDE_PREC_FP64 the FP64 product.  Needs set_model and
 * set_grid; the coefficients of the context are left unchanged.  Errors as
 * bsde_solve, and BSDE_ERR_INVALID_ARG when cap < p * p. */
BSDE_API int bsde_gram_matrix(bsde_ctx* ctx, const bsde_solve_params* params, int k, double* A_out,
                              int cap);

/* ------------------------------------------------------------------------
 * Point sharding (Section 4.2: the loop over the points of an iteration is
 * parallel, and the paper's master/slave scheme of Section 4.3 distributes
 * it).  With nranks > 1, rank `rank` of a group of contexts (normally one
 * process per GPU) runs the path kernel and the per-point reduction only on
 * its block of points [i0, i1) = bsde_shard_block(n, rank, nranks): blocks
 * of nb = ceil(n / nranks) consecutive points, the last one shorter.  Every
 * rank draws all n points itself (they depend on (seed, k) only) and builds
 * the basis matrix, the Gram matrices and their factors of all n points, so
 * the only data that crosses ranks is the corrections c_i: once per
 * iteration, after its block's c_i are written (stream-ordered) to
 * c_dev[i0 .. i1), the library calls on the host
 *     exchange(c_dev, nb, rank, nranks, stream, user)
 * which must enqueue on `stream`, or make `stream` wait for, an operation
 * after which c_dev[q nb .. q nb + nb) holds the block of every rank q
 * (an all-gather of nb doubles per rank, e.g. ncclAllGather in place with
 * sendbuff = c_dev + rank nb); it returns 0, or nonzero to make the solve
 * fail with BSDE_ERR_EXCHANGE.  The refit then uses all n corrections
 * exactly as the unsharded solve does: every rank ends with the same
 * coefficients, equal bit for bit to those of the unsharded solve.
 *   c_dev, c_len: device buffer of the caller (c_len doubles, at least
 *   nranks * nb for the grid of the solve), read and written on the
 *   context's stream; it must stay valid while the setting holds.
 * nranks = 1 turns sharding off (c_dev and exchange may then be NULL).
 * While sharded, solves run as direct launches (use_graph is ignored: the
 * exchange is a host call in every iteration).  Errors:
 * BSDE_ERR_INVALID_ARG (rank out of range, missing buffer or hook). */
typedef int (*bsde_exchange_fn)(double* c_dev, int nb, int rank, int nranks, void* stream,
                                void* user);
BSDE_API int bsde_set_shard(bsde_ctx* ctx, int rank, int nranks, double* c_dev, size_t c_len,
                            bsde_exchange_fn exchange, void* user);
/* The block [*i0, *i1) of rank `rank` (host only, no GPU). */
BSDE_API int bsde_shard_block(int n, int rank, int nranks, int* i0, int* i1);

/* The same sharding with the exchange done on the devices by peer stores,
 * for GPUs that address each other's memory (NVLink peers of one node, with
 * peer access enabled or the buffers mapped by the caller).  Every rank owns
 * a correction buffer of c_len >= 2 * nranks * nb doubles and an array of
 * nranks uint32 arrival counters, zeroed before the first solve; px gives,
 * for every rank q, the addresses of q's buffer and counters as this
 * context's device sees them.  In each iteration, after its block of
 * corrections is computed (into its own buffer), this rank stores the block
 * into every other rank's buffer at the same offset and then raises its
 * counter in their arrays to the iteration's exchange number (stream-ordered
 * kernels); it then waits on the device until every other rank's counter in
 * its own array has reached that number, at most wait_ms milliseconds
 * (0: 1000).  If the bound passes (a rank that failed or never joined) the
 * solve completes without further waits and returns BSDE_ERR_TIMEOUT; the
 * context stays usable.  Buffers alternate between two halves from one
 * exchange to the next, so a rank one exchange ahead never overwrites data
 * that another still reads.  pushed (optional) is called on the host after
 * this rank's push has been enqueued and before the wait is, with this
 * rank's buffer (as bsde_exchange_fn: its return value is ignored unless
 * nonzero, which fails the solve with BSDE_ERR_EXCHANGE).  The result
 * equals the unsharded solve bit for bit, as with bsde_set_shard.  The
 * exchange numbers count on from the previous solves of the context, so
 * every rank must run the same sequence of solves.  nranks = 1 or
 * bsde_set_shard(ctx, 0, 1, ...) turns sharding off. */
#define BSDE_MAX_RANKS 64
typedef struct {
  double* c[BSDE_MAX_RANKS];      /* rank q's correction buffer              */
  uint32_t* flag[BSDE_MAX_RANKS]; /* rank q's arrival counters (nranks each) */
  size_t c_len;                   /* doubles in each correction buffer       */
  double wait_ms;                 /* bound of the device wait (0: 1000 ms)   */
  bsde_exchange_fn pushed;        /* optional host call between push and wait */
  void* user;                     /* passed back to pushed                   */
} bsde_peer_exchange;
BSDE_API int bsde_set_shard_peers(bsde_ctx* ctx, int rank, int nranks, const bsde_peer_exchange* px);

/* Basis size p of the current solve parameters, and the multi-indices in
 * the library's order (p x (d+1) ints, graded, lexicographically descending
 * with the time variate first).  Host-only; needs no GPU. */
BSDE_API int bsde_basis_size(int d, int eta, double q, int* p_out);
BSDE_API int bsde_basis_indices(int d, int eta, double q, int* nu_out, int cap_rows);

/* Copy the current coefficients alpha (p values in the order of
 * bsde_basis_indices) to the host; cap is the capacity of out. */
BSDE_API int bsde_get_coeffs(bsde_ctx* ctx, double* out, int cap);

/* Replace the coefficients (checkpoint / resume: the state after iteration
 * k is (alpha^k, k, seed)); p must match the basis of the last solve or of
 * the parameters given. */
BSDE_API int bsde_set_coeffs(bsde_ctx* ctx, const bsde_solve_params* params, const double* alpha, int p);

/* Evaluate the fitted u at q query points: price[i] = u(t[i], log S[i,:])
 * and delta[i*d + j] = (du/dx_j)/S[i,j] (NULL to skip).  S is q x d
 * row-major prices.  Requires a completed solve or bsde_set_coeffs
 * (BSDE_ERR_STATE otherwise). */
BSDE_API int bsde_eval_price_delta(bsde_ctx* ctx, int q, const double* t, const double* S, double* price,
                          double* delta);

/* ------------------------------------------------------------------------
 * No-allocation entry point.  The paper has no counterpart: it serves
 * callers of this library that cannot allocate device memory themselves or
 * through the library -- code that runs inside a fixed device-memory arena,
 * a plugin whose host process forbids cudaMalloc/cudaFree, or a steady-state
 * service loop that must never enter the allocator.
 *
 * bsde_corrections_noalloc computes the Monte Carlo corrections c^k_i of
 * eq. chat (Algorithm 2) at n given points with the path kernel, like
 * c_out of bsde_iterate with eval_mode 1, and calls no allocating routine
 * (no cudaMalloc, cudaFree, PyTorch or other allocator).  Inputs and outputs
 * are the caller's device buffers: t_dev (n), x_dev (d x n, row j holding
 * x_j of every point), alpha_dev (p FP64 coefficients in the order of
 * bsde_basis_indices for (d, eta, q)) and c_dev (n outputs).  The model and
 * the box (lo, hi: d+1 host values each) are as in bsde_set_model and
 * bsde_set_grid; M, N_steps, seed and the iteration index k as in a solve;
 * precision is BSDE_PREC_FP64 or BSDE_PREC_MIXED.  Works on the current
 * CUDA device and on `stream` (NULL: the legacy default stream); it returns
 * after the stream has finished the work.
 *
 * The kernel's scratch (per-chunk partial sums, the packed basis table, the
 * FP32 coefficient copy, the Philox key) is one static 4 MiB device array
 * that every GPU loading the library holds until the process exits.  Limits:
 * p <= 4096 basis functions and n * ceil(M / C) <= 503808, where C is the
 * number of paths per chunk that the path kernel uses (512 in MIXED and 256
 * in FP64 precision when M >= 256 and the basis tables fit; fewer for small
 * M or large bases); larger problems are rejected with BSDE_ERR_NOMEM
 * before any device work.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not call this entry point on a device after a
 * cudaDeviceReset of that device in the same process (the array may then
 * live at another address).  Each call blocks until its work is done.  Every call uses the same array
 * and the array keeps the last call's contents; each call rewrites every
 * scratch word it reads, so nothing needs clearing, but calls that overlap
 * on the GPU (other streams, other host threads) race on the array and must
 * be serialised by the caller.  errbuf (optional, errbuf_len bytes) receives
 * a message on failure.  Errors: BSDE_ERR_INVALID_ARG, BSDE_ERR_NOMEM (too
 * large for the scratch), BSDE_ERR_CUDA. */
BSDE_API int bsde_corrections_noalloc(const bsde_sigma* sigma, double r, const bsde_payoff* payoff,
                                      const bsde_penalty* penalty, const double* lo,
                                      const double* hi, int n, const double* t_dev,
                                      const double* x_dev, int eta, double q,
                                      const double* alpha_dev, int M, int N_steps, uint64_t seed,
                                      int k, int precision, double* c_dev, void* stream,
                                      char* errbuf, size_t errbuf_len);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching server of pricing requests.  Requests of
 * uneven d, n, M, N and degree are admitted while device memory (the
 * server's budget) and slots allow; each keeps its coefficients and points
 * resident across its Picard iterations; the iterations of all admitted
 * requests run concurrently on the device (requests with less work than the
 * average so far on high-priority streams); a finished request frees its
 * slot for the next one in the queue.
 * ---------------------------------------------------------------------- */
typedef struct bsde_server bsde_server;

#define BSDE_POLICY_FIFO 0     /* admit in arrival order                        */
#define BSDE_POLICY_SHORTEST 1 /* admit the queued request with the fewest
                                  path-steps (K_it n M N) first             */
#define BSDE_POLICY_RESPONSE_RATIO 2 /* admit the queued request with the
                                  highest (wait + service) / service, the
                                  service time estimated from its path-steps
                                  and the server's measured throughput: short
                                  requests go first, long ones rise as they
                                  wait (no starvation)                      */
#define BSDE_POLICY_SIZE_LANES 3 /* arrival order in two lanes: a request with
                                  less work than the average so far is
                                  admitted at once (high-priority stream);
                                  one with at least the average work waits
                                  while large_slots others of its lane run,
                                  and the smaller requests behind it pass it */

typedef struct {
  int device;
  int max_slots;        /* requests resident at once (1..64)             */
  size_t mem_budget;    /* device bytes for resident requests            */
  int precision;        /* BSDE_PREC_*                                   */
  int policy;           /* BSDE_POLICY_*                                 */
  int large_slots;      /* BSDE_POLICY_SIZE_LANES: requests of the large
                           lane resident at once (0: 2)                  */
} bsde_server_opts;

typedef struct {
  bsde_sigma sigma;
  double r;
  bsde_payoff payoff;
  bsde_penalty penalty;
  int n;
  double lo[BSDE_MAX_D + 1], hi[BSDE_MAX_D + 1];
  bsde_solve_params params;
} bsde_request;

typedef struct {
  uint64_t completed, queued, running;
  double p50_ms, p99_ms;     /* latency from submit to completion          */
  double path_steps;         /* over completed requests                    */
  double busy_s;             /* wall time with at least one request running */
  double path_steps_per_s;   /* path_steps / busy_s                         */
} bsde_server_stats;

BSDE_API int bsde_server_create(bsde_server** out, const bsde_server_opts* opts);
/* Copy the request and queue it; *id identifies it in poll. */
BSDE_API int bsde_server_submit(bsde_server* srv, const bsde_request* req, uint64_t* id);
/* 1 and the report when request id is done, 0 while it is queued or
 * running, <0 on error (unknown id).  A done request is forgotten after it
 * has been polled. */
BSDE_API int bsde_server_poll(bsde_server* srv, uint64_t id, bsde_report* report);
/* Block until every submitted request is done (timeout_ms <= 0: no limit);
 * BSDE_ERR_TIMEOUT when the limit passes first. */
BSDE_API int bsde_server_drain(bsde_server* srv, double timeout_ms);
BSDE_API int bsde_server_stats_get(bsde_server* srv, bsde_server_stats* stats);
BSDE_API void bsde_server_destroy(bsde_server* srv);
BSDE_API const char* bsde_server_last_error(const bsde_server* srv);

#ifdef __cplusplus
}
#endif
#endif
