// runtime.cu -- host runtime of one resident BSDE problem (see runtime.h).
#include "runtime.h"

#include <cmath>
#include <cstring>
#include <mutex>
#include <sstream>

#include "multiindex.h"

// Without caller hooks, memory comes from a library-private stream-ordered
// pool per device: cudaFree would synchronise the whole device, which in the
// serving loop stalls every resident request at each completion.  The pool
// keeps up to 2 GiB of freed memory for reuse.
namespace {
constexpr int POOL_DEVICES = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[POOL_DEVICES] = {};
bool g_pool_tried[POOL_DEVICES] = {};

cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= POOL_DEVICES) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pool_tried[dev]) {
    g_pool_tried[dev] = true;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&g_pool[dev], &props) != cudaSuccess) {
      cudaGetLastError();
      g_pool[dev] = nullptr;
    } else {
      uint64_t keep = (uint64_t)2 << 30;
      cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  return g_pool[dev];
}
}  // namespace

void* Allocator::get(size_t bytes, cudaStream_t st) {
  if (alloc) return alloc(bytes, (void*)st, user);
  void* p = nullptr;
  cudaMemPool_t pool = device_pool();
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void Allocator::put(void* p, cudaStream_t st) {
  if (!p) return;
  if (alloc) {
    if (free) free(p, (void*)st, user);
  } else if (device_pool()) {
    cudaFreeAsync(p, st);
  } else {
    cudaFree(p);
  }
}

int device_sm_count() {
  static std::mutex mu;
  static int cache[POOL_DEVICES] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= POOL_DEVICES) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> g(mu);
  if (cache[dev] == 0) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      return 1;
    }
    cache[dev] = sms;
  }
  return cache[dev];
}

void shard_block(int n, int rank, int nranks, int& i0, int& i1) {
  const int nb = (n + nranks - 1) / nranks;
  const long long a = (long long)rank * nb, b = a + nb;
  i0 = (int)(a < n ? a : n);
  i1 = (int)(b < n ? b : n);
}

static bool is_fin(double v) { return std::isfinite(v); }

// Cholesky-Banachiewicz of the d x d correlation (C = L L^*, Section 6.2)
static bool cholesky_host(int d, const double* C, double* L) {
  for (int i = 0; i < d * d; ++i) L[i] = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = C[i * d + j];
      for (int q = 0; q < j; ++q) s -= L[i * d + q] * L[j * d + q];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i * d + i] = std::sqrt(s);
      } else {
        L[i * d + j] = s / L[j * d + j];
      }
    }
  return true;
}

int bsde_set_model_impl(ModelHost& m, const bsde_sigma* sg, double r, const bsde_payoff* pf,
                        const bsde_penalty* pen, std::string& err) {
  if (!sg || !pf || !pen) {
    err = "set_model: NULL argument";
    return BSDE_ERR_INVALID_ARG;
  }
  const int d = sg->d;
  if (d < 1 || d > BSDE_MAX_D) {
    err = "set_model: d out of range";
    return BSDE_ERR_INVALID_ARG;
  }
  if (sg->kind < 0 || sg->kind > 3 || (pf->kind != 0 && pf->kind != 1) ||
      (pen->obstacle != 0 && pen->obstacle != 1)) {
    err = "set_model: unknown volatility, payoff or obstacle kind";
    return BSDE_ERR_INVALID_ARG;
  }
  if (!pf->S0) {
    err = "set_model: payoff.S0 is required";
    return BSDE_ERR_INVALID_ARG;
  }
  ModelHost t;
  memset(&t, 0, sizeof(t));  // padding too: models are compared bytewise
  t.d = d;
  t.vol_kind = sg->kind;
  t.payoff = pf->kind;
  t.obstacle = pen->obstacle;
  t.T = pf->T;
  t.r = r;
  t.lambda = pen->lambda;
  t.K = pf->K;
  t.b = sg->b;
  t.s_dupire = sg->s_dupire;
  bool ok = is_fin(t.T) && t.T > 0 && is_fin(r) && is_fin(t.lambda) && t.lambda >= 0 &&
            is_fin(t.K) && is_fin(t.b) && is_fin(t.s_dupire);
  for (int j = 0; j < d; ++j) {
    t.a[j] = sg->a ? sg->a[j] : sg->a_scalar;
    t.kappa[j] = sg->kappa ? sg->kappa[j] : sg->kappa_scalar;
    t.div[j] = sg->div ? sg->div[j] : 0.0;
    t.w[j] = pf->weights ? pf->weights[j] : 1.0 / d;
    t.S0[j] = pf->S0[j];
    ok = ok && is_fin(t.a[j]) && is_fin(t.kappa[j]) && is_fin(t.div[j]) && is_fin(t.w[j]) &&
         is_fin(t.S0[j]) && t.S0[j] > 0;
  }
  if (!ok) {
    err = "set_model: a parameter is not finite or out of range";
    return BSDE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      t.C[i * d + j] = sg->corr ? sg->corr[i * d + j] : (i == j ? 1.0 : sg->rho);
  if (!cholesky_host(d, t.C, t.L)) {
    err = "set_model: correlation matrix is not positive definite";
    return BSDE_ERR_INVALID_ARG;
  }
  m = t;
  return BSDE_OK;
}

int bsde_set_grid_impl(GridHost& g, int d, int n, const double* lo, const double* hi, int resample,
                       std::string& err) {
  if (n < 1 || !lo || !hi) {
    err = "set_grid: n < 1 or NULL box";
    return BSDE_ERR_INVALID_ARG;
  }
  GridHost t;
  memset(&t, 0, sizeof(t));
  t.n = n;
  t.resample = resample ? 1 : 0;
  for (int v = 0; v <= d; ++v) {
    if (!(is_fin(lo[v]) && is_fin(hi[v]) && hi[v] > lo[v])) {
      err = "set_grid: box needs finite lo < hi in every variate";
      return BSDE_ERR_INVALID_ARG;
    }
    t.lo[v] = lo[v];
    t.hi[v] = hi[v];
  }
  g = t;
  return BSDE_OK;
}

Problem::~Problem() {
  destroy_graph();
  for (auto e : events) cudaEventDestroy(e);
}

void Problem::destroy_graph() {
  if (gexec) cudaGraphExecDestroy(gexec);
  gexec = nullptr;
  graph_key.clear();
}

void Problem::ensure_events(int count) {
  while ((int)events.size() < count) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) break;
    events.push_back(e);
  }
}

// launch shape of the path kernel: threads per CTA and paths per thread,
// limited by the shared memory of the per-thread Chebyshev tables
int Problem::choose_launch(int d, int p, int eta, int N, int M, bool mx, bool dense, int& tpb,
                           int& ppt) {
  tpb = mx ? 128 : 64;
  while (tpb > 32 && paths_smem_bytes(d, p, eta, N, tpb, mx, dense) > 220 * 1024) tpb >>= 1;
  if (paths_smem_bytes(d, p, eta, N, tpb, mx, dense) > 220 * 1024) return BSDE_ERR_INVALID_ARG;
  // about 512 paths per CTA, fewer for small M
  ppt = 4;
  while (ppt > 1 && (long long)tpb * ppt > 2LL * M) ppt >>= 1;
  return BSDE_OK;
}

int Problem::fact_group(int p, int K_it, bool resample, bool qr) {
  if (qr || !resample) return 1;
  const size_t per = fact_block_bytes(p, 1);
  const size_t cap = (size_t)256 << 20;
  int g = per > 0 ? (int)(cap / per) : K_it;
  if (g < 1) g = 1;
  return g < K_it ? g : K_it;
}

// A and A^{-1} (p x p each), dinv and the original diagonal (p each), per slot
size_t Problem::fact_block_bytes(int p, int nfact) {
  return (size_t)nfact * ((size_t)2 * p * p + (size_t)2 * p) * 8 + 256;
}

size_t Problem::estimate_bytes(int d, int n, int p, int M, int N, bool mx, int tpb, int ppt, int pm,
                               int conv_nnz, bool qr, int nfact, int splits) {
  (void)N;
  const int n_pad = (n + 31) / 32 * 32;
  const int p_pad = (p + 127) / 128 * 128;
  const int chunks = (M + tpb * ppt - 1) / (tpb * ppt);
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
  add((size_t)n * 8);
  add((size_t)d * n * 8);
  add((size_t)p * n_pad * 8);
  if (mx) {
    add((size_t)p_pad * n_pad * 4);
    add((size_t)p_pad * n_pad * 4);
    add(gram_tc_part_bytes(p_pad, n_pad, gram_tc_splits(p_pad, n_pad, splits)));
  }
  add((size_t)n * chunks * 8);
  add((size_t)n * 8);
  add((size_t)p * 8 * 4);
  add((size_t)(n > p ? n : p) * 8);
  add((size_t)p * 8);
  add((size_t)p * 4);
  add((size_t)p * 8);
  add((size_t)p);
  add(64);
  add((OUT_SIZE + 1 + 2 * BSDE_DMAX) * 8);
  if (pm > 0) {
    add((size_t)pm * 8);
    add((size_t)pm * 4);
    add((size_t)(pm + 1) * 4);
    add((size_t)conv_nnz * 4);
    add((size_t)conv_nnz * 8);
  }
  if (qr) {
    add((size_t)p * n_pad * 8);
    add((size_t)n * 8);
    add((size_t)p * 8 * 2);
    add((size_t)p * 4 + 16);
  }
  return b + fact_block_bytes(p, nfact);
}

int Problem::prepare(const bsde_solve_params& prm, Allocator& al, size_t budget, cudaStream_t st) {
  if (!has_model || !has_grid) {
    err = "solve: set_model and set_grid must come first";
    return BSDE_ERR_STATE;
  }
  const int d = model.d;
  if (prm.M < 1 || prm.N_steps < 1 || prm.eta < 0 || prm.eta > 15 || !(prm.q > 0.0) ||
      prm.q > 1.0 || prm.K_it < 1 || prm.K_it > BSDE_MAX_IT || prm.k_start < 0 ||
      prm.k_start + prm.K_it >= (1 << 24)) {
    err = "solve: parameter out of range (M, N_steps >= 1; 0 <= eta <= 15; 0 < q <= 1; "
          "1 <= K_it <= 64)";
    return BSDE_ERR_INVALID_ARG;
  }
  if (!paths_supported_d(d)) {
    err = "solve: the path kernel is compiled for d = 1..10";
    return BSDE_ERR_INVALID_ARG;
  }
  // basis (cached per (d, eta, q))
  const auto nu_new = build_multi_indices(d + 1, prm.eta, prm.q);
  if (nu_new != nus) {
    nus = nu_new;
    int mdeg = 0;
    if (!pack_multi_indices(nus, pairs, nnz, mdeg)) {
      err = "solve: basis needs more than 8 active variates or a degree above 15";
      nus.clear();
      return BSDE_ERR_INVALID_ARG;
    }
    eta_used = mdeg;
    coeffs_valid = false;
    // monomial (dense) evaluation: Horner loops for total degree <= 3 (any
    // d) or 4 (d <= 5); with FP32 paths, the prefix-tree recursion for
    // degree 4 (d <= 10) and degrees 5 and 6 (d <= 5); beyond that the
    // per-thread Chebyshev tables
    int deg_max = 0;
    for (const auto& nu : nus) {
      int deg = 0;
      for (int e : nu) deg += e;
      deg_max = deg > deg_max ? deg : deg_max;
    }
    tree_deg = 0;
    if (deg_max <= 3 || (deg_max == 4 && d <= 5)) {
      pm = build_cheb_to_mono(nus, d + 1, 4, conv_row, conv_l, conv_c, mono_deg);
    } else if (mixed && ((deg_max == 4 && d <= 10) || (deg_max <= 6 && d <= 5))) {
      pm = build_cheb_to_mono_tree(nus, d + 1, conv_row, conv_l, conv_c, mono_deg);
      tree_deg = pm > 0 ? mono_deg : 0;
    } else {
      pm = -1;
    }
    if (pm < 0) pm = 0;
  }
  const int p = (int)nus.size();
  const int n = grid.n;
  if (!prm.allow_underdetermined && 2 * p > n) {
    std::ostringstream os;
    os << "solve: basis size p = " << p << " exceeds n/2 = " << n / 2;
    err = os.str();
    return BSDE_ERR_ILLPOSED;
  }
  Shape s;
  s.d = d;
  s.n = n;
  s.n_pad = (n + 31) / 32 * 32;
  s.p = p;
  s.p_pad = (p + 127) / 128 * 128;
  s.eta = eta_used < 1 ? 1 : eta_used;
  s.M = prm.M;
  s.N = prm.N_steps;
  s.mixed = mixed;
  if (prm.eval_mode == 2 && pm == 0) {
    err = "solve: eval_mode 2 (dense) needs a basis of total degree <= 3, <= 4 (d <= 5; with "
          "FP32 paths d <= 10) or, with FP32 paths, <= 6 (d <= 5)";
    return BSDE_ERR_INVALID_ARG;
  }
  // the dense evaluation needs a constant correlation (all off-diagonal
  // entries equal)
  bool const_corr = true;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (i != j && model.C[i * d + j] != model.C[1]) const_corr = false;
  if (prm.eval_mode == 2 && !const_corr) {
    err = "solve: eval_mode 2 (dense) needs a constant correlation";
    return BSDE_ERR_INVALID_ARG;
  }
  s.dense = pm > 0 && const_corr && prm.eval_mode != 1;
  s.dense4 = s.dense && tree_deg == 0 && mono_deg == 4;
  s.tree = s.dense ? tree_deg : 0;
  if (prm.ls_mode != 0 && prm.ls_mode != 1) {
    err = "solve: ls_mode must be 0 (normal equations) or 1 (pivoted QR)";
    return BSDE_ERR_INVALID_ARG;
  }
  s.qr = prm.ls_mode == 1;
  s.pm = s.dense ? pm : 0;
  if (choose_launch(d, s.dense ? pm : p, s.eta, s.N, s.M, mixed, s.dense, s.tpb, s.ppt) != BSDE_OK) {
    err = "solve: basis and step count too large for the shared-memory tables";
    return BSDE_ERR_INVALID_ARG;
  }
  // the large tree evaluations (d >= 6): 8 warps enter each evaluation
  // together (measured at d = 10, degree 4: 6.8 ms against 7.4 ms with 4)
  if (s.tree && d >= 6 && s.M >= 512) {
    s.tpb = 256;
    s.ppt = 2;
  }
  if (prm.paths_tpb) {
    if (prm.paths_tpb < 32 || prm.paths_tpb > 256 || prm.paths_tpb % 32 ||
        paths_smem_bytes(d, s.dense ? pm : p, s.eta, s.N, prm.paths_tpb, mixed, s.dense) > 220 * 1024) {
      err = "solve: paths_tpb must be a multiple of 32 in 32..256 within the shared memory";
      return BSDE_ERR_INVALID_ARG;
    }
    s.tpb = prm.paths_tpb;
  }
  if (prm.paths_ppt) {
    if (prm.paths_ppt < 1 || prm.paths_ppt > 16) {
      err = "solve: paths_ppt must be in 1..16";
      return BSDE_ERR_INVALID_ARG;
    }
    s.ppt = prm.paths_ppt;
  }
  s.chunks = (s.M + s.tpb * s.ppt - 1) / (s.tpb * s.ppt);
  if (prm.gram_splits < 0 || prm.gram_splits > 4096) {
    err = "solve: gram_splits must be in 0..4096";
    return BSDE_ERR_INVALID_ARG;
  }
  s.splits = mixed ? gram_tc_splits(s.p_pad, s.n_pad, prm.gram_splits) : 0;
  const int nf = fact_group(p, prm.K_it, grid.resample != 0, s.qr);
  {
    const size_t total = estimate_bytes(d, n, p, s.M, s.N, mixed, s.tpb, s.ppt, s.pm,
                                        s.dense ? (int)conv_l.size() : 0, s.qr, nf, s.splits);
    if (budget && total > budget) {
      std::ostringstream os;
      os << "solve: needs " << total << " bytes of device memory, budget " << budget;
      err = os.str();
      return BSDE_ERR_NOMEM;
    }
  }
  if (!block || !(s == alloc_shape)) {
    const size_t need = estimate_bytes(d, n, p, s.M, s.N, mixed, s.tpb, s.ppt, s.pm,
                                       s.dense ? (int)conv_l.size() : 0, s.qr, 0, s.splits);
    destroy_graph();
    if (block) al.put(block, st);
    block = nullptr;
    block_bytes = 0;
    void* b = al.get(need, st);
    if (!b) {
      release(al, st);  // a failed call leaves the context holding no device memory
      err = "solve: device allocation failed";
      return BSDE_ERR_NOMEM;
    }
    block = b;
    block_bytes = need;
    alloc_shape = s;
    if (cudaMemsetAsync(block, 0, need, st) != cudaSuccess) {
      err = "solve: cudaMemsetAsync failed";
      return BSDE_ERR_CUDA;
    }
    char* c = (char*)block;
    auto take = [&](size_t x) {
      char* r = c;
      c += (x + 255) / 256 * 256;
      return (void*)r;
    };
    ProblemDev P;
    P.n = n;
    P.n_pad = s.n_pad;
    P.p = p;
    P.p_pad = s.p_pad;
    P.eta = s.eta;
    P.chunks = s.chunks;
    P.t = (double*)take((size_t)n * 8);
    P.x = (double*)take((size_t)d * n * 8);
    P.B = (double*)take((size_t)p * s.n_pad * 8);
    if (mixed) {
      P.Bhi = (float*)take((size_t)s.p_pad * s.n_pad * 4);
      P.Blo = (float*)take((size_t)s.p_pad * s.n_pad * 4);
      P.gram_splits = s.splits;
      P.gram_part = (float*)take(gram_tc_part_bytes(s.p_pad, s.n_pad, s.splits));
    }
    P.partial = (double*)take((size_t)n * s.chunks * 8);
    P.c = (double*)take((size_t)n * 8);
    c_own = P.c;
    P.rhs = (double*)take((size_t)p * 8 * 4);
    P.delta = P.rhs + p;
    P.res = P.rhs + 2 * p;
    P.v = (double*)take((size_t)(n > p ? n : p) * 8);
    P.alpha = (double*)take((size_t)p * 8);
    P.alpha32 = (float*)take((size_t)p * 4);
    P.pairs = (uint2*)take((size_t)p * 8);
    P.nnz = (uint8_t*)take((size_t)p);
    P.key = (uint32_t*)take(64);
    P.status = (int*)(P.key + 4);
    P.out = (double*)take((OUT_SIZE + 1 + 2 * BSDE_DMAX) * 8);
    if (s.dense) {
      P.dense = true;
      P.dense4 = s.dense4;
      P.tree = s.tree;
      P.pm = s.pm;
      P.beta = (double*)take((size_t)s.pm * 8);
      P.beta32 = (float*)take((size_t)s.pm * 4);
      P.conv_row = (int*)take((size_t)(s.pm + 1) * 4);
      P.conv_l = (int*)take(conv_l.size() * 4);
      P.conv_c = (double*)take(conv_c.size() * 8);
    }
    if (s.qr) {
      P.qr_W = (double*)take((size_t)p * s.n_pad * 8);
      P.qr_y = (double*)take((size_t)n * 8);
      P.qr_nrm = (double*)take((size_t)p * 8 * 2);
      P.qr_tau = P.qr_nrm + p;
      P.qr_perm = (int*)take((size_t)p * 4 + 16);
      P.qr_rank = P.qr_perm + p;
    }
    dev = P;
    coeffs_valid = false;
    nfact = 0;  // the factor block is laid out for p again below
  }
  // factor block: kept across solves (and across reallocations of the main
  // block, which do not touch it) while it is large enough
  const size_t fneed = fact_block_bytes(p, nf);
  if (!fact || fact_bytes < fneed || nfact != nf || dev.A == nullptr) {
    if (!fact || fact_bytes < fneed) {
      destroy_graph();
      if (fact) al.put(fact, st);
      fact = al.get(fneed, st);
      fact_bytes = fact ? fneed : 0;
      if (!fact) {
        release(al, st);
        err = "solve: device allocation failed (Gram factors)";
        return BSDE_ERR_NOMEM;
      }
    }
    double* f = (double*)fact;
    const size_t pp = (size_t)p * p;
    dev.A = f;
    dev.Ainv = f + (size_t)nf * pp;
    dev.dinv = f + (size_t)2 * nf * pp;
    dev.diag0 = dev.dinv + (size_t)nf * p;
    nfact = nf;
  }
  shape = s;
  dev.chunks = s.chunks;
  // point sharding: this rank's block, and the corrections in the caller's
  // exchange buffer
  dev.c = c_own;
  dev.shard_i0 = 0;
  dev.shard_n = 0;
  if (sh_n > 1) {
    const int nb = (n + sh_n - 1) / sh_n;
    const size_t need_len = (size_t)nb * sh_n * (sh_peer ? 2 : 1);
    if (!sh_buf || sh_len < need_len) {
      err = sh_peer ? "solve: the peer exchange buffers hold fewer than 2 * nranks * ceil(n / nranks) values"
                    : "solve: the shard exchange buffer holds fewer than nranks * ceil(n / nranks) values";
      return BSDE_ERR_INVALID_ARG;
    }
    int i0, i1;
    shard_block(n, sh_rank, sh_n, i0, i1);
    dev.c = sh_buf;
    dev.shard_i0 = i0;
    dev.shard_n = i1 - i0;
  }
  // tables, read-out point, key
  cudaError_t e = cudaMemcpyAsync(dev.pairs, pairs.data(), (size_t)p * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev.nnz, nnz.data(), (size_t)p, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && dev.dense) {
    e = cudaMemcpyAsync(dev.conv_row, conv_row.data(), conv_row.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dev.conv_l, conv_l.data(), conv_l.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dev.conv_c, conv_c.data(), conv_c.size() * 8, cudaMemcpyHostToDevice, st);
  }
  double logS0[BSDE_DMAX];
  for (int j = 0; j < d; ++j) logS0[j] = std::log(model.S0[j]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev.out + OUT_SIZE + 1 + BSDE_DMAX, logS0, (size_t)d * 8,
                        cudaMemcpyHostToDevice, st);
  uint32_t key[2] = {(uint32_t)(prm.seed & 0xffffffffu), (uint32_t)(prm.seed >> 32)};
  dev.seed_key[0] = key[0];
  dev.seed_key[1] = key[1];
  if (e == cudaSuccess) e = cudaMemcpyAsync(dev.key, key, 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev.status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // key/logS0 live on this stack
  if (e != cudaSuccess) {
    err = std::string("solve: upload failed: ") + cudaGetErrorString(e);
    return BSDE_ERR_CUDA;
  }
  return BSDE_OK;
}

// event record that also works inside stream capture (an external event
// node of the graph, so that elapsed times can be read after a replay)
static void record(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  cudaEventRecordWithFlags(e, st,
                           cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// The Gram matrix of iteration k depends only on the points of iteration k,
// which depend only on (seed, k): the matrices of a group of iterations are
// built and factorised together before the group's path kernels, batched
// over the group (blockIdx.y of the factorisation kernels).  The path kernel
// then runs alone on the device, and the refit after it is a product with
// the stored inverse plus FP64 refinement.
int Problem::enqueue_factors(int k0, int nb, cudaStream_t st) {
  const size_t pp = (size_t)shape.p * shape.p;
  for (int j = 0; j < nb; ++j) {
    const uint32_t kp = grid.resample ? (uint32_t)(k0 + j) : 0u;
    launch_points(model, grid, dev, kp, st);
    launch_basis(model, grid, dev, mixed, st);
    ProblemDev Pj = dev;
    Pj.A = dev.A + (size_t)j * pp;
    if (mixed) {
      const cudaError_t e = launch_gram_tc(Pj, st);
      if (e != cudaSuccess) {
        err = std::string("tensor-core Gram launch failed: ") + cudaGetErrorString(e);
        return BSDE_ERR_CUDA;
      }
    } else {
      launch_gram_f64(Pj, st);
    }
  }
  launch_cholesky(dev, nb, st);
  launch_inverse(dev, nb, st);
  return BSDE_OK;
}

int Problem::enqueue_gram(int k, cudaStream_t st) {
  if (nfact < 1 || dev.A == nullptr) {
    err = "gram: no factor block";
    return BSDE_ERR_STATE;
  }
  launch_points(model, grid, dev, grid.resample ? (uint32_t)k : 0u, st);
  launch_basis(model, grid, dev, mixed, st);
  if (mixed) {
    const cudaError_t e = launch_gram_tc(dev, st);
    if (e != cudaSuccess) {
      err = std::string("tensor-core Gram launch failed: ") + cudaGetErrorString(e);
      return BSDE_ERR_CUDA;
    }
  } else {
    launch_gram_f64(dev, st);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("gram: kernel launch failed: ") + cudaGetErrorString(e);
    return BSDE_ERR_CUDA;
  }
  return BSDE_OK;
}

int Problem::enqueue_iteration(const bsde_solve_params& prm, int k, cudaStream_t st,
                               cudaEvent_t* ev, int slot) {
  const bool rec = ev != nullptr;
  // peer exchange: this iteration's corrections live in the half of the
  // buffers that belongs to its exchange number
  const uint32_t epoch = sh_epoch + 1;
  size_t region_off = 0;
  if (sh_n > 1 && sh_peer) {
    region_off = (size_t)(epoch & 1u) * (size_t)sh_n * (size_t)((shape.n + sh_n - 1) / sh_n);
    dev.c = sh_buf + region_off;
  }
  const uint32_t kp = grid.resample ? (uint32_t)k : 0u;
  launch_points(model, grid, dev, kp, st);
  launch_basis(model, grid, dev, false, st);  // FP64 B for the refit (no TF32 split)
  if (dev.dense) launch_cheb2mono(dev, st);
  if (rec) record(ev[0], st);
  cudaError_t e = launch_paths(model, grid, dev, shape.M, shape.N, (uint32_t)k, mixed, shape.tpb,
                               shape.ppt, st);
  if (e != cudaSuccess) {
    err = std::string("path kernel launch failed: ") + cudaGetErrorString(e);
    return BSDE_ERR_CUDA;
  }
  if (rec) record(ev[1], st);
  launch_reduce_c(dev, shape.M, st);
  if (sh_n > 1) {
    // every rank's block of corrections into the exchange buffer
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      err = std::string("kernel launch failed: ") + cudaGetErrorString(e);
      return BSDE_ERR_CUDA;
    }
    const int nb = (shape.n + sh_n - 1) / sh_n;
    if (sh_peer) {
      e = launch_exchange_peers(dev.c, dev.shard_i0, dev.shard_n, sh_rank, sh_n, sh_pp, region_off,
                                epoch, st);
      if (e != cudaSuccess) {
        err = std::string("exchange launch failed: ") + cudaGetErrorString(e);
        return BSDE_ERR_CUDA;
      }
      if (sh_fn) {
        const int rc = sh_fn(dev.c, nb, sh_rank, sh_n, (void*)st, sh_user);
        if (rc != 0) {
          err = "solve: the exchange hook failed (status " + std::to_string(rc) + ")";
          return BSDE_ERR_EXCHANGE;
        }
      }
      e = launch_exchange_wait(sh_pp.flag[sh_rank], sh_rank, sh_n, epoch, sh_wait_ms, dev.status, st);
      if (e != cudaSuccess) {
        err = std::string("exchange launch failed: ") + cudaGetErrorString(e);
        return BSDE_ERR_CUDA;
      }
      sh_epoch = epoch;
    } else {
      const int rc = sh_fn(sh_buf, nb, sh_rank, sh_n, (void*)st, sh_user);
      if (rc != 0) {
        err = "solve: the exchange hook failed (status " + std::to_string(rc) + ")";
        return BSDE_ERR_EXCHANGE;
      }
    }
  }
  if (rec) record(ev[2], st);
  if (shape.qr) {
    // refit by pivoted QR on the design matrix (FP64)
    if (rec) record(ev[3], st);
    if (rec) record(ev[6], st);
    if (rec) record(ev[7], st);
    if (rec) record(ev[4], st);
    launch_qr_solve(dev, st);
  } else {
    ProblemDev Ps = dev;
    Ps.Ainv = dev.Ainv + (size_t)slot * shape.p * shape.p;
    launch_rhs(dev, st);
    if (rec) record(ev[4], st);
    launch_inv_gemv(Ps, dev.rhs, dev.delta, 0, st);
    const int refine = prm.refine_steps >= 0 ? prm.refine_steps : (mixed ? 2 : 1);
    for (int r = 0; r < refine; ++r) {
      launch_refine_residual(dev, st);
      launch_inv_gemv(Ps, dev.res, dev.delta, 1, st);
    }
  }
  if (rec) record(ev[5], st);
  launch_update(dev, k - prm.k_start, st);
  launch_eval_x0(model, grid, dev, k - prm.k_start, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("kernel launch failed: ") + cudaGetErrorString(e);
    return BSDE_ERR_CUDA;
  }
  return BSDE_OK;
}

int Problem::enqueue_block(const bsde_solve_params& prm, int k0, int count, cudaStream_t st,
                           cudaEvent_t* ev) {
  if (!shape.qr && nfact < 1) {
    err = "solve: no factor block";
    return BSDE_ERR_STATE;
  }
  int it = 0;
  while (it < count) {
    // a group of iterations whose Gram inverses are built first (with fixed
    // points: one inverse, built once, serves every iteration)
    const int g = (shape.qr || !grid.resample) ? count - it
                                               : (nfact < count - it ? nfact : count - it);
    for (int j = 0; j < g; ++j) {
      cudaEvent_t* e = ev ? ev + 8 * (it + j) : nullptr;
      // Gram + factorisation time: events 3 and 7 of the group's first
      // iteration (zero for the others); the QR refit records its own
      if (!shape.qr && e) record(e[3], st);
      if (!shape.qr && j == 0 && (grid.resample || it == 0)) {
        const int rc = enqueue_factors(k0 + it, grid.resample ? g : 1, st);
        if (rc != BSDE_OK) return rc;
      }
      if (!shape.qr && e) {
        record(e[6], st);
        record(e[7], st);
      }
      const int rc = enqueue_iteration(prm, k0 + it + j, st, e, grid.resample ? j : 0);
      if (rc != BSDE_OK) return rc;
    }
    it += g;
  }
  return BSDE_OK;
}

int Problem::enqueue_solve(const bsde_solve_params& prm, cudaStream_t st) {
  const int nev = prm.timing ? 8 * prm.K_it : 0;
  if (nev) ensure_events(nev);
  return enqueue_block(prm, prm.k_start, prm.K_it, st,
                       nev && (int)events.size() >= nev ? events.data() : nullptr);
}

int Problem::start(const bsde_solve_params& prm, Allocator& al, size_t budget, cudaStream_t st,
                   cudaEvent_t e0, cudaEvent_t e1) {
  int rc = prepare(prm, al, budget, st);
  if (rc != BSDE_OK) return rc;
  if (prm.k_start == 0) {
    if (cudaMemsetAsync(dev.alpha, 0, (size_t)shape.p * 8, st) != cudaSuccess ||
        cudaMemsetAsync(dev.alpha32, 0, (size_t)shape.p * 4, st) != cudaSuccess) {
      err = "solve: reset of the coefficients failed";
      return BSDE_ERR_CUDA;
    }
  } else if (!coeffs_valid) {
    err = "solve: k_start > 0 needs coefficients from bsde_set_coeffs or an earlier solve";
    return BSDE_ERR_STATE;
  }
  cudaMemsetAsync(dev.out + OUT_PRICE_IT, 0, 3 * 64 * 8, st);
  if (prm.use_graph && sh_n == 1) {
    std::ostringstream os;
    os << shape.d << ' ' << shape.n << ' ' << shape.p << ' ' << shape.M << ' ' << shape.N << ' '
       << prm.K_it << ' ' << prm.k_start << ' ' << prm.refine_steps << ' ' << prm.timing << ' '
       << mixed << ' ' << (void*)block << ' ' << prm.seed << ' ' << prm.eval_mode << ' '
       << prm.paths_tpb << ' ' << prm.paths_ppt << ' ' << prm.ls_mode << ' ' << fact << ' ' << nfact
       << ' ' << shape.splits;
    if (!gexec || os.str() != graph_key) {
      destroy_graph();
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        err = std::string("solve: stream capture failed: ") + cudaGetErrorString(e);
        return BSDE_ERR_CUDA;
      }
      rc = enqueue_solve(prm, st);
      e = cudaStreamEndCapture(st, &graph);
      if (rc == BSDE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (rc != BSDE_OK || e != cudaSuccess) {
        if (rc == BSDE_OK) err = std::string("solve: graph capture failed: ") + cudaGetErrorString(e);
        gexec = nullptr;
        cudaGetLastError();
        return rc != BSDE_OK ? rc : BSDE_ERR_CUDA;
      }
      graph_key = os.str();
    }
    cudaEventRecord(e0, st);
    cudaError_t e = cudaGraphLaunch(gexec, st);
    cudaEventRecord(e1, st);
    if (e != cudaSuccess) {
      err = std::string("solve: graph launch failed: ") + cudaGetErrorString(e);
      return BSDE_ERR_CUDA;
    }
  } else {
    cudaEventRecord(e0, st);
    rc = enqueue_solve(prm, st);
    cudaEventRecord(e1, st);
    if (rc != BSDE_OK) return rc;
  }
  return BSDE_OK;
}

int Problem::complete(const bsde_solve_params& prm, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                      bsde_report* rep) {
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) {
    err = std::string("solve: device error: ") + cudaGetErrorString(e);
    return BSDE_ERR_CUDA;
  }
  coeffs_valid = true;
  return finish_report(prm, st, rep, ms);
}

int Problem::solve(const bsde_solve_params& prm, Allocator& al, size_t budget, cudaStream_t st,
                   bsde_report* rep) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return BSDE_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BSDE_ERR_CUDA;
  }
  int rc = start(prm, al, budget, st, e0, e1);
  if (rc == BSDE_OK) rc = complete(prm, st, e0, e1, rep);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

int Problem::finish_report(const bsde_solve_params& prm, cudaStream_t st, bsde_report* rep,
                           float ms_total) {
  std::vector<double> out(OUT_SIZE);
  int status = 0, rank = shape.p;
  cudaError_t e = cudaMemcpyAsync(out.data(), dev.out, OUT_SIZE * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, dev.status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && shape.qr)
    e = cudaMemcpyAsync(&rank, dev.qr_rank, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    err = std::string("solve: report copy failed: ") + cudaGetErrorString(e);
    return BSDE_ERR_CUDA;
  }
  int rc = BSDE_OK;
  if (status & ST_NOT_PD) {
    err = "solve: the Gram matrix is not positive definite (Cholesky pivot <= 0)";
    rc = BSDE_ERR_NOT_PD;
  } else if (status & ST_TIMEOUT) {
    err = "solve: a bounded device wait gave up";
    rc = BSDE_ERR_TIMEOUT;
  }
  if (rep) {
    bsde_report r;
    memset(&r, 0, sizeof(r));
    r.status = rc;
    r.d = model.d;
    r.p = shape.p;
    r.K_it = prm.K_it;
    r.price = out[OUT_PRICE];
    for (int j = 0; j < model.d; ++j) {
      r.dudx[j] = out[OUT_DUDX + j];
      r.delta[j] = out[OUT_DUDX + j] / model.S0[j];
    }
    for (int k = 0; k < prm.K_it && k < BSDE_MAX_IT; ++k) {
      r.price_iter[k] = out[OUT_PRICE_IT + k];
      r.resid_l2[k] = out[OUT_RES2 + k];
      r.resid_linf[k] = out[OUT_RESI + k];
    }
    r.ms_total = ms_total;
    r.path_steps = (double)prm.K_it * shape.n * (double)shape.M * shape.N;
    r.path_steps_per_s = ms_total > 0 ? r.path_steps / (ms_total * 1e-3) : 0.0;
    r.path_launches = prm.K_it;
    r.rank = rank;
    // launches: per iteration points, basis, (monomial conversion), paths,
    // reduce, refit (QR: init, pivot + apply per step, solve; otherwise
    // rhs, inverse product, 3 per refinement step), update, read-out (3);
    // per factorised Gram matrix points, basis, Gram (+ split-K reduce in
    // mixed precision); per group save_diag, 3 per panel but the last
    // (diag, trsm, update), the last panel's diag, the batched inverse
    const int panels = (shape.p + 31) / 32;
    const int steps_qr = shape.p < shape.n ? shape.p : shape.n;
    const int refine2 = prm.refine_steps >= 0 ? prm.refine_steps : (mixed ? 2 : 1);
    const int refit = shape.qr ? (2 + 2 * steps_qr) : (2 + 3 * refine2);
    int groups = 0, mats = 0;
    if (!shape.qr) {
      groups = grid.resample ? (prm.K_it + nfact - 1) / nfact : 1;
      mats = grid.resample ? prm.K_it : 1;
    }
    r.kernel_launches = prm.K_it * (2 + (dev.dense ? 1 : 0) + 1 + 1 + refit + 1 + 3) +
                        mats * (2 + (mixed ? 2 : 1)) + groups * (3 * panels - 1 + 1);
    if (prm.timing && (int)events.size() >= 8 * prm.K_it) {
      // paths: ev0..ev1; Gram matrices, factors and inverses built ahead of
      // a group of iterations: ev3..ev7 of the group's first iteration;
      // refit after the paths: ev4..ev5
      double mp = 0, mg = 0, msv = 0;
      for (int k = 0; k < prm.K_it; ++k) {
        cudaEvent_t* e = &events[8 * k];
        float a = 0, b = 0, c = 0;
        if (cudaEventElapsedTime(&a, e[0], e[1]) == cudaSuccess) mp += a;
        if (cudaEventElapsedTime(&b, e[3], e[7]) == cudaSuccess) mg += b;
        if (cudaEventElapsedTime(&c, e[4], e[5]) == cudaSuccess) msv += c;
      }
      cudaGetLastError();
      r.ms_paths = mp;
      r.ms_gram = mg;
      r.ms_solve = msv;
    }
    *rep = r;
  }
  return rc;
}

void Problem::release(Allocator& al, cudaStream_t st) {
  destroy_graph();
  if (block) al.put(block, st);
  block = nullptr;
  c_own = nullptr;
  block_bytes = 0;
  if (fact) al.put(fact, st);
  fact = nullptr;
  fact_bytes = 0;
  nfact = 0;
  dev = ProblemDev();
  alloc_shape = Shape();
  coeffs_valid = false;
}
