// api.cu -- the C ABI of include/bsde.h on top of the runtime (runtime.h).
#include <cstring>
#include <exception>
#include <string>

#include "multiindex.h"
#include "runtime.h"

struct bsde_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Allocator al;
  size_t budget = 0;
  Problem prob;
  std::string err;
};

namespace {
thread_local std::string g_create_err;

int fail(bsde_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

bool set_device(bsde_ctx* c) { return cudaSetDevice(c->device) == cudaSuccess; }

#define API_GUARD(ctx, ...)                                   \
  try {                                                       \
    __VA_ARGS__                                               \
  } catch (const std::exception& ex) {                        \
    return fail(ctx, BSDE_ERR_INVALID_ARG, ex.what());        \
  } catch (...) {                                             \
    return fail(ctx, BSDE_ERR_INVALID_ARG, "unknown error");  \
  }
}  // namespace

extern "C" {

int bsde_create(bsde_ctx** out, const bsde_create_opts* o) {
  try {
    if (!out || !o) {
      g_create_err = "bsde_create: NULL argument";
      return BSDE_ERR_INVALID_ARG;
    }
    if (o->precision != BSDE_PREC_FP64 && o->precision != BSDE_PREC_MIXED) {
      g_create_err = "bsde_create: unknown precision";
      return BSDE_ERR_INVALID_ARG;
    }
    if ((o->alloc == nullptr) != (o->free == nullptr)) {
      g_create_err = "bsde_create: alloc and free hooks go together";
      return BSDE_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || o->device < 0 || o->device >= ndev) {
      cudaGetLastError();
      g_create_err = "bsde_create: no such CUDA device";
      return BSDE_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, o->device) != cudaSuccess || prop.major != 10 ||
        prop.minor != 3) {
      g_create_err = "bsde_create: the kernels are built for sm_103a (GB300)";
      return BSDE_ERR_CUDA;
    }
    bsde_ctx* c = new bsde_ctx();
    c->device = o->device;
    c->al.alloc = o->alloc;
    c->al.free = o->free;
    c->al.user = o->alloc_user;
    c->budget = o->mem_budget;
    c->prob.mixed = (o->precision == BSDE_PREC_MIXED);
    cudaSetDevice(c->device);
    if (o->stream) {
      c->stream = (cudaStream_t)o->stream;
    } else {
      if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        g_create_err = "bsde_create: cudaStreamCreate failed";
        return BSDE_ERR_CUDA;
      }
      c->own_stream = true;
    }
    *out = c;
    return BSDE_OK;
  } catch (...) {
    g_create_err = "bsde_create: out of host memory";
    return BSDE_ERR_NOMEM;
  }
}

void bsde_destroy(bsde_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  c->prob.release(c->al, c->stream);
  cudaStreamSynchronize(c->stream);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* bsde_last_error(const bsde_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

int bsde_set_model(bsde_ctx* c, const bsde_sigma* sigma, double r, const bsde_payoff* payoff,
                   const bsde_penalty* penalty) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  API_GUARD(c, {
    ModelHost m;
    const int rc = bsde_set_model_impl(m, sigma, r, payoff, penalty, c->err);
    if (rc != BSDE_OK) return rc;
    if (c->prob.has_grid && c->prob.model.d != m.d) c->prob.has_grid = false;
    // the captured graph bakes the model into its kernel arguments
    if (!c->prob.has_model || memcmp(&c->prob.model, &m, sizeof(m)) != 0) c->prob.destroy_graph();
    c->prob.model = m;
    c->prob.has_model = true;
    return BSDE_OK;
  })
}

int bsde_set_grid(bsde_ctx* c, int n, const double* lo, const double* hi, int resample) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  API_GUARD(c, {
    if (!c->prob.has_model) return fail(c, BSDE_ERR_STATE, "set_grid: set_model must come first");
    GridHost g;
    const int rc = bsde_set_grid_impl(g, c->prob.model.d, n, lo, hi, resample, c->err);
    if (rc != BSDE_OK) return rc;
    if (!c->prob.has_grid || memcmp(&c->prob.grid, &g, sizeof(g)) != 0) c->prob.destroy_graph();
    c->prob.grid = g;
    c->prob.has_grid = true;
    return BSDE_OK;
  })
}

int bsde_solve(bsde_ctx* c, const bsde_solve_params* prm, bsde_report* rep) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (!prm) return fail(c, BSDE_ERR_INVALID_ARG, "solve: NULL params");
  API_GUARD(c, {
    if (!set_device(c)) return fail(c, BSDE_ERR_CUDA, "solve: cudaSetDevice failed");
    const int rc = c->prob.solve(*prm, c->al, c->budget, c->stream, rep);
    if (rc != BSDE_OK) {
      c->err = c->prob.err;
      if (rep) rep->status = rc;
    }
    return rc;
  })
}

int bsde_iterate(bsde_ctx* c, const bsde_solve_params* prm, int k, const double* alpha_in,
                 double* t_out, double* x_out, double* c_out, double* alpha_out) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (!prm || k < 0 || k >= (1 << 24)) return fail(c, BSDE_ERR_INVALID_ARG, "iterate: bad arguments");
  API_GUARD(c, {
    if (!set_device(c)) return fail(c, BSDE_ERR_CUDA, "iterate: cudaSetDevice failed");
    bsde_solve_params p1 = *prm;
    p1.K_it = 1;
    p1.k_start = k;
    Problem& P = c->prob;
    int rc = P.prepare(p1, c->al, c->budget, c->stream);
    if (rc != BSDE_OK) return fail(c, rc, P.err);
    const int p = P.shape.p, n = P.shape.n, d = P.model.d;
    if (alpha_in) {
      std::vector<float> a32(p);
      for (int l = 0; l < p; ++l) a32[l] = (float)alpha_in[l];
      if (cudaMemcpyAsync(P.dev.alpha, alpha_in, (size_t)p * 8, cudaMemcpyHostToDevice, c->stream) !=
              cudaSuccess ||
          cudaMemcpyAsync(P.dev.alpha32, a32.data(), (size_t)p * 4, cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return fail(c, BSDE_ERR_CUDA, "iterate: coefficient upload failed");
    } else if (!P.coeffs_valid) {
      cudaMemsetAsync(P.dev.alpha, 0, (size_t)p * 8, c->stream);
      cudaMemsetAsync(P.dev.alpha32, 0, (size_t)p * 4, c->stream);
    }
    rc = P.enqueue_block(p1, k, 1, c->stream, nullptr);
    if (rc != BSDE_OK) return fail(c, rc, P.err);
    cudaError_t e = cudaSuccess;
    if (t_out) e = cudaMemcpyAsync(t_out, P.dev.t, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (x_out && e == cudaSuccess)
      e = cudaMemcpyAsync(x_out, P.dev.x, (size_t)n * d * 8, cudaMemcpyDeviceToHost, c->stream);
    if (c_out && e == cudaSuccess)
      e = cudaMemcpyAsync(c_out, P.dev.c, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (alpha_out && e == cudaSuccess)
      e = cudaMemcpyAsync(alpha_out, P.dev.alpha, (size_t)p * 8, cudaMemcpyDeviceToHost, c->stream);
    int status = 0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&status, P.dev.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, BSDE_ERR_CUDA, std::string("iterate: ") + cudaGetErrorString(e));
    P.coeffs_valid = true;
    if (status & ST_NOT_PD) return fail(c, BSDE_ERR_NOT_PD, "iterate: Gram matrix not positive definite");
    if (status & ST_TIMEOUT) return fail(c, BSDE_ERR_TIMEOUT, "iterate: a bounded device wait gave up");
    return BSDE_OK;
  })
}

int bsde_gram_matrix(bsde_ctx* c, const bsde_solve_params* prm, int k, double* A_out, int cap) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (!prm || !A_out || k < 0 || k >= (1 << 24))
    return fail(c, BSDE_ERR_INVALID_ARG, "gram: bad arguments");
  API_GUARD(c, {
    if (!set_device(c)) return fail(c, BSDE_ERR_CUDA, "gram: cudaSetDevice failed");
    bsde_solve_params p1 = *prm;
    p1.K_it = 1;
    p1.k_start = k;
    Problem& P = c->prob;
    int rc = P.prepare(p1, c->al, c->budget, c->stream);
    if (rc != BSDE_OK) return fail(c, rc, P.err);
    const int p = P.shape.p;
    if ((long long)cap < (long long)p * p)
      return fail(c, BSDE_ERR_INVALID_ARG, "gram: capacity below p * p");
    rc = P.enqueue_gram(k, c->stream);
    if (rc != BSDE_OK) return fail(c, rc, P.err);
    int status = 0;
    cudaError_t e =
        cudaMemcpyAsync(A_out, P.dev.A, (size_t)p * p * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&status, P.dev.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, BSDE_ERR_CUDA, std::string("gram: ") + cudaGetErrorString(e));
    if (status & ST_TIMEOUT) return fail(c, BSDE_ERR_TIMEOUT, "gram: a bounded device wait gave up");
    return BSDE_OK;
  })
}

int bsde_set_shard(bsde_ctx* c, int rank, int nranks, double* c_dev, size_t c_len,
                   bsde_exchange_fn exchange, void* user) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (nranks < 1 || rank < 0 || rank >= nranks)
    return fail(c, BSDE_ERR_INVALID_ARG, "set_shard: rank out of range");
  if (nranks > 1 && (!c_dev || !exchange))
    return fail(c, BSDE_ERR_INVALID_ARG, "set_shard: nranks > 1 needs a buffer and an exchange hook");
  Problem& P = c->prob;
  P.destroy_graph();
  P.sh_rank = nranks > 1 ? rank : 0;
  P.sh_n = nranks;
  P.sh_buf = nranks > 1 ? c_dev : nullptr;
  P.sh_len = nranks > 1 ? c_len : 0;
  P.sh_fn = nranks > 1 ? exchange : nullptr;
  P.sh_user = user;
  P.sh_peer = false;
  return BSDE_OK;
}

int bsde_set_shard_peers(bsde_ctx* c, int rank, int nranks, const bsde_peer_exchange* px) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (nranks < 1 || nranks > BSDE_MAX_RANKS || rank < 0 || rank >= nranks)
    return fail(c, BSDE_ERR_INVALID_ARG, "set_shard_peers: rank out of range");
  if (nranks == 1) return bsde_set_shard(c, 0, 1, nullptr, 0, nullptr, nullptr);
  if (!px) return fail(c, BSDE_ERR_INVALID_ARG, "set_shard_peers: NULL peer table");
  for (int q = 0; q < nranks; ++q)
    if (!px->c[q] || !px->flag[q])
      return fail(c, BSDE_ERR_INVALID_ARG, "set_shard_peers: missing buffer or counters of a rank");
  if (!(px->wait_ms >= 0.0) || px->wait_ms > 3.6e6)
    return fail(c, BSDE_ERR_INVALID_ARG, "set_shard_peers: wait_ms out of range");
  Problem& P = c->prob;
  P.destroy_graph();
  P.sh_rank = rank;
  P.sh_n = nranks;
  P.sh_buf = px->c[rank];
  P.sh_len = px->c_len;
  P.sh_fn = px->pushed;
  P.sh_user = px->user;
  P.sh_peer = true;
  P.sh_wait_ms = px->wait_ms > 0.0 ? px->wait_ms : 1000.0;
  for (int q = 0; q < BSDE_RANKS_MAX; ++q) {
    P.sh_pp.c[q] = q < nranks ? px->c[q] : nullptr;
    P.sh_pp.flag[q] = q < nranks ? px->flag[q] : nullptr;
  }
  return BSDE_OK;
}

int bsde_shard_block(int n, int rank, int nranks, int* i0, int* i1) {
  if (n < 0 || nranks < 1 || rank < 0 || rank >= nranks || !i0 || !i1) return BSDE_ERR_INVALID_ARG;
  shard_block(n, rank, nranks, *i0, *i1);
  return BSDE_OK;
}

int bsde_basis_size(int d, int eta, double q, int* p_out) {
  if (d < 1 || d > BSDE_MAX_D || eta < 0 || eta > 15 || !(q > 0.0) || q > 1.0 || !p_out)
    return BSDE_ERR_INVALID_ARG;
  try {
    *p_out = (int)build_multi_indices(d + 1, eta, q).size();
    return BSDE_OK;
  } catch (...) {
    return BSDE_ERR_NOMEM;
  }
}

int bsde_basis_indices(int d, int eta, double q, int* nu_out, int cap_rows) {
  if (d < 1 || d > BSDE_MAX_D || eta < 0 || eta > 15 || !(q > 0.0) || q > 1.0 || !nu_out)
    return BSDE_ERR_INVALID_ARG;
  try {
    const auto nus = build_multi_indices(d + 1, eta, q);
    if ((int)nus.size() > cap_rows) return BSDE_ERR_INVALID_ARG;
    for (size_t l = 0; l < nus.size(); ++l)
      for (int v = 0; v <= d; ++v) nu_out[l * (d + 1) + v] = nus[l][v];
    return BSDE_OK;
  } catch (...) {
    return BSDE_ERR_NOMEM;
  }
}

int bsde_get_coeffs(bsde_ctx* c, double* out, int cap) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (!out) return fail(c, BSDE_ERR_INVALID_ARG, "get_coeffs: NULL output");
  if (!c->prob.coeffs_valid) return fail(c, BSDE_ERR_STATE, "get_coeffs: no solve yet");
  const int p = c->prob.shape.p;
  if (cap < p) return fail(c, BSDE_ERR_INVALID_ARG, "get_coeffs: capacity below p");
  cudaSetDevice(c->device);
  if (cudaMemcpyAsync(out, c->prob.dev.alpha, (size_t)p * 8, cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(c, BSDE_ERR_CUDA, "get_coeffs: copy failed");
  return BSDE_OK;
}

int bsde_set_coeffs(bsde_ctx* c, const bsde_solve_params* prm, const double* alpha, int p) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (!prm || !alpha) return fail(c, BSDE_ERR_INVALID_ARG, "set_coeffs: NULL argument");
  API_GUARD(c, {
    if (!set_device(c)) return fail(c, BSDE_ERR_CUDA, "set_coeffs: cudaSetDevice failed");
    Problem& P = c->prob;
    int rc = P.prepare(*prm, c->al, c->budget, c->stream);
    if (rc != BSDE_OK) return fail(c, rc, P.err);
    if (p != P.shape.p) return fail(c, BSDE_ERR_INVALID_ARG, "set_coeffs: p does not match the basis");
    std::vector<float> a32(p);
    for (int l = 0; l < p; ++l) a32[l] = (float)alpha[l];
    if (cudaMemcpyAsync(P.dev.alpha, alpha, (size_t)p * 8, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(P.dev.alpha32, a32.data(), (size_t)p * 4, cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return fail(c, BSDE_ERR_CUDA, "set_coeffs: upload failed");
    P.coeffs_valid = true;
    return BSDE_OK;
  })
}

int bsde_eval_price_delta(bsde_ctx* c, int q, const double* t, const double* S, double* price,
                          double* delta) {
  if (!c) return BSDE_ERR_INVALID_ARG;
  if (q < 1 || !t || !S || !price) return fail(c, BSDE_ERR_INVALID_ARG, "eval: bad arguments");
  API_GUARD(c, {
    Problem& P = c->prob;
    if (!P.coeffs_valid) return fail(c, BSDE_ERR_STATE, "eval: no coefficients (solve first)");
    if (!set_device(c)) return fail(c, BSDE_ERR_CUDA, "eval: cudaSetDevice failed");
    const int d = P.model.d;
    std::vector<double> hx((size_t)q * d);
    for (size_t e = 0; e < hx.size(); ++e) {
      if (!(S[e] > 0.0)) return fail(c, BSDE_ERR_INVALID_ARG, "eval: prices must be positive");
      hx[e] = std::log(S[e]);
    }
    const size_t bytes = (size_t)q * 8 * (2 + 2 * d);
    double* buf = (double*)c->al.get(bytes, c->stream);
    if (!buf) return fail(c, BSDE_ERR_NOMEM, "eval: device allocation failed");
    double* dt = buf;
    double* dx = dt + q;
    double* dp = dx + (size_t)q * d;
    double* dg = dp + q;
    std::vector<double> g((size_t)q * d);
    cudaError_t e = cudaMemcpyAsync(dt, t, (size_t)q * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dx, hx.data(), (size_t)q * d * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
      launch_eval_points(P.model, P.grid, P.dev, q, dt, dx, dp, dg, c->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(price, dp, (size_t)q * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.data(), dg, (size_t)q * d * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->al.put(buf, c->stream);
    if (e != cudaSuccess) return fail(c, BSDE_ERR_CUDA, std::string("eval: ") + cudaGetErrorString(e));
    if (delta)
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < d; ++j) delta[(size_t)i * d + j] = g[(size_t)i * d + j] / S[(size_t)i * d + j];
    return BSDE_OK;
  })
}

}  // extern "C"
