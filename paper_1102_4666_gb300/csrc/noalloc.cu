// noalloc.cu -- bsde_corrections_noalloc: the per-point Monte Carlo
// corrections of the path kernel for callers that cannot allocate device
// memory (see include/bsde.h).
//
// Such callers (code that runs inside a fixed device-memory arena, a plugin
// whose host forbids cudaMalloc/cudaFree, or a process that must not touch
// the allocator in its steady state) pass every input and output buffer
// themselves.  The kernel's own scratch -- the per-(point, chunk) partial
// sums, the packed basis table, the FP32 coefficient copy and the Philox key
// -- lives in one file-scope device array of fixed size instead of memory
// obtained from an allocator.  Host code cannot use the array's name as a
// device address (in host code it is only a stand-in for the symbol), so the
// device address is looked up once per device with cudaGetSymbolAddress.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "multiindex.h"
#include "runtime.h"

namespace {

constexpr size_t SCRATCH_BYTES = 4u << 20;  // 4 MiB, held by every device that loads the library
constexpr int NOALLOC_MAX_P = 4096;          // basis functions
constexpr size_t TABLE_BYTES = 160u << 10;   // key, status, basis table, FP32 coefficients
constexpr size_t PARTIAL_MAX = (SCRATCH_BYTES - TABLE_BYTES) / sizeof(double);  // n * chunks

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_dev[MAX_DEVICES] = {nullptr};

void set_msg(char* buf, size_t len, const std::string& m) {
  if (buf && len) {
    strncpy(buf, m.c_str(), len - 1);
    buf[len - 1] = '\0';
  }
}

// device address of g_scratch on the current device (looked up once)
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> g(g_mu);
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

__global__ void k_to_f32(int p, const double* __restrict__ a, float* __restrict__ b) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < p) b[l] = (float)a[l];
}

}  // namespace

extern "C" BSDE_API int bsde_corrections_noalloc(
    const bsde_sigma* sigma, double r, const bsde_payoff* payoff, const bsde_penalty* penalty,
    const double* lo, const double* hi, int n, const double* t_dev, const double* x_dev, int eta,
    double q, const double* alpha_dev, int M, int N_steps, uint64_t seed, int k, int precision,
    double* c_dev, void* stream, char* errbuf, size_t errbuf_len) {
  try {
    std::string err;
    ModelHost m;
    int rc = bsde_set_model_impl(m, sigma, r, payoff, penalty, err);
    if (rc != BSDE_OK) {
      set_msg(errbuf, errbuf_len, err);
      return rc;
    }
    GridHost g;
    rc = bsde_set_grid_impl(g, m.d, n, lo, hi, 1, err);
    if (rc != BSDE_OK) {
      set_msg(errbuf, errbuf_len, err);
      return rc;
    }
    if (!t_dev || !x_dev || !alpha_dev || !c_dev || M < 1 || N_steps < 1 || eta < 0 || eta > 15 ||
        !(q > 0.0) || q > 1.0 || k < 0 || k >= (1 << 24) ||
        (precision != BSDE_PREC_FP64 && precision != BSDE_PREC_MIXED) || !paths_supported_d(m.d)) {
      set_msg(errbuf, errbuf_len,
              "corrections_noalloc: bad argument (NULL buffer, M or N_steps < 1, eta outside "
              "0..15, q outside (0,1], k outside 0..2^24-1, unknown precision or d outside 1..10)");
      return BSDE_ERR_INVALID_ARG;
    }
    const auto nus = build_multi_indices(m.d + 1, eta, q);
    std::vector<uint32_t> pairs;
    std::vector<uint8_t> nnz;
    int max_deg = 0;
    if (!pack_multi_indices(nus, pairs, nnz, max_deg)) {
      set_msg(errbuf, errbuf_len, "corrections_noalloc: basis needs more than 8 active variates");
      return BSDE_ERR_INVALID_ARG;
    }
    const int p = (int)nus.size();
    const bool mixed = precision == BSDE_PREC_MIXED;
    const int eta_t = max_deg < 1 ? 1 : max_deg;
    // launch shape of the path kernel, as the context runtime chooses it
    int tpb = mixed ? 128 : 64;
    while (tpb > 32 && paths_smem_bytes(m.d, p, eta_t, N_steps, tpb, mixed, false) > 220 * 1024) tpb >>= 1;
    int ppt = 4;
    while (ppt > 1 && (long long)tpb * ppt > 2LL * M) ppt >>= 1;
    const long long chunks = (M + tpb * ppt - 1) / (tpb * ppt);
    if (p > NOALLOC_MAX_P || (long long)n * chunks > (long long)PARTIAL_MAX ||
        paths_smem_bytes(m.d, p, eta_t, N_steps, tpb, mixed, false) > 220 * 1024) {
      char msg[256];
      snprintf(msg, sizeof(msg),
               "corrections_noalloc: problem exceeds the static scratch (p = %d, limit %d; "
               "n * ceil(M / %d) = %lld, limit %zu)",
               p, NOALLOC_MAX_P, tpb * ppt, (long long)n * chunks, PARTIAL_MAX);
      set_msg(errbuf, errbuf_len, msg);
      return BSDE_ERR_NOMEM;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      set_msg(errbuf, errbuf_len, "corrections_noalloc: no current CUDA device");
      return BSDE_ERR_CUDA;
    }
    void* base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess) {
      set_msg(errbuf, errbuf_len, std::string("corrections_noalloc: cudaGetSymbolAddress failed: ") +
                                      cudaGetErrorString(e));
      return BSDE_ERR_CUDA;
    }
    // carve the scratch: key + status | pairs | nnz | alpha32 | partial sums
    char* s = (char*)base;
    ProblemDev P;
    P.n = n;
    P.p = p;
    P.eta = eta_t;
    P.chunks = (int)chunks;
    P.t = const_cast<double*>(t_dev);
    P.x = const_cast<double*>(x_dev);
    P.alpha = const_cast<double*>(alpha_dev);
    P.key = (uint32_t*)s;
    P.status = (int*)(s + 16);
    P.pairs = (uint2*)(s + 256);
    P.nnz = (uint8_t*)(s + 256 + (size_t)NOALLOC_MAX_P * 8);
    P.alpha32 = (float*)(s + 256 + (size_t)NOALLOC_MAX_P * 9 + 256);
    P.partial = (double*)(s + TABLE_BYTES);
    P.c = c_dev;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    P.seed_key[0] = key[0];
    P.seed_key[1] = key[1];
    // every scratch word the kernels read is rewritten here; the partial
    // sums are all overwritten by the path kernel before they are read
    e = cudaMemcpyAsync(P.key, key, sizeof(key), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.pairs, pairs.data(), (size_t)p * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.nnz, nnz.data(), (size_t)p, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && mixed) {
      k_to_f32<<<(p + 127) / 128, 128, 0, st>>>(p, alpha_dev, P.alpha32);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_paths(m, g, P, M, N_steps, (uint32_t)k, mixed, tpb, ppt, st);
    if (e == cudaSuccess) {
      launch_reduce_c(P, M, st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host tables above live on this stack
    if (e != cudaSuccess) {
      set_msg(errbuf, errbuf_len, std::string("corrections_noalloc: CUDA error: ") + cudaGetErrorString(e));
      return BSDE_ERR_CUDA;
    }
    return BSDE_OK;
  } catch (...) {
    set_msg(errbuf, errbuf_len, "corrections_noalloc: out of host memory");
    return BSDE_ERR_NOMEM;
  }
}
