// runtime.h -- host runtime of one resident BSDE problem: device memory
// (one arena from the caller's allocator), the per-iteration launch sequence
// of Algorithm 2 and the captured CUDA graph of a whole solve.  Used by the
// C ABI (api.cu) and by the serving loop (server.cu).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bsde.h"
#include "common.cuh"

struct Allocator {
  bsde_alloc_fn alloc = nullptr;
  bsde_free_fn free = nullptr;
  void* user = nullptr;
  void* get(size_t bytes, cudaStream_t st);
  void put(void* p, cudaStream_t st);
};

struct Shape {
  int d = 0, n = 0, n_pad = 0, p = 0, p_pad = 0, eta = 0, M = 0, N = 0;
  int chunks = 0, tpb = 0, ppt = 0, splits = 0, pm = 0, tree = 0;
  bool mixed = false, dense = false, dense4 = false, qr = false;
  bool operator==(const Shape& o) const {
    return d == o.d && n == o.n && p == o.p && eta == o.eta && M == o.M && N == o.N &&
           tpb == o.tpb && ppt == o.ppt && mixed == o.mixed && dense == o.dense &&
           dense4 == o.dense4 && tree == o.tree && pm == o.pm && qr == o.qr && splits == o.splits;
  }
};

class Problem {
 public:
  ModelHost model;
  GridHost grid;
  bool has_model = false, has_grid = false, coeffs_valid = false;
  bool mixed = true;
  Shape shape;
  ProblemDev dev;
  std::vector<uint32_t> pairs;
  std::vector<uint8_t> nnz;
  std::vector<std::vector<int>> nus;
  int eta_used = 0;  // largest single-variate degree present
  // Chebyshev -> monomial map of the dense evaluation (pm > 0; mono_deg:
  // the largest monomial degree; tree_deg > 0: prefix-tree order)
  int pm = 0, mono_deg = 3, tree_deg = 0;
  std::vector<int> conv_row, conv_l;
  std::vector<double> conv_c;
  std::string err;
  // point sharding (bsde_set_shard): rank sh_rank of sh_n, the caller's
  // correction buffer and exchange hook
  int sh_rank = 0, sh_n = 1;
  double* sh_buf = nullptr;
  size_t sh_len = 0;
  bsde_exchange_fn sh_fn = nullptr;
  void* sh_user = nullptr;
  // peer exchange (bsde_set_shard_peers): every rank's buffer and counters,
  // the wait bound and the exchange number of the last exchange
  bool sh_peer = false;
  PeerPtrs sh_pp;
  double sh_wait_ms = 1000.0;
  uint32_t sh_epoch = 0;

  ~Problem();
  // validate params, build the basis, (re)allocate device memory; BSDE_OK or an error
  int prepare(const bsde_solve_params& prm, Allocator& al, size_t budget, cudaStream_t st);
  // launch iterations k0 .. k0 + count - 1 (no synchronisation), each
  // group of them after the factorisation of its Gram matrices; ev: 8
  // timing events per iteration or nullptr
  int enqueue_block(const bsde_solve_params& prm, int k0, int count, cudaStream_t st,
                    cudaEvent_t* ev);
  // full solve: alpha reset (k_start == 0), K_it iterations, report
  int solve(const bsde_solve_params& prm, Allocator& al, size_t budget, cudaStream_t st,
            bsde_report* rep);
  int enqueue_solve(const bsde_solve_params& prm, cudaStream_t st);  // after prepare
  // points, basis matrix and Gram matrix of iteration k into factor slot 0
  // (after prepare)
  int enqueue_gram(int k, cudaStream_t st);
  // asynchronous halves of solve(): start() enqueues (graph or launches)
  // between events e0 and e1; complete() waits for e1 and builds the report
  int start(const bsde_solve_params& prm, Allocator& al, size_t budget, cudaStream_t st,
            cudaEvent_t e0, cudaEvent_t e1);
  int complete(const bsde_solve_params& prm, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
               bsde_report* rep);
  int finish_report(const bsde_solve_params& prm, cudaStream_t st, bsde_report* rep,
                    float ms_total);
  void release(Allocator& al, cudaStream_t st);
  void destroy_graph();  // after a model or grid change
  size_t bytes() const { return block_bytes + fact_bytes; }
  static size_t estimate_bytes(int d, int n, int p, int M, int N, bool mixed, int tpb, int ppt,
                               int pm = 0, int conv_nnz = 0, bool qr = false, int nfact = 1,
                               int splits = 0);
  // Gram matrices factorised together ahead of their iterations: all K_it
  // of a solve while their factors and inverses fit in 256 MiB (one when
  // the points are not redrawn, none for the QR refit)
  static int fact_group(int p, int K_it, bool resample, bool qr);
  static size_t fact_block_bytes(int p, int nfact);

 private:
  void* block = nullptr;
  size_t block_bytes = 0;
  double* c_own = nullptr;  // the corrections in the context's own arena
  Shape alloc_shape;
  // Gram matrices, Cholesky factors and inverses of up to nfact iterations
  void* fact = nullptr;
  size_t fact_bytes = 0;
  int nfact = 0;
  // graph of a whole solve
  cudaGraphExec_t gexec = nullptr;
  std::string graph_key;
  std::vector<cudaEvent_t> events;  // 8 per iteration when timing
  int choose_launch(int d, int p, int eta, int N, int M, bool mixed, bool dense, int& tpb,
                    int& ppt);
  void ensure_events(int count);
  // points, basis and Gram matrix of iterations k0 .. k0 + nb - 1 into the
  // nb slots of the factor block, then their batched factorisation and inverses
  int enqueue_factors(int k0, int nb, cudaStream_t st);
  // one iteration k -> k + 1 whose Gram inverse is in slot `slot`
  int enqueue_iteration(const bsde_solve_params& prm, int k, cudaStream_t st, cudaEvent_t* ev,
                        int slot);
};

int bsde_set_model_impl(ModelHost& m, const bsde_sigma* sigma, double r, const bsde_payoff* payoff,
                        const bsde_penalty* penalty, std::string& err);
int bsde_set_grid_impl(GridHost& g, int d, int n, const double* lo, const double* hi,
                       int resample, std::string& err);
// block [i0, i1) of the points of rank `rank` of nranks: nb = ceil(n / nranks)
void shard_block(int n, int rank, int nranks, int& i0, int& i1);
