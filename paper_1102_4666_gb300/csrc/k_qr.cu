// k_qr.cu -- least-squares refit of eq. alpha by Householder QR with column
// pivoting on the design matrix, in FP64: the role the paper gives to
// LAPACK's dgelsy (Section 3.2.2: the Gram matrix is often ill-conditioned,
// so the paper avoids Cholesky).  Selected by bsde_solve_params.ls_mode = 1.
//
// The design matrix X[i][l] = B_l(t_i, x_i) is stored column by column
// (B[l][i], point index fastest), which is the layout Householder needs.
// Step j: pick the remaining column of largest norm, swap it to position j,
// build the reflector H_j = I - tau v v^T (v_0 = 1) that zeroes it below the
// diagonal, apply H_j to the remaining columns and to the right-hand side c,
// and refresh the remaining columns' norms.  Columns whose diagonal |R_jj|
// falls below 1e-13 |R_00| are treated as dependent (rank truncation); the
// solution is the basic solution R_11 delta_1 = (Q^T c)_1, delta_2 = 0,
// scattered back through the column permutation.
#include "common.cuh"

namespace {

// copy B -> W, c -> y, squared column norms
__global__ void k_qr_init(int n, int n_pad, int p, const double* __restrict__ B,
                          const double* __restrict__ c, double* __restrict__ W,
                          double* __restrict__ y, double* __restrict__ nrm, int* __restrict__ perm) {
  const int l = blockIdx.x;  // column (p of them) or the right-hand side (l == p)
  const double* src = (l < p) ? B + (size_t)l * n_pad : c;
  double* dst = (l < p) ? W + (size_t)l * n_pad : y;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = src[i];
    dst[i] = v;
    s += v * v;
  }
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0 && l < p) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    nrm[l] = t;
    perm[l] = l;
  }
}

// step j: pivot (largest remaining norm, first index on ties), swap, reflector
__global__ void __launch_bounds__(256) k_qr_pivot(int n, int n_pad, int p, int j,
                                                  double* __restrict__ W, double* __restrict__ nrm,
                                                  int* __restrict__ perm, double* __restrict__ tau) {
  __shared__ double sv[256];
  __shared__ int si[256];
  __shared__ double s_beta, s_scale;
  const int tid = threadIdx.x;
  double best = -1.0;
  int bi = j;
  for (int l = j + tid; l < p; l += 256) {
    const double v = nrm[l];
    if (v > best) {
      best = v;
      bi = l;
    }
  }
  sv[tid] = best;
  si[tid] = bi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) {
      const double a = sv[tid], b = sv[tid + o];
      const int ia = si[tid], ib = si[tid + o];
      if (b > a || (b == a && ib < ia)) {
        sv[tid] = b;
        si[tid] = ib;
      }
    }
    __syncthreads();
  }
  const int piv = si[0];
  if (piv != j) {
    double* cj = W + (size_t)j * n_pad;
    double* cp = W + (size_t)piv * n_pad;
    for (int i = tid; i < n; i += 256) {
      const double t = cj[i];
      cj[i] = cp[i];
      cp[i] = t;
    }
    if (tid == 0) {
      const double t = nrm[j];
      nrm[j] = nrm[piv];
      nrm[piv] = t;
      const int q = perm[j];
      perm[j] = perm[piv];
      perm[piv] = q;
    }
  }
  __syncthreads();
  // Householder vector of x = W[j][j:n]
  double* x = W + (size_t)j * n_pad;
  double s = 0.0;
  for (int i = j + 1 + tid; i < n; i += 256) s += x[i] * x[i];
  sv[tid] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) sv[tid] += sv[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    const double x0 = x[j], sig = sv[0];
    if (sig == 0.0 || j >= n) {
      tau[j] = 0.0;
      s_beta = x0;
      s_scale = 0.0;
    } else {
      const double nx = sqrt(x0 * x0 + sig);
      const double beta = x0 <= 0.0 ? nx : -nx;
      tau[j] = (beta - x0) / beta;
      s_beta = beta;
      s_scale = 1.0 / (x0 - beta);
    }
  }
  __syncthreads();
  const double sc = s_scale;
  for (int i = j + 1 + tid; i < n; i += 256) x[i] *= sc;  // v (v_0 = 1 implied)
  if (tid == 0) x[j] = s_beta;                             // R_jj
}

// step j: apply H_j to column l > j (block l - j - 1) or to y (last block),
// then refresh the squared norm of the column below row j
__global__ void __launch_bounds__(256) k_qr_apply(int n, int n_pad, int p, int j,
                                                  double* __restrict__ W, double* __restrict__ y,
                                                  double* __restrict__ nrm,
                                                  const double* __restrict__ tau) {
  __shared__ double red[8];
  __shared__ double s_f;
  const int l = j + 1 + blockIdx.x;
  double* col = (l < p) ? W + (size_t)l * n_pad : y;
  const double* v = W + (size_t)j * n_pad;
  const int tid = threadIdx.x;
  double s = 0.0;
  for (int i = j + 1 + tid; i < n; i += 256) s += v[i] * col[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double t = col[j];  // v_0 = 1
    for (int w = 0; w < 8; ++w) t += red[w];
    const double f = tau[j] * t;
    s_f = f;
    col[j] -= f;
  }
  __syncthreads();
  const double f = s_f;
  double q = 0.0;
  for (int i = j + 1 + tid; i < n; i += 256) {
    const double v2 = col[i] - f * v[i];
    col[i] = v2;
    q += v2 * v2;
  }
  if (l < p) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = q;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      nrm[l] = t;
    }
  }
}

// basic solution: rank r from |R_jj| > 1e-13 |R_00|, R_11 d = y_1 by back
// substitution (one CTA, column-oriented), delta[perm[j]] = d_j (0 beyond r)
__global__ void __launch_bounds__(256) k_qr_solve(int n_pad, int p, const double* __restrict__ W,
                                                  const double* __restrict__ y,
                                                  const int* __restrict__ perm,
                                                  double* __restrict__ delta,
                                                  double* __restrict__ work, int* __restrict__ rank_out) {
  __shared__ int s_rank;
  __shared__ double s_x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const double r00 = fabs(W[0]);
    int r = 0;
    while (r < p && fabs(W[(size_t)r * n_pad + r]) > 1e-13 * r00) ++r;
    s_rank = r;
    *rank_out = r;
  }
  __syncthreads();
  const int r = s_rank;
  for (int q = tid; q < p; q += 256) work[q] = (q < r) ? y[q] : 0.0;
  __syncthreads();
  for (int c = r - 1; c >= 0; --c) {
    if (tid == 0) {
      s_x = work[c] / W[(size_t)c * n_pad + c];
      work[c] = s_x;
    }
    __syncthreads();
    const double xc = s_x;
    for (int q = tid; q < c; q += 256) work[q] -= W[(size_t)c * n_pad + q] * xc;  // R_qc = W[c][q]
    __syncthreads();
  }
  for (int q = tid; q < p; q += 256) delta[perm[q]] = work[q];
}

}  // namespace

// delta = argmin |c - X delta| by pivoted QR; the workspace (W: p x n_pad,
// y: n, norms, tau, perm, rank) is P.qr_*
void launch_qr_solve(const ProblemDev& P, cudaStream_t st) {
  k_qr_init<<<P.p + 1, 256, 0, st>>>(P.n, P.n_pad, P.p, P.B, P.c, P.qr_W, P.qr_y, P.qr_nrm,
                                     P.qr_perm);
  const int steps = P.p < P.n ? P.p : P.n;
  for (int j = 0; j < steps; ++j) {
    k_qr_pivot<<<1, 256, 0, st>>>(P.n, P.n_pad, P.p, j, P.qr_W, P.qr_nrm, P.qr_perm, P.qr_tau);
    k_qr_apply<<<P.p - j, 256, 0, st>>>(P.n, P.n_pad, P.p, j, P.qr_W, P.qr_y, P.qr_nrm, P.qr_tau);
  }
  k_qr_solve<<<1, 256, 0, st>>>(P.n_pad, P.p, P.qr_W, P.qr_y, P.qr_perm, P.delta, P.res,
                                P.qr_rank);
}
