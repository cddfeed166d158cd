// k_linalg.cu -- the least-squares refit of Algorithm 2 (eq. alpha) through
// the normal equations A alpha = sum_i y_i B(t_i, x_i) (eq. alphasys,
// Section 3.2.2), in the correction form alpha^{k+1} = alpha^k + delta with
// A delta = B^T c^k (the fit of u^k + c^k equals alpha^k plus the fit of c^k
// because u^k lies in the span of the basis).  The paper solves with LAPACK
// dgelsy; here the Gram matrix is factored by an FP64 Cholesky on the GPU,
// with an optional FP64 iterative refinement of the normal equations.
// Also: the per-point reduction of eq. chat, the coefficient update and the
// price / delta read-out of Section 5.3.
#include "common.cuh"

namespace {

// eq. chat: c_i = (1/M) sum of the per-chunk sums, in chunk order
__global__ void k_reduce_c(int i0, int count, int chunks, int M, const double* __restrict__ partial,
                           double* __restrict__ c) {
  const int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= i0 + count) return;
  double s = 0.0;
  for (int q = 0; q < chunks; ++q) s += partial[(size_t)i * chunks + q];
  c[i] = s / (double)M;
}

// CTA of 128 threads per basis function: out[l] = sum_i B[l][i] y[i], each
// thread over i = tid mod 128, then a fixed shuffle tree and the four warp
// sums in order; with sub != nullptr, out[l] = sub[l] - that sum
__global__ void __launch_bounds__(128) k_bt_times(int n, int n_pad, int p,
                                                  const double* __restrict__ B,
                                                  const double* __restrict__ y,
                                                  const double* __restrict__ sub,
                                                  double* __restrict__ out) {
  __shared__ double ws[4];
  const int l = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* row = B + (size_t)l * n_pad;
  double s = 0.0;
  for (int i = tid; i < n; i += 128) s += row[i] * y[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) ws[warp] = s;
  __syncthreads();
  if (tid == 0) {
    const double tot = (ws[0] + ws[1]) + (ws[2] + ws[3]);
    out[l] = sub ? (sub[l] - tot) : tot;
  }
}

// v[i] = sum_l B[l][i] x[l]: CTA of 32 points x 8 slices of the basis
// functions (coalesced rows of B per warp), the slice sums added in order
__global__ void __launch_bounds__(256) k_b_times(int n, int n_pad, int p,
                                                 const double* __restrict__ B,
                                                 const double* __restrict__ x,
                                                 double* __restrict__ v) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const int per = (p + 7) / 8;
  const int l0 = slice * per, l1 = min(p, l0 + per);
  double s = 0.0;
  if (i < n)
    for (int l = l0; l < l1; ++l) s += B[(size_t)l * n_pad + i] * x[l];
  part[slice][lane] = s;
  __syncthreads();
  if (slice == 0 && i < n) {
    double tot = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) tot += part[q][lane];
    v[i] = tot;
  }
}

// FP64 Gram A = B B^T on CUDA cores: one 32x32 upper tile per CTA, written
// to both triangles.
__global__ void __launch_bounds__(256) k_gram_f64(int n, int n_pad, int p,
                                                  const double* __restrict__ B,
                                                  double* __restrict__ A) {
  __shared__ double As[32][33], Bs[32][33];
  // decode the upper tile (ti <= tj) from blockIdx.x
  const int T = (p + 31) / 32;
  int t = blockIdx.x, ti = 0;
  while (t >= T - ti) {
    t -= T - ti;
    ++ti;
  }
  const int tj = ti + t;
  const int r0 = ti * 32, c0 = tj * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int q = threadIdx.x; q < 32 * 32; q += 256) {
      const int rr = q >> 5, kk = q & 31;
      const int kg = k0 + kk;
      As[rr][kk] = (r0 + rr < p && kg < n) ? B[(size_t)(r0 + rr) * n_pad + kg] : 0.0;
      Bs[rr][kk] = (c0 + rr < p && kg < n) ? B[(size_t)(c0 + rr) * n_pad + kg] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double b = Bs[tx][kk];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][kk] * b;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + ty + 8 * q, c = c0 + tx;
    if (r < p && c < p) {
      A[(size_t)r * p + c] = acc[q];
      A[(size_t)c * p + r] = acc[q];
    }
  }
}

// The factorisation kernels work on a batch of Gram matrices, one per
// blockIdx.y: matrix z is A + z p^2, with its original diagonal at
// diag0 + z p, its reciprocal factor diagonal at dinv + z p and its inverse
// at Ainv + z p^2.

// original diagonal of A, for the relative pivot test of the factorisation
__global__ void k_save_diag(const double* __restrict__ A, int p, double* __restrict__ diag0) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t z = blockIdx.y;
  if (j < p) diag0[z * p + j] = A[z * p * p + (size_t)j * p + j];
}

// Right-looking blocked Cholesky, panel width 32, lower factor in place.
// Panel step 1: one warp factors the 32x32 diagonal block in shared memory
// and stores the reciprocals of its diagonal in dinv.  A pivot below 1e-13
// of its original diagonal entry (or not finite) marks the matrix as
// numerically singular: ST_NOT_PD, and the pivot becomes NaN.
__global__ void __launch_bounds__(32) k_chol_diag(double* __restrict__ A, int p, int j0,
                                                  int* __restrict__ status,
                                                  const double* __restrict__ diag0,
                                                  double* __restrict__ dinv) {
  __shared__ double Dg[32][33];
  const size_t z = blockIdx.y;
  A += z * p * p;
  diag0 += z * p;
  dinv += z * p;
  const int nb = min(32, p - j0);
  const int lane = threadIdx.x;
  for (int q = lane; q < 32 * 32; q += 32) {
    const int r = q >> 5, c = q & 31;
    Dg[r][c] = (r < nb && c < nb && c <= r) ? A[(size_t)(j0 + r) * p + (j0 + c)] : 0.0;
  }
  __syncwarp();
  for (int c = 0; c < nb; ++c) {
    double inv = 0.0;
    if (lane == 0) {
      const double piv = Dg[c][c];
      if (!(piv > 1e-13 * diag0[j0 + c]) || !isfinite(piv)) {
        atomicOr(status, ST_NOT_PD);
        Dg[c][c] = nan("");
        inv = nan("");
      } else {
        const double dcc = sqrt(piv);
        Dg[c][c] = dcc;
        inv = 1.0 / dcc;
      }
      dinv[j0 + c] = inv;
    }
    inv = __shfl_sync(0xffffffffu, inv, 0);
    __syncwarp();
    if (lane > c && lane < nb) Dg[lane][c] *= inv;
    __syncwarp();
    // rank-1 update of the trailing block: lane handles row r = lane
    if (lane > c && lane < nb) {
      const double lrc = Dg[lane][c];
      for (int s2 = c + 1; s2 <= lane; ++s2) Dg[lane][s2] -= lrc * Dg[s2][c];
    }
    __syncwarp();
  }
  for (int q = lane; q < 32 * 32; q += 32) {
    const int r = q >> 5, c = q & 31;
    if (r < nb && c <= r) A[(size_t)(j0 + r) * p + (j0 + c)] = Dg[r][c];
  }
}

// Panel step 2: rows below the diagonal block solve x L_jj^T = a (forward
// substitution with the reciprocal diagonal), one thread per row.
__global__ void __launch_bounds__(32) k_chol_trsm(double* __restrict__ A, int p, int j0,
                                                  const double* __restrict__ dinv) {
  __shared__ double Dg[32][33];
  __shared__ double di[32];
  const size_t z = blockIdx.y;
  A += z * p * p;
  dinv += z * p;
  const int nb = min(32, p - j0);
  for (int q = threadIdx.x; q < 32 * 32; q += 32) {
    const int r = q >> 5, c = q & 31;
    Dg[r][c] = (r < nb && c < nb && c <= r) ? A[(size_t)(j0 + r) * p + (j0 + c)] : 0.0;
  }
  di[threadIdx.x] = threadIdx.x < nb ? dinv[j0 + threadIdx.x] : 0.0;
  __syncthreads();
  const int row = j0 + nb + 32 * blockIdx.x + threadIdx.x;
  if (row >= p) return;
  double xr[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) xr[c] = (c < nb) ? A[(size_t)row * p + j0 + c] : 0.0;
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    if (c < nb) {
      double acc = xr[c];
#pragma unroll
      for (int q = 0; q < c; ++q) acc -= xr[q] * Dg[c][q];
      xr[c] = acc * di[c];
    }
  }
#pragma unroll
  for (int c = 0; c < 32; ++c)
    if (c < nb) A[(size_t)row * p + j0 + c] = xr[c];
}

// trailing update A22 -= L21 L21^T on the lower triangle, 32x32 tiles
__global__ void __launch_bounds__(256) k_chol_update(double* __restrict__ A, int p, int j0) {
  __shared__ double Lr[32][33], Lc[32][33];
  A += (size_t)blockIdx.y * p * p;
  const int nb = min(32, p - j0);
  const int base = j0 + nb;
  const int m = p - base;
  const int T = (m + 31) / 32;
  int t = blockIdx.x, ti = 0;  // lower tiles (tj <= ti), row-major
  while (t > ti) {
    t -= ti + 1;
    ++ti;
  }
  const int tj = t;
  if (ti >= T) return;
  const int r0 = base + 32 * ti, c0 = base + 32 * tj;
  for (int q = threadIdx.x; q < 32 * 32; q += 256) {
    const int rr = q >> 5, kk = q & 31;
    Lr[rr][kk] = (r0 + rr < p && kk < nb) ? A[(size_t)(r0 + rr) * p + j0 + kk] : 0.0;
    Lc[rr][kk] = (c0 + rr < p && kk < nb) ? A[(size_t)(c0 + rr) * p + j0 + kk] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rr = ty + 8 * q;
    const int r = r0 + rr, c = c0 + tx;
    if (r < p && c < p && c <= r) {
      double s = 0.0;
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) s += Lr[rr][kk] * Lc[tx][kk];
      A[(size_t)r * p + c] -= s;
    }
  }
}

// x (+)= A^{-1} b with the Cholesky factor L in the lower triangle of A and
// its reciprocal diagonal in dinv: L y = b, then L^T x = y, by blocks of 32.
// Warp 0 solves each 32x32 diagonal block with shuffles; all threads then
// update the rest of the vector with that block's 32 columns (forward: a
// row segment per thread; backward: coalesced column reads).  One CTA.
// With b == nullptr, CTA (j, z) solves A_z x = e_j and writes column j of
// A_z^{-1} to x + z p^2 + j p (the inverses used by the refit).
__global__ void __launch_bounds__(256) k_chol_solve(const double* __restrict__ A, int p,
                                                    const double* __restrict__ dinv,
                                                    const double* __restrict__ b,
                                                    double* __restrict__ x, int accumulate) {
  extern __shared__ double yv[];  // p
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t z = blockIdx.y;
  A += z * p * p;
  dinv += z * p;
  if (b == nullptr) x += z * p * p + (size_t)blockIdx.x * p;
  for (int r = tid; r < p; r += blockDim.x) yv[r] = b ? b[r] : (r == (int)blockIdx.x ? 1.0 : 0.0);
  __syncthreads();
  const int nblk = (p + 31) / 32;
  // for b = e_j the forward solution is zero above row j: start at its block
  for (int blk = b ? 0 : (int)blockIdx.x / 32; blk < nblk; ++blk) {
    const int c0 = blk * 32, nb = min(32, p - c0);
    if (warp == 0) {
      double yi = lane < nb ? yv[c0 + lane] : 0.0;
      for (int c = 0; c < nb; ++c) {
        if (lane == c) yi *= dinv[c0 + c];
        const double yc = __shfl_sync(0xffffffffu, yi, c);
        if (lane > c && lane < nb) yi -= A[(size_t)(c0 + lane) * p + c0 + c] * yc;
      }
      if (lane < nb) yv[c0 + lane] = yi;
    }
    __syncthreads();
    for (int r = c0 + nb + tid; r < p; r += blockDim.x) {
      const double* row = A + (size_t)r * p + c0;
      double acc = 0.0;
      for (int c = 0; c < nb; ++c) acc += row[c] * yv[c0 + c];
      yv[r] -= acc;
    }
    __syncthreads();
  }
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int c0 = blk * 32, nb = min(32, p - c0);
    if (warp == 0) {
      double xi = lane < nb ? yv[c0 + lane] : 0.0;
      for (int c = nb - 1; c >= 0; --c) {
        if (lane == c) xi *= dinv[c0 + c];
        const double xc = __shfl_sync(0xffffffffu, xi, c);
        if (lane < c) xi -= A[(size_t)(c0 + c) * p + c0 + lane] * xc;
      }
      if (lane < nb) yv[c0 + lane] = xi;
    }
    __syncthreads();
    for (int r = tid; r < c0; r += blockDim.x) {
      double acc = 0.0;
      for (int c = 0; c < nb; ++c) acc += A[(size_t)(c0 + c) * p + r] * yv[c0 + c];
      yv[r] -= acc;
    }
    __syncthreads();
  }
  for (int r = tid; r < p; r += blockDim.x) x[r] = accumulate ? (x[r] + yv[r]) : yv[r];
}

// alpha += delta; ||delta||_2, ||delta||_inf into the report block; FP32 copy
__global__ void __launch_bounds__(256) k_update(int p, int k, double* __restrict__ alpha,
                                                float* __restrict__ alpha32,
                                                const double* __restrict__ delta,
                                                double* __restrict__ out) {
  __shared__ double s2[256], si[256];
  double a2 = 0.0, ai = 0.0;
  for (int l = threadIdx.x; l < p; l += 256) {
    const double dl = delta[l];
    const double al = alpha[l] + dl;
    alpha[l] = al;
    if (alpha32) alpha32[l] = (float)al;
    a2 += dl * dl;
    ai = fmax(ai, fabs(dl));
  }
  s2[threadIdx.x] = a2;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s2[threadIdx.x] += s2[threadIdx.x + o];
      si[threadIdx.x] = fmax(si[threadIdx.x], si[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && k >= 0 && k < 64) {
    out[OUT_RES2 + k] = sqrt(s2[0]);
    out[OUT_RESI + k] = si[0];
  }
}

struct EvalArgs {
  int d, p, n_query;
  double ctr[BSDE_DMAX + 1], sc[BSDE_DMAX + 1];
};

// u and du/dx_j at query points (Section 5.3: price V = u, Delta = grad_x V):
// one CTA per point, threads over basis functions, fixed-order reduction.
__global__ void __launch_bounds__(256) k_eval(const __grid_constant__ EvalArgs ea,
                                              const double* __restrict__ alpha,
                                              const uint2* __restrict__ pairs,
                                              const uint8_t* __restrict__ nnz,
                                              const double* __restrict__ qt,
                                              const double* __restrict__ qx,
                                              double* __restrict__ price,
                                              double* __restrict__ dudx) {
  __shared__ double red[256][BSDE_DMAX + 1];
  const int qi = blockIdx.x;
  const int d = ea.d;
  double xi[BSDE_DMAX + 1];
  xi[0] = (qt[qi] - ea.ctr[0]) * ea.sc[0];
  for (int j = 0; j < d; ++j) xi[j + 1] = (qx[(size_t)qi * d + j] - ea.ctr[j + 1]) * ea.sc[j + 1];
  double u = 0.0, g[BSDE_DMAX];
  for (int j = 0; j < d; ++j) g[j] = 0.0;
  for (int l = threadIdx.x; l < ea.p; l += 256) {
    const uint2 pr = pairs[l];
    const int nz = nnz[l];
    double tv[BSDE_NNZ_MAX], dv[BSDE_NNZ_MAX];
    int var[BSDE_NNZ_MAX];
    for (int a = 0; a < nz; ++a) {
      const uint32_t byte = ((a < 4 ? pr.x >> (8 * a) : pr.y >> (8 * (a - 4)))) & 0xffu;
      const int v = (int)(byte >> 4), e = (int)(byte & 15u);
      const double z = xi[v];
      double t0 = 1.0, t1 = z, d0 = 0.0, d1 = 1.0;
      for (int q = 2; q <= e; ++q) {
        const double t2 = 2.0 * z * t1 - t0, d2 = 2.0 * t1 + 2.0 * z * d1 - d0;
        t0 = t1; t1 = t2; d0 = d1; d1 = d2;
      }
      tv[a] = t1;
      dv[a] = d1;
      var[a] = v;
    }
    double val = 1.0;
    for (int a = 0; a < nz; ++a) val *= tv[a];
    u += alpha[l] * val;
    for (int a = 0; a < nz; ++a) {
      if (var[a] == 0) continue;
      double gd = dv[a];
      for (int c = 0; c < nz; ++c)
        if (c != a) gd *= tv[c];
      g[var[a] - 1] += alpha[l] * gd * ea.sc[var[a]];
    }
  }
  red[threadIdx.x][0] = u;
  for (int j = 0; j < d; ++j) red[threadIdx.x][j + 1] = g[j];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int j = 0; j <= d; ++j) red[threadIdx.x][j] += red[threadIdx.x + o][j];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    price[qi] = red[0][0];
    if (dudx)
      for (int j = 0; j < d; ++j) dudx[(size_t)qi * d + j] = red[0][j + 1];
  }
}

// read-out point (0, log S0) written into the report block
__global__ void k_x0(int d, double t0, const double* __restrict__ logS0, double* __restrict__ qt,
                     double* __restrict__ qx) {
  if (threadIdx.x == 0) qt[0] = t0;
  if (threadIdx.x < d) qx[threadIdx.x] = logS0[threadIdx.x];
}

__global__ void k_copy_price(int k, int d, double* __restrict__ out) {
  // out[OUT_PRICE] and dudx were written by k_eval; keep the per-iteration price
  if (threadIdx.x == 0 && k >= 0 && k < 64) out[OUT_PRICE_IT + k] = out[OUT_PRICE];
}

// monomial coefficients of u^k (basis of total degree <= 3): beta_m =
// sum over the CSR row m of coef * alpha_l, in FP64, with an FP32 copy
__global__ void k_cheb2mono(int pm, const int* __restrict__ row, const int* __restrict__ lidx,
                            const double* __restrict__ coef, const double* __restrict__ alpha,
                            double* __restrict__ beta, float* __restrict__ beta32) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= pm) return;
  double s = 0.0;
  for (int e = row[m]; e < row[m + 1]; ++e) s += coef[e] * alpha[lidx[e]];
  beta[m] = s;
  beta32[m] = (float)s;
}

// x (+)= Ainv b: warp per row, fixed shuffle order
__global__ void k_inv_gemv(int p, const double* __restrict__ Ainv, const double* __restrict__ b,
                           double* __restrict__ x, int accumulate) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= p) return;
  const double* a = Ainv + (size_t)row * p;
  double s = 0.0;
  for (int c = lane; c < p; c += 32) s += a[c] * b[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = accumulate ? x[row] + s : s;
}

}  // namespace

void launch_inverse(const ProblemDev& P, int nb, cudaStream_t st) {
  const size_t smem = (size_t)P.p * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chol_solve<<<dim3(P.p, nb), 256, smem, st>>>(P.A, P.p, P.dinv, nullptr, P.Ainv, 0);
}

void launch_inv_gemv(const ProblemDev& P, const double* b, double* x, int accumulate,
                     cudaStream_t st) {
  k_inv_gemv<<<(P.p * 32 + 255) / 256, 256, 0, st>>>(P.p, P.Ainv, b, x, accumulate);
}

void launch_cheb2mono(const ProblemDev& P, cudaStream_t st) {
  k_cheb2mono<<<(P.pm + 127) / 128, 128, 0, st>>>(P.pm, P.conv_row, P.conv_l, P.conv_c, P.alpha,
                                                   P.beta, P.beta32);
}

void launch_reduce_c(const ProblemDev& P, int M, cudaStream_t st) {
  const int count = P.shard_n > 0 ? P.shard_n : P.n;
  if (count <= 0) return;
  k_reduce_c<<<(count + 255) / 256, 256, 0, st>>>(P.shard_i0, count, P.chunks, M, P.partial, P.c);
}

void launch_gram_f64(const ProblemDev& P, cudaStream_t st) {
  const int T = (P.p + 31) / 32;
  k_gram_f64<<<T * (T + 1) / 2, 256, 0, st>>>(P.n, P.n_pad, P.p, P.B, P.A);
}

void launch_rhs(const ProblemDev& P, cudaStream_t st) {
  k_bt_times<<<P.p, 128, 0, st>>>(P.n, P.n_pad, P.p, P.B, P.c, nullptr, P.rhs);
}

void launch_cholesky(const ProblemDev& P, int nb, cudaStream_t st) {
  k_save_diag<<<dim3((P.p + 255) / 256, nb), 256, 0, st>>>(P.A, P.p, P.diag0);
  for (int j0 = 0; j0 < P.p; j0 += 32) {
    k_chol_diag<<<dim3(1, nb), 32, 0, st>>>(P.A, P.p, j0, P.status, P.diag0, P.dinv);
    const int m = P.p - j0 - 32;
    if (m > 0) {
      k_chol_trsm<<<dim3((m + 31) / 32, nb), 32, 0, st>>>(P.A, P.p, j0, P.dinv);
      const int T = (m + 31) / 32;
      k_chol_update<<<dim3(T * (T + 1) / 2, nb), 256, 0, st>>>(P.A, P.p, j0);
    }
  }
}

void launch_refine_residual(const ProblemDev& P, cudaStream_t st) {
  k_b_times<<<(P.n + 31) / 32, 256, 0, st>>>(P.n, P.n_pad, P.p, P.B, P.delta, P.v);
  k_bt_times<<<P.p, 128, 0, st>>>(P.n, P.n_pad, P.p, P.B, P.v, P.rhs, P.res);
}

void launch_update(const ProblemDev& P, int k, cudaStream_t st) {
  k_update<<<1, 256, 0, st>>>(P.p, k, P.alpha, P.alpha32, P.delta, P.out);
}

static EvalArgs eval_args(const ModelHost& m, const GridHost& g, const ProblemDev& P, int q) {
  EvalArgs ea;
  memset(&ea, 0, sizeof(ea));
  ea.d = m.d;
  ea.p = P.p;
  ea.n_query = q;
  for (int v = 0; v <= m.d; ++v) {
    ea.ctr[v] = 0.5 * (g.lo[v] + g.hi[v]);
    ea.sc[v] = 2.0 / (g.hi[v] - g.lo[v]);
  }
  return ea;
}

// price and du/dx at (0, log S0) after iteration k; the query point lives in
// the tail of the report block (OUT_SIZE .. OUT_SIZE + 1 + 2 d)
void launch_eval_x0(const ModelHost& m, const GridHost& g, const ProblemDev& P, int k,
                    cudaStream_t st) {
  double* qt = P.out + OUT_SIZE;
  double* qx = qt + 1;
  double* logS0 = qx + BSDE_DMAX;
  k_x0<<<1, 32, 0, st>>>(m.d, 0.0, logS0, qt, qx);
  const EvalArgs ea = eval_args(m, g, P, 1);
  k_eval<<<1, 256, 0, st>>>(ea, P.alpha, P.pairs, P.nnz, qt, qx, P.out + OUT_PRICE,
                            P.out + OUT_DUDX);
  k_copy_price<<<1, 32, 0, st>>>(k, m.d, P.out);
}

void launch_eval_points(const ModelHost& m, const GridHost& g, const ProblemDev& P, int q,
                        const double* t, const double* x, double* price, double* dudx,
                        cudaStream_t st) {
  const EvalArgs ea = eval_args(m, g, P, q);
  k_eval<<<q, 256, 0, st>>>(ea, P.alpha, P.pairs, P.nnz, t, x, price, dudx);
}
