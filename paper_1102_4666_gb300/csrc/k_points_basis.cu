// k_points_basis.cu -- the random points of Algorithm 2 and the basis matrix
// B_l(t_i, x_i) of the least-squares extrapolation (eq. lspb, Section 3.2.2).
#include "common.cuh"

namespace {

struct BoxArgs {
  double lo[BSDE_DMAX + 1], hi[BSDE_DMAX + 1];
};

// Algorithm 2, first step of iteration k: point i takes coordinate c from
// lane c%4 of the Philox block (c/4, i, 0, TAG_PTS<<24 | k) and maps the
// uniform u = (w + 1/2) 2^-32 onto [lo_c, hi_c].  Explicit _rn operations
// keep every rounding as written (no FMA contraction).
__global__ void k_points(int n, int dp, const uint32_t* __restrict__ key, uint32_t k,
                         const __grid_constant__ BoxArgs box, double* __restrict__ t,
                         double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Philox ph{key[0], key[1]};
  for (int blk = 0; blk * 4 < dp; ++blk) {
    const uint4 o = ph((uint32_t)blk, (uint32_t)i, 0u, (TAG_PTS << 24) | k);
    const uint32_t w[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
    for (int lane = 0; lane < 4; ++lane) {
      const int c = blk * 4 + lane;
      if (c >= dp) break;
      const double u = __dmul_rn((double)w[lane] + 0.5, 2.3283064365386962890625e-10);
      const double y = __dadd_rn(box.lo[c], __dmul_rn(__dsub_rn(box.hi[c], box.lo[c]), u));
      if (c == 0)
        t[i] = y;
      else
        x[(size_t)(c - 1) * n + i] = y;
    }
  }
}

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// B[l][i] = prod over the active variates v of T_{nu_lv}(xi_v(t_i, x_i)),
// xi_v = (2 y_v - (lo_v + hi_v)) / (hi_v - lo_v), Chebyshev T_e by the
// three-term recurrence.  Each thread first tabulates T_0..T_eta of its
// point's dp reduced coordinates in shared memory ([v][e][thread], read back
// only by the same thread), so that the FP64 division and recurrence run
// once per (point, variate) instead of once per (point, basis function,
// active variate); the products are then formed in the same order as the
// definition.  With split != 0 also writes the 3xTF32 operands of the
// tensor-core Gram: hi = tf32(fp32(B)), lo = tf32(fp32(B) - hi).
__global__ void k_basis(int n, int n_pad, int p, int dp, int eta, const uint2* __restrict__ pairs,
                        const uint8_t* __restrict__ nnz, const double* __restrict__ t,
                        const double* __restrict__ x, const __grid_constant__ BoxArgs box,
                        double* __restrict__ B, float* __restrict__ Bhi,
                        float* __restrict__ Blo, int split) {
  extern __shared__ double cheb[];
  const int tid = threadIdx.x, tpb = blockDim.x;
  const int i = blockIdx.x * tpb + tid;
  if (i >= n) return;
  const int ne = eta + 1;
  for (int v = 0; v < dp; ++v) {
    const double y = (v == 0) ? t[i] : x[(size_t)(v - 1) * n + i];
    const double xi = __ddiv_rn(__dsub_rn(__dmul_rn(2.0, y), __dadd_rn(box.lo[v], box.hi[v])),
                                __dsub_rn(box.hi[v], box.lo[v]));
    double* tv = cheb + (size_t)v * ne * tpb + tid;
    tv[0] = 1.0;
    if (eta >= 1) tv[tpb] = xi;
    double tm1 = 1.0, tc = xi;
    for (int e = 2; e <= eta; ++e) {
      const double tn = __dsub_rn(__dmul_rn(__dmul_rn(2.0, xi), tc), tm1);
      tm1 = tc;
      tc = tn;
      tv[(size_t)e * tpb] = tc;
    }
  }
  const int l0 = blockIdx.y * 32;
  const int l1 = min(p, l0 + 32);
  for (int l = l0; l < l1; ++l) {
    const uint2 pr = pairs[l];
    const int nz = nnz[l];
    double val = 1.0;
    for (int a = 0; a < nz; ++a) {
      const uint32_t byte = ((a < 4 ? pr.x >> (8 * a) : pr.y >> (8 * (a - 4)))) & 0xffu;
      const int v = (int)(byte >> 4), e = (int)(byte & 15u);
      val = __dmul_rn(val, cheb[((size_t)v * ne + e) * tpb + tid]);
    }
    B[(size_t)l * n_pad + i] = val;
    if (split) {
      const float b32 = __double2float_rn(val);
      const float hi = to_tf32(b32);
      const float lo = to_tf32(b32 - hi);
      Bhi[(size_t)l * n_pad + i] = hi;
      Blo[(size_t)l * n_pad + i] = lo;
    }
  }
}

}  // namespace

void launch_points(const ModelHost& m, const GridHost& g, const ProblemDev& P, uint32_t k,
                   cudaStream_t st) {
  BoxArgs box;
  for (int v = 0; v <= m.d; ++v) {
    box.lo[v] = g.lo[v];
    box.hi[v] = g.hi[v];
  }
  const int tpb = 128;
  k_points<<<(P.n + tpb - 1) / tpb, tpb, 0, st>>>(P.n, m.d + 1, P.key, k, box, P.t, P.x);
}

void launch_basis(const ModelHost& m, const GridHost& g, const ProblemDev& P, bool mixed,
                  cudaStream_t st) {
  BoxArgs box;
  for (int v = 0; v <= m.d; ++v) {
    box.lo[v] = g.lo[v];
    box.hi[v] = g.hi[v];
  }
  const int dp = m.d + 1, eta = P.eta < 1 ? 1 : P.eta;
  // Chebyshev table of T_0..T_eta per variate and thread, within 48 KB
  int tpb = 128;
  while (tpb > 32 && (size_t)dp * (eta + 1) * tpb * sizeof(double) > 48 * 1024) tpb >>= 1;
  const size_t smem = (size_t)dp * (eta + 1) * tpb * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_basis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((P.n + tpb - 1) / tpb, (P.p + 31) / 32);
  k_basis<<<grid, tpb, smem, st>>>(P.n, P.n_pad, P.p, dp, eta, P.pairs, P.nnz, P.t, P.x, box, P.B,
                                   P.Bhi, P.Blo, mixed ? 1 : 0);
}
