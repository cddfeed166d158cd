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
// three-term recurrence.  A CTA takes 32 consecutive points and a range of
// basis functions: its threads first tabulate T_0..T_eta of the points' dp
// reduced coordinates in shared memory ([v][e][point]), so that the FP64
// division and recurrence run once per (point, variate) and CTA; then each
// warp forms the basis functions l = warp, warp + warps, ... of the range,
// one lane per point (a 256-byte row segment of B per store), the products
// in the order of the definition.  With split != 0 also writes the 3xTF32
// operands of the tensor-core Gram: hi = tf32(fp32(B)), lo = tf32(fp32(B) -
// hi).  The basis functions are split over gridDim.y ranges only as far as
// needed for two CTAs per SM.
constexpr int BASIS_PTS = 32;  // points per CTA of k_basis, one per lane

__global__ void k_basis(int n, int n_pad, int p, int l_per, int dp, int eta,
                        const uint2* __restrict__ pairs, const uint8_t* __restrict__ nnz,
                        const double* __restrict__ t, const double* __restrict__ x,
                        const __grid_constant__ BoxArgs box, double* __restrict__ B,
                        float* __restrict__ Bhi, float* __restrict__ Blo, int split) {
  extern __shared__ double cheb[];  // [v][e][point]
  const int tid = threadIdx.x, nth = blockDim.x;
  const int i0 = blockIdx.x * BASIS_PTS;
  const int ne = eta + 1;
  for (int idx = tid; idx < dp * BASIS_PTS; idx += nth) {
    const int v = idx / BASIS_PTS, q = idx - v * BASIS_PTS;
    const int i = i0 + q;
    if (i >= n) continue;
    const double y = (v == 0) ? t[i] : x[(size_t)(v - 1) * n + i];
    const double xi = __ddiv_rn(__dsub_rn(__dmul_rn(2.0, y), __dadd_rn(box.lo[v], box.hi[v])),
                                __dsub_rn(box.hi[v], box.lo[v]));
    double* tv = cheb + (size_t)v * ne * BASIS_PTS + q;
    tv[0] = 1.0;
    if (eta >= 1) tv[BASIS_PTS] = xi;
    double tm1 = 1.0, tc = xi;
    for (int e = 2; e <= eta; ++e) {
      const double tn = __dsub_rn(__dmul_rn(__dmul_rn(2.0, xi), tc), tm1);
      tm1 = tc;
      tc = tn;
      tv[(size_t)e * BASIS_PTS] = tc;
    }
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int i = i0 + lane;
  if (i >= n) return;
  const int l0 = blockIdx.y * l_per;
  const int l1 = min(p, l0 + l_per);
  for (int l = l0 + warp; l < l1; l += nw) {
    const uint2 pr = pairs[l];
    const int nz = nnz[l];
    double val = 1.0;
    for (int a = 0; a < nz; ++a) {
      const uint32_t byte = ((a < 4 ? pr.x >> (8 * a) : pr.y >> (8 * (a - 4)))) & 0xffu;
      const int v = (int)(byte >> 4), e = (int)(byte & 15u);
      val = __dmul_rn(val, cheb[((size_t)v * ne + e) * BASIS_PTS + lane]);
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
  const int tpb = 128;
  const size_t smem = (size_t)dp * (eta + 1) * BASIS_PTS * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_basis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int gx = (P.n + BASIS_PTS - 1) / BASIS_PTS;
  const int want = (2 * device_sm_count() + gx - 1) / gx;
  int gy = (P.p + 31) / 32;
  if (gy > want) gy = want;
  if (gy < 1) gy = 1;
  const int l_per = (P.p + gy - 1) / gy;
  gy = (P.p + l_per - 1) / l_per;
  k_basis<<<dim3(gx, gy), tpb, smem, st>>>(P.n, P.n_pad, P.p, l_per, dp, eta, P.pairs, P.nnz, P.t, P.x,
                                            box, P.B, P.Bhi, P.Blo, mixed ? 1 : 0);
}
