// k_paths.cuh -- the hot kernel of Algorithm 2: for every point (t_i, x_i)
// and every path m, the Monte Carlo sample
//     a_m = (T - t_i) g1(tau, X_tau) + Phi(X_T) - u^k(T, X_T),
//     g1  = f(tau, X_tau, u^k) + d_t u^k + L^N u^k,   f(t,x,y) = -r y + lambda (Phi - y)^+
// (eq. psiN with g1 = f_{u^k} + (d_t + L^N) u^k and g2 = Phi - u^k, Section 3.1;
// penalised driver of eq. bsde-penal-2), summed per point.
//
// GB300 mapping: one CTA per (point, chunk of paths); each thread runs PPT
// paths one after the other, keeping the d-dimensional state in registers
// (D is a template parameter, so every per-asset loop is unrolled).  The
// normals of the Euler steps come from Philox4x32-10 in groups of G steps
// whose G*D normals are a whole number of Philox blocks, so the counter of
// every normal is a compile-time offset.  The time factors of the local
// volatility, the coefficients alpha and the multi-index table are staged
// in shared memory once per CTA.  The random time tau falls inside step s*;
// the main loop only records the states before and after step s* (behind a
// warp vote where registers allow, so that a warp none of whose paths is at
// its step s* skips the copies), and X_tau is drawn after the loop through a
// Brownian bridge.  u^k and its derivatives at (tau, X_tau) and u^k(T, X_T)
// come from per-thread Chebyshev tables in shared memory (layout
// [slot][thread], conflict-free), or from the monomial coefficients beta of
// u^k (converted from the Chebyshev coefficients once per iteration, constant
// correlation only): Horner loops for total degree <= 3 (EV_DENSE3) and for
// degree 4 at d <= 5 (EV_DENSE4), a compile-time recursion over the prefix
// tree of variate multisets for degree 4 at d >= 6 and degrees 5 and 6 at
// d <= 5 (EV_TREE4..6, FP32 paths); every index is a compile-time constant,
// so u and its derivatives stay in registers.  The warps of a CTA enter the
// larger of these evaluations together (a barrier before them) to share
// their instruction fetches.  Per-path samples are accumulated in FP64; the
// CTA reduces them by a fixed warp-shuffle tree into partial[i][chunk], so
// the result does not depend on scheduling.
#pragma once
#include "common.cuh"

namespace paths {

// volatility families: constant, a + phi(t) tanh(x - kappa) (sin/tanh),
// Dupire's, and a + phi(t) |tanh(x - kappa)| (abs/tanh)
enum { VK_CONST = 0, VK_TANH = 1, VK_DUPIRE = 2, VK_TANH_ABS = 3 };
// evaluation of u^k along the paths: per-thread Chebyshev tables, dense
// monomial Horner loops for total degree <= 3 (any d) or 4 (d <= 5), or the
// prefix-tree recursion for total degree EV (EV_TREE4..EV_TREE6)
enum { EV_TABLES = 0, EV_DENSE3 = 1, EV_DENSE4 = 2, EV_TREE4 = 4, EV_TREE5 = 5, EV_TREE6 = 6 };

// monomials of total degree <= 3 in dp variates: C(dp + 3, 3)
__host__ __device__ constexpr int ncubic(int dp) { return (dp + 3) * (dp + 2) * (dp + 1) / 6; }
// index of (a, b), a <= b, in the row-major upper triangle of a dp x dp matrix
__host__ __device__ constexpr int sym(int dp, int a, int b) { return a * dp - a * (a - 1) / 2 + (b - a); }

template <typename R, int D>
struct Args {
  R T, r, lam, K, s_dupire;
  // the per-asset constants read in pairs by packed FP32x2 instructions
  // start on 16-byte boundaries of the parameter bank
  alignas(16) R rd[D];  // r - delta_j
  R w[D];
  alignas(16) R va[D];
  R kappa[D];
  R L[D][D];        // lower Cholesky factor of the correlation
  alignas(16) R Ld[D];  // constant correlation: diagonal of L and its constant column below it
  alignas(16) R Lc[D];
  R Cp[D + 1][D + 1];  // correlation padded with a zero time row/column
  R ctr[D + 1], sc[D + 1];  // xi_v = (y_v - ctr_v) sc_v
  int N, M, n, p, eta, chunks, tpb, ppt, tab_stride;
  int i0;           // first point of the launch (a block of the points when sharded)
  int payoff, obstacle, vol_sin;
  R vb;
  R rho;  // constant correlation (dense evaluation)
  alignas(16) R kc[D];  // -2 log2(e) kappa_j: e^{2 (x - kappa)} = 2^{x 2 log2(e) + kc}
  uint32_t k;
  uint32_t key0, key1;  // Philox key
  uint32_t rk0[10], rk1[10];  // its ten round keys (kernel-parameter constants)
  const double* pt;
  const double* px;
  const R* alpha;
  const uint2* pairs;
  const uint8_t* nnz;
  double* partial;
};

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

template <typename R>
__device__ __forceinline__ R uniform_frac(uint32_t w);
template <>
__device__ __forceinline__ float uniform_frac<float>(uint32_t w) {
  return fmaf(__uint2float_rn(w), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}
template <>
__device__ __forceinline__ double uniform_frac<double>(uint32_t w) {
  return ((double)w + 0.5) * 2.3283064365386962890625e-10;
}

// Philox4x32-10 with the round keys read from the kernel parameters (the
// same function as Philox in common.cuh; the xor with the round key then
// takes its operand from the constant bank instead of a key-schedule add)
template <typename R, int D>
__device__ __forceinline__ uint4 philox_rk(const Args<R, D>& a, uint32_t c0, uint32_t c1,
                                           uint32_t c2, uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u;
    const uint64_t p1 = (uint64_t)c2 * 0xCD9E8D57u;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ a.rk0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ a.rk1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Philox4x32-10 for a stream of counters (c0, c1, c2, c3) of which only c0
// varies along a path: the parts of rounds 1 and 2 that depend on c1 = m
// (the path) and c2 = i are computed once per path (PhiloxFixed); the parts
// that depend on c0, c2 and c3 only are shared by the paths of a point
// (philox_prep, below).
struct PhiloxFixed {
  uint32_t n0;    // round 1: hi(c2 M1) ^ c1 ^ k0
  uint32_t lo1;   // round 1: lo(c2 M1)
  uint32_t hiA;   // round 2: hi(n0 M0)
  uint32_t loA;   // round 2: lo(n0 M0)
  uint32_t c3k;   // round 1: c3 ^ k1
};

template <typename R, int D>
__device__ __forceinline__ PhiloxFixed philox_fix(const Args<R, D>& a, uint32_t c1, uint32_t c2,
                                                  uint32_t c3) {
  PhiloxFixed f;
  const uint64_t p1 = (uint64_t)c2 * 0xCD9E8D57u;
  f.n0 = (uint32_t)(p1 >> 32) ^ c1 ^ a.rk0[0];
  f.lo1 = (uint32_t)p1;
  const uint64_t pA = (uint64_t)f.n0 * 0xD2511F53u;
  f.hiA = (uint32_t)(pA >> 32);
  f.loA = (uint32_t)pA;
  f.c3k = c3 ^ a.rk1[0];
  return f;
}

// The normals' blocks (b, m, i, tag) of all the paths of one point share
// (b, i, tag): rounds 1-3 of Philox4x32-10 contain products and xors of those
// words alone, which philox_prep computes once per block index and point
// (a table in shared memory), leaving each path one wide multiply and three
// xors for rounds 1-3 besides its own PhiloxFixed words:
//   round 1: (n0, lo(i M1), hi(b M0) ^ tag ^ k1_0, lo(b M0))
//   round 2: (hi(R1_2 M1) ^ lo(i M1) ^ k0_1, lo(R1_2 M1), hiA ^ V, loA),
//            V = lo(b M0) ^ k1_1
//   round 3: (hi(R2_2 M1) ^ W, lo(R2_2 M1), U1 ^ loA, U3),
//            W = lo(R1_2 M1) ^ k0_2, U1 = hi(R2_0 M0) ^ k1_2, U3 = lo(R2_0 M0)
// (R1_2 = round 1's word 2, R2_* = round 2's words); table entry (V, W, U1, U3).
template <typename R, int D>
__device__ __forceinline__ uint4 philox_prep(const Args<R, D>& a, uint32_t b, uint32_t c2,
                                             uint32_t c3) {
  const uint64_t p0 = (uint64_t)b * 0xD2511F53u;
  const uint32_t r1_2 = (uint32_t)(p0 >> 32) ^ c3 ^ a.rk1[0];
  const uint32_t r1_3 = (uint32_t)p0;
  const uint32_t r1_1 = (uint32_t)((uint64_t)c2 * 0xCD9E8D57u);
  const uint64_t p1 = (uint64_t)r1_2 * 0xCD9E8D57u;
  const uint32_t r2_0 = (uint32_t)(p1 >> 32) ^ r1_1 ^ a.rk0[1];
  const uint32_t r2_1 = (uint32_t)p1;
  const uint64_t q0 = (uint64_t)r2_0 * 0xD2511F53u;
  return make_uint4(r1_3 ^ a.rk1[1], r2_1 ^ a.rk0[2], (uint32_t)(q0 >> 32) ^ a.rk1[2], (uint32_t)q0);
}

// the block (b, m, i, tag) of a path from its PhiloxFixed words and the
// table entry of philox_prep for b: the same outputs as philox_rk
template <typename R, int D>
__device__ __forceinline__ uint4 philox_tab(const Args<R, D>& a, const PhiloxFixed& f, uint4 pre) {
  const uint64_t q1 = (uint64_t)(f.hiA ^ pre.x) * 0xCD9E8D57u;
  uint32_t c0 = (uint32_t)(q1 >> 32) ^ pre.y;
  uint32_t c1 = (uint32_t)q1;
  uint32_t c2 = pre.z ^ f.loA;
  uint32_t c3 = pre.w;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint64_t q0 = (uint64_t)c0 * 0xD2511F53u;
    const uint64_t qq = (uint64_t)c2 * 0xCD9E8D57u;
    const uint32_t n0 = (uint32_t)(qq >> 32) ^ c1 ^ a.rk0[r];
    const uint32_t n2 = (uint32_t)(q0 >> 32) ^ c3 ^ a.rk1[r];
    c1 = (uint32_t)qq;
    c3 = (uint32_t)q0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

// r = 1 / (e^{2 y} + 1), so that tanh(y) = 1 - 2 r, with y = x - kappa_j
// (ABS: y = |x - kappa_j|, since |tanh(x - kappa)| = tanh(|x - kappa|))
template <bool ABS, typename R, int D>
__device__ __forceinline__ R tanh_r(const Args<R, D>& a, int j, R xj) {
  if constexpr (sizeof(R) == 4) {
    float e, r;
    const float t = fmaf(xj, 2.8853900817779268f, a.kc[j]);  // 2 log2(e) (x - kappa)
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(ABS ? fabsf(t) : t));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.0f));
    return r;
  } else {
    const double y = xj - a.kappa[j];
    return 1.0 / (::exp(2.0 * (ABS ? ::fabs(y) : y)) + 1.0);
  }
}

// local volatility of asset j at the step whose table row is tabs.  The
// tanh families keep (A, B) = (a + phi, -2 phi) per step and asset, with phi
// the time factor, and sigma = A + B r: a + phi tanh(y) = a + phi (1 - 2 r).
template <int VK, typename R, int D>
__device__ __forceinline__ R sigma_j(const Args<R, D>& a, const R* tabs, int j, R xj) {
  if constexpr (VK == VK_CONST) {
    return a.va[j];
  } else if constexpr (VK == VK_TANH || VK == VK_TANH_ABS) {
    const R r = tanh_r<VK == VK_TANH_ABS>(a, j, xj);
    R A, B;
    if constexpr (sizeof(R) == 4) {
      A = tabs[4 * (j >> 1) + (j & 1)];
      B = tabs[4 * (j >> 1) + 2 + (j & 1)];
    } else {
      A = tabs[2 * j];
      B = tabs[2 * j + 1];
    }
    return A + B * r;
  } else {
    const R dev = Math<R>::exp(xj) * tabs[2] - a.s_dupire;
    return tabs[0] - tabs[1] * Math<R>::exp(R(-0.001) * dev * dev);
  }
}

template <typename R, int D>
__device__ __forceinline__ R basket_value(const Args<R, D>& a, const R* x, bool positive) {
  R s = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) s += a.w[j] * Math<R>::exp(x[j]);
  const R v = (a.payoff == 0) ? (a.K - s) : (s - a.K);
  return positive ? Math<R>::fmax(v, R(0)) : v;
}

// contribution of one basis function with NZ active variates
template <int NZ, typename R>
__device__ __forceinline__ void term(const R* __restrict__ tb, int S, int eta, int tpb, int tid,
                                     uint2 pr, const R* __restrict__ Cp, int dp, R al, R& u,
                                     R& g, R& uT) {
  if constexpr (NZ == 0) {
    u += al;
    uT += al;
  } else {
    R tv[NZ], td[NZ], s1[NZ], s2[NZ], tt[NZ];
    int var[NZ];
#pragma unroll
    for (int a = 0; a < NZ; ++a) {
      const uint32_t byte = (a < 4 ? (pr.x >> (8 * a)) : (pr.y >> (8 * (a - 4)))) & 0xffu;
      const int v = (int)(byte >> 4), e = (int)(byte & 15u);
      var[a] = v;
      const int base = (v * eta + e - 1) * tpb + tid;
      tv[a] = tb[base];
      td[a] = tb[base + S];
      s1[a] = tb[base + 2 * S];
      s2[a] = tb[base + 3 * S];
      tt[a] = tb[base + 4 * S];
    }
    R pre[NZ + 1], suf[NZ + 1];
    pre[0] = R(1);
    suf[NZ] = R(1);
#pragma unroll
    for (int a = 0; a < NZ; ++a) pre[a + 1] = pre[a] * tv[a];
#pragma unroll
    for (int a = NZ - 1; a >= 0; --a) suf[a] = suf[a + 1] * tv[a];
    R valT = tt[0];
#pragma unroll
    for (int a = 1; a < NZ; ++a) valT *= tt[a];
    R gen = 0;
#pragma unroll
    for (int a = 0; a < NZ; ++a) {
      const R ex = pre[a] * suf[a + 1];
      gen += (td[a] + R(0.5) * s2[a]) * ex;
    }
#pragma unroll
    for (int a = 0; a < NZ; ++a) {
#pragma unroll
      for (int b = a + 1; b < NZ; ++b) {
        R ex2 = R(1);
#pragma unroll
        for (int c = 0; c < NZ; ++c)
          if (c != a && c != b) ex2 *= tv[c];
        gen += Cp[var[a] * dp + var[b]] * s1[a] * s1[b] * ex2;
      }
    }
    u += al * pre[NZ];
    g += al * gen;
    uT += al * valT;
  }
}

// u^k, (d_t + L^N) u^k at z (the reduced (tau, X_tau)) and u^k at zT (the
// reduced (T, X_T)) from the monomial coefficients of total degree <= 3,
// ordered: constant, linear (a), quadratic (a <= b), cubic (a <= b <= c),
// each group lexicographic.  Nested Horner form
//   u = c + sum_i z_i (g_i + sum_{j>=i} z_j (q_ij + sum_{k>=j} t_ijk z_k)),
// evaluated on numbers carrying (value, derivative along bt, derivative and
// second derivative along st), where bt = (d xi_0/dt, b_j d xi_j/dx_j) and
// st = (0, sigma_j d xi_j/dx_j).  With a constant correlation rho,
//   1/2 sum_{jl} st_j st_l C_jl d2_jl u
//     = 1/2 [(1 - rho) sum_j st_j^2 d2_jj u + rho d2_st u],
// and the diagonal second derivatives come from the few monomials with a
// repeated variate.  Every loop runs over all DP variates with the
// triangle selected by a test on the indices: the trip counts are then
// compile-time constants at every nesting level, so the loops unroll
// completely and the vectors z, zT, bt and st stay in registers.
// CS = 2 (FP32 paths only): every coefficient is stored twice, and the four
// accumulations of the innermost level, (av, aT) += t (z_k, zT_k) and
// (ab, as) += t (bt_k, st_k), run as two packed FP32x2 multiply-adds on a
// (t, t) load (the same IEEE operations; st_0 = 0 adds an exact zero); the
// next level's (bv, bT) and (bb, bs) as three more (the sums of bb and bs
// then associate as (b + bt_j av) + z_j ab).
template <typename R, int D, int CS = 1>
__device__ __forceinline__ void eval_dense3(const Args<R, D>& a, const R* __restrict__ beta,
                                            const R (&z)[D + 1], const R (&zT)[D + 1],
                                            const R (&bt)[D + 1], const R (&st)[D + 1], R& u,
                                            R& gen, R& uT) {
  static_assert(CS == 1 || (CS == 2 && sizeof(R) == 4), "paired coefficients are FP32 only");
  constexpr int DP = D + 1;
  constexpr int NQ = DP * (DP + 1) / 2;
  const R* bg = beta + CS;
  const R* bq = bg + CS * DP;
  const R* bc3 = bq + CS * NQ;
  // one pass over the coefficients for both points: value, d_bt, d_st,
  // d2_st and the weighted Hessian diagonal at (tau, X_tau), value at (T, X_T)
  R uv = beta[0], ub = R(0), us = R(0), uss = R(0), diag = R(0), sT = beta[0];
  int iq = 0, it = 0;
#pragma unroll
  for (int i = 0; i < DP; ++i) {
    R bv = bg[CS * i], bb = R(0), bs = R(0), bss = R(0), bT = bg[CS * i];
    float2 BVT = make_float2(bv, bT), BBS = make_float2(0.f, 0.f);  // CS = 2: (bv, bT), (bb, bs)
#pragma unroll
    for (int j = 0; j < DP; ++j) {
      if (j < i) continue;
      const R q = bq[CS * iq++];
      R av = q, ab = R(0), as = R(0), aT = q;
      float2 AVT = make_float2(q, q), ABS = make_float2(0.f, 0.f);  // CS = 2: (av, aT), (ab, as)
      if (i == j && i > 0) diag += R(2) * st[i] * st[i] * q;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        if (k < j) continue;
        const R t = bc3[CS * it];
        if constexpr (CS == 2) {
          const float2 tt = reinterpret_cast<const float2*>(bc3)[it];
          AVT = __ffma2_rn(tt, make_float2(z[k], zT[k]), AVT);
          ABS = __ffma2_rn(tt, make_float2(bt[k], st[k]), ABS);
        } else {
          av += t * z[k];
          ab += t * bt[k];
          if (k > 0) as += t * st[k];
          aT += t * zT[k];
        }
        ++it;
        if (i == j && j < k && i > 0) diag += R(2) * st[i] * st[i] * t * z[k];
        if (i < j && j == k && j > 0) diag += R(2) * st[j] * st[j] * t * z[i];
        if (i == j && j == k && i > 0) diag += R(6) * st[i] * st[i] * t * z[i];
      }
      if constexpr (CS == 2) {
        av = AVT.x;
        aT = AVT.y;
        ab = ABS.x;
        as = ABS.y;
      }
      // (z_j, bt_j, st_j, 0) * (av, ab, as, 0)
      if constexpr (CS == 2) {
        // (bv, bT) += (z_j, zT_j) (av, aT); (bb, bs) += (bt_j, st_j) av + z_j (ab, as)
        BVT = __ffma2_rn(make_float2(z[j], zT[j]), make_float2(av, aT), BVT);
        BBS = __ffma2_rn(make_float2(bt[j], st[j]), make_float2(av, av), BBS);
        BBS = __ffma2_rn(make_float2(z[j], z[j]), make_float2(ab, as), BBS);
        if (j > 0) bss += R(2) * st[j] * as;
      } else {
        bv += z[j] * av;
        bb += z[j] * ab + bt[j] * av;
        if (j > 0) {
          bs += z[j] * as + st[j] * av;
          bss += R(2) * st[j] * as;
        } else {
          bs += z[j] * as;
        }
        bT += zT[j] * aT;
      }
      // keep the coefficient loads of one (i, j) group together: without
      // this fence the scheduler hoists all of them and runs out of registers
      asm volatile("" ::: "memory");
    }
    if constexpr (CS == 2) {
      bv = BVT.x;
      bT = BVT.y;
      bb = BBS.x;
      bs = BBS.y;
    }
    // (z_i, bt_i, st_i, 0) * (bv, bb, bs, bss)
    uv += z[i] * bv;
    ub += z[i] * bb + bt[i] * bv;
    if (i > 0) {
      us += z[i] * bs + st[i] * bv;
      uss += z[i] * bss + R(2) * st[i] * bs;
    } else {
      us += z[i] * bs;
      uss += z[i] * bss;
    }
    sT += zT[i] * bT;
  }
  uT = sT;
  (void)us;
  u = uv;
  gen = ub + R(0.5) * ((R(1) - a.rho) * diag + a.rho * uss);
}

// The same for a basis of total degree <= 4 (d <= 5), one more Horner level:
//   u = c + sum_i z_i (g_i + sum_{j>=i} z_j (q_ij + sum_{k>=j} z_k (t_ijk
//         + sum_{l>=k} f_ijkl z_l))),
// monomials ordered constant, linear, quadratic, cubic, quartic, each group
// lexicographic.  The weighted Hessian diagonal sum_v st_v^2 d2_vv u takes,
// from each monomial with a variate v repeated e >= 2 times, e (e - 1)
// st_v^2 times the product of its other factors; the index patterns are
// compile-time constants, so each coefficient gets only its own terms.
// CS = 2 (FP32 paths only): every coefficient is stored twice, and the four
// accumulations of the innermost level, (ev, eT) += f (z_l, zT_l) and
// (eb, es) += f (bt_l, st_l), run as two packed FP32x2 multiply-adds on an
// (f, f) load -- the same IEEE operations (st_0 = 0 adds an exact zero).
template <typename R, int D, int CS = 1>
__device__ __forceinline__ void eval_dense4(const Args<R, D>& a, const R* __restrict__ beta,
                                            const R (&z)[D + 1], const R (&zT)[D + 1],
                                            const R (&bt)[D + 1], const R (&st)[D + 1], R& u,
                                            R& gen, R& uT) {
  static_assert(CS == 1 || (CS == 2 && sizeof(R) == 4), "paired coefficients are FP32 only");
  constexpr int DP = D + 1;
  constexpr int NQ = DP * (DP + 1) / 2;
  constexpr int NC = DP * (DP + 1) * (DP + 2) / 6;
  const R* bg = beta + CS;
  const R* bq = bg + CS * DP;
  const R* bc3 = bq + CS * NQ;
  const R* bc4 = bc3 + CS * NC;
  R s2[DP];  // st_v^2
#pragma unroll
  for (int v = 0; v < DP; ++v) s2[v] = st[v] * st[v];
  R uv = beta[0], ub = R(0), us = R(0), uss = R(0), diag = R(0), sT = beta[0];
  int iq = 0, ic = 0, i4 = 0;
#pragma unroll
  for (int i = 0; i < DP; ++i) {
    R bv = bg[CS * i], bb = R(0), bs = R(0), bss = R(0), bT = bg[CS * i];
#pragma unroll
    for (int j = 0; j < DP; ++j) {
      if (j < i) continue;
      const R q = bq[CS * iq++];
      R av = q, ab = R(0), as = R(0), ass = R(0), aT = q;
      if (i == j && i > 0) diag += R(2) * s2[i] * q;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        if (k < j) continue;
        const R t = bc3[CS * ic++];
        R ev = t, eb = R(0), es = R(0), eT = t;
        float2 EVT = make_float2(t, t), EBS = make_float2(0.f, 0.f);  // CS = 2: (ev, eT), (eb, es)
        if (i == j && j < k && i > 0) diag += R(2) * s2[i] * t * z[k];
        if (i < j && j == k && j > 0) diag += R(2) * s2[j] * t * z[i];
        if (i == j && j == k && i > 0) diag += R(6) * s2[i] * t * z[i];
#pragma unroll
        for (int l = 0; l < DP; ++l) {
          if (l < k) continue;
          const R f = bc4[CS * i4];
          if constexpr (CS == 2) {
            const float2 ff = reinterpret_cast<const float2*>(bc4)[i4];
            EVT = __ffma2_rn(ff, make_float2(z[l], zT[l]), EVT);
            EBS = __ffma2_rn(ff, make_float2(bt[l], st[l]), EBS);
          } else {
            ev += f * z[l];
            eb += f * bt[l];
            if (l > 0) es += f * st[l];
            eT += f * zT[l];
          }
          ++i4;
          if (i == j && j == k && k == l) {
            if (i > 0) diag += R(12) * s2[i] * f * z[i] * z[i];
          } else if (i == j && j == k) {  // k < l
            if (i > 0) diag += R(6) * s2[i] * f * z[i] * z[l];
          } else if (j == k && k == l) {  // i < j
            if (j > 0) diag += R(6) * s2[j] * f * z[i] * z[j];
          } else if (i == j && k == l) {  // j < k
            if (i > 0) diag += R(2) * s2[i] * f * z[k] * z[k];
            if (k > 0) diag += R(2) * s2[k] * f * z[i] * z[i];
          } else if (i == j) {  // j < k < l
            if (i > 0) diag += R(2) * s2[i] * f * z[k] * z[l];
          } else if (j == k) {  // i < j, k < l
            if (j > 0) diag += R(2) * s2[j] * f * z[i] * z[l];
          } else if (k == l) {  // i < j < k
            if (k > 0) diag += R(2) * s2[k] * f * z[i] * z[j];
          }
        }
        if constexpr (CS == 2) {
          ev = EVT.x;
          eT = EVT.y;
          eb = EBS.x;
          es = EBS.y;
        }
        // (z_k, bt_k, st_k, 0) * (ev, eb, es, 0)
        av += z[k] * ev;
        ab += z[k] * eb + bt[k] * ev;
        if (k > 0) {
          as += z[k] * es + st[k] * ev;
          ass += R(2) * st[k] * es;
        } else {
          as += z[k] * es;
        }
        aT += zT[k] * eT;
        // keep the coefficient loads of one (i, j, k) group together
        asm volatile("" ::: "memory");
      }
      // (z_j, bt_j, st_j, 0) * (av, ab, as, ass)
      bv += z[j] * av;
      bb += z[j] * ab + bt[j] * av;
      if (j > 0) {
        bs += z[j] * as + st[j] * av;
        bss += z[j] * ass + R(2) * st[j] * as;
      } else {
        bs += z[j] * as;
        bss += z[j] * ass;
      }
      bT += zT[j] * aT;
    }
    // (z_i, bt_i, st_i, 0) * (bv, bb, bs, bss)
    uv += z[i] * bv;
    ub += z[i] * bb + bt[i] * bv;
    if (i > 0) {
      us += z[i] * bs + st[i] * bv;
      uss += z[i] * bss + R(2) * st[i] * bs;
    } else {
      us += z[i] * bs;
      uss += z[i] * bss;
    }
    sT += zT[i] * bT;
  }
  uT = sT;
  (void)us;
  u = uv;
  gen = ub + R(0.5) * ((R(1) - a.rho) * diag + a.rho * uss);
}

// ---------------------------------------------------------------------------
// Dense evaluation of a basis of any total degree ETA by recursion over the
// prefix tree of sorted variate multisets: node N (a multiset ending with
// variate w) carries Q_N = beta_N + sum_{x >= w} z_x Q_{N+x}, so that u is
// Q at the root.  Besides the value, its derivative along bt and its first
// and second derivatives along st (as in the loops above), each node
// returns
//   DG_N = sum_v st_v^2 d2_vv Q_N = sum_x (z_x DG_{N+x} + 2 st_x^2 SD_{N+x}),
//   SD_N = d_w Q_N = Q_{N+w} + z_w SD_{N+w},
// the derivative of Q_N with respect to its own last variate (only the child
// that repeats w depends on z_w).  The coefficients are stored in the
// depth-first pre-order of the tree; every index is a compile-time constant.
// ---------------------------------------------------------------------------
template <typename R>
struct TreeAcc {
  R v, b, s, ss, dg, sd, t;
};

// sorted multisets of size <= m over nvar variates: C(nvar + m, m)
__host__ __device__ constexpr int tree_size(int nvar, int m) {
  int r = 1;
  for (int i = 1; i <= m; ++i) r = r * (nvar + i) / i;
  return r;
}

template <typename R, int DP, int ETA, int DEPTH, int W, int IDX>
__device__ __forceinline__ void tree_node(const R* __restrict__ beta, const R (&z)[DP],
                                          const R (&zT)[DP], const R (&bt)[DP], const R (&st)[DP],
                                          const R (&s2x2)[DP], TreeAcc<R>& a);

// fold the children x = X .. DP-1 of a node at depth DEPTH (last variate W)
template <typename R, int DP, int ETA, int DEPTH, int W, int X, int IDX>
__device__ __forceinline__ void tree_children(const R* __restrict__ beta, const R (&z)[DP],
                                              const R (&zT)[DP], const R (&bt)[DP],
                                              const R (&st)[DP], const R (&s2x2)[DP],
                                              TreeAcc<R>& a) {
  if constexpr (X < DP) {
    TreeAcc<R> c;
    tree_node<R, DP, ETA, DEPTH + 1, X, IDX>(beta, z, zT, bt, st, s2x2, c);
    a.v += z[X] * c.v;
    a.b += z[X] * c.b + bt[X] * c.v;
    if constexpr (X > 0) {
      a.s += z[X] * c.s + st[X] * c.v;
      a.ss += z[X] * c.ss + R(2) * st[X] * c.s;
      a.dg += z[X] * c.dg + s2x2[X] * c.sd;
    } else {  // the time variate has no diffusion
      a.s += z[X] * c.s;
      a.ss += z[X] * c.ss;
      a.dg += z[X] * c.dg;
    }
    if constexpr (DEPTH > 0 && X == W) a.sd = c.v + z[X] * c.sd;
    a.t += zT[X] * c.t;
    tree_children<R, DP, ETA, DEPTH, W, X + 1, IDX + tree_size(DP - X, ETA - DEPTH - 1)>(
        beta, z, zT, bt, st, s2x2, a);
  }
}

template <typename R, int DP, int ETA, int DEPTH, int W, int IDX>
__device__ __forceinline__ void tree_node(const R* __restrict__ beta, const R (&z)[DP],
                                          const R (&zT)[DP], const R (&bt)[DP], const R (&st)[DP],
                                          const R (&s2x2)[DP], TreeAcc<R>& a) {
  const R c0 = beta[IDX];
  a.v = c0;
  a.t = c0;
  a.b = a.s = a.ss = a.dg = a.sd = R(0);
  if constexpr (DEPTH < ETA) {
    tree_children<R, DP, ETA, DEPTH, W, (DEPTH == 0 ? 0 : W), IDX + 1>(beta, z, zT, bt, st, s2x2,
                                                                      a);
    // keep the coefficient loads of one group of leaves together
    if constexpr (DEPTH == ETA - 1) asm volatile("" ::: "memory");
  }
}

template <typename R, int D, int ETA>
__device__ __forceinline__ void eval_tree(const Args<R, D>& a, const R* __restrict__ beta,
                                          const R (&z)[D + 1], const R (&zT)[D + 1],
                                          const R (&bt)[D + 1], const R (&st)[D + 1], R& u,
                                          R& gen, R& uT) {
  constexpr int DP = D + 1;
  R s2x2[DP];
#pragma unroll
  for (int v = 0; v < DP; ++v) s2x2[v] = R(2) * st[v] * st[v];
  TreeAcc<R> r;
  tree_node<R, DP, ETA, 0, 0, 0>(beta, z, zT, bt, st, s2x2, r);
  u = r.v;
  uT = r.t;
  gen = r.b + R(0.5) * ((R(1) - a.rho) * r.dg + a.rho * r.ss);
}

// The tree recursion with FP32 paths, the leaves folded in packed FP32x2: a
// leaf carries only its coefficient c (every derivative of its Q is zero), so
// its parent adds (z_x, zT_x) c to (Q, T) and (bt_x, st_x) c to (B, S) in two
// __ffma2_rn, the coefficients stored twice in shared memory so that one
// 64-bit load gives (c, c).  The interior folds are those of tree_children.
// The same IEEE operations as tree_node up to additions of exact zeros (the
// leaves' zero derivatives, st_0 = 0), so the same results.
struct TreeAcc2 {
  float2 vt;  // (Q, T): value at (tau, X_tau) and at (T, X_T)
  float2 bs;  // (B, S): derivatives along bt and st
  float ss, dg, sd;
};

template <int DP, int ETA, int DEPTH, int W, int IDX>
__device__ __forceinline__ void tree_node2(const float2* __restrict__ beta2, const float2 (&PVT)[DP],
                                           const float2 (&PBS)[DP], const float (&s2x2)[DP],
                                           TreeAcc2& a);

template <int DP, int ETA, int DEPTH, int W, int X, int IDX>
__device__ __forceinline__ void tree_children2(const float2* __restrict__ beta2, const float2 (&PVT)[DP],
                                               const float2 (&PBS)[DP], const float (&s2x2)[DP],
                                               TreeAcc2& a) {
  if constexpr (X < DP) {
    if constexpr (DEPTH + 1 == ETA) {
      const float2 cc = beta2[IDX];
      a.vt = __ffma2_rn(PVT[X], cc, a.vt);
      a.bs = __ffma2_rn(PBS[X], cc, a.bs);
      if constexpr (DEPTH > 0 && X == W) a.sd = cc.x;
    } else {
      TreeAcc2 c;
      tree_node2<DP, ETA, DEPTH + 1, X, IDX>(beta2, PVT, PBS, s2x2, c);
      const float zx = PVT[X].x, zTx = PVT[X].y, btx = PBS[X].x, stx = PBS[X].y;
      a.vt.x += zx * c.vt.x;
      a.bs.x += zx * c.bs.x + btx * c.vt.x;
      if constexpr (X > 0) {
        a.bs.y += zx * c.bs.y + stx * c.vt.x;
        a.ss += zx * c.ss + 2.f * stx * c.bs.y;
        a.dg += zx * c.dg + s2x2[X] * c.sd;
      } else {  // the time variate has no diffusion
        a.bs.y += zx * c.bs.y;
        a.ss += zx * c.ss;
        a.dg += zx * c.dg;
      }
      if constexpr (DEPTH > 0 && X == W) a.sd = c.vt.x + zx * c.sd;
      a.vt.y += zTx * c.vt.y;
    }
    tree_children2<DP, ETA, DEPTH, W, X + 1, IDX + tree_size(DP - X, ETA - DEPTH - 1)>(beta2, PVT, PBS,
                                                                                      s2x2, a);
  }
}

template <int DP, int ETA, int DEPTH, int W, int IDX>
__device__ __forceinline__ void tree_node2(const float2* __restrict__ beta2, const float2 (&PVT)[DP],
                                           const float2 (&PBS)[DP], const float (&s2x2)[DP],
                                           TreeAcc2& a) {
  const float c0 = beta2[IDX].x;
  a.vt = make_float2(c0, c0);
  a.bs = make_float2(0.f, 0.f);
  a.ss = a.dg = a.sd = 0.f;
  if constexpr (DEPTH < ETA) {
    tree_children2<DP, ETA, DEPTH, W, (DEPTH == 0 ? 0 : W), IDX + 1>(beta2, PVT, PBS, s2x2, a);
    // keep the coefficient loads of one group of leaves together
    if constexpr (DEPTH == ETA - 1) asm volatile("" ::: "memory");
  }
}

// PVT[v] = (z_v, zT_v), PBS[v] = (bt_v, st_v): the reduced coordinates of
// both evaluation points and the drift and diffusion directions
template <int D, int ETA>
__device__ __forceinline__ void eval_tree_x2(const Args<float, D>& a, const float2* __restrict__ beta2,
                                             const float2 (&PVT)[D + 1], const float2 (&PBS)[D + 1],
                                             float& u, float& gen, float& uT) {
  constexpr int DP = D + 1;
  float s2x2[DP];
#pragma unroll
  for (int v = 0; v < DP; ++v) s2x2[v] = 2.f * PBS[v].y * PBS[v].y;
  TreeAcc2 r;
  tree_node2<DP, ETA, 0, 0, 0>(beta2, PVT, PBS, s2x2, r);
  u = r.vt.x;
  uT = r.vt.y;
  gen = r.bs.x + 0.5f * ((1.f - a.rho) * r.dg + a.rho * r.ss);
}

// correlated increment y = sqrt(h) (L Z)_j of asset j (prefix sum `pre` of
// the constant-correlation factor, or the triangular product)
template <bool CC, int G, typename R, int D>
__device__ __forceinline__ R corr_inc(const Args<R, D>& a, const R (&z)[G * D], int gs, int j, R& pre) {
  if constexpr (CC) {
    const R y = a.Ld[j] * z[gs * D + j] + pre;
    pre += a.Lc[j] * z[gs * D + j];
    return y;
  } else {
    R y = 0;
#pragma unroll
    for (int q = 0; q <= j; ++q) y += a.L[j][q] * z[gs * D + q];
    return y;
  }
}

// One Euler step of every asset of X (in place), with the sqrt(h)-scaled
// normals z[gs D .. gs D + D) of a group of G steps and the volatility row
// tabs of the step: X_j += h (r - delta_j) + sigma_j (y_j - h sigma_j / 2),
// y = sqrt(h) (L Z)_j, sigma_j at (t_s, X_s).  The main loop and the
// reconstruction of the states around the random time both call it, so the
// two compute the same numbers.
template <int VK, bool CC, int G, typename R, int D>
__device__ __forceinline__ void euler_step(const Args<R, D>& a, const R* tabs, const R (&z)[G * D],
                                           int gs, R nhh, R h, R (&X)[D]) {
  R pre = 0;  // running sum of the constant-correlation factor
  if constexpr ((VK == VK_TANH || VK == VK_TANH_ABS) && sizeof(R) == 4) {
    // FP32 tanh families: assets in pairs, the pair's table row
    // (A_j, A_j+1, B_j, B_j+1) in one 128-bit load, and the pair's
    // arithmetic in packed FP32x2 instructions (the same IEEE operations as
    // the scalar form, half the instructions)
#pragma unroll
    for (int j = 0; j < D; j += 2) {
      const float4 q4 = reinterpret_cast<const float4*>(tabs)[j >> 1];
      if (j + 1 < D) {
        float y0, y1;
        if constexpr (CC) {
          // (y_j, y_j+1) = (Ld_j, Ld_j+1) (z_j, z_j+1) + (pre, pre + Lc_j z_j)
          const float p1 = fmaf(a.Lc[j], z[gs * D + j], pre);
          const float2 yy = __ffma2_rn(make_float2(a.Ld[j], a.Ld[j + 1]),
                                       make_float2(z[gs * D + j], z[gs * D + j + 1]), make_float2(pre, p1));
          pre = fmaf(a.Lc[j + 1], z[gs * D + j + 1], p1);
          y0 = yy.x;
          y1 = yy.y;
        } else {
          y0 = corr_inc<CC, G>(a, z, gs, j, pre);
          y1 = corr_inc<CC, G>(a, z, gs, j + 1, pre);
        }
        const float2 xx = make_float2(X[j], X[j + 1]);
        float2 t = __ffma2_rn(xx, make_float2(2.8853900817779268f, 2.8853900817779268f),
                              make_float2(a.kc[j], a.kc[j + 1]));  // 2 log2(e) (x - kappa)
        if constexpr (VK == VK_TANH_ABS) t = make_float2(fabsf(t.x), fabsf(t.y));
        float e0, e1, r0, r1;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(t.x));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(t.y));
        const float2 ep = __fadd2_rn(make_float2(e0, e1), make_float2(1.0f, 1.0f));
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(ep.x));
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(ep.y));
        const float2 sig = __ffma2_rn(make_float2(q4.z, q4.w), make_float2(r0, r1), make_float2(q4.x, q4.y));
        // X + h rd_j + sigma (y - h sigma / 2)
        const float2 in = __ffma2_rn(make_float2(nhh, nhh), sig, make_float2(y0, y1));
        const float2 base = __ffma2_rn(make_float2(h, h), make_float2(a.rd[j], a.rd[j + 1]), xx);
        const float2 xn = __ffma2_rn(sig, in, base);
        X[j] = xn.x;
        X[j + 1] = xn.y;
      } else {
        const R y0 = corr_inc<CC, G>(a, z, gs, j, pre);
        const R r = tanh_r<VK == VK_TANH_ABS>(a, j, X[j]);
        const R sig = q4.x + q4.z * r;
        X[j] = sig * (nhh * sig + y0) + (h * a.rd[j] + X[j]);
      }
    }
  } else if constexpr (VK == VK_CONST && sizeof(R) == 4) {
    // constant volatilities: the update of a pair of assets in packed FP32x2
#pragma unroll
    for (int j = 0; j < D; j += 2) {
      const R y0 = corr_inc<CC, G>(a, z, gs, j, pre);
      if (j + 1 < D) {
        const R y1 = corr_inc<CC, G>(a, z, gs, j + 1, pre);
        const float2 xx = make_float2(X[j], X[j + 1]);
        const float2 sig = make_float2(a.va[j], a.va[j + 1]);
        const float2 in = __ffma2_rn(make_float2(nhh, nhh), sig, make_float2(y0, y1));
        const float2 base = __ffma2_rn(make_float2(h, h), make_float2(a.rd[j], a.rd[j + 1]), xx);
        const float2 xn = __ffma2_rn(sig, in, base);
        X[j] = xn.x;
        X[j + 1] = xn.y;
      } else {
        const R sig = a.va[j];
        X[j] = sig * (nhh * sig + y0) + (h * a.rd[j] + X[j]);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const R y = corr_inc<CC, G>(a, z, gs, j, pre);
      const R sig = sigma_j<VK>(a, tabs, j, X[j]);
      // X + (r - delta_j - sigma^2/2) h + sigma y = X + h rd_j + sigma (y - h sigma / 2)
      X[j] = sig * (nhh * sig + y) + (h * a.rd[j] + X[j]);
    }
  }
}

// The states before and after the step s* that contains the random time
// tau (the Brownian bridge needs both) are kept one of three ways:
// * in shared memory (copy_smem): a predicated 128-bit store per four assets
//   before and after every step, no registers held for the copies;
// * behind a warp vote (copy_vote), which skips the copies in the ~3/4 of
//   the steps where no lane of the warp is at its s*; with FP32 paths the
//   state is then copied once per group of G steps and the group's steps are
//   taken again after the loop (its normals drawn again);
// * as predicated register moves before and after every step.
// The same function takes each step, so the results do not depend on which.
// Measured per launch (FP32): the shared-memory copies against the register
// moves d = 10 degree 3 17.18 -> 16.84 ms, d = 6 degree 3 0.896 -> 0.887 ms,
// d = 10 degree 4 4.84 -> 4.77 ms; against the vote and second pass d = 5
// degree 4 3.42 -> 3.31 ms, degree 5 3.38 -> 3.26 ms, degree 6 4.63 -> 4.54
// ms, but d = 4 degree 4 2.08 -> 2.14 ms (G = 1: the second pass is one
// step) and d = 3 degree 3 0.104 -> 0.106 ms; FP64 paths keep the registers
// (and the vote).
__host__ __device__ constexpr bool copy_vote(int ev, int d) {
  return d >= 3 && ev != EV_DENSE3 && !(ev >= EV_TREE4 && d >= 6);
}
__host__ __device__ constexpr bool copy_smem(int ev, bool fp32, int d) {
  return fp32 && ev != EV_TABLES && d >= 4 && !(copy_vote(ev, d) && d % 4 == 0);
}

// A thread's d-dimensional FP32 state as ceil(d / 4) float4 in a
// [quad][thread] array of row length `stride` (zero padding past d).
template <int D, typename R>
__device__ __forceinline__ void store_state(float4* p, int stride, const R (&X)[D]) {
#pragma unroll
  for (int q = 0; q < (D + 3) / 4; ++q) {
    const int j = 4 * q;
    p[(size_t)q * stride] = make_float4(X[j], j + 1 < D ? X[j + 1] : 0.f, j + 2 < D ? X[j + 2] : 0.f,
                                        j + 3 < D ? X[j + 3] : 0.f);
  }
}
template <int D, typename R>
__device__ __forceinline__ void load_state(const float4* p, int stride, R (&X)[D]) {
#pragma unroll
  for (int q = 0; q < (D + 3) / 4; ++q) {
    const float4 v = p[(size_t)q * stride];
    const int j = 4 * q;
    X[j] = v.x;
    if (j + 1 < D) X[j + 1] = v.y;
    if (j + 2 < D) X[j + 2] = v.z;
    if (j + 3 < D) X[j + 3] = v.w;
  }
}

// One CTA's work: a point and a chunk of its paths (the kernels below).
template <int VK, int EV, bool CC, typename R, int D>
__device__ __forceinline__ void paths_cta(const Args<R, D>& a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int DP = D + 1;
  const int tid = threadIdx.x;
  const int tpb = a.tpb;
  const int item = blockIdx.x;
  const int il = item / a.chunks;
  const int chunk = item - il * a.chunks;
  const int i = a.i0 + il;

  // shared memory carve-up (dense evaluation: no multi-index or Chebyshev
  // tables; alpha holds the monomial coefficients, p of them)
  // the dense evaluations with FP32 paths keep every coefficient twice
  // (eval_tree_x2, eval_dense3 and eval_dense4 with CS = 2)
  constexpr bool PAIRS = EV != EV_TABLES && sizeof(R) == 4;
  R* tab = reinterpret_cast<R*>(smem_raw);                         // N x tab_stride
  R* s_alpha;                                                       // p (2 p with PAIRS)
  R* s_cp;                                                          // DP x DP
  size_t off;
  if constexpr (PAIRS) {
    // 16-byte aligned for the float2 loads of the coefficient pairs
    const size_t aoff = ((size_t)a.N * a.tab_stride * sizeof(R) + 15) & ~(size_t)15;
    s_alpha = reinterpret_cast<R*>(smem_raw + aoff);
    s_cp = s_alpha + 2 * a.p;
    off = aoff + ((size_t)2 * a.p + DP * DP) * sizeof(R);
  } else {
    s_alpha = tab + (size_t)a.N * a.tab_stride;
    s_cp = s_alpha + a.p;
    off = ((size_t)a.N * a.tab_stride + a.p + DP * DP) * sizeof(R);
  }
  off = (off + 15) & ~(size_t)15;
  uint2* s_pairs = reinterpret_cast<uint2*>(smem_raw + off);
  uint8_t* s_nnz = smem_raw + off;
  R* cheb = reinterpret_cast<R*>(smem_raw + off);                  // 5 x DP x eta x tpb
  const int S = DP * a.eta * tpb;
  if constexpr (EV == EV_TABLES) {
    off += (size_t)a.p * sizeof(uint2);
    s_nnz = smem_raw + off;
    off += ((size_t)a.p + 15) & ~(size_t)15;
    cheb = reinterpret_cast<R*>(smem_raw + off);
    off += (size_t)5 * S * sizeof(R);
    off = (off + 15) & ~(size_t)15;
  }
  double* red = reinterpret_cast<double*>(smem_raw + off);          // 32
  // rounds 1-3 of the normals' Philox blocks (philox_prep), per block index
  uint4* s_ph = reinterpret_cast<uint4*>(smem_raw + off + 32 * sizeof(double));
  // the states before and after step s* (copy_smem): [copy][quad][thread]
  // float4 after the Philox table
  constexpr bool XCOPY = copy_smem(EV, sizeof(R) == 4, D);
  constexpr int NQ = (D + 3) / 4;
  float4* s_xc = reinterpret_cast<float4*>(s_ph + (a.N + (4 / gcd_c(D, 4)) - 1) / (4 / gcd_c(D, 4)) *
                                                     ((4 / gcd_c(D, 4)) * D / 4));

  const R ti = (R)a.pt[i];
  R x0[D];
#pragma unroll
  for (int j = 0; j < D; ++j) x0[j] = (R)a.px[(size_t)j * a.n + i];
  const R h = (a.T - ti) / (R)a.N;
  const R sqh = Math<R>::sqrt(h);
  const R bmk = Math<R>::bm_factor(sqh);  // Box-Muller radius factor of the step normals
  const R bm1 = Math<R>::bm_factor(R(1));

  // per-step coefficients of the local volatility (in the precision of the
  // path: accurate sinf/expf for FP32, sin/exp for FP64)
  for (int idx = tid; idx < a.N * a.tab_stride; idx += tpb) {
    const int s = idx / a.tab_stride, c = idx - s * a.tab_stride;
    const R ts = ti + (R)s * h;
    R v = 0;
    if constexpr (VK == VK_TANH || VK == VK_TANH_ABS) {
      // FP32 rows: (A_j, A_j+1, B_j, B_j+1) per pair of assets, so that one
      // 128-bit load gives the pair's A and B as two float2; FP64 rows:
      // (A_j, B_j) per asset
      const int j = sizeof(R) == 4 ? 2 * (c >> 2) + (c & 1) : c >> 1;
      const bool isB = sizeof(R) == 4 ? ((c >> 1) & 1) != 0 : (c & 1) != 0;
      const R phi = a.vol_sin ? a.vb * Math<R>::sin((R)(j + 1) + ts) : a.vb * Math<R>::exp_acc(-ts);
      v = isB ? R(-2) * phi : a.va[j < D ? j : 0] + phi;
    } else if constexpr (VK == VK_DUPIRE) {
      const R ew = Math<R>::exp_acc(R(-0.05) * Math<R>::sqrt(ts));
      v = (c == 0) ? R(0.72) * ew
                   : (c == 1) ? R(0.6) * Math<R>::exp_acc(R(-0.1) * ts) * ew : Math<R>::exp_acc(a.r * ts);
    }
    tab[idx] = v;
  }
  for (int l = tid; l < a.p; l += tpb) {
    if constexpr (PAIRS) {
      s_alpha[2 * l] = a.alpha[l];
      s_alpha[2 * l + 1] = a.alpha[l];
    } else {
      s_alpha[l] = a.alpha[l];
    }
    if constexpr (EV == EV_TABLES) {
      s_pairs[l] = a.pairs[l];
      s_nnz[l] = a.nnz[l];
    }
  }
  for (int q = tid; q < DP * DP; q += tpb) s_cp[q] = (&a.Cp[0][0])[q];
  const uint32_t tagU = (TAG_U << 24) | a.k, tagZ = (TAG_Z << 24) | a.k, tagB = (TAG_B << 24) | a.k;
  constexpr int G = 4 / gcd_c(D, 4);  // steps per group: G*D normals = whole Philox blocks
  constexpr int NB = G * D / 4;
  constexpr int NBB = (D + 3) / 4;
  {
    const int nblk = (a.N + G - 1) / G * NB;
    for (int b = tid; b < nblk; b += tpb) s_ph[b] = philox_prep(a, (uint32_t)b, (uint32_t)i, tagZ);
  }
  __syncthreads();
  const int ppc = tpb * a.ppt;
  double acc = 0.0;

  // The degree-4 and prefix-tree evaluations are tens of kilobytes of
  // straight-line code run once per path: the warps of a CTA enter them
  // together (a barrier before them), so that one warp's instruction fetches
  // serve the others.  The loop then runs the same number of paths on every
  // thread of the CTA; threads past the last path compute one that is
  // discarded.  (Measured: d = 10 degree 4 16.1 -> 7.4 ms, d = 5 degree 4
  // 4.02 -> 3.75 ms; the degree-3 loops at d = 10 lose 2 % with it.)
  constexpr bool SYNC_EVAL = EV == EV_DENSE4 || EV >= EV_TREE4;
  for (int jp = 0; jp < a.ppt; ++jp) {
    const int m = chunk * ppc + jp * tpb + tid;
    if constexpr (SYNC_EVAL) {
      if (chunk * ppc + jp * tpb >= a.M) break;  // no path left in the CTA
    } else {
      if (m >= a.M) break;
    }
    // the uniform random time: U = (s* + theta) / N from one 32-bit word
    const uint4 ou = philox_rk(a, 0u, (uint32_t)m, (uint32_t)i, tagU);
    const uint64_t wN = (uint64_t)ou.x * (uint64_t)a.N;
    const int sstar = (int)(wN >> 32);
    const R theta = uniform_frac<R>((uint32_t)wN);

    // the states before and after step s* (copy_vote, copy_smem); the vote
    // is over the lanes that reach a copy together, and a lane whose copy is
    // due always votes for itself, so it is never skipped
    constexpr bool VOTE = copy_vote(EV, D) && !XCOPY;
    constexpr bool REBUILD = sizeof(R) == 4 && VOTE;
    const int g_hit = sstar - sstar % G;  // first step of the group that contains s*
    R X[D], Xg[D], Xs[D], Xn[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      X[j] = x0[j];
      Xg[j] = x0[j];
      Xs[j] = x0[j];
      Xn[j] = x0[j];
    }
    const R nhh = R(-0.5) * h;
    const PhiloxFixed pz = philox_fix(a, (uint32_t)m, (uint32_t)i, tagZ);
    for (int s0 = 0; s0 < a.N; s0 += G) {
      R z[G * D];  // normals of G steps, scaled by sqrt(h)
      const uint32_t blk0 = (uint32_t)(s0 / G) * (uint32_t)NB;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const uint4 o = philox_tab(a, pz, s_ph[blk0 + b]);
        Math<R>::box_muller(o.x, o.y, z[4 * b + 0], z[4 * b + 1], bmk);
        Math<R>::box_muller(o.z, o.w, z[4 * b + 2], z[4 * b + 3], bmk);
      }
      if constexpr (REBUILD) {
        const bool hit = (s0 == g_hit);
        const bool any_hit = VOTE ? __any_sync(__activemask(), hit) : true;
        if (any_hit) {
#pragma unroll
          for (int j = 0; j < D; ++j)
            if (hit) Xg[j] = X[j];
        }
      }
#pragma unroll
      for (int gs = 0; gs < G; ++gs) {
        const int s = s0 + gs;
        if (s < a.N) {
          if constexpr (REBUILD) {
            euler_step<VK, CC, G>(a, tab + s * a.tab_stride, z, gs, nhh, h, X);
          } else if constexpr (XCOPY) {
            const bool hit = (s == sstar);
            if (hit) store_state<D>(s_xc + tid, tpb, X);
            euler_step<VK, CC, G>(a, tab + s * a.tab_stride, z, gs, nhh, h, X);
            if (hit) store_state<D>(s_xc + (size_t)NQ * tpb + tid, tpb, X);
          } else {
            const bool hit = (s == sstar);
            const bool any_hit = VOTE ? __any_sync(__activemask(), hit) : true;
            if (any_hit) {
#pragma unroll
              for (int j = 0; j < D; ++j)
                if (hit) Xs[j] = X[j];
            }
            euler_step<VK, CC, G>(a, tab + s * a.tab_stride, z, gs, nhh, h, X);
            if (any_hit) {
#pragma unroll
              for (int j = 0; j < D; ++j)
                if (hit) Xn[j] = X[j];
            }
          }
        }
      }
    }

    if constexpr (REBUILD) {
      // X before and after step s*: the group's normals drawn again (the
      // same counters) and its steps taken again from the copy at its start
      R zr[G * D];
      const uint32_t blk0 = (uint32_t)(g_hit / G) * (uint32_t)NB;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const uint4 o = philox_tab(a, pz, s_ph[blk0 + b]);
        Math<R>::box_muller(o.x, o.y, zr[4 * b + 0], zr[4 * b + 1], bmk);
        Math<R>::box_muller(o.z, o.w, zr[4 * b + 2], zr[4 * b + 3], bmk);
      }
#pragma unroll
      for (int j = 0; j < D; ++j) Xs[j] = Xg[j];
#pragma unroll
      for (int gs = 0; gs < G; ++gs) {
        // steps past s* (and past the last step) are not needed; their table
        // row is clamped so that every read stays in the table
        const int s = g_hit + gs;
        const int row = s < a.N ? s : a.N - 1;
        if (gs > 0) {
#pragma unroll
          for (int j = 0; j < D; ++j)
            if (s <= sstar) Xs[j] = Xg[j];
        }
        euler_step<VK, CC, G>(a, tab + row * a.tab_stride, zr, gs, nhh, h, Xg);
#pragma unroll
        for (int j = 0; j < D; ++j)
          if (s == sstar) Xn[j] = Xg[j];
      }
    }

    if constexpr (XCOPY) {
      load_state<D>(s_xc + tid, tpb, Xs);
      load_state<D>(s_xc + (size_t)NQ * tpb + tid, tpb, Xn);
    }

    // X at tau: Brownian bridge inside step s*, coefficients frozen at t_{s*}
    R zb[NBB * 4];
#pragma unroll
    for (int b = 0; b < NBB; ++b) {
      const uint4 o = philox_rk(a, (uint32_t)b, (uint32_t)m, (uint32_t)i, tagB);
      Math<R>::box_muller(o.x, o.y, zb[4 * b + 0], zb[4 * b + 1], bm1);
      Math<R>::box_muller(o.z, o.w, zb[4 * b + 2], zb[4 * b + 3], bm1);
    }
    const R* tab_s = tab + sstar * a.tab_stride;
    const R bb = Math<R>::sqrt(theta * (R(1) - theta) * h);
    R Xtau[D], sig_s[D], drift_s[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      R y = 0;
#pragma unroll
      for (int q = 0; q <= j; ++q) y += a.L[j][q] * zb[q];
      sig_s[j] = sigma_j<VK>(a, tab_s, j, Xs[j]);
      drift_s[j] = a.rd[j] - R(0.5) * sig_s[j] * sig_s[j];
      Xtau[j] = Xs[j] + theta * (Xn[j] - Xs[j]) + sig_s[j] * bb * y;
    }
    const R tau = ti + ((R)sstar + theta) * h;
    if constexpr (SYNC_EVAL) __syncthreads();

    R u = 0, gsum = 0, uT = 0;
    if constexpr (PAIRS && EV >= EV_TREE4) {
      float2 PVT[DP], PBS[DP];
      PVT[0] = make_float2((tau - a.ctr[0]) * a.sc[0], (a.T - a.ctr[0]) * a.sc[0]);
      PBS[0] = make_float2(a.sc[0], 0.f);
#pragma unroll
      for (int v = 1; v < DP; ++v) {
        PVT[v] = make_float2((Xtau[v - 1] - a.ctr[v]) * a.sc[v], (X[v - 1] - a.ctr[v]) * a.sc[v]);
        PBS[v] = make_float2(drift_s[v - 1] * a.sc[v], sig_s[v - 1] * a.sc[v]);
      }
      eval_tree_x2<D, EV>(a, reinterpret_cast<const float2*>(s_alpha), PVT, PBS, u, gsum, uT);
    } else if constexpr (EV != EV_TABLES) {
      R z[DP], zT[DP], bt[DP], st[DP];
      z[0] = (tau - a.ctr[0]) * a.sc[0];
      zT[0] = (a.T - a.ctr[0]) * a.sc[0];
      bt[0] = a.sc[0];
      st[0] = R(0);
#pragma unroll
      for (int v = 1; v < DP; ++v) {
        z[v] = (Xtau[v - 1] - a.ctr[v]) * a.sc[v];
        zT[v] = (X[v - 1] - a.ctr[v]) * a.sc[v];
        bt[v] = drift_s[v - 1] * a.sc[v];
        st[v] = sig_s[v - 1] * a.sc[v];
      }
      if constexpr (EV >= EV_TREE4)
        eval_tree<R, D, EV>(a, s_alpha, z, zT, bt, st, u, gsum, uT);
      else if constexpr (EV == EV_DENSE4)
        eval_dense4<R, D, PAIRS ? 2 : 1>(a, s_alpha, z, zT, bt, st, u, gsum, uT);
      else
        eval_dense3<R, D, PAIRS ? 2 : 1>(a, s_alpha, z, zT, bt, st, u, gsum, uT);
    } else {
      // per-thread Chebyshev tables: value, drift- and diffusion-scaled
      // derivatives at (tau, X_tau), value at (T, X_T)
      R* tb = cheb + tid;
  #pragma unroll
      for (int v = 0; v < DP; ++v) {
        const R xi = (v == 0) ? (tau - a.ctr[0]) * a.sc[0] : (Xtau[v - 1] - a.ctr[v]) * a.sc[v];
        const R xT = (v == 0) ? (a.T - a.ctr[0]) * a.sc[0] : (X[v - 1] - a.ctr[v]) * a.sc[v];
        const R bt = (v == 0) ? a.sc[0] : drift_s[v - 1] * a.sc[v];
        const R st = (v == 0) ? R(0) : sig_s[v - 1] * a.sc[v];
        R t0 = 1, t1 = xi, d0 = 0, d1 = 1, e0 = 0, e1 = 0, T0 = 1, T1 = xT;
        for (int e = 1; e <= a.eta; ++e) {
          if (e >= 2) {
            const R t2 = R(2) * xi * t1 - t0;
            const R d2 = R(2) * t1 + R(2) * xi * d1 - d0;
            const R e2 = R(4) * d1 + R(2) * xi * e1 - e0;
            const R T2 = R(2) * xT * T1 - T0;
            t0 = t1; t1 = t2; d0 = d1; d1 = d2; e0 = e1; e1 = e2; T0 = T1; T1 = T2;
          }
          const int base = (v * a.eta + e - 1) * tpb;
          tb[base] = t1;
          tb[base + S] = bt * d1;
          tb[base + 2 * S] = st * d1;
          tb[base + 3 * S] = st * st * e1;
          tb[base + 4 * S] = T1;
        }
      }
      const R* tbr = cheb;
      for (int l = 0; l < a.p; ++l) {
        const R al = s_alpha[l];
        const uint2 pr = s_pairs[l];
        switch (s_nnz[l]) {
          case 0: term<0, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          case 1: term<1, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          case 2: term<2, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          case 3: term<3, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          case 4: term<4, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          case 5: term<5, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          case 6: term<6, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          case 7: term<7, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
          default: term<8, R>(tbr, S, a.eta, tpb, tid, pr, s_cp, DP, al, u, gsum, uT); break;
        }
      }
    }
    const R obs = basket_value<R, D>(a, Xtau, a.obstacle == 0);
    const R f = -a.r * u + a.lam * Math<R>::fmax(obs - u, R(0));
    const R phiT = basket_value<R, D>(a, X, true);
    const R am = (a.T - ti) * (f + gsum) + phiT - uT;
    if (!SYNC_EVAL || m < a.M) acc += (double)am;
  }

  // fixed-order CTA reduction of the per-thread sums
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int warp = tid >> 5, lane = tid & 31;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int wv = 0; wv < (tpb >> 5); ++wv) s += red[wv];
    a.partial[(size_t)i * a.chunks + chunk] = s;
  }
}


// The path kernel.  FP32 paths with the dense degree-3 and degree-4
// evaluations run with at most 96 registers per thread at d >= 8 (five
// 128-thread CTAs per SM, a few values spilled outside the step loop) and 80
// below (six), the prefix-tree evaluations at d <= 6 with at most 80 (three
// 256-thread CTAs); FP64 paths, the Chebyshev tables and the prefix-tree
// evaluations at d >= 7 (whose 256-thread CTAs share the instruction fetches
// of their long straight-line evaluation, and which spill hundreds of bytes
// under a cap: d = 10 degree 4 4.67 -> 4.84 ms with 96 registers, d = 8
// even) at two 256-thread CTAs with up to 128.  Measured per
// launch at the best shape: d = 10 degree 3 17.41 -> 17.18 ms (80 registers:
// 17.40), d = 5 degree 4 3.51 -> 3.41 ms, d = 6 degree 3 0.911 -> 0.896 ms
// (96 registers: 0.914), d = 5 degree 6 4.79 -> 4.64 ms, d = 2 degree 6
// 1.22 -> 1.18 ms (64 registers: slower), d = 6 degree 4 1.62 -> 1.57 ms.
template <int VK, int EV, bool CC, typename R, int D>
__global__ void __launch_bounds__(256, 2) k_paths(const __grid_constant__ Args<R, D> a) {
  paths_cta<VK, EV, CC, R, D>(a);
}
template <int VK, int EV, bool CC, typename R, int D>
__global__ void __maxnreg__(D >= 8 ? 96 : 80) k_paths_lr(const __grid_constant__ Args<R, D> a) {
  paths_cta<VK, EV, CC, R, D>(a);
}
template <int EV, typename R, int D>
constexpr bool paths_lr() {
  return sizeof(R) == 4 && (EV == EV_DENSE3 || EV == EV_DENSE4 || (EV >= EV_TREE4 && D <= 6));
}

// dynamic shared memory of the path kernel; dense: p is the number of
// monomial coefficients and there are no per-thread tables
inline size_t smem_bytes(int d, int p, int eta, int N, int tpb, size_t rsize, bool dense,
                         int tab_stride, bool pairs, bool xcopy) {
  const int dp = d + 1;
  // the volatility table, 16-byte aligned; the coefficients (twice when
  // `pairs`: the prefix-tree evaluation with FP32 paths reads them in pairs)
  size_t off = (size_t)N * tab_stride * rsize;
  if (pairs) off = (off + 15) & ~(size_t)15;
  off += ((size_t)p * (pairs ? 2 : 1) + dp * dp) * rsize;
  off = (off + 15) & ~(size_t)15;
  if (!dense) {
    off += (size_t)p * sizeof(uint2);
    off += ((size_t)p + 15) & ~(size_t)15;
    off += (size_t)5 * dp * eta * tpb * rsize;
    off = (off + 15) & ~(size_t)15;
  }
  off += 32 * sizeof(double);
  // the Philox table of the normals: 16 bytes per block, ceil(N / G) G d / 4
  // blocks with G = 4 / gcd(d, 4) steps per group
  const int gcd = (d % 4 == 0) ? 4 : (d % 2 == 0) ? 2 : 1;
  const int G = 4 / gcd, NB = G * d / 4;
  off += (size_t)((N + G - 1) / G) * NB * 16;
  // `xcopy` (copy_smem): the states before and after step s*, one row of
  // ceil(d / 4) float4 per thread and copy
  if (xcopy) off += (size_t)2 * ((d + 3) / 4) * tpb * 16;
  return off;
}

template <typename R, int D>
cudaError_t launch_kernel(void (*kern)(Args<R, D>), const Args<R, D>& a, unsigned grid, int tpb,
                          size_t smem, cudaStream_t st) {
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<grid, tpb, smem, st>>>(a);
  return cudaGetLastError();
}

template <int VK, int EV, bool CC, typename R, int D>
cudaError_t launch_one(const Args<R, D>& a, unsigned grid, int tpb, size_t smem, cudaStream_t st) {
  // only the kernel that runs is instantiated
  if constexpr (paths_lr<EV, R, D>())
    return launch_kernel<R, D>(k_paths_lr<VK, EV, CC, R, D>, a, grid, tpb, smem, st);
  else
    return launch_kernel<R, D>(k_paths<VK, EV, CC, R, D>, a, grid, tpb, smem, st);
}

template <int EV, bool CC, typename R, int D>
cudaError_t launch_ev(int vk, const Args<R, D>& a, unsigned grid, int tpb, size_t smem,
                      cudaStream_t st) {
  switch (vk) {
    case VK_CONST: return launch_one<VK_CONST, EV, CC>(a, grid, tpb, smem, st);
    case VK_TANH: return launch_one<VK_TANH, EV, CC>(a, grid, tpb, smem, st);
    case VK_TANH_ABS: return launch_one<VK_TANH_ABS, EV, CC>(a, grid, tpb, smem, st);
    default: return launch_one<VK_DUPIRE, EV, CC>(a, grid, tpb, smem, st);
  }
}

// the prefix-tree evaluations (FP32 paths only: FP64 solves of these bases
// use the tables), compiled in translation units of their own
template <typename R, int D>
cudaError_t launch_tree(int eta, int vk, const Args<R, D>& a, unsigned grid, int tpb, size_t smem,
                        cudaStream_t st) {
  switch (eta) {
    case 4:
      if constexpr (D >= 6 && sizeof(R) == 4)
        return launch_ev<EV_TREE4, true>(vk, a, grid, tpb, smem, st);
      return cudaErrorInvalidValue;
    case 5:
      if constexpr (D <= 5 && sizeof(R) == 4)
        return launch_ev<EV_TREE5, true>(vk, a, grid, tpb, smem, st);
      return cudaErrorInvalidValue;
    case 6:
      if constexpr (D <= 5 && sizeof(R) == 4)
        return launch_ev<EV_TREE6, true>(vk, a, grid, tpb, smem, st);
      return cudaErrorInvalidValue;
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename R, int D>
cudaError_t launch(const ModelHost& m, const GridHost& g, const ProblemDev& P, int M, int N,
                   uint32_t k, int tpb, int ppt, cudaStream_t st) {
  Args<R, D> a;
  memset(&a, 0, sizeof(a));
  a.T = (R)m.T;
  a.r = (R)m.r;
  a.lam = (R)m.lambda;
  a.K = (R)m.K;
  a.s_dupire = (R)m.s_dupire;
  a.vb = (R)m.b;
  a.rho = (R)(m.d > 1 ? m.C[1] : 0.0);
  bool cc = true;
  for (int j = 0; j < D; ++j)
    for (int q = 0; q < D; ++q)
      if (j != q && m.C[j * D + q] != m.C[D > 1 ? 1 : 0]) cc = false;
  for (int j = 0; j < D; ++j) {
    a.Ld[j] = (R)m.L[j * D + j];
    a.Lc[j] = (R)(j + 1 < D ? m.L[(j + 1) * D + j] : 0.0);
    a.kc[j] = (R)(-2.8853900817779268 * m.kappa[j]);
    a.rd[j] = (R)(m.r - m.div[j]);
    a.w[j] = (R)m.w[j];
    a.va[j] = (R)m.a[j];
    a.kappa[j] = (R)m.kappa[j];
    for (int q = 0; q < D; ++q) {
      a.L[j][q] = (R)m.L[j * D + q];
      a.Cp[j + 1][q + 1] = (R)m.C[j * D + q];
    }
  }
  for (int v = 0; v <= D; ++v) {
    a.ctr[v] = (R)(0.5 * (g.lo[v] + g.hi[v]));
    a.sc[v] = (R)(2.0 / (g.hi[v] - g.lo[v]));
  }
  a.N = N;
  a.M = M;
  a.n = P.n;
  a.p = P.p;
  a.eta = P.eta < 1 ? 1 : P.eta;
  a.tpb = tpb;
  a.ppt = ppt;
  a.chunks = P.chunks;
  a.i0 = P.shard_i0;
  // tanh families: (A_j, B_j) pairs, rows padded to 4 values (16 bytes in
  // FP32) so that one 128-bit load fetches two assets' pairs
  a.tab_stride = (m.vol_kind == 1 || m.vol_kind == 2) ? ((2 * D + 3) & ~3) : (D < 3 ? 3 : D);
  a.payoff = m.payoff;
  a.obstacle = m.obstacle;
  a.vol_sin = (m.vol_kind == 2) ? 1 : 0;
  a.k = k;
  a.key0 = P.seed_key[0];
  a.key1 = P.seed_key[1];
  for (int r = 0; r < 10; ++r) {
    a.rk0[r] = a.key0 + (uint32_t)r * 0x9E3779B9u;
    a.rk1[r] = a.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  a.pt = P.t;
  a.px = P.x;
  if constexpr (sizeof(R) == 4)
    a.alpha = reinterpret_cast<const R*>(P.alpha32);
  else
    a.alpha = reinterpret_cast<const R*>(P.alpha);
  a.pairs = P.pairs;
  a.nnz = P.nnz;
  a.partial = P.partial;
  const bool dense = P.dense;
  if (dense) {
    a.p = P.pm;
    if constexpr (sizeof(R) == 4)
      a.alpha = reinterpret_cast<const R*>(P.beta32);
    else
      a.alpha = reinterpret_cast<const R*>(P.beta);
  }
  const size_t smem = smem_bytes(D, a.p, a.eta, N, tpb, sizeof(R), dense, a.tab_stride,
                                dense && sizeof(R) == 4,
                                dense && copy_smem(P.tree > 0 ? EV_TREE4 : P.dense4 ? EV_DENSE4 : EV_DENSE3,
                                                   sizeof(R) == 4, D));
  const int vk = (m.vol_kind == 0)   ? VK_CONST
                 : (m.vol_kind == 1) ? VK_TANH_ABS
                 : (m.vol_kind == 3) ? VK_DUPIRE
                                     : VK_TANH;
  // the points of this launch: all n, or the block [shard_i0, shard_i0 + shard_n)
  const int npts = P.shard_n > 0 ? P.shard_n : P.n;
  if (npts <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)npts * (unsigned)P.chunks;
  if (dense) {  // implies a constant correlation
    // the host selects: degree <= 3 loops (any d), degree-4 loops (d <= 5),
    // the tree recursion of degree 4 (d >= 6) or 5 and 6 (d <= 5)
    switch (P.tree) {
      case 0:
        if (P.dense4) {
          if constexpr (D <= 5) return launch_ev<EV_DENSE4, true>(vk, a, grid, tpb, smem, st);
          return cudaErrorInvalidValue;
        }
        return launch_ev<EV_DENSE3, true>(vk, a, grid, tpb, smem, st);
      default:
        return launch_tree<R, D>(P.tree, vk, a, grid, tpb, smem, st);
    }
  }
  if (cc) return launch_ev<EV_TABLES, true>(vk, a, grid, tpb, smem, st);
  return launch_ev<EV_TABLES, false>(vk, a, grid, tpb, smem, st);
}

}  // namespace paths

// one translation unit per (d, precision), so that the build compiles them
// in parallel; the FP32 prefix-tree kernels in one more per d
#define BSDE_PATHS_INSTANTIATE(DV, R, SUF)                                                    \
  extern template cudaError_t paths::launch_tree<R, DV>(int, int, const paths::Args<R, DV>&, \
                                                        unsigned, int, size_t, cudaStream_t); \
  cudaError_t launch_paths_d##DV##_##SUF(const ModelHost& m, const GridHost& g,               \
                                         const ProblemDev& P, int M, int N, uint32_t k,       \
                                         int tpb, int ppt, cudaStream_t st) {                 \
    return paths::launch<R, DV>(m, g, P, M, N, k, tpb, ppt, st);                              \
  }

#define BSDE_PATHS_INSTANTIATE_TREE(DV)                                                     \
  template cudaError_t paths::launch_tree<float, DV>(int, int, const paths::Args<float, DV>&, \
                                                     unsigned, int, size_t, cudaStream_t);    \
  template cudaError_t paths::launch_tree<double, DV>(int, int, const paths::Args<double, DV>&, \
                                                      unsigned, int, size_t, cudaStream_t);
