"""FP32 operation counts of the path kernel (csrc/k_paths.cuh), counted from
its source for the roofline of the benchmark.

The path kernel computes, for every path of every point, the Euler steps of
the local-volatility diffusion (Section 3.1, eq. eqs3) and once per path
the evaluation of u^k, d_t u^k + L^N u^k at (tau, X_tau) and u^k(T, X_T)
with the driver and the sample a_m (eq. psiN).  The functions below walk the
same loops as the kernel's FP32 code (mixed precision, constant
correlation, the tanh volatility families, the dense monomial evaluation of
a total-degree-3 basis: the d = 10 benchmark kernel) and add up its
floating-point operations:
  * an FMA counts 2 flops, a multiply, add, subtract or max 1;
  * MUFU operations (ex2, lg2, rcp, sqrt, sin, cos) are counted apart, as
    transcendental operations, not flops;
  * integer work (Philox4x32-10, the counter arithmetic) is not counted;
  * expressions the compiler hoists out of the path loop (per point or per
    CTA: h, sqrt(h), the reduced time at T) and dead code (the unused
    derivative along sigma of eval_dense3) are not counted.
The counts change when the kernel's arithmetic changes; they are the ones of
the source they sit beside.
"""


def step_flops(d, vol="tanh"):
    """FP32 flops and MUFU operations of one Euler step of one path
    (k_paths main loop): Box-Muller normals, the correlated increment by the
    constant-correlation prefix sum, the tabulated local volatility and the
    fused Euler update.  Returns (flops, mufu)."""
    pairs = d / 2.0  # Box-Muller pairs per step (normals are drawn in whole pairs)
    # u0 = fma(w0, 2^-32, 2^-33); r2 = lg * k; ang = fma(w1, .., -pi);
    # z0 = -rad * c; z1 = -rad * s      -> 2 FMA + 3 MUL; lg2, sqrt, sin, cos
    bm = pairs * (2 * 2 + 3)
    bm_mufu = pairs * 4
    # y = Ld_j z_j + pre; pre += Lc_j z_j   -> 2 FMA per asset
    corr = d * 2 * 2
    if vol == "tanh":
        # t = fma(x, 2 log2 e, kc); e = ex2(t); r = rcp(e + 1); sig = A + B r
        vol_f, vol_mufu = d * (2 + 1 + 2), d * 2
    elif vol == "const":
        vol_f, vol_mufu = 0, 0
    else:
        raise ValueError("counted for the constant and tanh volatility families")
    # X = sig (nhh sig + y) + (h rd_j + X)   -> 3 FMA per asset
    update = d * 3 * 2
    return bm + corr + vol_f + update, bm_mufu + vol_mufu


def eval_dense3_flops(d):
    """FP32 flops of eval_dense3 (nested Horner on dual numbers, one pass
    over the monomial coefficients of total degree <= 3 for both points)."""
    dp = d + 1
    f = 0
    for i in range(dp):
        for j in range(i, dp):
            if i == j and i > 0:
                f += 4          # diag += 2 st_i st_i q
            for k in range(j, dp):
                f += 2 + 2 + 2  # av, ab, aT: one FMA each
                if k > 0:
                    f += 2      # as += t st_k
                if i == j and j < k and i > 0:
                    f += 5      # diag += 2 st_i st_i t z_k
                if i < j and j == k and j > 0:
                    f += 5
                if i == j and j == k and i > 0:
                    f += 5
            f += 2 + 4 + 2      # bv, bb (2 FMA), bT
            if j > 0:
                f += 4 + 3      # bs (2 FMA), bss (MUL + FMA)
            else:
                f += 2          # bs
        f += 2 + 4 + 2          # uv, ub (2 FMA), sT
        f += 5 if i > 0 else 2  # uss
    f += 6                      # gen = ub + 1/2 ((1 - rho) diag + rho uss)
    return f


def path_flops(d, vol="tanh"):
    """FP32 flops and MUFU operations of the once-per-path work besides
    eval_dense3: the random time, the Brownian bridge to X_tau (general
    triangular L times the bridge normals, sigma and drift frozen at the
    step s*), the reduced coordinates of both evaluation points, the two
    basket values, the penalised driver and the sample a_m.  Returns
    (flops, mufu)."""
    nbb = (d + 3) // 4            # Philox blocks of bridge normals
    theta = 2                     # fma(w, 2^-32, 2^-33)
    bridge_bm = nbb * 2 * 7       # two Box-Muller pairs per block
    bridge_bm_mufu = nbb * 2 * 4
    bb = 3                        # theta (1 - theta) h, then sqrt
    per_asset = 0
    for j in range(d):
        per_asset += 2 * (j + 1)  # y = sum_{q <= j} L_jq zb_q
        per_asset += 5 if vol == "tanh" else 0   # sigma at (t_s*, X_s*)
        per_asset += 3            # drift = rd - sig^2 / 2
        per_asset += 6            # Xtau = Xs + theta (Xn - Xs) + sig bb y
    vol_mufu = 2 * d if vol == "tanh" else 0
    tau = 3
    coords = 2 + 6 * d            # z_0; z, zT, bt, st of each asset
    basket = 2 * (3 * d + 2)      # two basket values: exp, weighted sum, K - s, max
    driver = 5 + 5                # f = -r u + lambda (obs - u)^+; a_m
    flops = theta + bridge_bm + bb + per_asset + tau + coords + basket + driver
    mufu = bridge_bm_mufu + 1 + vol_mufu + 2 * d
    return flops, mufu


def per_path_step(d, N, vol="tanh"):
    """Flops per path-step with and without the once-per-path evaluation
    amortised over the N steps of a path, and MUFU operations per
    path-step: a dict."""
    sf, sm = step_flops(d, vol)
    pf, pmu = path_flops(d, vol)
    ef = eval_dense3_flops(d)
    return {"step_flops": sf, "eval_flops_per_path": ef, "other_flops_per_path": pf,
            "flops_steps_only": sf, "flops_with_eval": sf + (ef + pf) / float(N),
            "mufu_per_step": sm + pmu / float(N)}
