"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs and the same Philox counters.

Tolerances:
  * points: bit-exact (both sides round the same IEEE operations);
  * FP64 mode: 1e-9 relative on coefficients and corrections, where the two
    sides differ only by libm ulps and summation order;
  * mixed mode: 1e-4 relative on price and delta; the corrections c_i agree
    to a tolerance derived from FP32 rounding along the path (see
    MIXED_C_TOL below).
For the penalised (American) configurations the Picard map amplifies a
perturbation by up to lambda (T - t) per iteration, so those are compared
one iteration at a time from the same alpha^k ("teacher forcing").
"""
import math
import os

import numpy as np
import pytest

import workloads
from oracle import bsde_oracle as O

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 1
# FP32 relative rounding u = 2^-24; a path of N steps accumulates about
# sqrt(N) u relative error in X, the Box-Muller/exp/tanh approximations add a
# few 1e-7; the evaluation of u^k sums p terms of size |alpha_l| (error about
# p u max|alpha|).  The mean over M paths averages the random part.  A bound
# of 2e-5 times the scale of the integrand (max of |Phi|, |u|, T |g1|) covers
# all the configurations below with margin.
MIXED_C_TOL = 2e-5


@pytest.fixture(scope="module")
def G():
    import paper_1102_4666_gb300 as G
    return G


def solver(G, cfg, prec):
    return G.Solver(cfg, precision=prec)


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1e-300, np.max(np.abs(np.asarray(b))))


# ---------------------------------------------------------------------------
# points and basis
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_points_bit_exact(G, prec):
    cfg = workloads.config("c3", n=1000, M=8, N=2, eta=2)
    s = solver(G, cfg, prec)
    nu = O.multi_index_set(6, 2)
    t, x, c, a1 = s.iterate(3, np.zeros(len(nu)))
    s.close()
    to, xo = O.points(cfg, 3)
    assert np.array_equal(t, to)
    assert np.array_equal(x, xo)


# ---------------------------------------------------------------------------
# config 1 (European put d=1): whole solve
# ---------------------------------------------------------------------------

def test_c1_fp64_full_trajectory(G):
    cfg = workloads.config("c1")
    s = solver(G, cfg, "fp64")
    rep = s.solve(use_graph=1)
    alpha = s.coeffs()
    s.close()
    ref = O.solve(cfg, nthreads=NTH)
    assert rel(alpha, ref["alpha"]) < 1e-9
    assert abs(rep.price - ref["price"]) < 1e-9 * abs(ref["price"])
    assert abs(rep.delta[0] - ref["delta"][0]) < 1e-9 * abs(ref["delta"][0])
    for k, h in enumerate(ref["history"]):
        assert abs(rep.price_iter[k] - h["price"]) < 1e-9 * abs(h["price"])


def test_c1_mixed_price_delta(G):
    cfg = workloads.config("c1")
    s = solver(G, cfg, "mixed")
    rep = s.solve(use_graph=1)
    s.close()
    ref = O.solve(cfg, nthreads=NTH)
    assert abs(rep.price - ref["price"]) <= 1e-4 * abs(ref["price"])
    assert abs(rep.delta[0] - ref["delta"][0]) <= 1e-4 * abs(ref["delta"][0])


@pytest.mark.parametrize("name,K_it", [("c3", 10), ("c4", 4)])
def test_full_size_mixed_price_delta_against_fp64(G, name, K_it):
    """The d = 5 and d = 10 American basket puts at their full sizes with the
    paper's penalty weight omega = 1: the mixed-precision solve's price and
    deltas at (0, x0) within 1e-4 relative of the FP64 solve (the FP64 path is
    pinned to the oracle at 1e-9 by the tests above; a full FP64 oracle solve
    at these sizes would take hours on the CPU).  Both use the same random
    numbers, so the difference is the FP32 arithmetic alone."""
    cfg = workloads.config(name, K_it=K_it, **{"lambda": 1.0})
    out = {}
    for prec in ("mixed", "fp64"):
        s = solver(G, cfg, prec)
        r = s.solve(use_graph=1)
        s.close()
        assert r.status == G.OK
        out[prec] = (r.price, np.array(r.delta[:cfg["d"]]))
    (pm, dm), (pf, df) = out["mixed"], out["fp64"]
    assert abs(pm - pf) <= 1e-4 * abs(pf)
    assert np.max(np.abs(dm - df)) <= 1e-4 * np.max(np.abs(df))


# ---------------------------------------------------------------------------
# one iteration from the same alpha^k (teacher forcing)
# ---------------------------------------------------------------------------

CASES = {
    # name: (config, overrides)
    "c2_small": ("c2", dict(n=300, M=400, N=50, eta=6)),
    "c3_small": ("c3", dict(n=480, M=200, N=25, eta=4)),
    "c4_small": ("c4", dict(n=800, M=128, N=20, eta=3)),
    "d2_ragged": ("c3", dict(d=2, n=70, M=77, N=7, eta=3)),
    "d3_call": ("c3", dict(d=3, n=90, M=130, N=9, eta=3, payoff="call")),
    "d10_tail": ("c4", dict(n=200, M=33, N=7, eta=2)),
    "d1_raw_obstacle": ("c2", dict(n=120, M=200, N=13, eta=5, obstacle="raw")),
    # degenerate sizes: one Euler step and one path per point; an odd step
    # count (the last group of two steps is half full) and a few paths
    "d10_one_step_one_path": ("c4", dict(n=160, M=1, N=1, eta=2)),
    "d5_odd_steps": ("c3", dict(n=60, M=5, N=3, eta=2)),
    # dense evaluation by the prefix-tree recursion: degree 4 at d = 10
    # (p = 1365) and degree 5 at d = 5 (p = 462)
    "d10_degree4": ("c4", dict(n=2800, M=16, N=5, eta=4)),
    "d5_degree5": ("c3", dict(n=940, M=40, N=6, eta=5)),
    "d5_degree6": ("c3", dict(n=1900, M=24, N=4, eta=6)),
    # a full correlation matrix (no constant correlation): the general
    # triangular product L Z in the Euler step and the correlation-weighted
    # cross terms of the per-thread table evaluation
    "d3_full_corr": ("c3", dict(d=3, n=90, M=130, N=9, eta=3,
                                corr=[[1.0, 0.3, -0.1], [0.3, 1.0, 0.5], [-0.1, 0.5, 1.0]])),
    # hyperbolic index sets (eq. hyper_set, q < 1): d = 10 degree 5 with
    # q = 0.6 (p = 221, per-thread tables), d = 10 degree 4 with q = 0.7
    # (p = 210, prefix-tree recursion over the kept monomials in FP32) and
    # d = 5 degree 6 with q = 0.75 (p = 237, degree-6 prefix tree in FP32)
    "d10_hyperbolic": ("c4", dict(n=460, M=24, N=5, eta=5, q=0.6)),
    "d10_hyperbolic_deg4": ("c4", dict(n=430, M=16, N=4, eta=4, q=0.7)),
    "d5_hyperbolic_deg6": ("c3", dict(n=480, M=24, N=5, eta=6, q=0.75)),
    # a call with the raw obstacle of the penalty (both differ from the
    # put with the payoff obstacle in the driver)
    "d2_call_raw": ("c3", dict(d=2, n=64, M=90, N=6, eta=3, payoff="call", obstacle="raw")),
}


def _case(name):
    base, over = CASES[name]
    cfg = workloads.config(base)
    d = over.get("d", cfg["d"])
    if d != cfg["d"]:
        cfg = workloads.make(d=d, T=cfg["T"], r=cfg["r"], K=cfg["K"], S0=100.0, vol=cfg["vol"],
                             rho=cfg["rho"], lam=cfg["lambda"], n=cfg["n"], M=cfg["M"], N=cfg["N"],
                             eta=cfg["eta"], K_it=1, seed=cfg["seed"])
    for k, v in over.items():
        if k != "d":
            cfg[k] = v
    return cfg


def _alpha(cfg, nu, scale=2.0, seed=3):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(len(nu)) * scale / np.sqrt(1 + nu.sum(axis=1)) ** 2
    a[0] += 5.0
    return a


def _nu(cfg):
    return O.multi_index_set(cfg["d"] + 1, cfg["eta"], cfg.get("q", 1.0))


def _phi_scale(cfg):
    """Size of the payoff (and of the obstacle in the penalty) by payoff kind:
    a put (K - basket)^+ never exceeds K; a call (basket - K)^+ reaches
    sum_j w_j e^{hi_j} - K at the top corner of the box.  The raw obstacle
    K - basket (put) or basket - K (call) has the same upper end."""
    if cfg["payoff"] == "put":
        return cfg["K"]
    return max(1.0, float(np.dot(cfg["weights"], np.exp(cfg["hi"][1:]))) - cfg["K"])


def _scale(cfg, nu, alpha, t, x):
    """Scale of the integrand a_m = (T - t)(-r u + lambda (Phi - u)^+ + d_t u + L u)
    + Phi - u (eq. psiN with the driver of eq. bsde-penal-2): both u and the
    payoff Phi enter multiplied by up to 1 + lambda T."""
    u = O.basis_matrix(cfg, nu, t, x) @ alpha
    return max(1.0, _phi_scale(cfg), np.max(np.abs(u))) * (1.0 + cfg["lambda"] * cfg["T"])


# (case, eval_mode): 0 automatic (dense monomial form for total degree <= 3,
# <= 4 at d <= 10 or <= 6 at d <= 5, and a constant correlation), 1
# per-thread Chebyshev tables -- both forms wherever the dense one applies
def _dense_applies(name):
    cfg = _case(name)
    if cfg.get("corr") is not None:
        return False
    return cfg["eta"] <= 3 or (cfg["eta"] == 4 and cfg["d"] <= 10) or (cfg["eta"] <= 6 and cfg["d"] <= 5)


EVAL_CASES = [(n, 0) for n in CASES] + [(n, 1) for n in CASES if _dense_applies(n)]


@pytest.mark.parametrize("name,ev", EVAL_CASES)
def test_teacher_forced_iteration_fp64(G, name, ev):
    cfg = _case(name)
    nu = _nu(cfg)
    a0 = _alpha(cfg, nu)
    s = solver(G, cfg, "fp64")
    t, x, c, a1 = s.iterate(2, a0, eval_mode=ev)
    s.close()
    it = O.iteration(cfg, nu, a0, 2, nthreads=NTH)
    sc = _scale(cfg, nu, a0, t, x)
    assert np.max(np.abs(c - it["c"])) < 1e-9 * sc
    # the coefficients alpha^{k+1} to 1e-9 relative, and the increment too
    assert rel(a1, it["alpha"]) < 1e-9
    assert rel(a1 - a0, it["alpha"] - a0) < 1e-9


@pytest.mark.parametrize("name,ev", EVAL_CASES)
def test_teacher_forced_iteration_mixed(G, name, ev):
    cfg = _case(name)
    nu = _nu(cfg)
    a0 = _alpha(cfg, nu)
    s = solver(G, cfg, "mixed")
    t, x, c, a1 = s.iterate(2, a0, eval_mode=ev)
    s.close()
    it = O.iteration(cfg, nu, a0, 2, nthreads=NTH)
    sc = _scale(cfg, nu, a0, t, x)
    assert np.max(np.abs(c - it["c"])) < MIXED_C_TOL * sc
    # price and delta of alpha^{k+1}
    pg, dg = O.price_delta(cfg, nu, a1)
    po, do = O.price_delta(cfg, nu, it["alpha"])
    assert abs(pg - po) <= 1e-4 * max(abs(po), 1.0)
    assert np.max(np.abs(dg - do)) <= 1e-4 * max(np.max(np.abs(do)), 1e-2)


# The path kernels are instantiated per dimension d; the cases above reach
# d = 1, 2, 3, 5 and 10.  These reach the rest: d = 4 and 8 (one Euler step
# per group of Philox blocks), 6 (two steps per group) and 7 and 9 (four),
# with a degree-2 basis (dense degree-3 loops in FP32, tables in FP64) and a
# degree-4 one (dense degree-4 loops at d = 4, the prefix-tree recursion at
# d >= 6 in FP32; tables in FP64), n just above 2 p.
DIM_CASES = [(d, eta, prec) for d in (4, 6, 7, 8, 9) for eta in (2, 4) for prec in ("fp64", "mixed")]


@pytest.mark.parametrize("d,eta,prec", DIM_CASES)
def test_teacher_forced_iteration_every_dimension(G, d, eta, prec):
    p = workloads.basis_size(d, eta)
    base = workloads.config("c3")
    cfg = workloads.make(d=d, T=base["T"], r=base["r"], K=base["K"], S0=100.0, vol=base["vol"],
                         rho=base["rho"], lam=base["lambda"], n=2 * p + 9, M=5 if eta == 4 else 37,
                         N=3 if eta == 4 else 6, eta=eta, K_it=1, seed=40 + d)
    nu = O.multi_index_set(d + 1, eta)
    a0 = _alpha(cfg, nu)
    s = solver(G, cfg, prec)
    t, x, c, a1 = s.iterate(1, a0)
    s.close()
    it = O.iteration(cfg, nu, a0, 1, nthreads=NTH)
    sc = _scale(cfg, nu, a0, t, x)
    tol = 1e-9 if prec == "fp64" else MIXED_C_TOL
    assert np.max(np.abs(c - it["c"])) < tol * sc


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_refit_solves_the_normal_equations(G, prec):
    """alpha^{k+1} - alpha^k is the least-squares fit of the GPU's own c on
    the (bit-exact) points: isolates the Gram matrix (tensor cores in mixed
    mode), the Cholesky solve and the refinement."""
    cfg = workloads.config("c4", n=900, M=64, N=4, eta=3)
    nu = O.multi_index_set(11, 3)
    a0 = _alpha(cfg, nu)
    s = solver(G, cfg, prec)
    t, x, c, a1 = s.iterate(1, a0)
    s.close()
    B = O.basis_matrix(cfg, nu, t, x)
    delta = O.fit(B, c)
    assert rel(a1 - a0, delta) < 1e-9


# the launch shapes the autotuner can give bench.py (dense evaluation), and
# the library's default shape for the per-thread-table evaluation
_FULL_SIZE = [(0, shape) for shape in __import__(
    "paper_1102_4666_gb300.autotune", fromlist=["CANDIDATES"]).CANDIDATES["mixed"]] + [(1, None)]


@pytest.mark.parametrize("ev,shape", _FULL_SIZE)
def test_full_size_c4_sampled_points(G, ev, shape):
    """c4 at its full size (n=4000, M=4000, N=100, p=364), one mixed
    iteration in each launch configuration bench.py can time (threads per
    CTA x paths per thread); the oracle recomputes c_i at the 256 points
    i = 0, 15, 30, ... (1e8 path-steps of FP64 oracle work per case)."""
    cfg = workloads.config("c4")
    nu = O.multi_index_set(11, 3)
    a0 = _alpha(cfg, nu, scale=1.0)
    s = solver(G, cfg, "mixed")
    kw = {} if shape is None else {"paths_tpb": shape[0], "paths_ppt": shape[1]}
    t, x, c, a1 = s.iterate(5, a0, eval_mode=ev, **kw)
    s.close()
    # the 256-point subset i = 0, 15, 30, ... of the d = 10 configuration
    idx = np.arange(0, 15 * 256, 15)
    co = O.correction(cfg, nu, a0, 5, idx, t[idx], x[:, idx], nthreads=NTH)
    sc = _scale(cfg, nu, a0, t, x)
    assert np.max(np.abs(c[idx] - co)) < MIXED_C_TOL * sc
    # the refit at full size: normal equations of the GPU's own c
    B = O.basis_matrix(cfg, nu, t, x)
    assert rel(a1 - a0, O.fit(B, c)) < 1e-8


def test_full_size_c4_sampled_points_fp64(G):
    """The plain FP64 path at the full d = 10 size: one iteration; the oracle
    recomputes c_i at a sample of points to 1e-9 of the integrand's scale."""
    cfg = workloads.config("c4")
    nu = O.multi_index_set(11, 3)
    a0 = _alpha(cfg, nu, scale=1.0)
    s = solver(G, cfg, "fp64")
    t, x, c, a1 = s.iterate(5, a0)
    s.close()
    idx = np.arange(0, 4000, 500)
    co = O.correction(cfg, nu, a0, 5, idx, t[idx], x[:, idx], nthreads=NTH)
    sc = _scale(cfg, nu, a0, t, x)
    assert np.max(np.abs(c[idx] - co)) < 1e-9 * sc
    B = O.basis_matrix(cfg, nu, t, x)
    assert rel(a1 - a0, O.fit(B, c)) < 1e-9


def test_full_size_c3_sampled_points(G):
    """c3 at its full size (d = 5, n = 2000, M = 5000, N = 50, total degree 4:
    p = 210, per-thread Chebyshev tables), one mixed iteration; the oracle
    recomputes c_i at a sample of points, and the refit solves the normal
    equations of the GPU's own c."""
    cfg = workloads.config("c3")
    nu = O.multi_index_set(6, 4)
    a0 = _alpha(cfg, nu, scale=1.0)
    s = solver(G, cfg, "mixed")
    t, x, c, a1 = s.iterate(3, a0)
    s.close()
    idx = np.arange(0, 2000, 250)
    co = O.correction(cfg, nu, a0, 3, idx, t[idx], x[:, idx], nthreads=NTH)
    sc = _scale(cfg, nu, a0, t, x)
    assert np.max(np.abs(c[idx] - co)) < MIXED_C_TOL * sc
    B = O.basis_matrix(cfg, nu, t, x)
    assert rel(a1 - a0, O.fit(B, c)) < 1e-8


# ---------------------------------------------------------------------------
# vol families, outputs, determinism, errors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["const", "abs_tanh", "sin_tanh", "dupire"])
@pytest.mark.parametrize("prec,ev", [("fp64", 0), ("fp64", 1), ("mixed", 0), ("mixed", 1)])
def test_vol_families(G, kind, prec, ev):
    """Every volatility family, in both precisions and both evaluation forms
    of u^k (dense monomial, per-thread Chebyshev tables)."""
    cfg = workloads.config("c3", n=80, M=96, N=9, eta=2)
    if kind == "const":
        cfg["vol"] = {"kind": "const", "a": [0.15, 0.2, 0.25, 0.3, 0.35]}
    elif kind == "abs_tanh":
        cfg["vol"] = {"kind": "abs_tanh", "a": 0.15, "b": 0.1, "kappa": math.log(100.0)}
    elif kind == "dupire":
        cfg["vol"] = {"kind": "dupire", "s": 100.0}
    cfg["div"] = [0.0, 0.01, 0.02, 0.03, 0.1]
    nu = O.multi_index_set(6, 2)
    a0 = _alpha(cfg, nu)
    s = solver(G, cfg, prec)
    t, x, c, a1 = s.iterate(0, a0, eval_mode=ev)
    s.close()
    it = O.iteration(cfg, nu, a0, 0, nthreads=NTH)
    tol = 1e-9 if prec == "fp64" else MIXED_C_TOL
    assert np.max(np.abs(c - it["c"])) < tol * _scale(cfg, nu, a0, t, x)


def test_eval_price_delta_matches_oracle(G):
    cfg = workloads.config("c3", n=400, M=64, N=5, eta=3, K_it=2)
    s = solver(G, cfg, "fp64")
    s.solve(use_graph=0)
    alpha = s.coeffs()
    rng = np.random.default_rng(8)
    q = 17
    tq = rng.uniform(0, 1, q)
    S = 100.0 * np.exp(rng.uniform(-0.5, 0.5, (q, 5)))
    price, delta = s.eval(tq, S)
    s.close()
    nu = O.multi_index_set(6, 3)
    u, g = O.eval_u(cfg, nu, alpha, tq, np.log(S).T)
    assert np.allclose(price, u, rtol=1e-12, atol=1e-12)
    assert np.allclose(delta, (g / S.T).T, rtol=1e-11, atol=1e-13)


def test_graph_and_direct_launch_agree_and_are_deterministic(G):
    cfg = workloads.config("c4", n=200, M=300, N=10, K_it=3, eta=2)
    s = solver(G, cfg, "mixed")
    r1 = s.solve(use_graph=1)
    a1 = s.coeffs()
    r2 = s.solve(use_graph=0)
    a2 = s.coeffs()
    r3 = s.solve(use_graph=1)
    a3 = s.coeffs()
    s.close()
    assert np.array_equal(a1, a2) and np.array_equal(a1, a3)
    assert r1.price == r2.price == r3.price


def test_library_memory_pool_matches_caller_allocator(G):
    """Without allocation hooks the context takes its memory from the
    library's stream-ordered pool; results are those of a context on
    PyTorch's caching allocator, also after the factor block is laid out
    again for a different number of iterations and after one iteration
    through bsde_iterate."""
    cfg = workloads.config("c4", n=200, M=300, N=10, K_it=3, eta=2)
    out = []
    for torch_memory in (True, False):
        s = G.Solver(cfg, precision="mixed", torch_memory=torch_memory)
        r3 = s.solve(use_graph=1)
        r5 = s.solve(use_graph=1, K_it=5)
        a5 = s.coeffs()
        _, _, c1, a1 = s.iterate(1)
        r3b = s.solve(use_graph=1)
        s.close()
        out.append((r3.price, r5.price, a5, c1, a1, r3b.price))
    (p3, p5, a5, c1, a1, p3b), (q3, q5, b5, d1, b1, q3b) = out
    assert p3 == q3 == p3b == q3b and p5 == q5
    assert np.array_equal(a5, b5) and np.array_equal(c1, d1) and np.array_equal(a1, b1)


def test_checkpoint_resume_reproduces_the_run(G):
    cfg = workloads.config("c3", n=300, M=200, N=10, eta=3, K_it=4)
    s = solver(G, cfg, "mixed")
    s.solve()
    full = s.coeffs()
    s.solve(K_it=2)
    half = s.coeffs()
    s.close()
    s2 = solver(G, cfg, "mixed")
    s2.set_coeffs(half)
    s2.solve(K_it=2, k_start=2)
    resumed = s2.coeffs()
    s2.close()
    assert np.array_equal(full, resumed)


def test_factorisation_groups_do_not_change_the_run(G):
    """A d = 10 degree-4 basis (p = 1365): the Gram factors and inverses of
    one group of iterations hold 8 iterations (256 MiB), so a 10-iteration
    solve factorises in two groups; it must equal the same run done as two
    solves of 5 iterations (one group each, resumed from the coefficients)."""
    cfg = workloads.config("c4", n=2800, M=16, N=3, eta=4, K_it=10, **{"lambda": 1.0})
    s = solver(G, cfg, "mixed")
    r = s.solve()
    full = s.coeffs()
    s.solve(K_it=5)
    half = s.coeffs()
    s.close()
    s2 = solver(G, cfg, "mixed")
    s2.set_coeffs(half)
    s2.solve(K_it=5, k_start=5)
    resumed = s2.coeffs()
    s2.close()
    assert r.status == G.OK and np.array_equal(full, resumed)


def test_maximum_iteration_count(G):
    """K_it = 64 (the largest the report holds): every per-iteration entry is
    written, and the iteration converges at the paper's omega = 1."""
    cfg = workloads.config("c1", n=100, M=100, N=5, eta=3, K_it=64)
    s = solver(G, cfg, "mixed")
    r = s.solve()
    s.close()
    assert r.status == G.OK and r.K_it == 64
    res = np.array(r.resid_l2[:64])
    assert np.all(np.isfinite(res)) and np.all(res > 0)
    assert np.all(np.array(r.price_iter[:64]) != 0.0)


def test_errors_are_status_codes(G):
    cfg = workloads.config("c3", n=20, M=10, N=3, eta=4)  # p = 210 > n/2
    s = solver(G, cfg, "fp64")
    rep = s.solve(check=False)
    assert rep.status == G.ERR_ILLPOSED
    # a basis larger than the point set: singular Gram matrix, no trap
    cfg2 = workloads.config("c3", n=40, M=16, N=3, eta=3, K_it=1)  # p = 56 > n
    s2 = solver(G, cfg2, "fp64")
    rep = s2.solve(check=False, allow_underdetermined=1)
    assert rep.status == G.ERR_NOT_PD
    s2.close()
    # the context stays usable after the error
    s.cfg = workloads.config("c3", n=40, M=16, N=3, eta=1, K_it=1)
    s.set_grid(s.cfg)
    rep = s.solve(check=False)
    assert rep.status == G.OK
    s.close()
    bad = workloads.make(d=11, T=1.0, r=0.01, K=100.0, S0=100.0, vol={"kind": "const", "a": 0.2}, rho=0.0,
                         lam=0.0, n=100, M=8, N=2, eta=1, K_it=1, seed=1)
    s3 = solver(G, bad, "fp64")
    assert s3.solve(check=False).status == G.ERR_INVALID_ARG
    s3.close()
    # paths too long for the path kernel's shared-memory tables (per-step
    # volatility coefficients and Philox words): refused before any launch,
    # and the context stays usable
    long_n = workloads.config("c4", n=200, M=64, N=20000, eta=2, K_it=1)
    s7 = solver(G, long_n, "mixed")
    assert s7.solve(check=False).status == G.ERR_INVALID_ARG
    assert "shared-memory" in G.lib().bsde_last_error(s7.h).decode()
    s7.cfg = workloads.config("c4", n=200, M=64, N=400, eta=2, K_it=1)
    assert s7.solve(check=False).status == G.OK
    s7.close()
    # empty inputs: no paths, no steps, K_it beyond the report
    s6 = solver(G, workloads.config("c1", n=100, M=10, N=3, eta=2, K_it=1), "mixed")
    for kw in (dict(M=0), dict(N_steps=0), dict(K_it=65)):
        p = G.solve_params(s6.cfg)
        for k, v in kw.items():
            setattr(p, k, v)
        assert G.lib().bsde_solve(s6.h, __import__("ctypes").byref(p),
                                  __import__("ctypes").byref(G.bsde_report())) == G.ERR_INVALID_ARG
    s6.close()
    # the dense evaluation forced where it does not apply: a full correlation
    # matrix, and a degree-5 basis with FP64 paths (tree kernels are FP32)
    full = _case("d3_full_corr")
    full["K_it"] = 1
    s4 = solver(G, full, "mixed")
    assert s4.solve(check=False, eval_mode=2).status == G.ERR_INVALID_ARG
    assert s4.solve(check=False, eval_mode=0).status == G.OK
    s4.close()
    deg5 = workloads.config("c3", n=940, M=16, N=3, eta=5, K_it=1)
    s5 = solver(G, deg5, "fp64")
    assert s5.solve(check=False, eval_mode=2).status == G.ERR_INVALID_ARG
    assert s5.solve(check=False, eval_mode=0).status == G.OK
    s5.close()
