"""Teacher-forced parity on seeded random configurations.

Besides the hand-picked cases of test_gpu_parity.py, one Picard iteration
(Algorithm 2) from the same alpha^k is compared with the FP64 oracle on
configurations drawn at random, with a fixed seed, over every axis the
kernels specialise on or branch over: the dimension d = 1..10 (one kernel
family per d, with its own grouping of Euler steps into Philox blocks), the
total degree (dense degree-3 and degree-4 loops, the prefix-tree recursion
of degrees 4 to 6, the per-thread Chebyshev tables), hyperbolic index sets
(eq. hyper_set), every volatility family, put and call payoffs, the payoff
and raw obstacles of the penalised driver (eq. bsde-penal-2), penalty
weights from 0 (European) to 100, positive and negative constant
correlations, dividends, maturities, strikes and rates, and ragged sizes
(n just above 2 p, M and N from 1).  Tolerances are those of the fixed
cases: 1e-9 of the integrand's scale in FP64, MIXED_C_TOL of it in mixed
precision, and 1e-9 relative on the FP64 coefficients alpha^{k+1}.  Whole
FP64 solves on random small configurations against the oracle's solve, and
whole mixed solves against FP64 ones, close the file.
"""
import random

import numpy as np
import pytest

import workloads
from oracle import bsde_oracle as O
from test_gpu_parity import MIXED_C_TOL, NTH, _alpha, _scale, rel

pytestmark = pytest.mark.gpu

N_CASES = 48


def _random_case(k):
    rng = random.Random(7000 + k)
    d = rng.randint(1, 10)
    eta = rng.randint(1, 6 if d <= 5 else 4)
    q = rng.choice([1.0, 1.0, 1.0, 0.75])
    nu = O.multi_index_set(d + 1, eta, q)
    p = len(nu)
    kind = rng.choice(["const", "abs_tanh", "sin_tanh", "dupire"])
    if kind == "const":
        vol = {"kind": "const", "a": [rng.uniform(0.1, 0.4) for _ in range(d)]}
    elif kind == "dupire":
        vol = {"kind": "dupire", "s": 100.0}
    else:
        vol = {"kind": kind, "a": rng.uniform(0.12, 0.25), "b": rng.uniform(0.02, 0.1),
               "kappa": float(np.log(rng.uniform(90.0, 110.0)))}
    # a constant correlation keeps the matrix positive definite above -1/(d-1)
    rho = 0.0 if d == 1 else rng.choice([0.0, 0.3, 0.6, -0.05])
    cfg = workloads.make(d=d, T=rng.choice([0.5, 1.0, 2.0]), r=rng.uniform(0.0, 0.05),
                         K=rng.uniform(80.0, 120.0), S0=100.0, vol=vol, rho=rho,
                         lam=rng.choice([0.0, 1.0, 100.0]), n=2 * p + rng.randint(1, 40),
                         M=rng.randint(1, 70), N=rng.randint(1, 9), eta=eta, K_it=1,
                         seed=rng.randint(1, 10**6), payoff=rng.choice(["put", "call"]), q=q,
                         div=[rng.uniform(0.0, 0.03) for _ in range(d)],
                         obstacle=rng.choice(["payoff", "raw"]))
    ev = rng.choice([0, 0, 1])  # automatic (dense where it applies) or the per-thread tables
    return cfg, nu, ev


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("k", range(N_CASES))
def test_random_configuration(k, prec):
    import paper_1102_4666_gb300 as G
    cfg, nu, ev = _random_case(k)
    a0 = _alpha(cfg, nu, seed=11 + k)
    it_k = k % 5
    s = G.Solver(cfg, precision=prec)
    t, x, c, a1 = s.iterate(it_k, a0, eval_mode=ev)
    s.close()
    it = O.iteration(cfg, nu, a0, it_k, nthreads=NTH)
    sc = _scale(cfg, nu, a0, t, x)
    tol = 1e-9 if prec == "fp64" else MIXED_C_TOL
    assert np.max(np.abs(c - it["c"])) < tol * sc, (cfg["d"], cfg["eta"], cfg["vol"]["kind"], ev)
    if prec == "fp64":
        assert rel(a1, it["alpha"]) < 1e-9


# Whole FP64 solves (several Picard iterations, points redrawn each time,
# refit and update on the device, with and without the captured graph)
# against the oracle's own solve, on seeded random small configurations.
# The penalty weight stays <= 1 (with maturities <= 2): there the Picard map
# contracts, so the rounding differences of the two sides (libm ulps,
# summation order) are not amplified past 1e-9 over the iterations.
N_SOLVES = 8


def _random_solve_case(k):
    rng = random.Random(9100 + k)
    d = rng.randint(1, 6)
    eta = rng.randint(1, 4 if d <= 3 else 3)
    p = workloads.basis_size(d, eta)
    kind = rng.choice(["const", "abs_tanh", "sin_tanh"])
    if kind == "const":
        vol = {"kind": "const", "a": [rng.uniform(0.1, 0.3) for _ in range(d)]}
    else:
        vol = {"kind": kind, "a": rng.uniform(0.12, 0.25), "b": rng.uniform(0.02, 0.1),
               "kappa": float(np.log(100.0))}
    cfg = workloads.make(d=d, T=rng.choice([0.5, 1.0, 2.0]), r=rng.uniform(0.0, 0.05),
                         K=rng.uniform(85.0, 115.0), S0=100.0, vol=vol,
                         rho=0.0 if d == 1 else rng.choice([0.0, 0.3]),
                         lam=rng.choice([0.0, 0.5, 1.0]), n=2 * p + rng.randint(5, 60),
                         M=rng.randint(8, 60), N=rng.randint(2, 8), eta=eta,
                         K_it=rng.randint(2, 3), seed=rng.randint(1, 10**6),
                         payoff=rng.choice(["put", "call"]))
    return cfg, rng.choice([0, 1])


@pytest.mark.parametrize("k", range(N_SOLVES))
def test_random_fp64_solve(k):
    import paper_1102_4666_gb300 as G
    cfg, use_graph = _random_solve_case(k)
    s = G.Solver(cfg, precision="fp64")
    rep = s.solve(use_graph=use_graph)
    alpha = s.coeffs()
    s.close()
    assert rep.status == G.OK
    ref = O.solve(cfg, nthreads=NTH)
    assert rel(alpha, ref["alpha"]) < 1e-9
    assert abs(rep.price - ref["price"]) <= 1e-9 * max(abs(ref["price"]), 1e-3)


# Whole mixed-precision solves against whole FP64 solves of the same random
# numbers (the FP64 path being pinned to the oracle above): the price and
# the deltas at (0, x0) within 1e-4 relative, on seeded random
# configurations of every dimension and evaluation form.
N_MIXED = 8


def _random_mixed_case(k):
    rng = random.Random(9300 + k)
    d = rng.randint(1, 10)
    eta = rng.randint(2, 6 if d <= 2 else (4 if d <= 5 else 3))
    p = workloads.basis_size(d, eta)
    kind = rng.choice(["const", "abs_tanh", "sin_tanh"])
    if kind == "const":
        vol = {"kind": "const", "a": [rng.uniform(0.1, 0.3) for _ in range(d)]}
    else:
        vol = {"kind": kind, "a": rng.uniform(0.12, 0.25), "b": rng.uniform(0.02, 0.1),
               "kappa": float(np.log(100.0))}
    return workloads.make(d=d, T=rng.choice([0.5, 1.0]), r=rng.uniform(0.0, 0.05),
                          K=rng.uniform(90.0, 110.0), S0=100.0, vol=vol,
                          rho=0.0 if d == 1 else rng.choice([0.0, 0.3]),
                          lam=rng.choice([0.0, 1.0]), n=2 * p + rng.randint(50, 300),
                          M=rng.randint(200, 600), N=rng.randint(8, 30), eta=eta, K_it=3,
                          seed=rng.randint(1, 10**6), payoff=rng.choice(["put", "call"]))


@pytest.mark.parametrize("k", range(N_MIXED))
def test_random_mixed_solve_against_fp64(k):
    import paper_1102_4666_gb300 as G
    cfg = _random_mixed_case(k)
    out = {}
    for prec in ("mixed", "fp64"):
        s = G.Solver(cfg, precision=prec)
        r = s.solve(use_graph=1)
        s.close()
        assert r.status == G.OK
        out[prec] = (r.price, np.array(r.delta[:cfg["d"]]))
    (pm, dm), (pf, df) = out["mixed"], out["fp64"]
    assert abs(pm - pf) <= 1e-4 * abs(pf)
    assert np.max(np.abs(dm - df)) <= 1e-4 * max(np.max(np.abs(df)), 1e-3)
