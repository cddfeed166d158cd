"""Pins of the oracle's least-squares extrapolation (eq. lspb / eq. alpha),
of one full iteration of Algorithm 2 and of the reference pricers.  CPU only."""
import math
import os

import numpy as np
import pytest

import workloads
from oracle import bsde_oracle as O
from oracle import closed_forms as CF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fit_reproduces_functions_in_the_span():
    cfg = workloads.config("c3")
    nu = O.multi_index_set(6, 4)
    t, x = O.points(cfg, 0, 900)
    B = O.basis_matrix(cfg, nu, t, x)
    alpha = np.random.default_rng(0).standard_normal(len(nu))
    assert np.allclose(O.fit(B, B @ alpha), alpha, rtol=1e-9, atol=1e-9)


def test_fit_of_a_line_is_the_textbook_regression():
    cfg = workloads.config("c1")
    nu = np.array([[0, 0], [0, 1]], dtype=np.int32)
    t, x = O.points(cfg, 0, 50)
    y = np.sin(x[0])
    xi = O.reduce_coords(cfg, t, x)[1]
    slope = np.sum((xi - xi.mean()) * (y - y.mean())) / np.sum((xi - xi.mean()) ** 2)
    icpt = y.mean() - slope * xi.mean()
    a = O.fit(O.basis_matrix(cfg, nu, t, x), y)
    assert a == pytest.approx([icpt, slope], rel=1e-12, abs=1e-12)


def test_black_scholes_textbook_values():
    with open(os.path.join(GOLDEN, "black_scholes_textbook.txt")) as f:
        rows = [list(map(float, l.split())) for l in f if l.strip() and not l.startswith("#")]
    for S, K, r, s, T, call, put in rows:
        assert round(CF.bs_call(S, K, r, s, T), 2) == call
        assert round(CF.bs_put(S, K, r, s, T), 2) == put
        # put-call parity
        assert CF.bs_call(S, K, r, s, T) - CF.bs_put(S, K, r, s, T) == pytest.approx(
            S - K * math.exp(-r * T), rel=1e-12)


def test_crr_tree():
    S, K, r, s, T = 100.0, 100.0, 0.02, 0.2, 1.0
    eu = CF.crr_put(S, K, r, s, T, 2000, american=False)
    am = CF.crr_put(S, K, r, s, T, 2000, american=True)
    assert abs(eu - CF.bs_put(S, K, r, s, T)) < 2e-3
    assert am > eu
    # no early exercise premium for a put when r = 0
    assert CF.crr_put(S, K, 0.0, s, T, 1000, True) == pytest.approx(
        CF.crr_put(S, K, 0.0, s, T, 1000, False), rel=1e-12)


def test_fd_penalised_put_brackets():
    S, K, r, s, T = 100.0, 100.0, 0.05, 0.2, 1.0
    eu = CF.fd_penalised_put(S, K, r, lambda t, x: s, T, 0.0, nx=400, nt=200)
    assert abs(eu - CF.bs_put(S, K, r, s, T)) < 0.02
    am = CF.crr_put(S, K, r, s, T, 2000, True)
    p10 = CF.fd_penalised_put(S, K, r, lambda t, x: s, T, 10.0, nx=400, nt=200)
    p1000 = CF.fd_penalised_put(S, K, r, lambda t, x: s, T, 1000.0, nx=400, nt=200)
    assert eu < p10 < p1000
    assert abs(p1000 - am) < 0.03


def test_first_iteration_is_the_projection_of_the_expected_payoff():
    """k = 0 with omega = 0: alpha^1 is the least-squares fit of c^0, whose
    mean at (t_i, x_i) is e^{r(T-t_i)} BS_put(S_i, T - t_i).  The price
    u^1(0, x0) must match the same fit of the exact values within four
    standard errors of the propagated Monte Carlo noise."""
    cfg = workloads.config("c1", n=120, M=4000)
    nu = O.multi_index_set(2, cfg["eta"])
    it = O.iteration(cfg, nu, np.zeros(len(nu)), 0)
    t, x, B = it["t"], it["x"], it["B"]
    exact = np.array([CF.bs_put(math.exp(x[0, i]), 100.0, 0.02, 0.2, 1 - t[i]) * math.exp(0.02 * (1 - t[i]))
                      for i in range(len(t))])
    a_exact = O.fit(B, exact)
    # standard error of each c_i from its samples
    se = np.array([O.samples(cfg, nu, np.zeros(len(nu)), t[i], x[:, i], 0, i).std(ddof=1)
                   for i in range(len(t))]) / math.sqrt(cfg["M"])
    b0 = O.basis_matrix(cfg, nu, np.array([0.0]), np.array([[math.log(100.0)]]))[0]
    w = B @ np.linalg.solve(B.T @ B, b0)
    sd = math.sqrt(np.sum((w * se) ** 2))
    p_fit = O.price_delta(cfg, nu, it["alpha"])[0]
    p_exact = O.price_delta(cfg, nu, a_exact)[0]
    assert abs(p_fit - p_exact) < 4 * sd


def test_european_solve_approaches_black_scholes():
    """Algorithm 2 end to end for a European put (omega = 0), degree 6 on
    log S0 +- 1: every iterate after the first within 4% of Black-Scholes,
    their mean within 2%, every delta within 0.02.  (Higher degrees on
    narrower boxes make the iteration unstable: paths leave the box where
    the fitted polynomial and its derivatives grow quickly.)"""
    cfg = workloads.make(d=1, T=1.0, r=0.02, K=100.0, S0=100.0, vol={"kind": "const", "a": 0.2},
                         rho=0.0, lam=0.0, n=600, M=4000, N=10, eta=6, K_it=4, seed=21,
                         half_width=1.0)
    res = O.solve(cfg)
    bs = CF.bs_put(100.0, 100.0, 0.02, 0.2, 1.0)
    bsd = CF.bs_put_delta(100.0, 100.0, 0.02, 0.2, 1.0)
    prices = [h["price"] for h in res["history"][1:]]
    assert all(abs(p - bs) < 0.04 * bs for p in prices)
    assert abs(np.mean(prices) - bs) < 0.02 * bs
    assert all(abs(h["delta"][0] - bsd) < 0.02 for h in res["history"][1:])


def _put_d1(lam, r, S0, K_it):
    return workloads.make(d=1, T=1.0, r=r, K=100.0, S0=S0, vol={"kind": "const", "a": 0.2},
                          rho=0.0, lam=lam, n=600, M=4000, N=10, eta=6, K_it=K_it, seed=21,
                          half_width=1.0)


def test_picard_residual_decreases():
    """The Picard map of Algorithm 2 contracts: with the driver's Lipschitz
    constant omega, the error after k iterations is bounded by
    (omega T)^k / k! times the first one (plus the Monte Carlo and
    projection floor).  European put (omega = 0): the second step is already
    at the floor, far below the first.  Penalised put with the paper's
    omega = 1: the steps shrink one after the other before reaching it."""
    eu = O.solve(_put_d1(0.0, 0.02, 100.0, 3))["history"]
    assert eu[1]["resid_l2"] < 0.1 * eu[0]["resid_l2"]
    assert eu[2]["resid_l2"] < 0.1 * eu[0]["resid_l2"]
    am = O.solve(_put_d1(1.0, 0.1, 90.0, 4))["history"]
    r = [h["resid_l2"] for h in am]
    assert r[0] > r[1] > r[2] > r[3]
    assert r[3] < 0.1 * r[0]


def test_penalised_price_lies_between_european_and_american():
    """The penalised BSDE (eq. bsde-penal-2) adds omega (Phi - Y)^+ >= 0 to
    the European driver and its solution increases to the American price as
    omega grows (Section 5.4), so for omega = 1:
    BS European <= Y^omega <= American (CRR tree, 2000 steps).  With
    r = 0.1 and S0 = 90 the bracket is wide (7.43 .. 10.43); the mean of the
    converged iterates also matches the finite-difference solution of the
    penalised PDE (8.46) within 10 % (Monte Carlo noise of four iterates,
    the degree-6 projection and the 10-step time grid: 8.96 here)."""
    res = O.solve(_put_d1(1.0, 0.1, 90.0, 8))
    prices = np.array([h["price"] for h in res["history"][4:]])
    eu = CF.bs_put(90.0, 100.0, 0.1, 0.2, 1.0)
    am = CF.crr_put(90.0, 100.0, 0.1, 0.2, 1.0, 2000, True)
    fd = CF.fd_penalised_put(90.0, 100.0, 0.1, lambda t, x: 0.2, 1.0, 1.0, nx=400, nt=200)
    assert np.all(prices > eu) and np.all(prices < am)
    assert abs(prices.mean() - fd) < 0.10 * fd


def test_penalised_limit_dominates_the_payoff():
    """The American price (the limit of the penalised solutions) is at least
    the payoff: the finite-difference penalised put at omega = 1000 is above
    max(K - S, 0) up to its O(1/omega) penalty gap, at, in and out of the money."""
    for S in (60.0, 80.0, 90.0, 100.0, 120.0):
        p = CF.fd_penalised_put(S, 100.0, 0.1, lambda t, x: 0.2, 1.0, 1000.0, nx=400, nt=200)
        assert p >= max(100.0 - S, 0.0) - 0.05
