"""Pins of the oracle's Euler paths, Brownian bridge, model functions and of
the Monte Carlo sample a_m of Algorithm 2 (eq. psiN).  CPU only.

The expectations below come from closed forms (log-normal laws, the
Black-Scholes formula) or from Dynkin's formula, which holds exactly for the
Euler scheme eqs3 because its coefficients are constant on each step: for any
polynomial u, E[u(T, X_T)] - u(t, x) = E[int_t^T (d_t + L^N) u(s, X_s) ds],
and the random-time sample (T - t) g(tau) is unbiased for the integral
(Section 3.1).  Each check allows four Monte Carlo standard errors.
"""
import math

import numpy as np
import pytest
from scipy import stats

import workloads
from oracle import bsde_oracle as O
from oracle import closed_forms as CF


def gbm_cfg(**kw):
    base = dict(d=1, T=1.0, r=0.05, K=100.0, S0=100.0, vol={"kind": "const", "a": 0.25},
                rho=0.0, lam=0.0, n=16, M=20000, N=8, eta=4, K_it=1, seed=9, half_width=1.0)
    base.update(kw)
    return workloads.make(**base)


def test_cholesky_factor():
    for d, rho in [(2, 0.3), (5, 0.3), (10, 0.2), (4, -0.2)]:
        C = np.full((d, d), rho); np.fill_diagonal(C, 1.0)
        L = O.cholesky(C)
        assert np.allclose(np.triu(L, 1), 0.0)
        assert np.allclose(L @ L.T, C, atol=1e-14)
    with pytest.raises(ValueError):
        C = np.full((3, 3), -0.6); np.fill_diagonal(C, 1.0)
        O.cholesky(C)


def test_vol_families_special_values():
    L = O.lib()
    cfg = workloads.config("c3")
    m = O.model(cfg)
    k = math.log(100.0)
    for j in range(5):
        assert L.orc_sigma(m, j, 0.4, k) == pytest.approx(0.2, abs=1e-15)  # tanh(0) = 0
        assert L.orc_sigma(m, j, 0.4, k + 50.0) == pytest.approx(0.2 + 0.05 * math.sin(j + 1.4), rel=1e-12)
    m2 = O.model(workloads.config("c2"))
    assert L.orc_sigma(m2, 0, 0.7, k + 0.3) == pytest.approx(L.orc_sigma(m2, 0, 0.7, k - 0.3), rel=1e-14)
    assert L.orc_sigma(m2, 0, 0.0, k + 40.0) == pytest.approx(0.25, rel=1e-12)
    dup = workloads.make(d=1, T=1.0, r=0.05, K=100.0, S0=100.0,
                         vol={"kind": "dupire", "s": 100.0}, rho=0.0, lam=0.0, n=1, M=1, N=1,
                         eta=1, K_it=1, seed=0)
    m3 = O.model(dup)
    assert L.orc_sigma(m3, 0, 0.0, math.log(100.0)) == pytest.approx(0.6 * 0.2, rel=1e-12)


def test_payoff_values():
    cfg = workloads.config("c3")
    m = O.model(cfg)
    L = O.lib()
    x = np.full(5, math.log(100.0))
    assert L.orc_payoff(m, O._dptr(x)) == 0.0
    x = np.log(np.array([50.0, 60.0, 70.0, 80.0, 90.0]))
    assert L.orc_payoff(m, O._dptr(x)) == pytest.approx(30.0, rel=1e-13)
    # the call (eq. call_payoff): (sum_j w_j S_j - K)^+, zero below the strike
    call = workloads.config("c3", payoff="call")
    mc = O.model(call)
    assert L.orc_payoff(mc, O._dptr(x)) == 0.0
    x = np.log(np.array([110.0, 120.0, 130.0, 140.0, 150.0]))
    assert L.orc_payoff(mc, O._dptr(x)) == pytest.approx(30.0, rel=1e-13)
    assert L.orc_payoff(m, O._dptr(x)) == 0.0
    # unequal weights enter as the basket sum_j w_j S_j
    w = workloads.config("c3", payoff="call", weights=[0.5, 0.2, 0.1, 0.1, 0.1])
    mw = O.model(w)
    assert L.orc_payoff(mw, O._dptr(x)) == pytest.approx(0.5 * 110 + 24 + 13 + 14 + 15 - 100.0, rel=1e-13)


def test_gbm_log_euler_is_exact_in_law():
    """Constant sigma: X_T ~ N(x + (r - s^2/2)(T-t), s^2 (T-t)) and, given tau,
    X_tau ~ N(x + (r - s^2/2)(tau-t), s^2 (tau-t))."""
    cfg = gbm_cfg(N=7)
    t0, x0 = 0.2, np.array([math.log(90.0)])
    XT, Xtau, tau = O.simulate(cfg, 0, 3, t0, x0, 40000)
    s, r = 0.25, 0.05
    z = (XT[:, 0] - x0[0] - (r - 0.5 * s * s) * (1 - t0)) / (s * math.sqrt(1 - t0))
    assert stats.kstest(z, "norm").pvalue > 1e-3
    zt = (Xtau[:, 0] - x0[0] - (r - 0.5 * s * s) * (tau - t0)) / (s * np.sqrt(tau - t0))
    assert stats.kstest(zt, "norm").pvalue > 1e-3
    assert stats.kstest((tau - t0) / (1 - t0), "uniform").pvalue > 1e-3
    # the pair (X_tau, X_T) has the Brownian covariance s^2 (tau - t)
    wT = XT[:, 0] - x0[0] - (r - 0.5 * s * s) * (1 - t0)
    wt = Xtau[:, 0] - x0[0] - (r - 0.5 * s * s) * (tau - t0)
    ratio = np.mean(wT * wt) / np.mean(s * s * (tau - t0))
    assert abs(ratio - 1.0) < 0.05


def test_correlated_increments():
    cfg = workloads.make(d=3, T=1.0, r=0.0, K=100.0, S0=100.0, vol={"kind": "const", "a": 0.3},
                         rho=0.5, lam=0.0, n=1, M=1, N=4, eta=1, K_it=1, seed=3)
    XT, _, _ = O.simulate(cfg, 0, 0, 0.0, np.full(3, math.log(100.0)), 30000)
    C = np.corrcoef(XT.T)
    se = (1 - 0.25) / math.sqrt(30000)
    assert np.all(np.abs(C[np.triu_indices(3, 1)] - 0.5) < 4 * se)


def _undiscounted_put(S, K, r, sig, tau):
    if tau <= 0:
        return max(K - S, 0.0)
    return CF.bs_put(S, K, r, sig, tau) * math.exp(r * tau)


def _undiscounted_call(S, K, r, sig, tau):
    if tau <= 0:
        return max(S - K, 0.0)
    return CF.bs_call(S, K, r, sig, tau) * math.exp(r * tau)


@pytest.mark.parametrize("payoff", ["put", "call"])
def test_first_correction_is_expected_payoff(payoff):
    """u^0 = 0, omega = 0: c^0(t,x) = E[Phi(X_T)], that is e^{r(T-t)} BS_put
    for the put and e^{r(T-t)} BS_call for the call (eq. call_payoff)."""
    cfg = gbm_cfg(payoff=payoff)
    nu = O.multi_index_set(2, 2)
    alpha = np.zeros(len(nu))
    expect = _undiscounted_put if payoff == "put" else _undiscounted_call
    for (t0, S) in [(0.0, 100.0), (0.5, 80.0), (0.9, 115.0)]:
        a = O.samples(cfg, nu, alpha, t0, np.array([math.log(S)]), 0, 0)
        ref = expect(S, 100.0, 0.05, 0.25, 1.0 - t0)
        se = a.std(ddof=1) / math.sqrt(len(a))
        assert abs(a.mean() - ref) < 4 * se


@pytest.mark.parametrize("name", ["gbm1", "corr2", "lv5"])
def test_dynkin_identity_control_variate(name):
    """r = 0, omega = 0, u^k an arbitrary polynomial: the paired difference
    a_m(alpha) - a_m(0) + u^k(t,x) has mean zero (the control variate
    cancels u^k exactly in expectation)."""
    if name == "gbm1":
        cfg = gbm_cfg(r=0.0, M=6000)
    elif name == "corr2":
        cfg = workloads.make(d=2, T=1.0, r=0.0, K=100.0, S0=100.0, vol={"kind": "const", "a": 0.3},
                             rho=0.4, lam=0.0, n=1, M=6000, N=6, eta=3, K_it=1, seed=5)
    else:
        cfg = workloads.config("c3", r=0.0, M=3000, N=10)
        cfg["lambda"] = 0.0
    d = cfg["d"]
    nu = O.multi_index_set(d + 1, cfg["eta"])
    rng = np.random.default_rng(2)
    alpha = rng.standard_normal(len(nu)) * 3.0
    t0 = 0.3
    x0 = np.log(np.full(d, 100.0)) + 0.1 * rng.standard_normal(d)
    a1 = O.samples(cfg, nu, alpha, t0, x0, 1, 7)
    a0 = O.samples(cfg, nu, np.zeros(len(nu)), t0, x0, 1, 7)
    u0 = O.basis_eval(cfg, nu, alpha, t0, x0)[0]
    diff = a1 - a0 + u0
    se = diff.std(ddof=1) / math.sqrt(len(diff))
    assert abs(diff.mean()) < 4 * se
    # a plausible mistake (dropping the 1/2 of the generator) breaks it
    assert se < 0.05 * np.abs(alpha).sum()


def test_discount_term_of_the_driver():
    """omega = 0, r > 0, constant sigma: E[a(alpha) - a(0)] =
    -u(t,x) - r int_t^T E[u(s, X_s)] ds, the integral by Gauss quadrature."""
    cfg = gbm_cfg(r=0.08, M=8000)
    nu = O.multi_index_set(2, 3)
    rng = np.random.default_rng(4)
    alpha = rng.standard_normal(len(nu))
    t0, x0 = 0.25, math.log(95.0)
    a1 = O.samples(cfg, nu, alpha, t0, np.array([x0]), 2, 1)
    a0 = O.samples(cfg, nu, np.zeros(len(nu)), t0, np.array([x0]), 2, 1)
    s, r = 0.25, 0.08
    gl_x, gl_w = np.polynomial.legendre.leggauss(20)
    gh_x, gh_w = np.polynomial.hermite_e.hermegauss(30)
    integral = 0.0
    for xs, ws in zip(gl_x, gl_w):
        sv = t0 + (1 - t0) * (xs + 1) / 2
        mean = x0 + (r - 0.5 * s * s) * (sv - t0)
        sd = s * math.sqrt(sv - t0)
        xx = mean + sd * gh_x
        u = O.eval_u(cfg, nu, alpha, np.full(len(xx), sv), xx[None, :])[0]
        integral += ws * (1 - t0) / 2 * np.sum(gh_w * u) / math.sqrt(2 * math.pi)
    u0 = O.basis_eval(cfg, nu, alpha, t0, np.array([x0]))[0]
    expect = -u0 - r * integral
    diff = a1 - a0
    se = diff.std(ddof=1) / math.sqrt(len(diff))
    assert abs(diff.mean() - expect) < 4 * se


def test_penalty_term_of_the_driver():
    """r = 0, u^k = c0 constant, put payoff: E[a] = E[Phi(X_T)] - c0 +
    lambda int_t^T E[(K - c0 - S_s)^+] ds, each expectation a Black-Scholes
    put (r = 0) and the time integral by Gauss-Legendre."""
    lam, c0 = 3.0, 4.0
    cfg = gbm_cfg(r=0.0, lam=lam, M=20000)
    nu = O.multi_index_set(2, 2)
    alpha = np.zeros(len(nu)); alpha[0] = c0
    t0, S = 0.4, 97.0
    a = O.samples(cfg, nu, alpha, t0, np.array([math.log(S)]), 0, 2)
    gl_x, gl_w = np.polynomial.legendre.leggauss(40)
    integral = sum(w * (1 - t0) / 2 * _undiscounted_put(S, 100.0 - c0, 0.0, 0.25,
                                                        (1 - t0) * (x + 1) / 2)
                   for x, w in zip(gl_x, gl_w))
    expect = _undiscounted_put(S, 100.0, 0.0, 0.25, 1 - t0) - c0 + lam * integral
    se = a.std(ddof=1) / math.sqrt(len(a))
    assert abs(a.mean() - expect) < 4 * se


@pytest.mark.parametrize("payoff", ["put", "call"])
@pytest.mark.parametrize("obstacle", ["payoff", "raw"])
def test_penalty_obstacle_forms_separate(payoff, obstacle):
    """The two obstacles of the penalty (eq. bsde-penal-2 and the literal
    form of the d = 1 American configuration) with a negative constant
    u^k = c0 < 0, r = 0, where they differ:
      payoff form  lambda (Phi(X) - c0)^+  = lambda (Phi(X) + |c0|), so the
                   time integral is lambda int (E[Phi(X_s)] + |c0|) ds;
      raw form     lambda (I(X) - c0)^+ with I = K - S (put) or S - K (call),
                   a put of strike K + |c0| or a call of strike K - |c0|.
    Each expectation is a Black-Scholes price (r = 0), the integral by
    Gauss-Legendre.  A sign or positive-part slip in either branch moves the
    mean by many standard errors."""
    lam, c0 = 3.0, -4.0
    cfg = gbm_cfg(r=0.0, lam=lam, M=20000, payoff=payoff, obstacle=obstacle)
    nu = O.multi_index_set(2, 2)
    alpha = np.zeros(len(nu)); alpha[0] = c0
    t0, S = 0.4, 97.0 if payoff == "put" else 103.0
    a = O.samples(cfg, nu, alpha, t0, np.array([math.log(S)]), 0, 3)
    price = _undiscounted_put if payoff == "put" else _undiscounted_call
    gl_x, gl_w = np.polynomial.legendre.leggauss(40)
    integral = 0.0
    for x, w in zip(gl_x, gl_w):
        tau = (1 - t0) * (x + 1) / 2
        if obstacle == "payoff":
            inner = price(S, 100.0, 0.0, 0.25, tau) - c0
        else:
            inner = price(S, 100.0 - c0 if payoff == "put" else 100.0 + c0, 0.0, 0.25, tau)
        integral += w * (1 - t0) / 2 * inner
    expect = price(S, 100.0, 0.0, 0.25, 1 - t0) - c0 + lam * integral
    se = a.std(ddof=1) / math.sqrt(len(a))
    assert abs(a.mean() - expect) < 4 * se
    # the other form's expectation is far outside the Monte Carlo error
    other = 0.0
    for x, w in zip(gl_x, gl_w):
        tau = (1 - t0) * (x + 1) / 2
        if obstacle == "raw":
            inner = price(S, 100.0, 0.0, 0.25, tau) - c0
        else:
            inner = price(S, 100.0 - c0 if payoff == "put" else 100.0 + c0, 0.0, 0.25, tau)
        other += w * (1 - t0) / 2 * inner
    assert abs(lam * (other - integral)) > 10 * se


def test_correction_is_the_mean_of_the_samples():
    cfg = workloads.config("c2", M=300, N=12)
    nu = O.multi_index_set(2, 3)
    alpha = np.random.default_rng(1).standard_normal(len(nu))
    t, x = O.points(cfg, 1, 6)
    c = O.correction(cfg, nu, alpha, 1, np.arange(6), t, x, nthreads=3)
    for i in range(6):
        a = O.samples(cfg, nu, alpha, t[i], x[:, i], 1, i)
        assert c[i] == pytest.approx(a.sum() / len(a), rel=1e-14, abs=1e-14)
