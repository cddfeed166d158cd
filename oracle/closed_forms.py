"""Reference prices used to pin the oracle end to end (test infrastructure).

  * Black-Scholes closed form of the European put/call and its delta (the
    omega = 0 case of Section 5.5 in one dimension with constant volatility);
  * the Cox-Ross-Rubinstein binomial tree for European and American puts
    (brute force for the American price of Section 5.2);
  * an implicit finite-difference solver of the penalised one-dimensional PDE
    d_t u + A u - r u + lambda (Phi - u)^+ = 0 (the PDE of eq. bsde-penal-2
    through the link of Section 2.2), i.e. the fixed point the Picard
    iteration targets.
"""
import math

import numpy as np


def norm_cdf(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def bs_d1d2(S, K, r, sigma, T, q=0.0):
    d1 = (math.log(S / K) + (r - q + 0.5 * sigma * sigma) * T) / (sigma * math.sqrt(T))
    return d1, d1 - sigma * math.sqrt(T)


def bs_put(S, K, r, sigma, T, q=0.0):
    d1, d2 = bs_d1d2(S, K, r, sigma, T, q)
    return K * math.exp(-r * T) * norm_cdf(-d2) - S * math.exp(-q * T) * norm_cdf(-d1)


def bs_call(S, K, r, sigma, T, q=0.0):
    d1, d2 = bs_d1d2(S, K, r, sigma, T, q)
    return S * math.exp(-q * T) * norm_cdf(d1) - K * math.exp(-r * T) * norm_cdf(d2)


def bs_put_delta(S, K, r, sigma, T, q=0.0):
    d1, _ = bs_d1d2(S, K, r, sigma, T, q)
    return -math.exp(-q * T) * norm_cdf(-d1)


def crr_put(S, K, r, sigma, T, steps, american=True):
    """Cox-Ross-Rubinstein tree, backward induction with early exercise."""
    dt = T / steps
    u = math.exp(sigma * math.sqrt(dt))
    dn = 1.0 / u
    disc = math.exp(-r * dt)
    pu = (math.exp(r * dt) - dn) / (u - dn)
    j = np.arange(steps + 1)
    ST = S * u ** (steps - j) * dn ** j
    V = np.maximum(K - ST, 0.0)
    for s in range(steps - 1, -1, -1):
        V = disc * (pu * V[:-1] + (1.0 - pu) * V[1:])
        if american:
            jj = np.arange(s + 1)
            Ss = S * u ** (s - jj) * dn ** jj
            V = np.maximum(V, K - Ss)
    return float(V[0])


def fd_penalised_put(S0, K, r, sigma_fn, T, lam, nx=800, nt=800, half_width=4.0):
    """Fully implicit finite differences in x = log S for
        u_t + 1/2 s^2 u_xx + (r - s^2/2) u_x - r u + lam (Phi - u)^+ = 0,
    u(T) = Phi = (K - e^x)^+, with the penalty linearised by a policy
    (Howard) iteration at each step.  sigma_fn(t, x) gives the local vol."""
    x0 = math.log(S0)
    x = np.linspace(x0 - half_width, x0 + half_width, nx + 1)
    dx = x[1] - x[0]
    dt = T / nt
    phi = np.maximum(K - np.exp(x), 0.0)
    u = phi.copy()
    for step in range(nt - 1, -1, -1):
        t = step * dt
        s = np.array([sigma_fn(t, xx) for xx in x])
        a = 0.5 * s * s / dx ** 2
        b = (r - 0.5 * s * s) / (2.0 * dx)
        lower = a - b
        upper = a + b
        diag_base = -2.0 * a - r
        rhs_base = u.copy()
        active = phi > u
        for _ in range(50):
            diag = 1.0 / dt - diag_base + lam * active
            rhs = rhs_base / dt + lam * phi * active
            # Dirichlet boundaries: deep ITM ~ intrinsic, deep OTM ~ 0
            A = np.zeros((3, nx + 1))
            A[1] = diag
            A[0, 1:] = -upper[:-1]
            A[2, :-1] = -lower[1:]
            A[1, 0] = 1.0; A[0, 1] = 0.0; rhs[0] = K * math.exp(-r * (T - t)) - math.exp(x[0]) \
                if lam == 0.0 else max(phi[0], K * math.exp(-r * (T - t)) - math.exp(x[0]))
            A[1, -1] = 1.0; A[2, -2] = 0.0; rhs[-1] = 0.0
            from scipy.linalg import solve_banded
            new = solve_banded((1, 1), A, rhs)
            new_active = phi > new
            if np.array_equal(new_active, active):
                u_next = new
                break
            active = new_active
            u_next = new
        u = u_next
    return float(np.interp(x0, x, u))
