"""Seeded synthetic workloads of the BSDE pricing problems.

This module holds input specifications only (model parameters, grid sizes,
seeds) and a seeded generator of the serving request mix.  It contains none
of the method's arithmetic and is shared by the CUDA library's tests and
bench and by the CPU oracle.

The four model configurations are synthetic basket-option problems of the
shape studied in Section 6 of Labart & Lelong (European and American basket
puts under Black-Scholes and local volatility, d up to 10, n ~ 10^3 points,
M ~ 10^3-10^4 paths, total-degree polynomial bases).  There is no dataset.
"""
import copy
import math
import random

# Every configuration is a plain dict; lists hold per-asset values.
#   vol kinds: "const"    sigma_j = a
#              "abs_tanh" sigma = a + b e^{-t} |tanh(x - log K)|
#              "sin_tanh" sigma_j = a + b sin(j + t) tanh(x_j - log K), j = 1..d
#              "dupire"   eq. vol_locale of the paper (Section 6.3)


def _box(T, S0, half_width):
    lo = [0.0] + [math.log(s) - half_width for s in S0]
    hi = [T] + [math.log(s) + half_width for s in S0]
    return lo, hi


def make(d, T, r, K, S0, vol, rho, lam, n, M, N, eta, K_it, seed, payoff="put", q=1.0,
         div=0.0, obstacle="payoff", half_width=1.5, weights=None, name=""):
    S0 = [float(S0)] * d if not isinstance(S0, (list, tuple)) else [float(s) for s in S0]
    lo, hi = _box(T, S0, half_width)
    return {
        "name": name,
        "d": d, "T": float(T), "r": float(r), "K": float(K), "S0": S0,
        "weights": list(weights) if weights is not None else [1.0 / d] * d,
        "payoff": payoff, "obstacle": obstacle,
        "vol": dict(vol), "rho": float(rho),
        "div": [float(div)] * d if not isinstance(div, (list, tuple)) else list(div),
        "lambda": float(lam),
        "lo": lo, "hi": hi,
        "n": int(n), "M": int(M), "N": int(N), "eta": int(eta), "q": float(q),
        "K_it": int(K_it), "seed": int(seed),
    }


LOG100 = math.log(100.0)

CONFIGS = {
    # European put d=1, GBM, checked against Black-Scholes
    "c1": make(d=1, T=1.0, r=0.02, K=100.0, S0=100.0,
               vol={"kind": "const", "a": 0.2}, rho=0.0, lam=0.0,
               n=200, M=500, N=20, eta=4, K_it=3, seed=1,
               name="european put d=1 GBM"),
    # American put d=1, penalised driver, local vol
    "c2": make(d=1, T=1.0, r=0.02, K=100.0, S0=100.0,
               vol={"kind": "abs_tanh", "a": 0.15, "b": 0.1, "kappa": LOG100},
               rho=0.0, lam=50.0, n=1000, M=2000, N=50, eta=6, K_it=8, seed=2,
               name="american put d=1 local vol lambda=50"),
    # American basket put d=5
    "c3": make(d=5, T=1.0, r=0.03, K=100.0, S0=100.0,
               vol={"kind": "sin_tanh", "a": 0.2, "b": 0.05, "kappa": LOG100},
               rho=0.3, lam=100.0, n=2000, M=5000, N=50, eta=4, K_it=10, seed=3,
               name="american basket put d=5 local vol lambda=100"),
    # American basket put d=10 (the throughput workload)
    "c4": make(d=10, T=1.0, r=0.03, K=100.0, S0=100.0,
               vol={"kind": "sin_tanh", "a": 0.2, "b": 0.05, "kappa": LOG100},
               rho=0.2, lam=100.0, n=4000, M=4000, N=100, eta=3, K_it=12, seed=4,
               name="american basket put d=10 local vol lambda=100"),
}


# The two workloads of the paper's timing tables (Section 6.4: American basket
# put, Black-Scholes with sigma = 0.2, rho = 0, r = 0.02, T = 1, S0 = 100,
# K = 95, N = 10 steps, K_it = 10 iterations, n = 2000 points, degree 3,
# q = 1, omega = 1): d = 3 with M = 1000 and d = 6 with M = 5000.  The paper
# does not give the domain D; these use log S0 +- 0.25, the box on which the
# paper's printed American prices are reproduced.
PAPER_TIMING = {
    "paper_d3": make(d=3, T=1.0, r=0.02, K=95.0, S0=100.0, vol={"kind": "const", "a": 0.2}, rho=0.0,
                     lam=1.0, n=2000, M=1000, N=10, eta=3, K_it=10, seed=31, half_width=0.25,
                     name="paper timing table: american put d=3"),
    "paper_d6": make(d=6, T=1.0, r=0.02, K=95.0, S0=100.0, vol={"kind": "const", "a": 0.2}, rho=0.0,
                     lam=1.0, n=2000, M=5000, N=10, eta=3, K_it=10, seed=32, half_width=0.25,
                     name="paper timing table: american put d=6"),
}
# the paper's wall times for them (seconds): on 8 processes, and the fastest
# of its process counts (d = 3: 64 processes; d = 6: 256 processes)
PAPER_TIMING_SECONDS = {"paper_d3": (543.677, 97.0629, 64), "paper_d6": (1196.79, 35.9239, 256)}


def config(name, **overrides):
    """A copy of a named configuration with some fields replaced."""
    cfg = copy.deepcopy(CONFIGS[name] if name in CONFIGS else PAPER_TIMING[name])
    for key, val in overrides.items():
        cfg[key] = val
    return cfg


def path_steps(cfg):
    """Euler path-steps of one full solve: K_it * n * M * N."""
    return cfg["K_it"] * cfg["n"] * cfg["M"] * cfg["N"]


def basis_size(d, eta):
    """Binomial(d + 1 + eta, eta): size of the total-degree basis."""
    return math.comb(d + 1 + eta, eta)


def serving_mix(n_requests=2000, seed=7, rate_hz=None):
    """Seeded Poisson stream of pricing requests of uneven size.

    Per request: d in {1,2,5,10}, strike K ~ U[80,120], maturity T ~ U[0.25,2],
    points n in 200..4000, paths M in 500..8000, total degree eta in 2..6
    restricted so that the basis size p <= n/2, lambda in {0, 100}, its own
    seed.  Fixed fill-ins: S0 = 100, r = 0.03, rho = 0.3, N = 50 Euler steps,
    K_it = 10 iterations, domain log S0 +- 1.5.  Arrival times are returned
    as offsets in seconds when rate_hz is given (exponential gaps).
    """
    rng = random.Random(seed)
    reqs = []
    t = 0.0
    for j in range(n_requests):
        d = rng.choice([1, 2, 5, 10])
        K = rng.uniform(80.0, 120.0)
        T = rng.uniform(0.25, 2.0)
        n = rng.randint(200, 4000)
        M = rng.randint(500, 8000)
        etas = [e for e in range(2, 7) if basis_size(d, e) <= n // 2]
        eta = rng.choice(etas)
        lam = rng.choice([0.0, 100.0])
        if d == 1:
            vol = {"kind": "abs_tanh", "a": 0.15, "b": 0.1, "kappa": math.log(K)}
        else:
            vol = {"kind": "sin_tanh", "a": 0.2, "b": 0.05, "kappa": math.log(K)}
        cfg = make(d=d, T=T, r=0.03, K=K, S0=100.0, vol=vol, rho=0.3 if d > 1 else 0.0,
                   lam=lam, n=n, M=M, N=50, eta=eta, K_it=10, seed=1000 + j,
                   name="serving request %d" % j)
        if rate_hz:
            t += rng.expovariate(rate_hz)
            cfg["arrival_s"] = t
        reqs.append(cfg)
    return reqs
