"""Pins of the oracle's polynomial basis (Section 3.2.2): multi-index sets,
Chebyshev values and derivatives, domain reduction.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import workloads
from oracle import bsde_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_basis_size_paper_example():
    with open(os.path.join(GOLDEN, "basis_size_example.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for dp, eta, p in rows:
        assert O.multi_index_set(int(dp), int(eta)).shape == (int(p), int(dp))


@pytest.mark.parametrize("dp,eta", [(2, 4), (2, 6), (6, 4), (11, 3), (3, 0), (1, 5), (4, 6)])
def test_total_degree_set_brute_force(dp, eta):
    nu = O.multi_index_set(dp, eta)
    assert nu.shape[0] == math.comb(dp + eta, eta)
    brute = {t for t in itertools.product(range(eta + 1), repeat=dp) if sum(t) <= eta}
    got = [tuple(r) for r in nu]
    assert len(set(got)) == len(got)
    assert set(got) == brute
    deg = nu.sum(axis=1)
    assert np.all(np.diff(deg) >= 0)  # graded
    for a, b in zip(got, got[1:]):  # descending lexicographic within a degree
        if sum(a) == sum(b):
            assert a > b


def test_hyperbolic_sets():
    full = {tuple(r) for r in O.multi_index_set(6, 4)}
    for q in (0.9, 0.75, 0.6, 0.5):
        hyp = {tuple(r) for r in O.multi_index_set(6, 4, q)}
        assert hyp <= full
        for v in range(6):  # single-variate terms always kept
            for e in range(5):
                t = [0] * 6; t[v] = e
                assert tuple(t) in hyp
        # (1,1,0,...) has pseudo-norm 2^{1/q}
        assert ((1, 1, 0, 0, 0, 0) in hyp) == (2.0 ** (1.0 / q) <= 4.0 + 1e-9)
    sizes = [len(O.multi_index_set(11, 5, q)) for q in (0.5, 0.6, 0.8, 1.0)]
    assert sizes == sorted(sizes)
    assert {tuple(r) for r in O.multi_index_set(6, 4, 1.0)} == full


def test_chebyshev_cosine_identity():
    """T_e(cos th) = cos(e th) through the oracle's C recurrence."""
    cfg = workloads.make(d=1, T=1.0, r=0.0, K=1.0, S0=1.0, vol={"kind": "const", "a": 0.2},
                         rho=0.0, lam=0.0, n=1, M=1, N=1, eta=7, K_it=1, seed=0, half_width=1.0)
    nu = np.array([[0, e] for e in range(8)], dtype=np.int32)
    for th in np.linspace(0.05, 3.0, 9):
        x = np.array([math.cos(th)])  # lo = -1, hi = 1 around log S0 = 0
        for e in range(8):
            alpha = np.zeros(8); alpha[e] = 1.0
            u, ut, ux, uxx = O.basis_eval(cfg, nu, alpha, 0.3, x)
            assert u == pytest.approx(math.cos(e * th), abs=1e-13)


def test_basis_eval_matches_numpy_and_finite_differences():
    cfg = workloads.config("c3")
    nu = O.multi_index_set(cfg["d"] + 1, cfg["eta"])
    rng = np.random.default_rng(11)
    alpha = rng.standard_normal(len(nu))
    t, x = O.points(cfg, 0, 5)
    B = O.basis_matrix(cfg, nu, t, x)  # numpy chebvander
    ug, gg = O.eval_u(cfg, nu, alpha, t, x)
    for i in range(5):
        xi = x[:, i].copy()
        u, ut, ux, uxx = O.basis_eval(cfg, nu, alpha, t[i], xi)
        assert u == pytest.approx(B[i] @ alpha, rel=1e-12, abs=1e-12)
        assert np.allclose(ux, gg[:, i], rtol=1e-11, atol=1e-11)
        # fourth-order central differences
        h = 1e-3

        def fd(f):
            return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

        assert ut == pytest.approx(fd(lambda s: O.basis_eval(cfg, nu, alpha, t[i] + s, xi)[0]),
                                   rel=1e-8, abs=1e-8)
        for j in range(cfg["d"]):
            e = np.zeros(cfg["d"]); e[j] = 1.0
            col = fd(lambda s: O.basis_eval(cfg, nu, alpha, t[i], xi + s * e)[2])
            assert np.allclose(uxx[j], col, rtol=1e-8, atol=1e-7)
        assert np.allclose(uxx, uxx.T, atol=1e-12)


def test_domain_reduction_maps_box_to_unit_cube():
    cfg = workloads.config("c4")
    lo, hi = np.array(cfg["lo"]), np.array(cfg["hi"])
    xi = O.reduce_coords(cfg, np.array([lo[0], hi[0]]), np.stack([lo[1:], hi[1:]], axis=1))
    assert np.allclose(xi[:, 0], -1.0) and np.allclose(xi[:, 1], 1.0)
