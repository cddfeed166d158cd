"""The pivoted-QR refit (ls_mode 1, the role of LAPACK dgelsy in the paper):
it solves the same least-squares problem as the normal equations on
well-conditioned bases, and still solves it where the Gram matrix is
numerically singular."""
import numpy as np
import pytest

import workloads
from oracle import bsde_oracle as O

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_qr_refit_matches_least_squares(prec):
    import paper_1102_4666_gb300 as G
    cfg = workloads.config("c4", n=900, M=64, N=4, eta=3)
    nu = O.multi_index_set(11, 3)
    a0 = np.random.default_rng(3).standard_normal(len(nu)) * 0.3
    s = G.Solver(cfg, precision=prec)
    t, x, c, a1 = s.iterate(1, a0, ls_mode=1)
    s.close()
    B = O.basis_matrix(cfg, nu, t, x)
    assert rel(a1 - a0, O.fit(B, c)) < 1e-9


def test_qr_handles_a_rank_deficient_basis():
    """p > n: the Gram matrix is singular (normal equations fail with
    NOT_PD); the pivoted QR returns a basic solution of rank n that fits the
    data exactly."""
    import paper_1102_4666_gb300 as G
    cfg = workloads.config("c3", n=40, M=16, N=3, eta=3, K_it=1)  # p = 84 > n = 40
    nu = O.multi_index_set(6, 3)
    a0 = np.zeros(len(nu))
    s = G.Solver(cfg, precision="fp64")
    t, x, c, a1 = s.iterate(0, a0, ls_mode=1, allow_underdetermined=1)
    rep = s.solve(check=False, allow_underdetermined=1, ls_mode=1)
    assert rep.status == G.OK and rep.rank == 40
    s.close()
    B = O.basis_matrix(cfg, nu, t, x)
    assert np.max(np.abs(B @ a1 - c)) < 1e-8 * max(1.0, np.max(np.abs(c)))


def test_qr_solve_matches_normal_equation_solve():
    import paper_1102_4666_gb300 as G
    cfg = workloads.config("c3", n=500, M=200, N=10, eta=3, K_it=3)
    s = G.Solver(cfg, precision="fp64")
    r0 = s.solve(ls_mode=0)
    a_chol = s.coeffs()
    r1 = s.solve(ls_mode=1)
    a_qr = s.coeffs()
    s.close()
    assert r1.rank == r1.p
    assert rel(a_qr, a_chol) < 1e-8
    assert abs(r1.price - r0.price) < 1e-8 * abs(r0.price)
