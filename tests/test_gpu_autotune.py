"""The launch-shape autotuner: it returns one of its candidates, stores it in
its cache, and a solve with the tuned shape gives the same coefficients as
the library's default shape up to the summation order of the per-point
reduction."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_tune_and_lookup(tmp_path, monkeypatch):
    monkeypatch.setenv("BSDE_TUNE_CACHE", str(tmp_path / "tune.json"))
    import paper_1102_4666_gb300 as G
    from paper_1102_4666_gb300 import autotune
    cfg = workloads.config("c3", n=300, M=600, N=10, eta=2, K_it=2)
    best = autotune.tune(cfg, "mixed", repeats=1)
    assert best in autotune.CANDIDATES["mixed"]
    assert autotune.lookup(cfg, "mixed") == best
    s = G.Solver(cfg, precision="mixed", launch_shape=best)
    r1 = s.solve()
    a1 = s.coeffs()
    s.launch_shape = None
    r0 = s.solve()
    a0 = s.coeffs()
    s.close()
    assert np.max(np.abs(a1 - a0)) <= 1e-9 * np.max(np.abs(a0))
    assert abs(r1.price - r0.price) <= 1e-9 * abs(r0.price)
