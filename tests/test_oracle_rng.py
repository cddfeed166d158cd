"""Pins of the oracle's random numbers: Philox4x32-10, uniforms, Box-Muller,
the points of Algorithm 2.  CPU only."""
import ctypes
import math
import os

import numpy as np
import pytest
from scipy import stats

import workloads
from oracle import bsde_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(tok, 16) for tok in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert O.philox(ctr, key) == expect


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
                  "/usr/local/cuda/targets/x86_64-linux/lib", ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4_32_10 generator, called (not read): with seed s
    its key is (s lo, s hi) and, in its default ordering, its j-th block of
    four words is the block of counter (0, 0, j, 0): subsequence j, offset 0."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 64
        buf = (ctypes.c_uint * n)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        got = [int(v) for v in buf]
    finally:
        lib.curandDestroyGenerator(gen)
    key = O.seed_key(seed)
    ours = []
    for blk in range(n // 4):
        ours += O.philox([0, 0, blk, 0], key)
    assert ours == got


def test_uniform_open_interval():
    L = O.lib()
    assert L.orc_uniform(0) == 2.0 ** -33
    assert L.orc_uniform(0xffffffff) == 1.0 - 2.0 ** -33
    assert L.orc_uniform(0x80000000) == 0.5 + 2.0 ** -33


def test_box_muller_polar_identities():
    """z0^2 + z1^2 = -2 ln u0 and atan2(z1, z0) = 2 pi u1 (mod 2 pi)."""
    rng = np.random.default_rng(5)
    for w0, w1 in rng.integers(0, 2 ** 32, size=(200, 2)):
        u0 = (int(w0) + 0.5) / 2 ** 32
        u1 = (int(w1) + 0.5) / 2 ** 32
        z0, z1 = O.box_muller(int(w0), int(w1))
        assert z0 * z0 + z1 * z1 == pytest.approx(-2.0 * math.log(u0), rel=1e-12, abs=1e-300)
        ang = math.atan2(z1, z0) % (2 * math.pi)
        assert min(abs(ang - 2 * math.pi * u1), 2 * math.pi - abs(ang - 2 * math.pi * u1)) < 1e-9


def test_path_normals_are_standard_normal():
    cfg = workloads.config("c3")
    z = np.concatenate([O.path_normals(cfg, 0, i, m, 400) for i in range(5) for m in range(50)])
    n = len(z)
    assert abs(z.mean()) < 4.0 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4.0 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 4.0 * math.sqrt(24.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # adjacent draws uncorrelated
    assert abs(np.corrcoef(z[:-1], z[1:])[0, 1]) < 4.0 / math.sqrt(n)


def test_points_uniform_on_box_and_reproducible():
    cfg = workloads.config("c3", n=4000)
    t, x = O.points(cfg, 3)
    lo, hi = np.array(cfg["lo"]), np.array(cfg["hi"])
    assert t.min() > lo[0] and t.max() < hi[0]
    for j in range(cfg["d"]):
        assert x[j].min() > lo[j + 1] and x[j].max() < hi[j + 1]
        assert stats.kstest((x[j] - lo[j + 1]) / (hi[j + 1] - lo[j + 1]), "uniform").pvalue > 1e-3
    assert stats.kstest(t / cfg["T"], "uniform").pvalue > 1e-3
    t2, x2 = O.points(cfg, 3)
    assert np.array_equal(t, t2) and np.array_equal(x, x2)
    t3, _ = O.points(cfg, 4)
    assert not np.array_equal(t, t3)
    # one coordinate from its counter
    w = O.philox([1, 17, 0, (1 << 24) | 3], O.seed_key(cfg["seed"]))[1]
    u = (w + 0.5) / 2 ** 32
    assert x[4, 17] == lo[5] + (hi[5] - lo[5]) * u
