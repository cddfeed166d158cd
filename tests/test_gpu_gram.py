"""Element-wise accuracy of the Gram matrix A = B^T B of the normal equations
(eq. alphasys, Section 3.2.2), read back through bsde_gram_matrix and
compared with the oracle's B^T B at the same (oracle-drawn) points.

The refit of a solve restores FP64 accuracy by iterative refinement against
the FP64 basis matrix, so the parity of the coefficients says little about A
itself; these tests bound A directly.

Error bound of the 3xTF32 tensor-core product (FP32 accumulation).  For one
product b b' of basis values (|.| below taken element-wise):
  * b32 = fl32(b):            |b32 - b|             <= 2^-24 |b|
  * hi = tf32(b32) (cvt.rna): |b32 - hi|            <= 2^-11 |b32|
  * lo = tf32(b32 - hi):      |lo - (b32 - hi)|     <= 2^-11 |b32 - hi| <= 2^-22 |b32|
  * the MMA forms hi hi' + hi lo' + lo hi' = (hi + lo)(hi' + lo') - lo lo'
    exactly (a TF32 x TF32 product fits an FP32 significand), and
    |lo lo'| <= 2^-22 |b b'| (1 + 2^-20)
so the three products equal b b' within (2 * 2^-24 + 3 * 2^-22)(1 + 2^-19)
|b b'| < 2^-20 |b b'| (U_SPLIT).  Within one slice of the points the tensor
core accumulates the 3 m products of the slice (m points) in FP32: at most
3 m additions, each rounding (or truncating) with a relative error below
2^-23 (U_ACC), so |error| <= 3 m 2^-23 sum |b b'| to first order.  The FP64
sum of the slices adds nothing visible.  Hence
    |A - B^T B| <= (2^-20 + 3 m_max 2^-23) (|B|^T |B|)      element-wise,
m_max the points of the longest slice (slices are whole K-blocks of 32).
The bound is a worst case, and the accumulation term grows with the slice:
at the automatic split of the d = 10 workload (160-point slices) it admits
errors near 6e-5 of |B|^T |B|, which catches any slip of a descriptor, a
swizzle or a tile index (errors of order one) but not the loss of one of the
three split products (its terms hi lo' have random signs; 2e-5 on the
diagonal there).  With one K-block of 32 points per slice (gram_splits =
n_pad / 32) the bound is 1.2e-5 and does catch it, by a factor 2.7 on the
same data (tests/test_gram_bound.py checks that on the CPU); the cases below
include that split.

The FP64 path (k_gram_f64) accumulates each entry by n fused multiply-adds:
|A - B^T B| <= n 2^-53 / (1 - n 2^-53) (|B|^T |B|).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import bsde_oracle as O

pytestmark = pytest.mark.gpu

U_SPLIT = 2.0 ** -20
U_ACC = 2.0 ** -23
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def G():
    import paper_1102_4666_gb300 as G
    return G


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _slice_points(n, p, splits):
    """Points of the longest slice of the tensor-core Gram: K-blocks of 32
    points split as evenly as integer division allows (0: one wave of the
    device's multiprocessors over the upper 128 x 128 tiles)."""
    n_pad = (n + 31) // 32 * 32
    kblocks = n_pad // 32
    side = (p + 127) // 128
    tiles = side * (side + 1) // 2
    s = splits if splits > 0 else _sms() // tiles
    s = max(1, min(s, kblocks))
    longest = max(((q + 1) * kblocks) // s - (q * kblocks) // s for q in range(s))
    return 32 * longest


def _oracle_gram(cfg, k):
    nu = O.multi_index_set(cfg["d"] + 1, cfg["eta"], cfg.get("q", 1.0))
    t, x = O.points(cfg, k)
    B = O.basis_matrix(cfg, nu, t, x)
    return B, B.T @ B, np.abs(B).T @ np.abs(B)


CASES = [
    # name, overrides, gram_splits
    ("c4", {}, 0),                          # the d = 10 workload: p = 364, n = 4000
    ("c4", {}, 1),                          # one slice: every point accumulated in FP32
    ("c4", {}, 7),                          # uneven slices
    ("c4", {}, 125),                        # one K-block of 32 points per slice
    ("c3", {}, 63),                         # the same for d = 5 (n_pad = 2016)
    ("c3", {}, 0),                          # d = 5, p = 210, n = 2000
    ("c4", dict(n=2801, eta=4), 0),         # p = 1365 (11 x 11 tiles), ragged n
    ("c2", dict(n=77), 0),                  # p = 28 < one tile, n not a multiple of 32
    ("c4", dict(n=700, eta=5, q=0.6), 3),   # hyperbolic set (eq. hyper_set), p = 221
]


@pytest.mark.parametrize("name,over,splits", CASES)
def test_tensor_core_gram_elementwise(G, name, over, splits):
    cfg = workloads.config(name, **over)
    k = 3
    s = G.Solver(cfg, precision="mixed")
    A = s.gram(k, gram_splits=splits)
    s.close()
    B, ref, absref = _oracle_gram(cfg, k)
    m = _slice_points(cfg["n"], B.shape[1], splits)
    bound = (U_SPLIT + 3 * m * U_ACC) * absref
    err = np.abs(A - ref)
    assert np.array_equal(A, A.T)
    worst = float(np.max(err / bound))
    assert worst <= 1.0, "Gram error %.3g of the 3xTF32 bound" % worst


@pytest.mark.parametrize("name,over", [("c4", {}), ("c3", dict(n=777, eta=3))])
def test_fp64_gram_elementwise(G, name, over):
    cfg = workloads.config(name, **over)
    s = G.Solver(cfg, precision="fp64")
    A = s.gram(2)
    s.close()
    B, ref, absref = _oracle_gram(cfg, 2)
    n = cfg["n"]
    bound = n * U64 / (1 - n * U64) * absref
    assert np.max(np.abs(A - ref) / bound) <= 1.0


def test_gram_is_the_refit_matrix(G):
    """The matrix bsde_gram_matrix returns is the one the refit of the same
    iteration solves with: alpha^{k+1} - alpha^k = A^{-1} B^T c to the
    refinement's accuracy, with A read back and B, c from the oracle points
    and the GPU's own corrections."""
    cfg = workloads.config("c4", n=900, M=32, N=4, eta=3)
    nu = O.multi_index_set(11, 3)
    a0 = np.zeros(len(nu)); a0[0] = 5.0
    s = G.Solver(cfg, precision="mixed")
    A = s.gram(1)
    t, x, c, a1 = s.iterate(1, a0)
    s.close()
    B = O.basis_matrix(cfg, nu, t, x)
    delta = np.linalg.solve(B.T @ B, B.T @ c)
    assert np.max(np.abs(a1 - a0 - delta)) <= 1e-9 * np.max(np.abs(delta))
    # A differs from B^T B only within the 3xTF32 bound
    m = _slice_points(cfg["n"], len(nu), 0)
    assert np.max(np.abs(A - B.T @ B) / ((U_SPLIT + 3 * m * U_ACC) * np.abs(B).T @ np.abs(B))) <= 1.0
