"""CPU check that the element-wise error bound of the 3xTF32 tensor-core Gram
matrix used in tests/test_gpu_gram.py (derivation there) is tight enough to
catch a plausible kernel mistake: leaving out one of the three split
products hi hi' + hi lo' + lo hi'.  The split is emulated in numpy (FP32,
then TF32 by round-to-nearest-away on the 13 low mantissa bits, as
cvt.rna.tf32.f32 does) on the oracle's basis matrix of the d = 10 workload.
"""
import numpy as np

import workloads
from oracle import bsde_oracle as O

U_SPLIT = 2.0 ** -20
U_ACC = 2.0 ** -23
# slices of one K-block of 32 points (gram_splits = n_pad / 32), where the
# worst-case bound is tight enough for this check
M_SLICE = 32


def _tf32(v):
    bits = v.view(np.uint32)
    return ((bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def test_bound_catches_a_dropped_product():
    cfg = workloads.config("c4")
    nu = O.multi_index_set(11, 3)
    t, x = O.points(cfg, 3)
    B = O.basis_matrix(cfg, nu, t, x)
    ref = B.T @ B
    bound = (U_SPLIT + 3 * M_SLICE * U_ACC) * (np.abs(B).T @ np.abs(B))
    b32 = B.astype(np.float32)
    hi = _tf32(b32)
    lo = _tf32((b32 - hi).astype(np.float32))
    assert np.all(np.abs(b32 - hi) <= 2.0 ** -11 * np.abs(b32))
    assert np.all(np.abs(b32 - hi - lo) <= 2.0 ** -22 * np.abs(b32))
    h, l = hi.astype(np.float64), lo.astype(np.float64)
    two = h.T @ h + h.T @ l
    assert np.max(np.abs(two - ref) / bound) > 1.0
    three = two + l.T @ h
    # the split itself (FP64 sums) uses a small part of the bound: the rest
    # is for the FP32 accumulation in the tensor core
    assert np.max(np.abs(three - ref) / bound) < 0.1
