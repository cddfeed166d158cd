"""The no-allocation entry point bsde_corrections_noalloc, for callers that
cannot allocate device memory (a fixed device-memory arena, a host process
that forbids cudaMalloc/cudaFree, an allocator-free steady state).  Its
corrections must match those of bsde_iterate (the entry point that owns its
memory) on the same points and coefficients, on two calls in a row.  This
file is collected last so that a failure here comes after every other
test; it needs nothing from them."""
import ctypes
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

# tolerances of the parity tests: FP64 1e-9, mixed 2e-5, relative to the
# scale of the integrand
TOL = {"fp64": 1e-9, "mixed": 2e-5}


def _call(G, cfg, t, x, alpha, k, prec, torch):
    sg, r, pf, pen, keep = G.model_structs(cfg)
    lo = (ctypes.c_double * (cfg["d"] + 1))(*cfg["lo"])
    hi = (ctypes.c_double * (cfg["d"] + 1))(*cfg["hi"])
    dev = torch.device("cuda", 0)
    t_d = torch.tensor(t, dtype=torch.float64, device=dev)
    x_d = torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)
    a_d = torch.tensor(alpha, dtype=torch.float64, device=dev)
    c_d = torch.full((len(t),), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    err = ctypes.create_string_buffer(512)
    rc = G.lib().bsde_corrections_noalloc(
        ctypes.byref(sg), r, ctypes.byref(pf), ctypes.byref(pen),
        ctypes.cast(lo, G._dptr), ctypes.cast(hi, G._dptr), len(t), t_d.data_ptr(), x_d.data_ptr(),
        cfg["eta"], cfg.get("q", 1.0), a_d.data_ptr(), cfg["M"], cfg["N"], cfg["seed"], k,
        G.PREC_MIXED if prec == "mixed" else G.PREC_FP64, c_d.data_ptr(),
        torch.cuda.current_stream(dev).cuda_stream, err, len(err))
    return rc, c_d.cpu().numpy(), err.value.decode()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_iterate_two_calls(prec):
    torch = pytest.importorskip("torch")
    import paper_1102_4666_gb300 as G
    cfg = workloads.config("c3", n=300, M=200, N=12, eta=3)
    p = len(G.basis_indices(cfg["d"], cfg["eta"]))
    rng = np.random.default_rng(4)
    s = G.Solver(cfg, precision=prec)
    for call, k in enumerate((1, 2)):
        alpha = rng.standard_normal(p) * 0.5
        alpha[0] += 5.0
        t, x, c_ref, _ = s.iterate(k, alpha, eval_mode=1)
        rc, c, msg = _call(G, cfg, t, x, alpha, k, prec, torch)
        assert rc == G.OK, msg
        scale = max(1.0, cfg["K"] * 0.5, float(np.max(np.abs(c_ref))))
        assert np.all(np.isfinite(c)), "call %d" % call
        assert np.max(np.abs(c - c_ref)) <= TOL[prec] * scale, "call %d" % call
    s.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import paper_1102_4666_gb300 as G
    cfg = workloads.config("c3", n=600000, M=4000, N=4, eta=1)
    t = np.zeros(4); x = np.zeros((5, 4))
    # the size check happens before any buffer is touched
    sg, r, pf, pen, keep = G.model_structs(cfg)
    lo = (ctypes.c_double * 6)(*cfg["lo"]); hi = (ctypes.c_double * 6)(*cfg["hi"])
    err = ctypes.create_string_buffer(512)
    rc = G.lib().bsde_corrections_noalloc(
        ctypes.byref(sg), r, ctypes.byref(pf), ctypes.byref(pen), ctypes.cast(lo, G._dptr),
        ctypes.cast(hi, G._dptr), cfg["n"], 1, 1, 1, 1.0, 1, cfg["M"], cfg["N"], 1, 0, G.PREC_MIXED, 1,
        None, err, len(err))
    assert rc == G.ERR_NOMEM
    assert "static scratch" in err.value.decode()
