"""Autotuner of the path kernel's launch shape.

The path kernel's throughput depends on its CTA size (threads per CTA) and
on the number of paths each thread runs: these set the occupancy (the
per-thread shared-memory tables of the Chebyshev evaluation scale with the
CTA size), the share of the per-CTA prologue (volatility tables, coefficient
staging) and the tail of the last chunk of each point.  tune() times a small
set of candidates with one-iteration solves through the C ABI
(bsde_solve_params.paths_tpb / paths_ppt) and keeps the fastest in a JSON
cache keyed by the problem class: precision, d, degree, q, N, a bucket of M
and the volatility family.
"""
import json
import os
import threading

_LOCK = threading.Lock()

CANDIDATES = {
    "mixed": [(128, 4), (256, 2), (256, 4), (128, 8), (64, 8)],
    "fp64": [(64, 4), (64, 8), (32, 8), (128, 2)],
}


def cache_path():
    return os.environ.get("BSDE_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune.json"))


def key(cfg, precision):
    m = cfg["M"]
    bucket = 1 << max(0, (m - 1).bit_length())  # next power of two
    return "%s:d%d:eta%d:q%.3f:N%d:M%d:%s" % (precision, cfg["d"], cfg["eta"], cfg.get("q", 1.0),
                                              cfg["N"], bucket, cfg["vol"]["kind"])


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(cfg, precision):
    """(tpb, ppt) tuned for this problem class, or None."""
    with _LOCK:
        v = _load().get(key(cfg, precision))
    return tuple(v["shape"]) if v else None


def tune(cfg, precision="mixed", candidates=None, repeats=2, n_points=None, store=True):
    """Time each candidate launch shape on the problem of cfg (one iteration,
    n_points points) and return the fastest (tpb, ppt)."""
    from . import Solver
    probe = dict(cfg)
    probe["K_it"] = 1
    if n_points:
        probe["n"] = n_points
    cands = candidates or CANDIDATES[precision]
    s = Solver(probe, precision=precision)
    times = {}
    try:
        for tpb, ppt in cands:
            try:
                s.solve(use_graph=0, timing=1, paths_tpb=tpb, paths_ppt=ppt)
                ms = min(s.solve(use_graph=0, timing=1, paths_tpb=tpb, paths_ppt=ppt).ms_paths
                         for _ in range(repeats))
            except Exception:
                continue
            times[(tpb, ppt)] = ms
    finally:
        s.close()
    if not times:
        return None
    best = min(times, key=times.get)
    if store:
        with _LOCK:
            data = _load()
            data[key(cfg, precision)] = {"shape": list(best), "ms_paths": times[best],
                                         "candidates": {"%dx%d" % k: v for k, v in times.items()}}
            os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
            tmp = cache_path() + ".%d.tmp" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, cache_path())
    return best
