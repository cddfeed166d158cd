"""Autotuner of the path kernel's launch shape and of the tensor-core Gram's
split count.

The path kernel's throughput depends on its CTA size (threads per CTA) and
on the number of paths each thread runs: these set the occupancy (the
per-thread shared-memory tables of the Chebyshev evaluation scale with the
CTA size), the share of the per-CTA prologue (volatility tables, coefficient
staging) and the tail of the last chunk of each point.  The Gram matrix's
time depends on how many slices of the points its CTAs split (one wave of
CTAs by default; more slices hide the TMA latency better, fewer slices
leave less to reduce).  tune() times a small set of candidates of each with
one-iteration solves through the C ABI (bsde_solve_params.paths_tpb /
paths_ppt / gram_splits) and keeps the fastest in a JSON cache keyed by the
problem class: precision, d, degree, q, N, a bucket of M and the volatility
family.  The serving binding looks the class of each request up at submit.
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


def lookup_gram_splits(cfg, precision):
    """Tuned split count of the tensor-core Gram for this class (0: the
    library's default, also when none was tuned)."""
    with _LOCK:
        v = _load().get(key(cfg, precision))
    return int(v.get("gram_splits", 0)) if v else 0


def gram_split_candidates(cfg, sms):
    """0 (one wave of CTAs over the upper 128 x 128 tiles) and half, twice
    and four times as many slices, each at least one K-block of 32 points."""
    side = (_basis_size(cfg) + 127) // 128
    tiles = side * (side + 1) // 2
    kblocks = (cfg["n"] + 31) // 32
    wave = max(1, sms // tiles)
    cands = [0] + sorted({min(kblocks, max(1, f)) for f in (wave // 2, 2 * wave, 4 * wave)} - {wave})
    return cands


def _sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _basis_size(cfg):
    from . import basis_indices
    return len(basis_indices(cfg["d"], cfg["eta"], cfg.get("q", 1.0)))


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
    # the Gram's split count (mixed precision: the tensor-core product),
    # timed by the Gram + factorisation time of a one-iteration solve (the
    # factorisation does not depend on it)
    gram = {}
    if precision == "mixed":
        sms = _sm_count()
        s = Solver(probe, precision=precision)
        try:
            for g in gram_split_candidates(probe, sms):
                try:
                    s.solve(use_graph=0, timing=1, gram_splits=g)
                    gram[g] = min(s.solve(use_graph=0, timing=1, gram_splits=g).ms_gram
                                  for _ in range(repeats))
                except Exception:
                    continue
        finally:
            s.close()
    gbest = min(gram, key=gram.get) if gram else 0
    if store:
        with _LOCK:
            data = _load()
            data[key(cfg, precision)] = {"shape": list(best), "ms_paths": times[best],
                                         "candidates": {"%dx%d" % k: v for k, v in times.items()},
                                         "gram_splits": gbest,
                                         "gram_candidates_ms": {str(k): v for k, v in gram.items()}}
            os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
            tmp = cache_path() + ".%d.tmp" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, cache_path())
    return best
