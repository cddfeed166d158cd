"""Host-side logic that needs no GPU: the autotuner's problem-class key and
JSON cache, the seeded request mix of the serving benchmark, and the
benchmark's arrival stream and weak-scaling arithmetic, the tuner's choice
of a launch shape and the timing-table workloads."""
import json
import math

import pytest

import workloads


def test_autotune_key_buckets_problem_classes():
    from paper_1102_4666_gb300 import autotune
    c4 = workloads.config("c4")
    # the bucket is the next power of two of M: 3000 and 4000 share a class
    assert autotune.key(workloads.config("c4", M=3000), "mixed") == autotune.key(c4, "mixed")
    assert autotune.key(workloads.config("c4", M=5000), "mixed") != autotune.key(c4, "mixed")
    assert autotune.key(c4, "fp64") != autotune.key(c4, "mixed")
    assert autotune.key(workloads.config("c4", eta=4), "mixed") != autotune.key(c4, "mixed")


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    from paper_1102_4666_gb300 import autotune
    path = tmp_path / "tune.json"
    monkeypatch.setenv("BSDE_TUNE_CACHE", str(path))
    c3 = workloads.config("c3")
    assert autotune.lookup(c3, "mixed") is None
    path.write_text(json.dumps({autotune.key(c3, "mixed"): {"shape": [256, 2], "ms_paths": 1.0}}))
    assert autotune.lookup(c3, "mixed") == (256, 2)
    assert autotune.lookup(workloads.config("c4"), "mixed") is None


def test_server_requests_take_the_tuned_shapes(tmp_path, monkeypatch):
    """The serving binding builds each request's parameters with the launch
    shape and Gram split count tuned for its problem class, and the library
    defaults (0) for a class that was not tuned."""
    import paper_1102_4666_gb300 as G
    from paper_1102_4666_gb300 import autotune
    path = tmp_path / "tune.json"
    monkeypatch.setenv("BSDE_TUNE_CACHE", str(path))
    c4 = workloads.config("c4")
    path.write_text(json.dumps({autotune.key(c4, "mixed"): {"shape": [64, 8], "ms_paths": 1.0,
                                                             "gram_splits": 50}}))
    rq, _ = G.request(c4, precision="mixed")
    assert (rq.params.paths_tpb, rq.params.paths_ppt, rq.params.gram_splits) == (64, 8, 50)
    assert autotune.lookup_gram_splits(c4, "mixed") == 50
    rq, _ = G.request(workloads.config("c3"), precision="mixed")
    assert (rq.params.paths_tpb, rq.params.paths_ppt, rq.params.gram_splits) == (0, 0, 0)
    rq, _ = G.request(c4, precision="fp64")
    assert (rq.params.paths_tpb, rq.params.paths_ppt) == (0, 0)


def test_gram_split_candidates():
    from paper_1102_4666_gb300 import autotune
    c4 = workloads.config("c4")  # p = 364: 6 upper tiles; n = 4000: 125 K-blocks
    assert autotune.gram_split_candidates(c4, 152) == [0, 12, 50, 100]
    small = workloads.config("c4", n=200, eta=2)  # p = 78: 1 tile; 7 K-blocks
    assert autotune.gram_split_candidates(small, 152) == [0, 7]


def test_serving_mix_is_seeded_and_respects_its_ranges():
    a = workloads.serving_mix(300, seed=7)
    b = workloads.serving_mix(300, seed=7)
    assert [r["n"] for r in a] == [r["n"] for r in b] and [r["eta"] for r in a] == [r["eta"] for r in b]
    assert [r["n"] for r in a] != [r["n"] for r in workloads.serving_mix(300, seed=8)]
    for r in a:
        assert r["d"] in (1, 2, 5, 10)
        assert 200 <= r["n"] <= 4000 and 500 <= r["M"] <= 8000 and 2 <= r["eta"] <= 6
        assert 80.0 <= r["K"] <= 120.0 and 0.25 <= r["T"] <= 2.0
        assert r["lambda"] in (0.0, 100.0)
        assert 2 * workloads.basis_size(r["d"], r["eta"]) <= r["n"]  # p <= n / 2
    assert {r["d"] for r in a} == {1, 2, 5, 10}


def test_basis_size_is_the_binomial_coefficient():
    assert workloads.basis_size(10, 3) == 364 and workloads.basis_size(5, 4) == 210
    assert workloads.basis_size(1, 6) == 28
    for d in range(1, 11):
        for eta in range(0, 7):
            assert workloads.basis_size(d, eta) == math.comb(d + 1 + eta, eta)


def test_arrival_stream_is_seeded_and_poisson_like():
    import bench
    t = bench.arrival_times(4000, 20.0, 7)
    assert t == bench.arrival_times(4000, 20.0, 7)
    gaps = [b - a for a, b in zip([0.0] + t[:-1], t)]
    assert all(g > 0 for g in gaps)
    mean = sum(gaps) / len(gaps)
    assert abs(mean - 1 / 20.0) < 4 * (1 / 20.0) / math.sqrt(len(gaps))  # 4 standard errors
    assert abs(sorted(gaps)[len(gaps) // 2] - math.log(2) / 20.0) < 0.1 / 20.0  # exponential median


def test_weak_scaling_value_single_rank():
    import bench
    value, ms = bench.weak_scaling_value(2000.0, 4, 1.92e10)
    assert ms == 2000.0
    assert value == pytest.approx(4 * 1.92e10 / 2.0)


def test_paper_timing_workloads_follow_the_captions():
    """The two timing-table workloads carry the captions' parameters (Section 6.4)."""
    for name, d, M in (("paper_d3", 3, 1000), ("paper_d6", 6, 5000)):
        c = workloads.config(name)
        assert (c["d"], c["M"], c["N"], c["n"], c["eta"], c["K_it"]) == (d, M, 10, 2000, 3, 10)
        assert (c["r"], c["K"], c["T"], c["rho"], c["lambda"], c["q"]) == (0.02, 95.0, 1.0, 0.0, 1.0, 1.0)
        assert c["vol"] == {"kind": "const", "a": 0.2} and c["S0"] == [100.0] * d
        t8, tbest, procs = workloads.PAPER_TIMING_SECONDS[name]
        assert t8 > tbest and procs in (64, 256)
    # the basis has d' = d + 1 variates: 35 functions at d = 3, 120 at d = 6
    assert workloads.basis_size(3, 3) == 35 and workloads.basis_size(6, 3) == 120


def test_autotune_keeps_the_fastest_shape_and_skips_failing_ones(tmp_path, monkeypatch):
    """tune() with the library's Solver replaced by a stand-in that reports
    fixed path-kernel times: it probes a one-iteration problem, keeps the
    fastest launch shape, skips shapes whose launch fails and writes the
    problem class's entry to the cache; with every shape failing it returns
    None and writes nothing."""
    import paper_1102_4666_gb300 as G
    from paper_1102_4666_gb300 import autotune
    path = tmp_path / "tune.json"
    monkeypatch.setenv("BSDE_TUNE_CACHE", str(path))
    times = {(128, 4): 5.0, (256, 2): 3.0, (64, 8): 4.0}
    gram_ms = {0: 0.5, 7: 0.3}
    probes = []

    class Report:
        def __init__(self, ms, ms_gram=1.0):
            self.ms_paths = ms
            self.ms_gram = ms_gram

    class StandIn:
        def __init__(self, cfg, precision="mixed"):
            probes.append((cfg["K_it"], cfg["n"], precision))

        def solve(self, use_graph=1, timing=0, paths_tpb=0, paths_ppt=0, gram_splits=None):
            if gram_splits is not None:
                return Report(1.0, gram_ms[gram_splits])
            if (paths_tpb, paths_ppt) not in times:
                raise RuntimeError("launch failed")
            return Report(times[(paths_tpb, paths_ppt)])

        def close(self):
            pass

    monkeypatch.setattr(G, "Solver", StandIn)
    monkeypatch.setattr(autotune, "_sm_count", lambda: 152)
    cfg = workloads.config("c3")
    # p = 210 (3 upper tiles: one wave is 50 slices) and 300 points (10 K-blocks):
    # candidates 0 and 10 slices ... capped by the K-blocks
    gram_ms[10] = 0.3
    best = autotune.tune(cfg, "mixed", candidates=[(128, 4), (256, 2), (32, 32), (64, 8)], n_points=300)
    assert best == (256, 2)
    assert probes == [(1, 300, "mixed"), (1, 300, "mixed")]
    assert autotune.lookup(cfg, "mixed") == (256, 2)
    entry = json.loads(path.read_text())[autotune.key(cfg, "mixed")]
    assert entry["ms_paths"] == 3.0 and set(entry["candidates"]) == {"128x4", "256x2", "64x8"}
    assert entry["gram_splits"] == 10 and autotune.lookup_gram_splits(cfg, "mixed") == 10

    path.unlink()
    assert autotune.tune(cfg, "mixed", candidates=[(32, 32)]) is None
    assert not path.exists()
