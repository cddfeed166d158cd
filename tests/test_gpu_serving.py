"""The continuous-batching server: each request's result is the same alone
(a dedicated solver) and in the mix (admitted next to others, sharing the
device), because every kernel reduces in a fixed order."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _mix():
    reqs = []
    base = workloads.serving_mix(8, seed=11)
    for j, r in enumerate(base):
        # keep the test short: small point sets and path counts
        r["n"] = max(2 * workloads.basis_size(r["d"], r["eta"]) + 8, 200)
        r["M"] = 300 + 50 * j
        r["K_it"] = 3
        reqs.append(r)
    return reqs


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_alone_equals_in_the_mix(precision):
    import paper_1102_4666_gb300 as G
    reqs = _mix()
    alone = []
    for r in reqs:
        s = G.Solver(r, precision=precision)
        rep = s.solve(use_graph=1)
        alone.append((rep.price, list(rep.delta[:r["d"]]), rep.status))
        s.close()
    srv = G.Server(max_slots=4, precision=precision)
    ids = [srv.submit(r) for r in reqs]
    assert srv.drain(120000.0) == G.OK
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["running"] == 0
    for r, rid, (p, d, stt) in zip(reqs, ids, alone):
        rep = srv.poll(rid)
        assert rep is not None and rep.status == stt == G.OK
        assert rep.price == p
        assert list(rep.delta[:r["d"]]) == d
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_admission_by_memory_budget():
    """With a budget that fits one request at a time, requests still all
    complete (queued until memory frees up); a request larger than the
    whole budget is refused at submit."""
    import paper_1102_4666_gb300 as G
    reqs = [r for r in _mix() if workloads.basis_size(r["d"], r["eta"]) <= 400][:4]
    srv = G.Server(max_slots=4, mem_budget=64 << 20, precision="mixed")
    ids = [srv.submit(r) for r in reqs]
    assert srv.drain(120000.0) == G.OK
    for rid in ids:
        rep = srv.poll(rid)
        assert rep is not None and rep.status == G.OK
    big = workloads.config("c4", eta=4)  # p = 1365: about 120 MB resident
    with pytest.raises(G.BsdeError):
        srv.submit(big)
    srv.close()


def _completion_order(policy, slots=1, large_slots=2):
    """Submit two long requests and then a short one to a server with `slots`
    slots and return the order in which they complete (0, 1: long; 2: short)."""
    import time

    import paper_1102_4666_gb300 as G
    long_req = workloads.config("c3", K_it=2)  # 1e9 path-steps
    short_req = workloads.config("c3", n=500, M=1000, K_it=1)
    srv = G.Server(max_slots=slots, precision="mixed", policy=policy, large_slots=large_slots)
    ids = [srv.submit(long_req), srv.submit(long_req, seed=99), srv.submit(short_req)]
    done = []
    t0 = time.monotonic()
    while len(done) < 3 and time.monotonic() - t0 < 120.0:
        for k in (2, 1, 0):  # the short request is looked at first in every sweep
            if k not in done:
                rep = srv.poll(ids[k])
                if rep is not None:
                    assert rep.status == G.OK
                    done.append(k)
        time.sleep(0.0005)
    srv.close()
    return done


def test_fifo_policy_admits_in_arrival_order():
    assert _completion_order("fifo") == [0, 1, 2]


def test_shortest_first_policy_overtakes_queued_long_requests():
    """The short request, queued behind a long one, is admitted as soon as
    the slot frees up, before the second long request."""
    order = _completion_order("shortest")
    assert sorted(order) == [0, 1, 2]
    assert order.index(2) < order.index(1)


def test_response_ratio_policy_serves_short_first_and_everyone():
    """Highest response ratio next: the short request queued behind a long
    one goes first (its ratio grows fastest), and every request completes."""
    order = _completion_order("response_ratio")
    assert sorted(order) == [0, 1, 2]
    assert order.index(2) < order.index(1)


def test_size_lanes_policy_runs_large_requests_one_at_a_time():
    """Two slots and one large-lane slot: the second long request (at least
    the average work) waits while the first runs, and the short one behind
    it passes it."""
    order = _completion_order("size_lanes", slots=2, large_slots=1)
    assert sorted(order) == [0, 1, 2]
    assert order.index(2) < order.index(1) and order.index(0) < order.index(1)
