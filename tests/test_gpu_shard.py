"""Point-sharded solves (bsde_set_shard; Section 4.2: the loop over the points
of an iteration is parallel) on one GPU.  R ranks run as host threads of one
process, each with its own context and stream; their exchange hook gathers
the blocks of corrections through host memory behind a host barrier, so no
kernel ever waits for another.  Every rank must end with the coefficients
and price of the unsharded solve, bit for bit: the blocks' corrections are
computed by the same kernels in the same order, and the refit is the same."""
import threading

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1102_4666_gb300 as G
    return G


class ThreadExchange:
    """All-gather of the blocks of R host threads through host memory."""

    def __init__(self, nranks, nb):
        self.barrier = threading.Barrier(nranks, timeout=120)
        self.host = np.full(nranks * nb, np.nan)

    def __call__(self, xbuf, nb, rank, nranks, stream):
        import torch
        s = torch.cuda.ExternalStream(int(stream))
        s.synchronize()
        self.host[rank * nb:(rank + 1) * nb] = xbuf[rank * nb:(rank + 1) * nb].cpu().numpy()
        self.barrier.wait()
        full = torch.from_numpy(self.host.copy())
        with torch.cuda.stream(s):
            xbuf[:nranks * nb].copy_(full)
        s.synchronize()
        self.barrier.wait()


def _sharded_solve(G, cfg, prec, nranks):
    import torch
    n = cfg["n"]
    nb = (n + nranks - 1) // nranks
    ex = ThreadExchange(nranks, nb)
    out = [None] * nranks
    errs = []

    def run(rank):
        try:
            torch.cuda.set_device(0)
            s = G.Solver(cfg, precision=prec)
            xbuf = torch.zeros(nranks * nb, dtype=torch.float64, device="cuda")
            s.set_shard(rank, nranks, xbuf, ex)
            rep = s.solve(use_graph=1)  # ignored while sharded: direct launches
            out[rank] = (rep.price, np.array(rep.delta[:cfg["d"]]), s.coeffs(), rep.status)
            s.close()
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)

    th = [threading.Thread(target=run, args=(r,)) for r in range(nranks)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("nranks", [2, 3])
def test_sharded_solve_equals_unsharded(G, prec, nranks):
    # n = 301 does not divide by 2 or 3: the last block is shorter
    cfg = workloads.config("c4", n=301, M=96, N=6, eta=2, K_it=3, **{"lambda": 1.0})
    s = G.Solver(cfg, precision=prec)
    ref = s.solve()
    a_ref = s.coeffs()
    s.close()
    for price, delta, alpha, status in _sharded_solve(G, cfg, prec, nranks):
        assert status == G.OK
        assert np.array_equal(alpha, a_ref)
        assert price == ref.price
        assert np.array_equal(delta, np.array(ref.delta[:cfg["d"]]))


def test_shard_blocks_tile_the_points(G):
    for n in (1, 5, 301, 4000):
        for R in (1, 2, 3, 7):
            blocks = [G.shard_block(n, r, R) for r in range(R)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[j][1] == blocks[j + 1][0] for j in range(R - 1))
            assert all(0 <= b - a <= (n + R - 1) // R for a, b in blocks)


def test_failed_exchange_is_reported_and_the_context_stays_usable(G):
    import torch
    cfg = workloads.config("c4", n=200, M=64, N=4, eta=2, K_it=2, **{"lambda": 1.0})
    s = G.Solver(cfg, precision="mixed")
    ref = s.solve()

    def broken(xbuf, nb, rank, nranks, stream):
        raise RuntimeError("peer lost")

    xbuf = torch.zeros(2 * 100, dtype=torch.float64, device="cuda")
    s.set_shard(0, 2, xbuf, broken)
    rep = s.solve(check=False)
    assert rep.status == G.ERR_EXCHANGE
    # too small an exchange buffer is refused before any device work
    s.set_shard(1, 2, xbuf[:150], broken)
    assert s.solve(check=False).status == G.ERR_INVALID_ARG
    s.set_shard(0, 1)
    again = s.solve()
    assert again.status == G.OK and again.price == ref.price
    s.close()


def test_torch_distributed_exchange_on_the_solve_stream(G, tmp_path):
    """The binding's NCCL exchange on a one-rank process group: the block
    is gathered into place on the given stream (ordering through
    torch.cuda.ExternalStream)."""
    import torch
    import torch.distributed as dist
    store = dist.FileStore(str(tmp_path / "store"), 1)
    dist.init_process_group("nccl", store=store, rank=0, world_size=1)
    try:
        ex = G.torch_distributed_exchange()
        st = torch.cuda.Stream()
        xbuf = torch.arange(10, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(st):
            xbuf.mul_(2.0)  # ordered before the exchange on the same stream
        ex(xbuf, 10, 0, 1, st.cuda_stream)
        st.synchronize()
        assert torch.equal(xbuf.cpu(), torch.arange(10, dtype=torch.float64) * 2.0)
    finally:
        dist.destroy_process_group()


def _peer_solve(G, cfg, prec, nranks):
    """R ranks as host threads sharing one GPU, exchanging by peer stores
    into each other's buffers.  The pushed hook holds every rank at a host
    barrier until all ranks' pushes and counters have completed, so each
    device-side wait finds its counters already raised: no kernel waits for
    another kernel."""
    import torch
    n = cfg["n"]
    nb = (n + nranks - 1) // nranks
    bufs = [torch.zeros(2 * nranks * nb, dtype=torch.float64, device="cuda") for _ in range(nranks)]
    flags = [torch.zeros(nranks, dtype=torch.int32, device="cuda") for _ in range(nranks)]
    barrier = threading.Barrier(nranks, timeout=120)
    out = [None] * nranks
    errs = []

    def pushed(nb_, rank, R, stream):
        torch.cuda.ExternalStream(int(stream)).synchronize()
        barrier.wait()

    def run(rank):
        try:
            torch.cuda.set_device(0)
            s = G.Solver(cfg, precision=prec)
            s.set_shard_peers(rank, nranks, bufs, flags, wait_ms=2000.0, pushed=pushed)
            rep = s.solve(use_graph=1)
            out[rank] = (rep.price, s.coeffs(), rep.status)
            s.close()
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)

    th = [threading.Thread(target=run, args=(r,)) for r in range(nranks)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return out, flags


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("nranks", [2, 3])
def test_peer_exchange_equals_unsharded(G, prec, nranks):
    cfg = workloads.config("c4", n=301, M=96, N=6, eta=2, K_it=3, **{"lambda": 1.0})
    s = G.Solver(cfg, precision=prec)
    ref = s.solve()
    a_ref = s.coeffs()
    s.close()
    out, flags = _peer_solve(G, cfg, prec, nranks)
    for price, alpha, status in out:
        assert status == G.OK
        assert np.array_equal(alpha, a_ref) and price == ref.price
    # every rank raised its counter at every other rank once per iteration
    for r in range(nranks):
        f = flags[r].cpu().numpy()
        assert all(f[q] == cfg["K_it"] for q in range(nranks) if q != r)


def test_peer_exchange_wait_runs_out_when_a_rank_never_joins(G):
    """Rank 0 of 2 alone: nobody raises its counter for rank 1, so its
    device-side wait gives up after wait_ms; the solve returns
    BSDE_ERR_TIMEOUT without waiting again in later iterations, and the
    context then solves unsharded as before."""
    import time
    import torch
    cfg = workloads.config("c4", n=200, M=64, N=4, eta=2, K_it=3, **{"lambda": 1.0})
    s = G.Solver(cfg, precision="mixed")
    ref = s.solve()
    nb = 100
    bufs = [torch.zeros(4 * nb, dtype=torch.float64, device="cuda") for _ in range(2)]
    flags = [torch.zeros(2, dtype=torch.int32, device="cuda") for _ in range(2)]
    s.set_shard_peers(0, 2, bufs, flags, wait_ms=50.0)
    t0 = time.monotonic()
    rep = s.solve(check=False)
    el = time.monotonic() - t0
    assert rep.status == G.ERR_TIMEOUT
    assert "bounded device wait" in G.lib().bsde_last_error(s.h).decode()
    assert el < 10.0
    # rank 0 did push to rank 1 and raise its counter there, once per iteration
    assert int(flags[1][0].item()) == cfg["K_it"]
    s.set_shard(0, 1)
    again = s.solve()
    assert again.status == G.OK and again.price == ref.price
    s.close()


def test_more_ranks_than_points_per_block(G):
    """Seven ranks over six points: nb = 1, and the last rank's block is
    empty (it launches no path kernel and sends nothing); the result is still
    the unsharded one bit for bit, with either exchange."""
    cfg = workloads.make(d=1, T=1.0, r=0.02, K=100.0, S0=100.0, vol={"kind": "const", "a": 0.2}, rho=0.0,
                         lam=0.0, n=6, M=64, N=4, eta=1, K_it=2, seed=21)
    s = G.Solver(cfg, precision="fp64")
    ref = s.solve()
    a_ref = s.coeffs()
    s.close()
    assert G.shard_block(6, 6, 7) == (6, 6)
    for price, delta, alpha, status in _sharded_solve(G, cfg, "fp64", 7):
        assert status == G.OK and np.array_equal(alpha, a_ref) and price == ref.price
    out, _ = _peer_solve(G, cfg, "fp64", 7)
    for price, alpha, status in out:
        assert status == G.OK and np.array_equal(alpha, a_ref) and price == ref.price
