"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
solves its own problem (its own seed, no data-path collective) and the job
value is all ranks' units over the slowest rank's time (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, lr = bench.env_rank()
    seed = bench.rank_seed(4, r)
    ms_local = 100.0 + 50.0 * r  # rank 1 is the slowest
    value, ms = bench.weak_scaling_value(ms_local, steps=3, units_per_step=1e9)
    dist.barrier()
    out.put((r, w, seed, value, ms))
    dist.destroy_process_group()


def test_weak_scaling_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, v0, m0), (r1, w1, s1, v1, m1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 != s1  # independent problems
    assert m0 == m1 == 150.0  # job time = slowest rank
    assert v0 == v1 == pytest.approx(2 * 3 * 1e9 / 0.150)


def _shard_worker(rank, world, port, out):
    """One rank of a point-sharded iteration on the CPU: its block of the
    corrections from the oracle, the exchange of the library's binding over
    gloo, and the replicated least-squares refit (eq. alpha)."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads
    import paper_1102_4666_gb300 as G
    from oracle import bsde_oracle as O
    cfg = workloads.make(d=2, T=1.0, r=0.03, K=100.0, S0=100.0, vol=workloads.config("c3")["vol"],
                         rho=0.3, lam=1.0, n=37, M=40, N=4, eta=2, K_it=2, seed=11)
    n = cfg["n"]
    nu = O.multi_index_set(3, 2)
    nb = (n + world - 1) // world
    exchange = G.torch_distributed_exchange()
    alpha = np.zeros(len(nu))
    blocks = []
    for k in range(cfg["K_it"]):
        t, x = O.points(cfg, k)
        i0, i1 = G.shard_block(n, rank, world)
        blocks.append((i0, i1))
        xbuf = torch.full((world * nb,), float("nan"), dtype=torch.float64)
        if i1 > i0:
            idx = np.arange(i0, i1)
            xbuf[i0:i1] = torch.from_numpy(O.correction(cfg, nu, alpha, k, idx, t[idx], x[:, idx],
                                                        nthreads=1))
        exchange(xbuf, nb, rank, world)
        c = xbuf[:n].numpy().copy()
        B = O.basis_matrix(cfg, nu, t, x)
        alpha = O.fit(B, B @ alpha + c)
    out.put((rank, blocks, alpha.tolist()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_point_sharded_iterations_gloo_ranks(world):
    """Point sharding (Section 4.2): every rank simulates its block of the
    points, one all-gather of the corrections per iteration, the refit
    replicated on every rank.  Every rank ends with the coefficients of the
    unsharded iteration, bit for bit, and the blocks tile the points."""
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import numpy as np
    import workloads
    from oracle import bsde_oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    base = workloads.config("c3")
    cfg = workloads.make(d=2, T=1.0, r=0.03, K=100.0, S0=100.0, vol=base["vol"], rho=0.3, lam=1.0,
                         n=37, M=40, N=4, eta=2, K_it=2, seed=11)
    ref = O.solve(cfg, nthreads=1)
    covered = []
    for rank, blocks, alpha in res:
        assert np.array_equal(np.array(alpha), ref["alpha"])
        covered.append(blocks[0])
    assert covered[0][0] == 0 and covered[-1][1] == cfg["n"]
    assert all(covered[j][1] == covered[j + 1][0] for j in range(world - 1))
