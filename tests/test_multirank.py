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
