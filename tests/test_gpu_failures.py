"""Failure injection on the host, without a GPU fault: an allocation hook
that refuses its k-th request.  The call that meets the refusal returns
BSDE_ERR_NOMEM, the context gives back every byte it holds (the hook's
live-byte count returns to zero), and the next call on the same context
succeeds with the result of an undisturbed run."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


class CountingAllocator:
    """PyTorch's caching allocator behind a counter: refuses request number
    fail_at (1-based; None: never) and tracks the bytes it has handed out."""

    def __init__(self, fail_at=None):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        dev = self.torch.cuda.current_device()
        ptr = int(self.torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0)))
        self.live[ptr] = int(nbytes)
        return ptr

    def free(self, ptr, stream):
        if ptr in self.live:
            del self.live[ptr]
            self.torch.cuda.caching_allocator_delete(int(ptr))

    def live_bytes(self):
        return sum(self.live.values())


@pytest.fixture(scope="module")
def G():
    import paper_1102_4666_gb300 as G
    return G


CFG = dict(n=300, M=64, N=5, eta=2, K_it=2)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("fail_at", [1, 2])
def test_solve_allocation_failure(G, prec, fail_at):
    """Request 1 is the problem's arena, request 2 its block of Gram factors."""
    cfg = workloads.config("c4", **CFG)
    ref = G.Solver(cfg, precision=prec)
    r0 = ref.solve()
    a0 = ref.coeffs()
    ref.close()
    al = CountingAllocator(fail_at)
    s = G.Solver(cfg, precision=prec, allocator=al)
    rep = s.solve(check=False)
    assert rep.status == G.ERR_NOMEM
    assert al.calls == fail_at
    assert al.live_bytes() == 0
    assert "allocation failed" in G.lib().bsde_last_error(s.h).decode()
    # the context stays usable: the next solve allocates again and succeeds
    al.fail_at = None
    rep = s.solve()
    assert rep.status == G.OK and rep.price == r0.price
    assert np.array_equal(s.coeffs(), a0)
    assert al.live_bytes() > 0
    s.close()
    assert al.live_bytes() == 0


def test_eval_allocation_failure(G):
    """bsde_eval_price_delta takes a temporary buffer for its query points:
    refused, the call fails with BSDE_ERR_NOMEM, nothing leaks, and the same
    evaluation succeeds next."""
    cfg = workloads.config("c4", **CFG)
    al = CountingAllocator()
    s = G.Solver(cfg, precision="mixed", allocator=al)
    s.solve()
    held = al.live_bytes()
    al.fail_at = al.calls + 1
    t = np.array([0.0, 0.5]); S = np.full((2, 10), 100.0)
    with pytest.raises(G.BsdeError) as ex:
        s.eval(t, S)
    assert ex.value.code == G.ERR_NOMEM
    assert al.live_bytes() == held
    al.fail_at = None
    price, delta = s.eval(t, S)
    assert np.all(np.isfinite(price)) and al.live_bytes() == held
    s.close()
    assert al.live_bytes() == 0


def test_memory_budget_refusal_leaves_the_context_usable(G):
    """A budget below the problem's footprint: BSDE_ERR_NOMEM before any
    allocation; a smaller problem on the same context then solves."""
    cfg = workloads.config("c4", **CFG)
    al = CountingAllocator()
    s = G.Solver(cfg, precision="mixed", allocator=al, mem_budget=1 << 20)
    rep = s.solve(check=False)
    assert rep.status == G.ERR_NOMEM and al.calls == 0
    small = workloads.config("c4", n=40, M=32, N=3, eta=1, K_it=1)
    s.cfg = small
    s.set_grid(small)
    assert s.solve().status == G.OK
    s.close()
    assert al.live_bytes() == 0
