"""Failure paths of the library, made without faulting the GPU.

- A bounded device wait that expires: while LTS_TEST_STALL_SORT is set, one
  tile of the sort's first digit pass waits on look-back words that nothing
  sets; its wait gives up after a short budget, the call returns
  LTS_ERR_TIMEOUT, and the next call on the same context is exact.
- An allocation that fails: while LTS_TEST_FAIL_ALLOC is set, every device
  allocation of the library fails as if the device were full.  Creating a
  context or a batch's extra workspaces gives LTS_ERR_OOM; served requests
  fall back to the context's own workspace; the context keeps working.
Both variables are read at call time by the library (test hooks only)."""
import os

import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OK, ERR_OOM, ERR_TIMEOUT = 0, 4, 6


@pytest.fixture(scope="module")
def lts():
    import paper_2009_00083_gb300 as lts_mod

    lts_mod.load()
    return lts_mod


class env:
    def __init__(self, name, value):
        self.name, self.value = name, value

    def __enter__(self):
        self.old = os.environ.get(self.name)
        os.environ[self.name] = self.value

    def __exit__(self, *a):
        if self.old is None:
            os.environ.pop(self.name, None)
        else:
            os.environ[self.name] = self.old


def _case(shape=(96, 112), seed=3):
    f = W.gaussian_field(shape, 8, 0.05, seed=seed)
    ids = oracle.authorized_by_persistence(f, 0.05)
    g, O = oracle.lts(f, ids, mode="both")
    return f, ids, g, O


def _exact(g, o, g_ref, o_ref):
    return np.array_equal(o, o_ref) and np.array_equal(g.view(np.uint32), g_ref.view(np.uint32))


def test_expired_sort_wait_returns_timeout_and_the_context_recovers(lts):
    f, ids, g_ref, o_ref = _case()
    assert f.size > 2 * 4096                        # the sort runs more than one tile
    dev = torch.device("cuda", 0)
    fd, idd = torch.from_numpy(f).to(dev), torch.from_numpy(ids).to(dev)
    ctx = lts.Context(f.size, device=0)
    try:
        with env("LTS_TEST_STALL_SORT", "1"):
            with pytest.raises(lts.LtsError) as e:
                ctx.simplify(fd, idd, "both")
            assert e.value.code == ERR_TIMEOUT
        for _ in range(2):
            g, o, _ = ctx.simplify(fd, idd, "both")
            torch.cuda.synchronize()
            assert _exact(g.cpu().numpy(), o.cpu().numpy(), g_ref, o_ref)
    finally:
        ctx.close()


def test_failed_allocations_give_oom_and_the_context_recovers(lts):
    cases = [_case((64 + 8 * k, 80), seed=10 + k) for k in range(3)]
    dev = torch.device("cuda", 0)
    fields = [torch.from_numpy(c[0]).to(dev) for c in cases]
    idss = [torch.from_numpy(c[1]).to(dev) for c in cases]
    outs = [(torch.empty_like(f), torch.empty(f.shape, dtype=torch.int32, device=dev)) for f in fields]
    grids = [lts.grid_of_shape(tuple(f.shape)) for f in fields]
    nmax = max(f.numel() for f in fields)

    with env("LTS_TEST_FAIL_ALLOC", "1"):
        with pytest.raises(lts.LtsError) as e:
            lts.lts_create(0, nmax)
        assert e.value.code == ERR_OOM
    ctx = lts.Context(nmax, device=0)

    def batch():
        return lts.lts_simplify_batch(ctx._ctx, grids, [f.data_ptr() for f in fields], [a.data_ptr() for a in idss],
                                      [a.numel() for a in idss], "both", [g.data_ptr() for g, _ in outs],
                                      [o.data_ptr() for _, o in outs])

    try:
        # the batch's extra workspaces cannot be allocated
        with env("LTS_TEST_FAIL_ALLOC", "1"):
            assert batch() == ERR_OOM
            assert "workspace" in lts.lts_last_error(ctx._ctx)
            # served requests fall back to the context's own workspace
            tickets = []
            for k, (f, a) in enumerate(zip(fields, idss)):
                g, o = outs[k]
                code, t = lts.lts_submit(ctx._ctx, grids[k], f.data_ptr(), a.data_ptr(), a.numel(), "both",
                                         g.data_ptr(), o.data_ptr())
                assert code == OK
                tickets.append(t)
            for t in tickets:
                done = False
                while not done:
                    code, done = lts.lts_poll(ctx._ctx, t)
                assert code == OK
            torch.cuda.synchronize()
            for (g, o), c in zip(outs, cases):
                assert _exact(g.cpu().numpy(), o.cpu().numpy(), c[2], c[3])
        # after the failures: a plain call and the batch are exact
        g, o, _ = ctx.simplify(fields[0], idss[0], "both")
        torch.cuda.synchronize()
        assert _exact(g.cpu().numpy(), o.cpu().numpy(), cases[0][2], cases[0][3])
        for g, o in outs:
            g.zero_()
            o.zero_()
        assert batch() == OK, lts.lts_last_error(ctx._ctx)
        torch.cuda.synchronize()
        for (g, o), c in zip(outs, cases):
            assert _exact(g.cpu().numpy(), o.cpu().numpy(), c[2], c[3])
    finally:
        ctx.close()
