"""Batches (lts_simplify_batch) and served requests (lts_submit / lts_poll)
through the C ABI, bit-exact against the oracle field by field, including a
failing field in the middle of each."""
import numpy as np
import pytest

import oracle
from paper_2009_00083_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lts():
    import paper_2009_00083_gb300 as lts_mod

    lts_mod.load()
    return lts_mod


def mixed_fields(seed, count):
    """2D and 3D fields of mixed sizes, heavy ties in some, with random authorized sets."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        if k % 2 == 0:
            shape = (int(rng.integers(8, 90)), int(rng.integers(8, 90)))
        else:
            shape = tuple(int(rng.integers(4, 26)) for _ in range(3))
        f = W.random_tiny_field(rng, shape, levels=None if k % 3 else 7)
        O = oracle.order_field(f).reshape(-1)
        ids = np.nonzero(rng.random(f.size) < 0.05)[0]
        ids = np.concatenate([ids, [np.argmax(O), np.argmin(O)]]).astype(np.int32)
        out.append((f, ids))
    return out


def to_dev(f, ids):
    dev = torch.device("cuda", 0)
    return torch.from_numpy(np.ascontiguousarray(f)).to(dev), torch.from_numpy(ids).to(dev)


def check(g, o, f, ids, what):
    g_ref, o_ref = oracle.lts(f, ids, mode="both")
    assert np.array_equal(o.cpu().numpy(), o_ref), f"order differs ({what})"
    assert np.array_equal(g.cpu().numpy().view(np.uint32), g_ref.view(np.uint32)), f"field differs ({what})"


@pytest.mark.parametrize("count", [1, 3, 13])
def test_batch_matches_oracle(lts, count):
    cases = mixed_fields(100 + count, count)
    ctx = lts.Context(max(f.size for f, _ in cases), device=0)
    try:
        dev = [to_dev(f, ids) for f, ids in cases]
        for rep in range(2):                        # the batch workspaces are reused on the second call
            outs, stats = ctx.simplify_batch([d[0] for d in dev], [d[1] for d in dev], "both")
            torch.cuda.synchronize()
            for i, ((f, ids), (g, o)) in enumerate(zip(cases, outs)):
                check(g, o, f, ids, f"rep {rep} field {i} {f.shape}")
                assert stats[i]["n_vertices"] == f.size
    finally:
        ctx.close()


def test_batch_reports_the_failing_field_and_finishes_the_others(lts):
    cases = mixed_fields(7, 9)
    f_bad = cases[3][0].copy()
    f_bad.reshape(-1)[5] = np.nan
    ctx = lts.Context(max(f.size for f, _ in cases), device=0)
    try:
        dev = [to_dev(f, ids) for f, ids in cases]
        dev[3] = to_dev(f_bad, cases[3][1])
        fields = [d[0] for d in dev]
        auth = [d[1] for d in dev]
        outs = [(torch.empty_like(f), torch.empty(f.shape, dtype=torch.int32, device=f.device)) for f in fields]
        code = lts.lts_simplify_batch(ctx._ctx, [lts.grid_of_shape(tuple(f.shape)) for f in fields],
                                      [f.data_ptr() for f in fields], [a.data_ptr() for a in auth],
                                      [a.numel() for a in auth], "both", [o[0].data_ptr() for o in outs],
                                      [o[1].data_ptr() for o in outs])
        assert code == 2
        assert "field 3" in lts.lts_last_error(ctx._ctx)
        torch.cuda.synchronize()
        for i, ((f, ids), (g, o)) in enumerate(zip(cases, outs)):
            if i != 3:
                check(g, o, f, ids, f"field {i}")
        # the failed field left no state behind
        outs2, _ = ctx.simplify_batch([d[0] for d in dev[:3]], [d[1] for d in dev[:3]], "both")
        for i in range(3):
            check(outs2[i][0], outs2[i][1], cases[i][0], cases[i][1], f"after failure, field {i}")
    finally:
        ctx.close()


def test_batch_argument_errors_name_the_field(lts):
    cases = mixed_fields(3, 3)
    ctx = lts.Context(max(f.size for f, _ in cases) - 1, device=0)
    try:
        dev = [to_dev(f, ids) for f, ids in cases]
        big = int(np.argmax([f.size for f, _ in cases]))
        with pytest.raises(lts.LtsError) as e:
            ctx.simplify_batch([d[0] for d in dev], [d[1] for d in dev])
        assert e.value.code == 1 and f"field {big}" in str(e.value)
    finally:
        ctx.close()


def test_submitted_requests_match_oracle_in_order_and_after_a_failure(lts):
    cases = mixed_fields(21, 12)
    f_bad = cases[5][0].copy()
    f_bad.reshape(-1)[0] = np.nan
    ctx = lts.Context(max(f.size for f, _ in cases), device=0)
    try:
        dev = [to_dev(f, ids) for f, ids in cases]
        dev[5] = to_dev(f_bad, cases[5][1])
        torch.cuda.synchronize()
        tickets = [ctx.submit(f, a, "both") for f, a in dev]
        assert tickets == list(range(tickets[0], tickets[0] + len(tickets)))
        results = {}
        for _ in range(200000):
            for i, t in enumerate(tickets):
                if i in results:
                    continue
                try:
                    r = ctx.poll(t)
                except lts.LtsError as err:
                    results[i] = err
                    continue
                if r is not None:
                    results[i] = r
            if len(results) == len(tickets):
                break
        assert len(results) == len(tickets)
        assert isinstance(results[5], lts.LtsError) and results[5].code == 2
        for i, (f, ids) in enumerate(cases):
            if i != 5:
                g, o = results[i]
                check(g, o, f, ids, f"request {i}")
        code, done = lts.lts_poll(ctx._ctx, tickets[-1] + 100)
        assert code == 1 and not done
    finally:
        ctx.close()


def test_full_batch_workload_against_stored_oracle_hashes(lts):
    """The 256-field batch workload (2D 64..1024 squares, 3D 32..160 cubes,
    125,571,267 vertices) in one lts_simplify_batch call: every field's g and
    order field hash equal the oracle's stored ones."""
    from tests.golden import store as mg

    rec = mg.load_record("mixed_batch_256")
    auth = mg.load_set_authorized("mixed_batch_256")
    specs = W.batch_specs(256)
    dev = torch.device("cuda", 0)
    fields, ids = [], []
    for spec, fr, a in zip(specs, rec["fields"], auth):
        f = W.batch_field(spec)
        assert W.sha256_of(f) == fr["field_sha256"]
        fields.append(torch.from_numpy(f).to(dev))
        ids.append(torch.from_numpy(a).to(dev))
    ctx = lts.Context(max(f.numel() for f in fields), device=0)
    try:
        outs, _ = ctx.simplify_batch(fields, ids, "both", with_stats=False)
        torch.cuda.synchronize()
        for k, ((g, o), fr) in enumerate(zip(outs, rec["fields"])):
            assert W.sha256_of(o.cpu().numpy()) == fr["order_sha256"], f"field {k} {fr['shape']}: order"
            assert W.sha256_of(g.cpu().numpy()) == fr["g_sha256"], f"field {k} {fr['shape']}: field"
    finally:
        ctx.close()


@pytest.mark.parametrize("concurrent", [0, 3, 15])
def test_served_pool_against_stored_oracle_hashes(lts, concurrent):
    """The first 16 served requests (3D cubes of side 32..256) through
    lts_submit / lts_poll, all queued at once, each twice (forwards, then
    backwards), on the context's own workspace one after another
    (concurrent = 0) or spread over 3 or 15 serving workspaces running side by
    side: every result equals the oracle's stored one, alone or in the mix."""
    from tests.golden import store as mg

    rec = mg.load_record("serve_pool_16")
    auth = mg.load_set_authorized("serve_pool_16")
    dev = torch.device("cuda", 0)
    reqs = []
    for spec, fr, a in zip(W.serve_specs(16), rec["fields"], auth):
        f = W.serve_field(spec)
        assert W.sha256_of(f) == fr["field_sha256"]
        reqs.append((torch.from_numpy(f).to(dev), torch.from_numpy(a).to(dev)))
    ctx = lts.Context(max(f.numel() for f, _ in reqs), device=0)
    try:
        ctx.serve_config(concurrent)
        torch.cuda.synchronize()
        order = list(range(16)) + list(range(15, -1, -1))
        tickets = [ctx.submit(*reqs[k], "both") for k in order]
        done = {}
        while len(done) < len(tickets):
            for i, t in enumerate(tickets):
                if i not in done:
                    r = ctx.poll(t)
                    if r is not None:
                        done[i] = r
        for i, k in enumerate(order):
            g, o = done[i]
            fr = rec["fields"][k]
            assert W.sha256_of(o.cpu().numpy()) == fr["order_sha256"], f"request {k} (#{i}): order"
            assert W.sha256_of(g.cpu().numpy()) == fr["g_sha256"], f"request {k} (#{i}): field"
    finally:
        ctx.close()


def test_serve_config_errors(lts):
    ctx = lts.Context(1 << 16, device=0)
    try:
        for bad in ((-1, 1 << 30), (16, 1 << 30), (2, -5)):
            with pytest.raises(lts.LtsError) as e:
                ctx.serve_config(*bad)
            assert e.value.code == 1
        # a zero budget allocates no serving workspace: requests run on the context's own
        ctx.serve_config(7, 0)
        f = W.make_config_field(0, shape=(64, 48))
        ids = oracle.authorized_by_persistence(f, 0.05)
        fd, idd = to_dev(f, ids)
        t = ctx.submit(fd, idd, "both")
        r = None
        while r is None:
            r = ctx.poll(t)
        check(r[0], r[1], f, ids, "zero budget")
    finally:
        ctx.close()
