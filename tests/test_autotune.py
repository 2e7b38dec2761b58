"""The autotuner's host logic (buckets, cache, coordinate descent) on the CPU
with a stand-in context; the GPU tests check that tunings change no result."""
import json

import pytest

from paper_2009_00083_gb300 import autotune as AT


def test_buckets_separate_dimensions_and_sizes():
    assert AT.bucket((256, 256)) == "2d:2^16"
    assert AT.bucket((64, 64, 64)) == "3d:2^18"
    assert AT.bucket((65, 64, 64)) == "3d:2^20"           # rounded up to an even power
    assert AT.bucket((512, 512, 512)) == "3d:2^28"
    assert AT.bucket((8, 8)) == "2d:2^12"                 # small grids share one bucket
    assert AT.bucket((1 << 12, 1 << 12)) != AT.bucket((256, 256, 256))


def test_cache_round_trip_and_lookup(tmp_path):
    p = str(tmp_path / "c.json")
    assert AT.load_cache(p) == {}
    cache = {}
    AT.record(cache, "GPU X", "3d:2^24", {"engine_blocks_per_sm": 6}, 0.0123, [({"engine_blocks_per_sm": 8}, 0.013)])
    AT.save_cache(cache, p)
    back = AT.load_cache(p)
    assert back == json.loads(json.dumps(cache))
    t = AT.lookup(back, "GPU X", "3d:2^24")
    assert t == {"engine_blocks_per_sm": 6, "team_blocks_per_sm": 12, "batch_workspaces": 32}
    assert AT.lookup(back, "GPU Y", "3d:2^24") is None
    assert AT.lookup(back, "GPU X", "2d:2^16") is None


class FakeCtx:
    def __init__(self):
        self.t = None
        self.device = "fake"

    def set_tuning(self, t):
        self.t = None if t is None else dict(t)

    def tuning(self):
        out = dict(AT.DEFAULTS)
        out.update(self.t or {})
        return out


def test_apply_sets_the_cached_tuning_or_the_defaults():
    cache = {}
    AT.record(cache, "GPU X", "batch", {"batch_workspaces": 16}, 0.5, [])
    ctx = FakeCtx()
    assert AT.apply(ctx, key="batch", cache=cache, gpu="GPU X")["batch_workspaces"] == 16
    assert AT.apply(ctx, shape=(32, 32, 32), cache=cache, gpu="GPU X") == AT.DEFAULTS
    assert AT.apply(ctx, key="batch", cache=cache, gpu="GPU Z") == AT.DEFAULTS


def test_descent_keeps_the_fastest_candidate_of_each_knob():
    ctx = FakeCtx()
    cost = {("engine_blocks_per_sm", 4): 3.0, ("engine_blocks_per_sm", 6): 1.0, ("engine_blocks_per_sm", 8): 2.0,
            ("team_blocks_per_sm", 8): 0.5, ("team_blocks_per_sm", 12): 0.7, ("team_blocks_per_sm", 16): 0.9}

    def timer(run):
        t = ctx.tuning()
        return cost[("engine_blocks_per_sm", t["engine_blocks_per_sm"])] + \
            cost[("team_blocks_per_sm", t["team_blocks_per_sm"])]

    best, sec, trials = AT._descend(ctx, AT.KNOBS, lambda: 1, lambda a, b: a == b, 1, lambda: None, timer)
    assert best == {"engine_blocks_per_sm": 6, "team_blocks_per_sm": 8}
    assert sec == pytest.approx(1.5)
    assert ctx.t == best
    assert len(trials) == 1 + 2 + 2


def test_descent_keeps_the_default_unless_a_candidate_is_clearly_faster():
    ctx = FakeCtx()
    cost = {4: 1.00, 6: 0.995, 8: 1.0}                   # 0.5% apart: noise

    def timer(run):
        return cost[ctx.tuning()["engine_blocks_per_sm"]]

    best, sec, _ = AT._descend(ctx, {"engine_blocks_per_sm": (4, 6, 8)}, lambda: 1, lambda a, b: a == b, 1,
                               lambda: None, timer)
    assert best == {"engine_blocks_per_sm": 8} and sec == 1.0
    cost[6] = 0.9
    best, sec, _ = AT._descend(ctx, {"engine_blocks_per_sm": (4, 6, 8)}, lambda: 1, lambda a, b: a == b, 1,
                               lambda: None, timer)
    assert best == {"engine_blocks_per_sm": 6} and sec == 0.9


def test_descent_refuses_a_tuning_that_changes_the_result():
    ctx = FakeCtx()
    with pytest.raises(RuntimeError):
        AT._descend(ctx, AT.KNOBS, lambda: ctx.tuning()["engine_blocks_per_sm"], lambda a, b: a == b, 1,
                    lambda: None, lambda run: 1.0)
