"""Host logic of the autotuner (no GPU): it keeps the fastest candidate,
caches the choice per key in JSON, and reuses it without timing again."""
import json

import pytest

from paper_1609_03782_gb300 import tune


def test_pick_fastest_and_cache(tmp_path):
    cost = {0: 5.0, 8: 2.0, 16: 3.0}
    calls = []

    def timer(fn, reps):
        fn()
        return cost[calls[-1]]

    t = tune.Tuner(str(tmp_path / "c.json"), timer=timer)
    best = t.pick("k1", [0, 8, 16], lambda c: calls.append(c))
    assert best == 8 and calls == [0, 8, 16]
    data = json.loads((tmp_path / "c.json").read_text())
    assert data["k1"]["choice"] == 8
    # a new tuner reads the cache and does not time again
    calls.clear()
    t2 = tune.Tuner(str(tmp_path / "c.json"), timer=timer)
    assert t2.pick("k1", [0, 8, 16], lambda c: calls.append(c)) == 8 and calls == []
    # tuple candidates survive the JSON round trip
    cost2 = {(1, 0): 4.0, (2, 16): 1.0}
    t2.timer = lambda fn, reps: (fn(), cost2[calls[-1]])[1]
    assert t2.pick("k2", [(1, 0), (2, 16)], lambda c: calls.append(c)) == (2, 16)
    t3 = tune.Tuner(str(tmp_path / "c.json"), timer=timer)
    assert t3.pick("k2", [(1, 0), (2, 16)], lambda c: 1 / 0) == (2, 16)


def test_keys_bucket_shapes():
    a = tune.shape_key("filter_ex", (200, 300, 500), "f16", "rational", 30)
    b = tune.shape_key("filter_ex", (256, 512, 512), "f16", "rational", 30)
    assert a == b
    assert a != tune.shape_key("filter_ex", (256, 512, 512), "f32", "rational", 30)
    k = tune.batch_key([(32, 40, 50), (100, 100, 100)], "f32", "rational", 20)
    assert k.startswith("batch|2 cubes|")


class _FakeAfd:
    """Records the knob settings a tuner applies (no GPU)."""

    def __init__(self, cost):
        self.cost, self.state, self.calls = cost, {}, []

    def afd_batch_set_tiles(self, b, kind):
        self.state["tiles"] = kind

    def afd_batch_set_zchunk(self, b, zc):
        self.state["zc"] = zc

    def afd_batch_filter(self, b, K, dt, n, cond, sp):
        self.calls.append((self.state["tiles"], self.state["zc"]))


def test_tune_batch_picks_tile_kind_and_zchunk(tmp_path):
    cost = {(t, z): 10.0 for t in tune.TILES for z in tune.BATCH_ZCHUNKS}
    cost[("64x32", 32)] = 3.0
    fake = _FakeAfd(cost)

    class B:
        shapes = [(32, 40, 50), (64, 64, 64)]
        storage = "f32"

    t = tune.Tuner(str(tmp_path / "c.json"), timer=lambda fn, reps: (fn(), cost[fake.calls[-1]])[1])
    best = t.tune_batch(fake, B(), [-1.5, -1.5], 0.125, 20)
    assert best == ("64x32", 32)
    assert fake.state == {"tiles": "64x32", "zc": 32}     # the choice is left applied
    ms = json.loads((tmp_path / "c.json").read_text())[tune.batch_key(B.shapes, "f32",
                                                                      "rational", 20)]["ms"]
    assert any("wide" in k for k in ms) and any("64x32" in k for k in ms)


class _FakeEx:
    """Records afd_filter_ex calls with the knobs applied (no GPU)."""

    def __init__(self):
        self.state, self.calls = {"zc": 0, "kernel": "auto"}, []

    def afd_set_stream_zchunk(self, ctx, zc):
        self.state["zc"] = zc

    def afd_set_kernel(self, ctx, k):
        self.state["kernel"] = k

    def afd_filter_ex(self, ctx, src, dst, storage, scale, K, dt, n, cond, sp, t):
        self.calls.append((t, self.state["zc"], self.state["kernel"]))


def test_tune_filter_ex_respects_min_depth_and_applies_route(tmp_path):
    class Src:
        shape = (64, 256, 256)

    fake = _FakeEx()
    cost = {}
    for t in tune.DEPTHS:
        for z in (0, 16):
            for r in tune.ROUTES:
                cost[(t, z, r)] = 10.0 - t - (0.5 if r == "two_stage" else 0.0)
    cost[(1, 0, "auto")] = 1.0                       # depth 1 fastest overall
    t = tune.Tuner(str(tmp_path / "c.json"), timer=lambda fn, reps: (fn(), cost[fake.calls[-1]])[1])
    assert t.tune_filter_ex(fake, None, Src(), None, "f16", 1.0, 1.0, 0.125, 20,
                            zchunks=(0, 16)) == 1
    # at least depth 4: the fastest of depths 4 and 8 over both routes
    fake.calls.clear()
    best = t.tune_filter_ex(fake, None, Src(), None, "f16", 1.0, 1.0, 0.125, 20,
                            zchunks=(0, 16), min_depth=4)
    assert best == 8 and fake.state == {"zc": 0, "kernel": "two_stage"}
    assert all(c[0] >= 4 for c in fake.calls)
    assert not any(c[0] == 1 and c[2] != "auto" for c in fake.calls)
    with pytest.raises(ValueError):
        t.tune_filter_ex(fake, None, Src(), None, "f16", 1.0, 1.0, 0.125, 20, min_depth=16)
