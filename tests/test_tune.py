"""Host logic of the autotuner (no GPU): it keeps the fastest candidate,
caches the choice per key in JSON, and reuses it without timing again."""
import json

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
