"""Host logic of the tile autotuner (no GPU: a fake batch and timer)."""
import json

from paper_2311_15242_gb300 import autotune as AT


class FakeBatch:
    storage = 1  # f32

    def __init__(self):
        self.calls = []

    def set_tiles(self, tx, ty, sor):
        self.calls.append((tx, ty, sor))


def fake_timer(cost):
    def t(b):
        return cost[b.calls[-1]]
    return t


def costs(best_cell=(64, 4), best_sor=2):
    c = {}
    for tx, ty in AT.CELL_TILES:
        for v in AT.SOR_TILES:
            c[(tx, ty, v)] = 10.0 + (0 if (tx, ty) == best_cell else 3.0 + tx / 100) + \
                (0 if v == best_sor else 1.0 + v / 10)
    return c


def test_width_class_and_key():
    assert AT.width_class([64, 64, 96]) == "w64"
    assert AT.width_class([64, 128, 192, 256, 256]) == "w256"
    assert AT.width_class([100]) == "w128"
    assert AT.cache_key("d2q9", 2, [64]) == "d2q9/f16/w64"


def test_coordinate_search_picks_the_fastest_and_applies_it(tmp_path):
    b = FakeBatch()
    path = str(tmp_path / "tiles.json")
    r = AT.tune(b, [96, 128, 128], timer=fake_timer(costs()), cache_path=path)
    assert (r["tx"], r["ty"], r["sor"]) == (64, 4, 2)
    assert r["source"] == "timed"
    assert b.calls[-1] == (64, 4, 2)
    # every cell tile once with SOR tile 0, then the other SOR tiles once
    assert len(r["timings"]) == len(AT.CELL_TILES) + len(AT.SOR_TILES) - 1
    saved = json.load(open(path))
    assert saved["d2q9/f32/w128"]["tx"] == 64


def test_cache_hit_skips_timing(tmp_path):
    path = str(tmp_path / "tiles.json")
    AT.tune(FakeBatch(), [128], timer=fake_timer(costs((32, 16), 1)), cache_path=path)
    b = FakeBatch()

    def no_timing(_):
        raise AssertionError("timed on a cache hit")
    r = AT.tune(b, [128, 100], timer=no_timing, cache_path=path)
    assert r["source"] == "cache"
    assert b.calls == [(32, 16, 1)]
    # another width class is timed again
    b2 = FakeBatch()
    r2 = AT.tune(b2, [256], timer=fake_timer(costs()), cache_path=path)
    assert r2["source"] == "timed" and len(json.load(open(path))) == 2


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tiles.json"
    path.write_text("{not json")
    r = AT.tune(FakeBatch(), [64], timer=fake_timer(costs()), cache_path=str(path))
    assert r["source"] == "timed"


class FakeSolver:
    storage = 1

    def __init__(self):
        self.calls = []

    def set_sor_tile(self, v):
        self.calls.append(v)


def test_single_context_sor_variant(tmp_path):
    path = str(tmp_path / "tiles.json")
    cost = {0: 5.0, 1: 6.0, 2: 7.0, 3: 4.0, 4: 4.5, 5: 4.2, 6: 4.8, 7: 4.9, 8: 5.5}
    s = FakeSolver()
    r = AT.tune_single(s, 256, timer=lambda b: cost[b.calls[-1]], cache_path=path)
    assert r["sor"] == 3 and s.calls[-1] == 3 and r["key"] == "d2q9/f32/w256/single"
    s2 = FakeSolver()
    r2 = AT.tune_single(s2, 200, timer=lambda b: 1 / 0, cache_path=path)
    assert r2["source"] == "cache" and s2.calls == [3]
