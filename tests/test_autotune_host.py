"""Host logic of the tile autotuner (no GPU): the coordinate search keeps the
fastest candidate of each parameter, writes the choice and its timings to
the cache under the shape/precision/GPU key, and a cached shape is answered
without building a solver. The solver is replaced by a stand-in whose stage
times are a known function of the tiles."""
import json

from paper_2103_08246_gb300 import autotune, binding, inputs

BEST = {"rhs_planes": 32, "rhs_stages": 6, "afx_planes": 64}


class FakeSolver:
    made = 0

    def __init__(self, wl, precision, tiles=None):
        FakeSolver.made += 1
        self.tiles = dict(tiles)

    def step(self, n=1, dt=None):
        pass

    def time_stage(self, stage, nrep=10):
        t = self.tiles
        if stage == "rhs":
            return 1.0 + abs(t["rhs_planes"] - BEST["rhs_planes"]) * 0.01 + abs(t["rhs_stages"] - BEST["rhs_stages"]) * 0.02
        assert stage == "af_x"
        return 0.5 + abs(t["afx_planes"] - BEST["afx_planes"]) * 0.001

    def close(self):
        pass


def test_search_picks_the_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setattr(binding, "Solver", FakeSolver)
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "test-gpu")
    wl = inputs.small(16, 8, 8)
    cache = tmp_path / "tiles.json"
    FakeSolver.made = 0
    tiles = autotune.tune(wl, binding.IBM_FP32, cache_path=str(cache), reps=1)
    assert tiles == BEST
    assert FakeSolver.made == sum(len(v) for v in autotune.CANDIDATES.values())
    stored = json.load(open(cache))
    key = f"{wl.nx}x{wl.ny}x{wl.nz}:p{binding.IBM_FP32}:test-gpu"
    assert stored[key]["tiles"] == BEST
    assert set(stored[key]["timings_ms"]) == {f"{k}={v}" for k, vs in autotune.CANDIDATES.items() for v in vs}
    # a cached shape needs no solver; another precision is a new key
    FakeSolver.made = 0
    assert autotune.tune(wl, binding.IBM_FP32, cache_path=str(cache)) == BEST
    assert FakeSolver.made == 0
    autotune.tune(wl, binding.IBM_MIXED, cache_path=str(cache), reps=1)
    assert FakeSolver.made > 0
    assert len(json.load(open(cache))) == 2


def test_unreadable_cache_is_ignored(tmp_path, monkeypatch):
    monkeypatch.setattr(binding, "Solver", FakeSolver)
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "test-gpu")
    cache = tmp_path / "tiles.json"
    cache.write_text("{not json")
    assert autotune.tune(inputs.small(16, 8, 8), binding.IBM_FP64, cache_path=str(cache), reps=1) == BEST
