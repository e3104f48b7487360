"""Tile-shape autotuner for the solver's streamed kernels.

The explicit stage (rhs_planes: x planes per block of the bulk-copy pipeline;
rhs_stages: depth of its shared-memory ring)
and the FP32 implicit x factor (afx_planes: x planes per block) have tile
parameters that change performance but not results. For a problem shape and
precision the tuner times each candidate with the library's stage timer on a
timing-only state, keeps the fastest, and caches the choice in a JSON file
keyed by shape, precision and GPU name.
"""
from __future__ import annotations

import json
import os

from . import binding

CANDIDATES = {
    "rhs_planes": (8, 16, 32, 64),
    "rhs_stages": (4, 5, 6, 8),
    "afx_planes": (16, 32, 64),   # 16: register segments; 32, 64: shared-memory segments
}
STAGE_OF = {"rhs_planes": "rhs", "rhs_stages": "rhs", "afx_planes": "af_x"}
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tile_cache.json")


def _gpu_name():
    import torch
    return torch.cuda.get_device_name()


def _key(wl, precision):
    return f"{wl.nx}x{wl.ny}x{wl.nz}:p{precision}:{_gpu_name()}"


def load_cache(path=DEFAULT_CACHE):
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except Exception:
            return {}
    return {}


def tune(wl, precision, cache_path=DEFAULT_CACHE, reps=5, use_cache=True):
    """Best tile parameters for this shape (coordinate search, cached)."""
    cache = load_cache(cache_path) if use_cache else {}
    key = _key(wl, precision)
    if key in cache:
        return dict(cache[key]["tiles"])
    tiles = {k: v[len(v) // 2] for k, v in CANDIDATES.items()}
    timings = {}
    for name, values in CANDIDATES.items():

        best = None
        for val in values:
            trial = dict(tiles, **{name: val})
            s = binding.Solver(wl, precision, tiles=trial)
            s.step(1)
            s.time_stage(STAGE_OF[name], 2)
            ms = s.time_stage(STAGE_OF[name], reps)
            s.close()
            timings[f"{name}={val}"] = ms
            if best is None or ms < best[0]:
                best = (ms, val)
        tiles[name] = best[1]
    cache = load_cache(cache_path)
    cache[key] = {"tiles": tiles, "timings_ms": timings}
    try:
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return tiles
