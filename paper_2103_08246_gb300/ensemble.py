"""Batched ensembles of independent cases of uneven size.

Each member is an ordinary solver state (its own grid, Re, bodies and
precision, with tile parameters from the autotuner); the ensemble advances
all of them with one CUDA graph launch per step in which every member's
captured step is an independent branch.
"""
from __future__ import annotations

from . import autotune, binding, inputs


def build(cases=None, precision=binding.IBM_MIXED, tuned=True, batched=False):
    """Create the members (seeded noise per case) and the ensemble; batched:
    the members' explicit stages in one persistent launch."""
    cases = inputs.ensemble_cases() if cases is None else cases
    solvers = []
    for wl in cases:
        tiles = autotune.tune(wl, precision) if tuned else None
        solvers.append(binding.Solver(wl, precision, noise=inputs.initial_noise(wl), tiles=tiles))
    return solvers, binding.Ensemble(solvers, batched=batched)
