"""Laminar flag validation (the paper's appendix, flapping flag in laminar
flow): the flag of the production workload in uniform inflow (no bars, Tu =
0) at Re = 200, its trailing-edge midpoint oscillation, Strouhal number and
amplitude, at two grid spacings. Also the comparison of the two bar-grid
forcings (delta-kernel markers against Eulerian volume-fraction forcing):
cost, velocity left inside the bars, and the wake downstream.

The comparison data of the appendix (an earlier three-dimensional flag study)
are not available here, so the run reports its own numbers and their
grid dependence: the flapping period at h = 1/32 against h = 1/64 (the
appendix states that its period and the reference one differ by about 2%).
All stepping runs in the library's kernels; the analysis is host-side.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding, inputs
from .inflow import strouhal


def flag_oscillation(t, te, length=1.0, speed=1.0):
    """Strouhal number, amplitude (half the peak-to-peak excursion) and rms of
    the trailing-edge midpoint's transverse motion; te [n, 3] sampled at t.
    The transverse direction is the one (y or z) that moves most."""
    te = np.asarray(te, dtype=float)
    comp = 1 + int(np.argmax(te[:, 1:].std(axis=0)))
    y = te[:, comp]
    St, rms = strouhal(t, y, length, speed)
    return {"strouhal": St, "period": length / (St * speed) if St > 0 else float("inf"),
            "amplitude": 0.5 * float(y.max() - y.min()), "rms": rms, "component": comp}


def laminar_workload(cells_per_length=64, base=inputs.PRODUCTION):
    """The production domain and flag without the bar grid, at spacing
    1 / cells_per_length (flag vertices at the grid spacing)."""
    n = cells_per_length
    ratio = n / (base.nx / base.lx)
    return base.replace(name=f"laminar-flag-h1/{n}", nx=int(round(base.nx * ratio)),
                        ny=int(round(base.ny * ratio)), nz=int(round(base.nz * ratio)), bars_on=False,
                        flag_ns=n + 1, flag_nt=n + 1)


def run(wl, steps, discard, precision=binding.IBM_FP32, every=2):
    s = binding.Solver(wl, precision, noise=inputs.initial_noise(wl))
    t, te = [], []
    t0 = time.perf_counter()
    s.step(discard, dt=-1.0)
    for k in range(0, steps - discard, every):
        s.step(every, dt=-1.0)
        st = s.stats()
        t.append(st["t"])
        te.append(list(st["te_mid"]))
    wall = time.perf_counter() - t0
    out = flag_oscillation(t, te, wl.flag_len, 1.0)
    out.update({"workload": wl.name, "cells": wl.cells, "steps": steps, "discard": discard,
                "t_end": float(t[-1]), "seconds": wall})
    s.close()
    return out


def _inside_rods(wl, comp, i):
    """Velocity nodes of component comp on plane i whose whole cell lies in
    the bars (the slab |x - bar_x| <= d/2 crossed with a rod of either
    family): a boolean (ny, nz) mask."""
    h = wl.lx / wl.nx
    d, M = wl.bar_width, wl.bar_mesh
    x = (i + (0.0 if comp == 0 else 0.5)) * h
    if abs(x - wl.bar_x) > 0.5 * d - 0.5 * h:
        return np.zeros((wl.ny, wl.nz), dtype=bool)
    y = (np.arange(wl.ny) + (0.0 if comp == 1 else 0.5)) * h
    z = (np.arange(wl.nz) + (0.0 if comp == 2 else 0.5)) * h

    def in_rod(c, period):
        off = np.abs(((c - 0.5 * M) % M + 0.5 * M) % M - 0.5 * M)   # distance to the nearest centre
        return off <= 0.5 * d - 0.5 * h
    return in_rod(y, wl.ly)[:, None] | in_rod(z, wl.lz)[None, :]


def bar_forcing_comparison(steps=2000, precision=binding.IBM_FP32):
    """Production workload without the flag, the bars forced by markers and
    by the Eulerian volume fraction: stage and step times, the rms velocity
    at the nodes whose cells lie wholly inside the bars (the slip left by the
    forcing after the projection), and the turbulence intensity at x = 2."""
    import torch
    out = {}
    for mode in ("markers", "eulerian"):
        wl = inputs.PRODUCTION.replace(flag_on=False, bar_forcing=mode)
        s = binding.Solver(wl, precision, noise=inputs.initial_noise(wl))
        s.step(steps, dt=-1.0)
        torch.cuda.synchronize()
        ib_ms = s.time_stage("ib", 10)
        step_ms = s.time_stage("step", 10)
        h = wl.lx / wl.nx
        i0, i1 = int((wl.bar_x - wl.bar_width) / h), int((wl.bar_x + wl.bar_width) / h) + 1
        sq, n = 0.0, 0
        for i in range(i0, i1 + 1):
            planes = s.plane(i)
            for comp in range(3):
                m = _inside_rods(wl, comp, i)
                sq += float((planes[comp][m] ** 2).sum())
                n += int(m.sum())
        u, v, w = s.plane(int(round(2.0 / h)))
        tu = float(np.sqrt((u.var() + v.var() + w.var()) / 3.0))
        out[mode] = {"ib_ms": ib_ms, "step_ms": step_ms, "inside_rms": float(np.sqrt(sq / max(n, 1))),
                     "inside_nodes": n, "tu_x2": tu, "markers": int(s.markers().shape[0]),
                     "t": s.stats()["t"]}
        s.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--discard", type=int, default=4000)
    ap.add_argument("--out", default="laminar_flag.json")
    ap.add_argument("--bars", action="store_true",
                    help="compare the two bar-grid forcings instead (production workload, no flag)")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.bars:
        res = bar_forcing_comparison()
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
        print(json.dumps(res, indent=1))
        return
    fine = run(laminar_workload(64), a.steps, a.discard)
    coarse = run(laminar_workload(32), a.steps // 2, a.discard // 2)
    res = {"h_1_64": fine, "h_1_32": coarse,
           "period_difference": abs(coarse["period"] - fine["period"]) / fine["period"]}
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
