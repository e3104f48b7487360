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
The precision comparison runs the laminar flag with the same fixed time
step in FP64, mixed precision and FP32 and states the errors of the last two
against the first (trailing-edge trajectory, Strouhal number, amplitude,
fields, divergence).

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


def cycle_statistics(t, y, hysteresis=0.5):
    """Period and amplitude of an oscillation from its upward crossings of
    the mean, with hysteresis: a crossing counts only after the signal has
    been below -hysteresis * rms since the last one and it is confirmed once
    the signal reaches +hysteresis * rms, so that harmonics and small
    wiggles near the mean add no crossings. Crossing times by linear
    interpolation; the period is the mean spacing of the crossings, the
    amplitude the mean over whole cycles of half the peak-to-peak
    excursion. Resolves the frequency to a fraction of the sampling interval
    over the record, where a periodogram resolves one bin (1 / record
    length)."""
    t = np.asarray(t, dtype=float)
    y = np.asarray(y, dtype=float)
    y = y - y.mean()
    band = hysteresis * float(np.sqrt(np.mean(y * y)))
    up, armed, cand = [], False, None
    for q in range(len(y) - 1):
        if y[q] < -band:
            armed, cand = True, None
        if armed and y[q] < 0 <= y[q + 1]:
            cand = q
        if armed and cand is not None and y[q + 1] > band:
            up.append(cand)
            armed, cand = False, None
    up = np.asarray(up, dtype=int)
    if up.size < 2:
        return {"period": float("nan"), "cycles": 0, "amplitude": float("nan")}
    tc = t[up] - y[up] * (t[up + 1] - t[up]) / (y[up + 1] - y[up])
    amps = [0.5 * float(y[a:b + 1].max() - y[a:b + 1].min()) for a, b in zip(up[:-1], up[1:])]
    per = np.diff(tc)
    return {"period": float(per.mean()), "period_std": float(per.std()), "cycles": int(per.size),
            "amplitude": float(np.mean(amps)), "amplitude_std": float(np.std(amps))}


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


def precision_comparison(steps=12000, discard=4000, cells_per_length=32, dt=6e-3, every=2, early=200,
                         precisions=("fp64", "mixed", "fp32")):
    """The laminar flag (production domain and flag, no bars, Re = 200) run
    with the same fixed time step in each precision. Errors of the mixed and
    FP32 runs are taken against the FP64 run (the path that matches the CPU
    oracle to 1e-9):
      * after `early` steps, u, v, w (relative to U), gauge-fixed p (relative
        to U^2) and the trailing-edge midpoint (relative to L);
      * the times at which the trailing-edge trajectories first differ by
        1e-4, 1e-3 and 1e-2 L (the self-excited flapping amplifies any
        difference until the runs drift apart in phase);
      * after `discard` steps, the flapping statistics: period and amplitude
        from zero crossings, Strouhal number St = L / (U T), rms;
      * the divergence left after the projection (h max |div u|)."""
    wl = laminar_workload(cells_per_length)
    prec = {"fp64": binding.IBM_FP64, "fp32": binding.IBM_FP32, "mixed": binding.IBM_MIXED}
    runs = {}
    for name in precisions:
        s = binding.Solver(wl, prec[name], noise=inputs.initial_noise(wl))
        t, te = [], []
        early_fields = None
        t0 = time.perf_counter()
        for k in range(0, steps, every):
            s.step(every, dt=dt)
            st = s.stats()
            t.append(st["t"])
            te.append(list(st["te_mid"]))
            if early_fields is None and k + every >= early:
                early_fields = s.fields()
        wall = time.perf_counter() - t0
        t, te = np.asarray(t), np.asarray(te)
        keep = slice(discard // every, None)
        comp = 1 + int(np.argmax(te[keep, 1:].std(axis=0)))
        cyc = cycle_statistics(t[keep], te[keep, comp])
        st = s.stats()
        runs[name] = {"t": t, "te": te, "cyc": cyc, "comp": comp, "seconds": wall,
                      "rms": float(te[keep, comp].std()), "h_max_div": st["max_div"] * wl.lx / wl.nx,
                      "early": early_fields}
        s.close()
    ref = runs["fp64"]
    out = {"workload": wl.name, "cells": wl.cells, "re": wl.re, "steps": steps, "discard": discard,
           "dt": dt, "early_steps": early, "t_end": float(ref["t"][-1]),
           "fp64": {"period": ref["cyc"]["period"], "strouhal": wl.flag_len / ref["cyc"]["period"],
                    "amplitude": ref["cyc"]["amplitude"], "rms": ref["rms"], "cycles": ref["cyc"]["cycles"],
                    "period_std": ref["cyc"].get("period_std"), "amplitude_std": ref["cyc"].get("amplitude_std"),
                    "h_max_div": ref["h_max_div"], "seconds": ref["seconds"]}}
    # sampling error of the mean period and amplitude (cycle-to-cycle spread / sqrt(cycles))
    for key in ("period", "amplitude"):
        sd = ref["cyc"].get(key + "_std")
        out["fp64"][key + "_sampling_err"] = (sd / np.sqrt(ref["cyc"]["cycles"])) if sd is not None else None
    # the trailing-edge trajectories, every 30th sample (t, fp64, and each other precision)
    sub = slice(None, None, 30)
    out["te_series"] = {"t": np.round(ref["t"][sub], 6).tolist(), "component": ref["comp"],
                        **{name: np.round(runs[name]["te"][sub, ref["comp"]], 6).tolist() for name in precisions}}
    for name in precisions:
        if name == "fp64":
            continue
        r = runs[name]
        st_r = wl.flag_len / r["cyc"]["period"]
        e = {"period": r["cyc"]["period"], "strouhal": st_r, "amplitude": r["cyc"]["amplitude"],
             "rms": r["rms"], "cycles": r["cyc"]["cycles"], "period_std": r["cyc"].get("period_std"),
             "amplitude_std": r["cyc"].get("amplitude_std"),
             "strouhal_rel_err": abs(st_r - out["fp64"]["strouhal"]) / out["fp64"]["strouhal"],
             "amplitude_rel_err": abs(r["cyc"]["amplitude"] - ref["cyc"]["amplitude"]) / ref["cyc"]["amplitude"],
             "rms_rel_err": abs(r["rms"] - ref["rms"]) / ref["rms"],
             "h_max_div": r["h_max_div"], "seconds": r["seconds"]}
        dte = np.abs(r["te"] - ref["te"]).max(axis=1) / wl.flag_len
        for thr in (1e-4, 1e-3, 1e-2):
            hit = np.nonzero(dte > thr)[0]
            e[f"t_diverge_{thr:g}"] = float(ref["t"][hit[0]]) if hit.size else None
        e["te_err_early"] = float(dte[early // every - 1])
        for q, a, b in zip("uvwp", r["early"], ref["early"]):
            if q == "p":
                a, b = a - a.mean(), b - b.mean()
            e[f"{q}_err_early"] = float(np.abs(a - b).max()) / max(float(np.abs(b).max()), 1.0)
        out[name] = e
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
    ap.add_argument("--precision", action="store_true",
                    help="compare the mixed and FP32 paths with the FP64 one on the laminar flag")
    ap.add_argument("--cells", type=int, default=32, help="cells per unit length of the precision comparison")
    ap.add_argument("--dt", type=float, default=6e-3, help="fixed time step of the precision comparison")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.precision:
        res = precision_comparison(a.steps, a.discard, cells_per_length=a.cells, dt=a.dt)
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
        print(json.dumps(res, indent=1))
        return
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
