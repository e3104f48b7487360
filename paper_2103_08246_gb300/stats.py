"""Virtual probes and the statistics of grid-generated turbulence (Sec. III).

Probe lines run along x at a 3 x 3 set of transverse positions; every few
steps the library gathers the cell-centred velocity of all probes into a
device buffer (``ibm_probe_sample``), so a run keeps full time histories at
negligible cost. From them, per streamwise station (host-side numpy):

* mean velocity U and rms fluctuations u', v', w' (time and transverse
  averages), turbulent kinetic energy k = (u'^2 + v'^2 + w'^2) / 2 and the
  large-scale anisotropy v_rms / u_rms (v, w averaged) of Sec. III;
* Taylor's frozen-turbulence hypothesis, d/dx = -(1/U) d/dt, for the
  longitudinal derivative: Taylor microscale lambda_f^2 = 2 u'^2 / <(du/dx)^2>,
  lambda_g = lambda_f / sqrt(2), dissipation eps = 15 nu <(du/dx)^2>
  (= 30 nu u'^2 / lambda_f^2 in isotropic turbulence), Kolmogorov scale
  eta = (nu^3 / eps)^(1/4), Re_lambda = u' lambda_g / nu, and the integral
  scale L = U * integral of the u' autocorrelation up to its first zero;
* the power-law decay k ~ (x - x0)^-n fitted over the decay region: from
  the station of largest k (the end of the production region behind the
  grid) to one length unit before the outflow (x0 the grid position).

Series are resampled to uniform time before derivatives and correlations
(the CFL step varies).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding, inputs


def probe_cells(wl, x_stride=4, x_start=None, n_transverse=3):
    """Probe cells (i, j, k): every x_stride-th x cell from x_start (default:
    just past the grid) at an n x n set of transverse positions placed
    between the bars' centre lines. Returns (ijk [n, 3], x of each station)."""
    h = wl.lx / wl.nx
    i0 = int(np.ceil((wl.bar_x + wl.bar_width) / h)) + 1 if x_start is None else int(round(x_start / h))
    ii = np.arange(i0, wl.nx, x_stride)
    frac = (np.arange(n_transverse) + 0.5) / n_transverse
    jj = np.minimum((frac * wl.ny).astype(int), wl.ny - 1)
    kk = np.minimum((frac * wl.nz).astype(int), wl.nz - 1)
    cells = np.array([(i, j, k) for i in ii for j in jj for k in kk], dtype=np.int32)
    return cells, (ii + 0.5) * h


def record(solver, cells, steps, every=4, warmup=0):
    """Step the solver, sampling the probes every `every` steps after
    `warmup` steps. Returns (times [T], series [T, n, 3] as float64)."""
    import torch
    if warmup:
        solver.step(warmup, dt=-1.0)
    solver.set_probes(cells)
    n = cells.shape[0]
    T = steps // every
    dtype = torch.float64 if solver.precision == binding.IBM_FP64 else torch.float32
    buf = torch.zeros((T, n, 3), dtype=dtype, device="cuda")
    torch.cuda.synchronize()
    esz = buf.element_size()
    times = []
    for t in range(T):
        solver.step(every, dt=-1.0)
        solver.probe_sample(buf.data_ptr() + t * n * 3 * esz)
        times.append(solver.stats()["t"])
    solver.stream.synchronize()
    return np.asarray(times), buf.double().cpu().numpy()


def _uniform(t, y):
    tu = np.linspace(t[0], t[-1], len(t))
    return tu, np.stack([np.interp(tu, t, y[:, q]) for q in range(y.shape[1])], axis=1)


def station_statistics(t, u, v, w, nu):
    """Statistics of one station from the histories u, v, w [T, m] of its m
    transverse probes (see the module docstring)."""
    U = float(u.mean())
    up = u - u.mean(axis=0)
    vp, wp = v - v.mean(axis=0), w - w.mean(axis=0)
    u2, v2, w2 = float((up ** 2).mean()), float((vp ** 2).mean()), float((wp ** 2).mean())
    tu_, uu = _uniform(t, up)
    dt = tu_[1] - tu_[0]
    dudx = -np.gradient(uu, dt, axis=0) / U
    g2 = float((dudx ** 2).mean())
    lam_f = float(np.sqrt(2.0 * u2 / g2)) if g2 > 0 else float("inf")
    lam_g = lam_f / np.sqrt(2.0)
    eps = 15.0 * nu * g2
    eta = float((nu ** 3 / eps) ** 0.25) if eps > 0 else float("inf")
    # integral scale: autocorrelation of u' averaged over the probes
    n = uu.shape[0]
    f = np.fft.rfft(uu - uu.mean(axis=0), n=2 * n, axis=0)
    ac = np.fft.irfft(np.abs(f) ** 2, axis=0)[:n].mean(axis=1)
    ac = ac / ac[0] if ac[0] > 0 else ac
    zero = np.argmax(ac <= 0.0) if np.any(ac <= 0.0) else n
    L = float(U * dt * (ac[:zero].sum() - 0.5 * ac[0]))
    urms = float(np.sqrt(u2))
    return {"U": U, "u_rms": urms, "v_rms": float(np.sqrt(0.5 * (v2 + w2))),
            "k": 0.5 * (u2 + v2 + w2), "anisotropy": float(np.sqrt(0.5 * (v2 + w2) / u2)) if u2 > 0 else 0.0,
            "lambda_f": lam_f, "lambda_g": lam_g, "eps": eps, "eta": eta,
            "re_lambda": urms * lam_g / nu, "L": L}


def decay_fit(x, k, x0, x_min, x_max=np.inf):
    """n and A of k = A (x - x0)^-n by least squares in log-log over
    x_min <= x <= x_max."""
    x = np.asarray(x, dtype=float)
    k = np.asarray(k, dtype=float)
    sel = (x >= x_min) & (x <= x_max) & (k > 0)
    slope, icpt = np.polyfit(np.log(x[sel] - x0), np.log(k[sel]), 1)
    return -slope, float(np.exp(icpt))


def analyse(t, series, x_st, per_station, nu, x0, x_max):
    out = []
    for s, x in enumerate(x_st):
        q = slice(s * per_station, (s + 1) * per_station)
        st = station_statistics(t, series[:, q, 0], series[:, q, 1], series[:, q, 2], nu)
        st["x"] = float(x)
        out.append(st)
    xs = np.array([o["x"] for o in out])
    ks = np.array([o["k"] for o in out])
    x_min = float(xs[int(np.argmax(ks))])
    n, A = decay_fit(xs, ks, x0, x_min, x_max)
    return {"stations": out, "decay_exponent": n, "decay_prefactor": A, "decay_range": [x_min, x_max]}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--re", type=float, default=None)
    ap.add_argument("--warmup", type=int, default=3000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--every", type=int, default=4)
    ap.add_argument("--out", default="grid_turbulence.json")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    wl = inputs.PRODUCTION.replace(flag_on=False)
    if a.re:
        wl = wl.replace(re=a.re)
    s = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl))
    cells, x_st = probe_cells(wl)
    t0 = time.perf_counter()
    t, series = record(s, cells, a.steps, a.every, a.warmup)
    wall = time.perf_counter() - t0
    s.close()
    res = analyse(t, series, x_st, 9, 1.0 / wl.re, wl.bar_x, wl.lx - 1.0)
    res.update({"re": wl.re, "probes": int(cells.shape[0]), "samples": int(len(t)), "t_span": float(t[-1] - t[0]),
                "seconds": wall})
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)
    short = [{k: round(v, 4) for k, v in st.items()} for st in res["stations"][::8]]
    print(json.dumps({"decay_exponent": res["decay_exponent"], "decay_range": res["decay_range"],
                      "stations": short}, indent=1))


if __name__ == "__main__":
    main()
