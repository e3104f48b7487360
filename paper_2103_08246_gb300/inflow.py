"""Learned inflow campaign: precursor record, generator training, driven runs
and their statistics.

Sec. V of the paper leaves open how a flag behaves when the grid-resolved
inflow turbulence (bars inside the domain, Sec. II.A) is replaced by a
synthetic one. This module runs that comparison with the solver and the
learned generator of the C ABI (``ibm_gen_*``):

1. precursor: the production workload without the flag; after a spin-up
   (3000 steps, about 5 time units, while the bar wakes reach x = 2 after
   about 1.5), that
   plane (u on the face, v, w on the cell centres) is recorded every step
   (device planes, FP32);
2. training: the generator learns keyframe steps q_{t+s} - q_t from
   (q_t, q_{t-s}), s = 10 recorded planes, on the first 90% of the record (Adam, cosine learning-rate decay; Gaussian
   noise on the inputs with the target taken from the noisy q_t, so that
   the rollout is pulled back towards the data), the last 10% is held out;
3. runs with the flag, each for the same number of steps:
   R  grid-resolved: the production workload (bars at 0.5, flag at 3);
   G  generated inflow: a 384 x 256 x 256 domain of length 6 without bars,
      flag at 1, inflow planes from the generator rollout: a keyframe every
      s steps (seeded with the last two recorded keyframes, relaxed towards
      the record's time-mean plane at 1% per keyframe), the planes in
      between interpolated linearly in time;
   U  uniform inflow on the same domain;
   W  white-noise inflow on the same domain: independent Gaussian planes
      with the record's per-component rms (matched turbulence intensity);
   the driven domain starts 2 length units downstream of R's (its inflow
   is R's plane x = 2), so station x in G, U, W is station x + 2 in R;
4. statistics: turbulence intensity at three stations upstream of the flag
   and its decay exponent (Tu^2 ~ (x - x0)^-n, x0 the bar grid, Sec. III),
   the one-dimensional spectrum of u' across z at the station ahead of the
   flag (Sec. III), and the flag's trailing-edge Strouhal number and rms
   displacement (Sec. IV).

Bounds on G against R are fixed before training (``BOUNDS``), and G is also
scored against U and W.

The statistics are host-side post-processing (numpy) of sampled planes and
diagnostics; every step of the solver and the generator runs in the
library's kernels.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding, inputs

# stations of the driven domain (length units; ahead of its flag at 1) and
# the offset of the driven domain inside R's
STATIONS_X = (0.03, 0.5, 0.89)
SHIFT_X = 2.0

# fixed before training (relative unless stated)
BOUNDS = {
    "tu_flag_station": 0.25,            # |Tu_G - Tu_R| / Tu_R at the station ahead of the flag
    "decay_exponent_abs": 0.5,          # |n_G - n_R|
    "spectrum_log10_mean_abs": 0.3,     # mean |log10 E_G - log10 E_R| over kappa index 1..32
    "strouhal": 0.15,                   # |St_G - St_R| / St_R
    "y_rms": 0.30,                      # |Y_G - Y_R| / Y_R
}


def shift_cells(base: inputs.Workload) -> int:
    return int(round(SHIFT_X * base.nx / base.lx))


def driven_workload(base: inputs.Workload = inputs.PRODUCTION) -> inputs.Workload:
    """The generated-inflow domain: R's domain without its first 2 length
    units and without bars (384 x 256 x 256, length 6, flag at x = 1 for the
    production workload)."""
    h = base.lx / base.nx
    nx = base.nx - shift_cells(base)
    return base.replace(name=f"driven-{nx}x{base.ny}x{base.nz}", nx=nx, lx=nx * h, bars_on=False,
                        flag_x_le=base.flag_x_le - shift_cells(base) * h)


class _DevArray:
    """Zero-copy view of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def device_planes(ptrs, ny, nz, fp64=False):
    import torch
    ts = "<f8" if fp64 else "<f4"
    return [torch.as_tensor(_DevArray(p, (ny, nz), ts), device="cuda") for p in ptrs]


def record_planes(solver, i_plane, n, spin=0):
    """Step the solver `spin` steps, then n steps recording plane i (u, v, w)
    after each into a device tensor [n, 3, ny, nz] (FP32)."""
    import torch
    wl = solver.wl
    if spin:
        solver.step(spin, dt=-1.0)
    rec = torch.empty((n, 3, wl.ny, wl.nz), dtype=torch.float32, device="cuda")
    fp64 = solver.precision == binding.IBM_FP64
    with torch.cuda.stream(solver.stream):
        for k in range(n):
            solver.step(1, dt=-1.0)
            views = device_planes(binding.ibm_plane_device(solver.state, i_plane), wl.ny, wl.nz, fp64)
            for c in range(3):
                rec[k, c].copy_(views[c])
    solver.stream.synchronize()
    return rec


def data_norm(planes, sample=256, seed=0):
    """Per-component mean and std of a record, the rms of the normalised
    planes with their plane mean removed (the rollout's target rms), and the
    time-mean plane [3, ny, nz] (the rollout's relaxation reference)."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(planes.shape[0], min(sample, planes.shape[0]), replace=False))
    a = planes[idx].double().cpu().numpy()
    mean = a.mean(axis=(0, 2, 3))
    std = a.std(axis=(0, 2, 3))
    q = (a - mean[None, :, None, None]) / std[None, :, None, None]
    q = q - q.mean(axis=(2, 3), keepdims=True)
    rms = np.sqrt((q ** 2).mean(axis=(0, 2, 3)))
    return mean, std, rms, a.mean(axis=0)


def data_spectrum(planes, std, mean_plane, sample=512, seed=2):
    """Mean 2-D Fourier power |FFT2(f)|^2 (unnormalised transform) of the
    recorded planes' fluctuation about the time-mean plane, in the
    generator's normalised units: the target of the rollout's spectral
    relaxation, [3, ny, nz]."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(planes.shape[0], min(sample, planes.shape[0]), replace=False))
    acc = np.zeros(mean_plane.shape)
    for i in idx:
        f = (planes[i].double().cpu().numpy() - mean_plane) / std[:, None, None]
        acc += np.abs(np.fft.fft2(f, axes=(1, 2))) ** 2
    return acc / len(idx)


def train(gen, planes, steps, lr0=5e-4, lr1=2e-5, train_frac=0.9, seed=0, log_every=100, pushforward=0.0):
    """Adam with cosine decay from lr0 to lr1; returns the loss history.
    Samples are keyframe triples (t - s, t, t + s), s = gen.stride. In the
    second half of the steps a fraction `pushforward` of them are pushforward
    steps (the input q_t replaced by the network's own prediction from
    (q_{t-s}, q_{t-2s}))."""
    n = planes.shape[0]
    s_ = gen.stride
    n_train = int(n * train_frac)
    rng = np.random.default_rng(seed)
    val_idx = np.arange(n_train + s_, n - s_)
    hist = {"step": [], "train": [], "val": []}
    t0 = time.perf_counter()
    for s in range(steps):
        lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + np.cos(np.pi * s / max(steps - 1, 1)))
        gen.set_lr(lr)
        log = (s % log_every == 0) or s == steps - 1
        if pushforward > 0 and 2 * s >= steps and rng.random() < pushforward:
            idx = rng.integers(2 * s_, n_train - s_, size=gen.batch)
            loss = gen.train_step_pushforward(planes, idx, with_loss=log)
        else:
            idx = rng.integers(s_, n_train - s_, size=gen.batch)
            loss = gen.train_step(planes, idx, with_loss=log)
        if log:
            vb = rng.choice(val_idx, size=gen.batch, replace=len(val_idx) < gen.batch)
            hist["step"].append(s)
            hist["train"].append(loss)
            hist["val"].append(gen.eval(planes, vb))
    gen.sync()
    hist["seconds"] = time.perf_counter() - t0
    return hist


def baselines(planes, mean, std, n_train, stride=1, count=64, seed=1):
    """Validation losses of two predictors without parameters, in the
    training loss's units: persistence (delta = 0) and linear extrapolation
    (delta = q_t - q_{t-s})."""
    rng = np.random.default_rng(seed)
    n = planes.shape[0]
    idx = rng.integers(n_train + stride, n - stride, size=count)
    s = std[:, None, None]
    m = mean[:, None, None]
    pers, lin = 0.0, 0.0
    for t in idx:
        q = [(planes[k].double().cpu().numpy() - m) / s for k in (t - stride, t, t + stride)]
        d = q[2] - q[1]
        pers += float(np.mean(d * d))
        e = d - (q[1] - q[0])
        lin += float(np.mean(e * e))
    return {"persistence": pers / count, "linear_extrapolation": lin / count}


def rollout_diagnostics(gen, planes, checkpoints=(1, 10, 100, 300, 800)):
    """Generator alone, seeded with the last two recorded keyframes: the u
    spectrum across z, the component rms and the correlation of u' with the
    seed plane after the given numbers of keyframes, and the record's mean u
    spectrum."""
    import torch
    ny, nz = planes.shape[2], planes.shape[3]
    gen.rollout_init(planes[-1 - gen.stride].cpu().numpy(), planes[-1].cpu().numpy())
    out = [torch.zeros((ny, nz), dtype=torch.float32, device="cuda") for _ in range(3)]
    torch.cuda.synchronize()
    seed_u = planes[-1, 0].double().cpu().numpy()
    seed_u = seed_u - seed_u.mean()
    res = {"step": [], "spectrum_u": [], "rms": [], "corr_seed_u": []}
    last = max(checkpoints)
    for k in range(1, last + 1):
        gen.rollout(*[o.data_ptr() for o in out], precision=binding.IBM_FP32)
        if k in checkpoints:
            gen.sync()
            a = [o.double().cpu().numpy() for o in out]
            u = a[0] - a[0].mean()
            res["step"].append(k)
            res["spectrum_u"].append(spectrum_z(a[0]).tolist())
            res["rms"].append([float(np.sqrt(np.mean((x - x.mean()) ** 2))) for x in a])
            res["corr_seed_u"].append(float(np.sum(u * seed_u) / np.sqrt(np.sum(u * u) * np.sum(seed_u * seed_u))))
    idx = np.linspace(0, planes.shape[0] - 1, 32).astype(int)
    res["data_spectrum_u"] = np.mean([spectrum_z(planes[i, 0].double().cpu().numpy()) for i in idx], axis=0).tolist()
    return res


# ------------------------------------------------------------- statistics
def spectrum_z(plane):
    """One-sided spectrum of a plane's fluctuation along z, averaged over y:
    E[k] for k = 0 .. nz/2, normalised so that sum(E) = mean(plane'^2)."""
    a = plane - plane.mean()
    nz = a.shape[-1]
    f = np.fft.rfft(a, axis=-1) / nz
    e = (np.abs(f) ** 2).mean(axis=0)
    e[1:(nz + 1) // 2] *= 2.0
    return e


def decay_exponent(x, tu2, x0):
    """n of Tu^2 = A (x - x0)^-n by least squares in log-log."""
    X = np.log(np.asarray(x, dtype=float) - x0)
    Y = np.log(np.asarray(tu2, dtype=float))
    slope, _ = np.polyfit(X, Y, 1)
    return -slope


def strouhal(t, y, length=1.0, speed=1.0):
    """Dominant frequency of a signal sampled at (possibly uneven) times t,
    as St = f L / U, and its rms about the mean: resampled uniformly,
    Hann-windowed, peak of the periodogram refined by a parabola."""
    t = np.asarray(t, dtype=float)
    y = np.asarray(y, dtype=float)
    n = len(t)
    tu = np.linspace(t[0], t[-1], n)
    yu = np.interp(tu, t, y)
    yu = yu - yu.mean()
    w = np.hanning(n)
    p = np.abs(np.fft.rfft(yu * w)) ** 2
    p[0] = 0.0
    k = int(np.argmax(p))
    if 0 < k < len(p) - 1:
        a, b, c = np.log(p[k - 1] + 1e-300), np.log(p[k] + 1e-300), np.log(p[k + 1] + 1e-300)
        den = a - 2 * b + c
        k = k + (0.5 * (a - c) / den if den != 0 else 0.0)
    dt = (tu[-1] - tu[0]) / (n - 1)
    f = k / (n * dt)
    return f * length / speed, float(np.sqrt(np.mean((y - y.mean()) ** 2)))


class StationStats:
    """Running per-station sums of sampled planes: component means and
    variances about the time-and-plane mean, and the u' spectrum along z."""

    def __init__(self, n_st, nz):
        self.n = 0
        self.s1 = np.zeros((n_st, 3))
        self.s2 = np.zeros((n_st, 3))
        self.spec = np.zeros((n_st, nz // 2 + 1))

    def add(self, planes):
        for k, (u, v, w) in enumerate(planes):
            for c, a in enumerate((u, v, w)):
                self.s1[k, c] += a.mean()
                self.s2[k, c] += (a * a).mean()
            self.spec[k] += spectrum_z(u)
        self.n += 1

    def tu(self, speed=1.0):
        m = self.s1 / self.n
        var = np.maximum(self.s2 / self.n - m * m, 0.0)
        return np.sqrt(var.mean(axis=1)) / speed

    def spectra(self):
        return self.spec / self.n


def run_flag(solver, steps, discard, stations, sample_every=10, flag_every=2, before_step=None):
    """Run with the flag; sample station planes (host) every `sample_every`
    steps and the trailing-edge midpoint every `flag_every` steps after
    `discard` steps. `before_step` (if given) is called before every step."""
    wl = solver.wl
    st = StationStats(len(stations), wl.nz)
    t_te, te = [], []
    t0 = time.perf_counter()
    for k in range(steps):
        if before_step is not None:
            before_step(k)
        solver.step(1, dt=-1.0)
        if k >= discard and (k - discard) % flag_every == 0:
            s = solver.stats()
            t_te.append(s["t"])
            te.append(list(s["te_mid"]))
        if k >= discard and (k - discard) % sample_every == 0:
            st.add([solver.plane(i) for i in stations])
    wall = time.perf_counter() - t0
    te = np.asarray(te)
    # flapping direction: the transverse component that moves most
    comp = 1 + int(np.argmax(te[:, 1:].std(axis=0)))
    St, y_rms = strouhal(t_te, te[:, comp], wl.flag_len, 1.0)
    return {"tu": st.tu().tolist(), "spectrum_u": st.spectra()[-1].tolist(), "strouhal": St,
            "y_rms": y_rms, "flap_component": comp, "samples": st.n, "flag_samples": len(t_te),
            "steps": steps, "discard": discard, "seconds": wall, "t_end": float(t_te[-1])}


def compare(res, x_st, x0):
    """Errors of G, U, W against R, and the bounds' verdicts for G."""
    R = res["R"]
    n_R = decay_exponent(x_st, np.square(R["tu"]), x0)
    out = {"n_R": n_R}
    kk = slice(1, 33)
    for key in ("G", "U", "W"):
        if key not in res:
            continue
        r = res[key]
        e = {"tu_flag_station": abs(r["tu"][-1] - R["tu"][-1]) / R["tu"][-1]}
        tu2 = np.square(r["tu"])
        if np.all(tu2 > 0):
            n = decay_exponent(x_st, tu2, x0)
            e["decay_exponent"] = n
            e["decay_exponent_abs"] = abs(n - n_R)
        ER, E = np.asarray(R["spectrum_u"])[kk], np.asarray(r["spectrum_u"])[kk]
        if np.all(E > 0):
            e["spectrum_log10_mean_abs"] = float(np.mean(np.abs(np.log10(E) - np.log10(ER))))
        e["strouhal"] = abs(r["strouhal"] - R["strouhal"]) / R["strouhal"]
        e["y_rms"] = abs(r["y_rms"] - R["y_rms"]) / R["y_rms"]
        out[key] = e
    if "G" in out:
        out["G_within_bounds"] = {k: (out["G"].get(k, np.inf) <= b) for k, b in BOUNDS.items()}
        gains = {}
        for k in ("tu_flag_station", "spectrum_log10_mean_abs", "y_rms", "strouhal"):
            for other in ("U", "W"):
                if other in out and k in out[other] and k in out["G"]:
                    gains[f"{k}_vs_{other}"] = bool(out["G"][k] < out[other][k])
        out["G_better_than"] = gains
    return out


def campaign(spin=3000, record=4000, train_steps=1500, run_steps=8000, discard=3000, blocks=13, batch=8,
             precision=binding.IBM_FP32, seed=0, log=print, base=inputs.PRODUCTION, sample_every=10,
             re=None, noise=0.03, stride=10, relax=0.01, spectral=0.0, pushforward=0.0):
    import torch
    prod = base if re is None else base.replace(re=float(re))
    out = {"bounds": BOUNDS, "workload": base.name, "re": prod.re, "train_noise": noise, "stride": stride,
           "relax": relax, "spectral": spectral, "pushforward": pushforward}
    h = prod.lx / prod.nx
    R_SHIFT = shift_cells(prod)
    i_rec = R_SHIFT
    # 1. precursor
    pre = binding.Solver(prod.replace(flag_on=False), precision, noise=inputs.initial_noise(prod))
    t0 = time.perf_counter()
    planes = record_planes(pre, i_rec, record, spin)
    out["precursor"] = {"spin": spin, "record": record, "plane_x": i_rec * h,
                        "seconds": time.perf_counter() - t0, "t_end": pre.stats()["t"]}
    pre.close()
    mean, std, rms, mean_plane = data_norm(planes)
    out["data"] = {"mean": mean.tolist(), "std": std.tolist(), "rms_normalised": rms.tolist()}
    log(f"precursor: {out['precursor']}, data {out['data']}")
    # 2. training
    gen = binding.Generator(prod.ny, prod.nz, blocks=blocks, in_channels=6, batch=batch, stride=stride)
    gen.set_params(inputs.generator_params(seed, 128, blocks, 6))
    gen.set_norm(mean, std, rms)
    gen.set_noise(noise, seed=seed + 17)
    out["train"] = train(gen, planes, train_steps, seed=seed, pushforward=pushforward)
    out["train"]["n_params"] = gen.n_params
    out["train"]["baselines"] = baselines(planes, mean, std, int(planes.shape[0] * 0.9), stride)
    power = data_spectrum(planes, std, mean_plane) if spectral > 0 else None
    diag_gen = binding.Generator(prod.ny, prod.nz, blocks=blocks, in_channels=6, batch=1, stride=stride)
    diag_gen.set_params(gen.params())
    diag_gen.set_norm(mean, std, rms)
    diag_gen.set_relax(mean_plane, relax)
    if power is not None:
        diag_gen.set_spectrum(power, spectral)
    out["rollout"] = rollout_diagnostics(diag_gen, planes,
                                         tuple(k for k in (1, 10, 100, 300, 800) if k * stride <= max(run_steps, 1)))
    diag_gen.close()
    log(f"training: final train {out['train']['train'][-1]:.4g} val {out['train']['val'][-1]:.4g} "
        f"in {out['train']['seconds']:.1f} s")
    seed_prev = planes[-1 - stride].clone()
    seed_cur = planes[-1].clone()
    del planes
    torch.cuda.empty_cache()
    # 3. runs
    drv = driven_workload(prod)
    st_d = [max(1, int(round(x / h))) for x in STATIONS_X]
    st_r = [i + R_SHIFT for i in st_d]
    res = {}
    s = binding.Solver(prod, precision, noise=inputs.initial_noise(prod))
    res["R"] = run_flag(s, run_steps, discard, st_r, sample_every)
    s.close()
    log(f"R: {res['R']['tu']} St {res['R']['strouhal']:.3f} Y {res['R']['y_rms']:.3f}")
    s = binding.Solver(drv, precision, noise=inputs.initial_noise(drv), inflow=True)
    # the generator shares the solver's stream: rollout k is ordered before step k
    gen_run = binding.Generator(prod.ny, prod.nz, blocks=blocks, in_channels=6, batch=1, stream=s.stream,
                                stride=stride)
    gen_run.set_params(gen.params())
    gen_run.set_norm(mean, std, rms)
    gen_run.set_relax(mean_plane, relax)
    if power is not None:
        gen_run.set_spectrum(power, spectral)
    gen.close()
    gen_run.rollout_init(seed_prev.cpu().numpy(), seed_cur.cpu().numpy())
    ptrs = binding.ibm_inflow_planes(s.state)
    fp64 = precision == binding.IBM_FP64
    def generated(k):
        # a keyframe every `stride` steps, planes in between interpolated in time
        if k % stride == 0:
            gen_run.rollout(None, None, None, precision=precision)
        gen_run.emit((k % stride) / stride, *ptrs, precision=precision)
    res["G"] = run_flag(s, run_steps, discard, st_d, sample_every, before_step=generated)
    s.close()
    gen_run.close()
    log(f"G: {res['G']['tu']} St {res['G']['strouhal']:.3f} Y {res['G']['y_rms']:.3f}")
    s = binding.Solver(drv, precision, noise=inputs.initial_noise(drv))
    res["U"] = run_flag(s, run_steps, discard, st_d, sample_every)
    s.close()
    log(f"U: {res['U']['tu']} St {res['U']['strouhal']:.3f} Y {res['U']['y_rms']:.3f}")
    s = binding.Solver(drv, precision, noise=inputs.initial_noise(drv), inflow=True)
    rng = np.random.default_rng(seed + 1)
    pool = []
    for _ in range(64):
        pl = mean[:, None, None] + (std * rms)[:, None, None] * rng.standard_normal((3, drv.ny, drv.nz))
        pool.append(torch.as_tensor(pl, dtype=torch.float64 if fp64 else torch.float32, device="cuda"))
    torch.cuda.synchronize()
    views = device_planes(binding.ibm_inflow_planes(s.state), drv.ny, drv.nz, fp64)

    def white(k):
        src = pool[int(rng.integers(len(pool)))]
        with torch.cuda.stream(s.stream):
            for c in range(3):
                views[c].copy_(src[c])
    res["W"] = run_flag(s, run_steps, discard, st_d, sample_every, before_step=white)
    s.close()
    log(f"W: {res['W']['tu']} St {res['W']['strouhal']:.3f} Y {res['W']['y_rms']:.3f}")
    out["runs"] = res
    x_st = [(i + R_SHIFT) * h for i in st_d]
    out["stations_x_R"] = x_st
    out["comparison"] = compare(res, x_st, prod.bar_x)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--spin", type=int, default=3000)
    ap.add_argument("--record", type=int, default=4000)
    ap.add_argument("--train-steps", type=int, default=1500)
    ap.add_argument("--run-steps", type=int, default=8000)
    ap.add_argument("--discard", type=int, default=3000)
    ap.add_argument("--blocks", type=int, default=13)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--re", type=float, default=None, help="Reynolds number of every run (default: the workload's)")
    ap.add_argument("--noise", type=float, default=0.03, help="training-input noise, normalised units")
    ap.add_argument("--stride", type=int, default=10, help="solver steps between generated keyframes")
    ap.add_argument("--relax", type=float, default=0.01,
                    help="rollout relaxation rate per keyframe towards the record's time-mean plane")
    ap.add_argument("--spectral", type=float, default=0.0,
                    help="rollout spectral relaxation exponent per keyframe towards the record's power spectrum")
    ap.add_argument("--pushforward", type=float, default=0.0,
                    help="fraction of pushforward steps in the second half of the training")
    ap.add_argument("--out", default="inflow_campaign.json")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    res = campaign(a.spin, a.record, a.train_steps, a.run_steps, a.discard, a.blocks, a.batch, re=a.re,
                   noise=a.noise, stride=a.stride, relax=a.relax, spectral=a.spectral,
                   pushforward=a.pushforward)
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1, default=lambda o: o.tolist() if hasattr(o, "tolist") else str(o))
    print(json.dumps(res["comparison"], indent=1, default=str))


if __name__ == "__main__":
    main()
