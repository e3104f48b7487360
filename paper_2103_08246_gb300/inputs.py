"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only describes workloads (grid sizes, domain, body parameters)
and draws the random numbers the method consumes (the initial velocity
perturbation). It holds none of the method's arithmetic, so that both sides
can take their inputs from one place without sharing any computation.

Workloads (all lengths in units of the flag length L = 1, velocities in units
of the inflow speed U = 1; Sec. II.A of the paper defines the geometry):

* ``tiny``        64x32x32 cells, domain 4x2x2, Re = 100, bar grid (mesh 0.5,
                  bar width 0.1) at x = 0.5, 1x1 flag hinged at x = 2 with
                  17x17 vertices, mass ratio 1, bending 0.01, dt = 2e-3.
* ``production``  512x256x256 cells, domain 8x4x4, Re = 200, same bar grid,
                  flag at x = 3 with 65x65 vertices, bending 0.005, CFL 0.3.

It also draws the inflow generator's initial weights (random numbers the
training consumes) and synthetic plane sequences for its tests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    re: float
    # passive bar grid (square rods along y and z in the plane x = bar_x)
    bars_on: bool = True
    bar_x: float = 0.5
    bar_mesh: float = 0.5
    bar_width: float = 0.1
    # "markers": delta-kernel markers filling the bars (the benchmark's
    # specification); "eulerian": volume-fraction direct forcing at the
    # Eulerian velocity nodes (the paper's treatment of the fixed grid)
    bar_forcing: str = "markers"
    # flexible flag hinged at its leading edge
    flag_on: bool = True
    flag_x_le: float = 2.0
    flag_len: float = 1.0
    flag_span: float = 1.0
    flag_ns: int = 17
    flag_nt: int = 17
    mass_ratio: float = 1.0
    bending: float = 0.01
    pitch0: float = 0.1 * math.pi
    stretch: float = 1000.0
    # time stepping: dt > 0 fixed, dt <= 0 means CFL-controlled
    dt: float = 2e-3
    cfl: float = 0.3
    steps: int = 100
    # initial perturbation U(-a, a) on interior faces
    noise_amp: float = 1e-3
    seed: int = 0

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


TINY = Workload(name="tiny-64x32x32", nx=64, ny=32, nz=32, lx=4.0, ly=2.0, lz=2.0,
                re=100.0, flag_x_le=2.0, flag_ns=17, flag_nt=17, bending=0.01,
                dt=2e-3, steps=100)

PRODUCTION = Workload(name="production-512x256x256", nx=512, ny=256, nz=256,
                      lx=8.0, ly=4.0, lz=4.0, re=200.0, flag_x_le=3.0,
                      flag_ns=65, flag_nt=65, bending=0.005, dt=-1.0, cfl=0.3,
                      steps=2000)


def small(nx=16, ny=8, nz=8, **kw) -> Workload:
    """A small case with the tiny workload's spacing rules (h = 1/4 by default)."""
    base = dict(name=f"small-{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz,
                lx=nx / 4.0, ly=ny / 4.0, lz=nz / 4.0, re=100.0,
                bars_on=False, flag_on=False, dt=2e-3, steps=10)
    base.update(kw)
    return Workload(**base)


def initial_noise(wl: Workload, seed: int | None = None, amp: float | None = None):
    """Uniform U(-a, a) perturbations for u, v, w, drawn from a seeded generator.

    Returns three float64 arrays of shape (nx+1, ny, nz) in x-slowest,
    z-fastest order. Entries that the method does not perturb (the inflow and
    outflow faces of u, the outflow ghost plane of v and w) are zero; the
    consumers rely on that and add the arrays as they are.
    """
    seed = wl.seed if seed is None else seed
    amp = wl.noise_amp if amp is None else amp
    rng = np.random.default_rng(seed)
    shape = (wl.nx + 1, wl.ny, wl.nz)
    out = []
    for comp in range(3):
        a = rng.uniform(-amp, amp, size=shape)
        if comp == 0:
            a[0] = 0.0
            a[wl.nx] = 0.0
        else:
            a[wl.nx] = 0.0
        out.append(a)
    return out


def random_field(shape, seed: int, lo=-1.0, hi=1.0):
    """A plain seeded uniform field (used by operator-level tests)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def ensemble_cases(n: int = 16, seed: int = 0):
    """Independent flag cases of uneven size (the batched-ensemble workload).

    Spacing h = 1/16 (17 x 17 flag vertices at the grid spacing); x from 64
    to 256 cells, y = z from {32, 64, 128} cells (power-of-two transverse
    sizes), domains scaled accordingly; bar grid (mesh 0.5, width 0.1) at
    x = 0.5; flag leading edge 1 to 4 bar meshes behind the grid; bending
    log-uniform in [1e-3, 1e-1]; Re uniform in [100, 400]; CFL 0.3.
    """
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        nyz = int(rng.choice([32, 64, 128]))
        nx = int(rng.integers(64, 257))
        h = 1.0 / 16.0
        dist = float(rng.uniform(1.0, 4.0))
        out.append(Workload(
            name=f"ensemble-{q}-{nx}x{nyz}x{nyz}", nx=nx, ny=nyz, nz=nyz,
            lx=nx * h, ly=nyz * h, lz=nyz * h, re=float(rng.uniform(100.0, 400.0)),
            flag_x_le=0.5 + 0.5 * dist, flag_ns=17, flag_nt=17,
            bending=float(10.0 ** rng.uniform(-3.0, -1.0)), dt=-1.0, cfl=0.3,
            steps=100, seed=seed + q))
    return out


def generator_param_count(width: int = 128, blocks: int = 13, in_channels: int = 6) -> int:
    """Parameters of the inflow generator: W_in, b_in, blocks x (W, b), W_out, b_out."""
    return 9 * width * in_channels + width + blocks * (9 * width * width + width) + 9 * 3 * width + 3


def generator_params(seed: int = 0, width: int = 128, blocks: int = 13, in_channels: int = 6,
                     block_scale: float = 0.1, out_scale: float = 0.1, bias_std: float = 0.0):
    """Seeded initial weights of the inflow generator, flat in the interface
    order (W_in, b_in, then W_l, b_l per block, then W_out, b_out; every W in
    [dy + 1][dz + 1][out][in] order). Weights are normal with standard
    deviation sqrt(2 / (9 in)) (He), scaled by ``block_scale`` in the residual
    blocks (an untrained network is close to h -> h) and by ``out_scale`` in
    the output layer; biases normal with ``bias_std`` (zero by default)."""
    rng = np.random.default_rng(seed)

    def he(o, c, scale):
        return (rng.standard_normal((3, 3, o, c)) * scale * np.sqrt(2.0 / (9 * c))).ravel()

    def bias(n):
        return rng.standard_normal(n) * bias_std if bias_std > 0 else np.zeros(n)
    parts = [he(width, in_channels, 1.0), bias(width)]
    for _ in range(blocks):
        parts += [he(width, width, block_scale), bias(width)]
    parts += [he(3, width, out_scale), bias(3)]
    out = np.concatenate(parts)
    assert out.size == generator_param_count(width, blocks, in_channels)
    return out


def advected_planes(n: int, ny: int, nz: int, seed: int = 0, shift: int = 1, modes: int = 3,
                    mean=(1.0, 0.0, 0.0), amp=(0.1, 0.05, 0.05)):
    """n planes [n, 3, ny, nz] of a smooth periodic random field carried
    ``shift`` cells in z per plane (frozen turbulence passing a fixed plane):
    plane t is f(y, z - shift t). f is a sum of random Fourier modes with
    wavenumbers below ``modes``, scaled per component to rms ``amp`` around
    ``mean``."""
    rng = np.random.default_rng(seed)
    y = np.arange(ny)[:, None]
    out = np.empty((n, 3, ny, nz))
    for c in range(3):
        coef = []
        for ky in range(-modes + 1, modes):
            for kz in range(0, modes):
                if ky == 0 and kz == 0:
                    continue
                coef.append((ky, kz, rng.standard_normal(), rng.uniform(0, 2 * np.pi)))
        for t in range(n):
            z = (np.arange(nz)[None, :] - shift * t)
            f = np.zeros((ny, nz))
            for ky, kz, a, ph in coef:
                f += a * np.cos(2 * np.pi * (ky * y / ny + kz * z / nz) + ph)
            out[t, c] = f
        rms = np.sqrt((out[:, c] ** 2).mean())
        out[:, c] = mean[c] + amp[c] * out[:, c] / rms
    return out
