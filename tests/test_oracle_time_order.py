"""Temporal order of the oracle's time step (Sec. II.B: AB2 for the explicit
terms, Crank-Nicolson for diffusion, fractional-step projection), without a
closed-form solution: a smooth, x-localised perturbation of the uniform inflow
on a 32 x 8 x 8 grid (h = 1/4, Re 100), run to T = 0.32 at successive halvings
of the step and compared with a run at a much smaller step.

* velocity: errors fall by ~4 per halving (second order) on a non-uniform
  step sequence (2/3 and 4/3 of the nominal step, alternating), which pins
  the variable-step AB2 weights alpha = 1 + dt/(2 dt_old),
  beta = -dt/(2 dt_old): with the constant weights 3/2, -1/2 planted instead
  (on the CPU, by resetting dt_old before each step) the ratio drops to ~2.6;
* pressure: the scheme's pressure belongs to the half step; compared with the
  reference interpolated to T - dt/2 its errors also fall by ~4 per halving.

The perturbation starts six length units upstream of the outflow, where the
first-order convective outflow condition would otherwise limit the order.
"""
import numpy as np

from oracle.solver import OracleSolver
from paper_2103_08246_gb300 import inputs

T = 0.32


def _initial(nx=32, ny=8, nz=8, amp=0.1):
    wl = inputs.small(nx, ny, nz)
    h = wl.lx / nx
    xf = np.arange(nx + 1) * h
    xc = (np.arange(nx + 1) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h
    zc = (np.arange(nz) + 0.5) * h
    g = lambda x: np.exp(-((x - 2.0) / 0.5) ** 2)
    cy, cz = np.cos(2 * np.pi * yc / wl.ly), np.cos(2 * np.pi * zc / wl.lz)
    sy, sz = np.sin(2 * np.pi * yc / wl.ly), np.sin(2 * np.pi * zc / wl.lz)
    u = 0.5 * amp * g(xf)[:, None, None] * cy[None, :, None] * cz[None, None, :]
    v = amp * g(xc)[:, None, None] * np.ones(ny)[None, :, None] * sz[None, None, :]
    w = amp * g(xc)[:, None, None] * sy[None, :, None] * np.ones(nz)[None, None, :]
    u[0] = 0.0
    u[nx] = 0.0
    v[nx] = 0.0
    w[nx] = 0.0
    return wl, [u, v, w]


def _run_variable(dt, constant_weights=False):
    wl, noise = _initial()
    s = OracleSolver(wl, noise)
    t, i = 0.0, 0
    while t < T - 1e-12:
        d = dt * (2.0 / 3.0 if i % 2 == 0 else 4.0 / 3.0)
        if constant_weights and s.n_prev is not None:
            s.dt_old = d            # planted mistake: AB2 weights as for a constant step
        s.step(d)
        t += d
        i += 1
    return s.v.copy()


def _velocity_ratios(constant_weights=False):
    ref = _run_variable(0.0025, constant_weights)
    err = [np.abs(_run_variable(dt, constant_weights) - ref).max() for dt in (0.04, 0.02, 0.01)]
    return [err[0] / err[1], err[1] / err[2]]


def test_velocity_second_order_with_variable_steps():
    r = _velocity_ratios()
    assert all(3.5 < x < 5.0 for x in r), r


def test_constant_ab2_weights_are_detected():
    r = _velocity_ratios(constant_weights=True)
    assert all(x < 3.0 for x in r), r


def test_pressure_second_order_at_the_half_step():
    def history(dt, n):
        wl, noise = _initial()
        s = OracleSolver(wl, noise)
        out = []
        for _ in range(n):
            s.step(dt)
            out.append(s.p - s.p.mean())
        return out

    dtr = 0.00125
    ref = history(dtr, int(round(T / dtr)))

    def ref_at(t):
        x = t / dtr + 0.5              # ref[k - 1] holds the pressure at (k - 1/2) dtr
        k = int(np.floor(x))
        f = x - k
        return (1 - f) * ref[k - 1] + f * ref[k]

    err = []
    for dt in (0.04, 0.02, 0.01):
        p = history(dt, int(round(T / dt)))[-1]
        err.append(np.abs(p - ref_at(T - dt / 2)).max())
    r = [err[0] / err[1], err[1] / err[2]]
    assert all(3.5 < x < 5.0 for x in r), r
