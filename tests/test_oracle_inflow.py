"""Pins for the oracle's prescribed (time-dependent) inflow.

* A uniform oblique flow (U, V0, W0) entering through matching inflow planes
  is an exact steady solution on the periodic channel: it must stay uniform
  to round-off (this fixes the ghost q_-1 = 2 q_in - q_0; a ghost that
  reflects without the inflow value, or adds it once, breaks it at once).
* Random time-dependent inflow planes: the inflow face is shifted to mean U,
  so Q_in = U Ly Lz exactly, the mass fix makes Q_out = Q_in, and the
  projected field is divergence-free to round-off every step.
* A uniform inflow plane equal to (U, 0, 0) reproduces the run without a
  prescribed inflow bit for bit.
"""
import numpy as np

from oracle import mac
from oracle.solver import OracleSolver
from paper_2103_08246_gb300 import inputs


def _wl(**kw):
    return inputs.small(12, 8, 8, **kw)


def test_uniform_oblique_inflow_is_steady():
    wl = _wl()
    V0, W0 = 0.3, -0.2
    shape = (wl.nx + 1, wl.ny, wl.nz)
    noise = (np.zeros(shape), np.full(shape, V0), np.full(shape, W0))
    s = OracleSolver(wl, noise=noise)
    s.v_in[:], s.w_in[:] = V0, W0      # the inflow at t = 0 matches the initial field
    s.set_inflow(np.ones((wl.ny, wl.nz)), np.full((wl.ny, wl.nz), V0), np.full((wl.ny, wl.nz), W0))
    s.run(15)
    assert np.abs(s.u - 1.0).max() < 1e-12
    assert np.abs(s.v - V0).max() < 1e-12
    assert np.abs(s.w - W0).max() < 1e-12
    assert np.abs(s.p - s.p.mean()).max() < 1e-10


def test_time_dependent_inflow_keeps_mass():
    wl = _wl()
    rng = np.random.default_rng(4)
    s = OracleSolver(wl, noise=inputs.initial_noise(wl, amp=0.05))
    h = s.h
    for step in range(6):
        pu = 1.0 + 0.1 * rng.standard_normal((wl.ny, wl.nz)) + 0.37   # mean is not U
        pv = 0.05 * rng.standard_normal((wl.ny, wl.nz))
        pw = 0.05 * rng.standard_normal((wl.ny, wl.nz))
        s.set_inflow(pu, pv, pw)
        s.step()
        q_in = s.u[0].sum() * h * h
        q_out = s.u[wl.nx].sum() * h * h
        assert abs(q_in - wl.ly * wl.lz) < 1e-12
        assert abs(q_out - q_in) < 1e-12
        np.testing.assert_allclose(s.u[0], pu - pu.mean() + 1.0, rtol=0, atol=1e-15)
        div = mac.divergence(s.u, s.v, s.w, h)
        assert np.abs(div).max() * h < 1e-11


def test_default_inflow_plane_reproduces_plain_run():
    wl = _wl(bars_on=True, bar_x=1.0)
    noise = inputs.initial_noise(wl, amp=0.05)
    a = OracleSolver(wl, noise=noise)
    b = OracleSolver(wl, noise=noise)
    b.set_inflow(np.ones((wl.ny, wl.nz)), np.zeros((wl.ny, wl.nz)), np.zeros((wl.ny, wl.nz)))
    a.run(5)
    b.run(5)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
