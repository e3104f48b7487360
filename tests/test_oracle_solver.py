"""Pins for the oracle's full time step (Sec. II.B order; Sec. II.A boundary
conditions).

* uniform inflow with no bodies stays exactly (U, 0, 0) with p = 0;
* after the mass fix the Poisson right-hand side sums to zero (compatibility
  of the Neumann problem) and the projected velocity is divergence-free to
  round-off;
* the discrete problem is symmetric under z -> Lz - z (bars and flag
  present), y -> Ly - y (bars present) and the y <-> z exchange (no bodies):
  stepping a mirrored initial field gives the mirrored result. A wrong sign
  or a shifted index in any y or z operator breaks one of these;
* the CFL time step follows its definition.
"""
import math

import numpy as np

from oracle import mac
from oracle.solver import OracleSolver
from paper_2103_08246_gb300 import inputs


def _wl(**kw):
    base = dict(bars_on=False, flag_on=False)
    base.update(kw)
    return inputs.small(16, 8, 8, **base)


def test_uniform_flow_is_preserved():
    s = OracleSolver(_wl())
    s.run(20)
    assert np.abs(s.u - 1.0).max() < 1e-13
    assert np.abs(s.v).max() < 1e-13 and np.abs(s.w).max() < 1e-13
    assert np.abs(s.p).max() < 1e-11


def test_mass_compatibility_and_divergence():
    wl = _wl(bars_on=True, bar_x=1.0, flag_on=True, flag_x_le=2.0, flag_ns=5, flag_nt=5,
             flag_len=1.0, flag_span=1.0)
    s = OracleSolver(wl, inputs.initial_noise(wl, amp=0.05))
    for _ in range(5):
        s.step()
        D = s.last_D
        assert abs(D.sum()) <= 1e-12 * np.abs(D).sum()
        div = mac.divergence(s.u, s.v, s.w, s.h)
        assert np.abs(div).max() <= 1e-12 * max(1.0, np.abs(D).max())
        q_in = s.u[0].sum()
        q_out = s.u[wl.nx].sum()
        assert abs(q_in - q_out) < 1e-12 * abs(q_in)


def _mirror_z(u, v, w, p):
    nz = u.shape[2]
    k_c = (nz - 1 - np.arange(nz))          # cell-centred z index
    k_f = (-np.arange(nz)) % nz             # z-face index
    return u[:, :, k_c], v[:, :, k_c], -w[:, :, k_f], p[:, :, k_c]


def _mirror_y(u, v, w, p):
    ny = u.shape[1]
    j_c = (ny - 1 - np.arange(ny))
    j_f = (-np.arange(ny)) % ny
    return u[:, j_c], -v[:, j_f], w[:, j_c], p[:, j_c]


def _swap_yz(u, v, w, p):
    t = lambda a: np.swapaxes(a, 1, 2)
    return t(u), t(w), t(v), t(p)


def _check_equivariance(wl, op, nsteps=6, flag_perm=None):
    noise = inputs.initial_noise(wl, amp=0.05)
    zero_p = np.zeros((wl.nx, wl.ny, wl.nz))
    mn = op(noise[0], noise[1], noise[2], zero_p)[:3]
    a = OracleSolver(wl, noise)
    b = OracleSolver(wl, list(mn))
    a.run(nsteps)
    b.run(nsteps)
    fa = op(*a.fields())
    for x, y in zip(fa, b.fields()):
        assert np.abs(x - y).max() < 1e-11 * max(1.0, np.abs(y).max())
    if flag_perm is not None:
        Xa = a.X.copy()
        Xa[:, 2] = wl.lz - Xa[:, 2]
        np.testing.assert_allclose(Xa[flag_perm], b.X, atol=1e-12)


def test_mirror_z_with_bars_and_flag():
    ns = nt = 5
    wl = _wl(bars_on=True, bar_x=1.0, flag_on=True, flag_x_le=2.0, flag_ns=ns, flag_nt=nt,
             flag_len=1.0, flag_span=1.0)
    perm = np.array([a * nt + (nt - 1 - b) for a in range(ns) for b in range(nt)])
    _check_equivariance(wl, _mirror_z, flag_perm=perm)


def test_mirror_y_with_bars():
    _check_equivariance(_wl(bars_on=True, bar_x=1.0), _mirror_y)


def test_swap_y_z_without_bodies():
    _check_equivariance(_wl(), _swap_yz)


def test_cfl_time_step():
    wl = _wl(dt=-1.0, cfl=0.3)
    s = OracleSolver(wl)
    assert math.isclose(s.next_dt(), 0.3 * s.h / 1.0, rel_tol=1e-14)
