"""Pin of the oracle's pressure update (A9) by the momentum balance the
fractional step must reproduce (Sec. II.B: AB2 + Crank--Nicolson with
approximate factorisation, then projection).

Eliminating the provisional velocity from the three sub-steps of one step
gives, at every velocity node away from the x boundaries (where the discrete
Laplacian and gradient commute),

    (u1 - u0)/dt + (alpha N^n + beta N^{n-1}) - (nu/2) L (u1 + u0) + G p1
        = -E du / dt,

    E  = a^2 (Lx Ly + Ly Lz + Lz Lx) - a^3 Lx Ly Lz,   a = nu dt / 2,
    du = u* - u0 = u1 - u0 + dt G phi,

i.e. the step is the Crank--Nicolson discretisation of the momentum equation
with the pressure p1 at the half step, up to the factorisation's splitting
term E. That holds only for p1 = p0 + phi - (nu dt/2) L phi: dropping the
correction term (or flipping its sign) leaves a residual of size
(nu dt / 2) G L phi, which the test shows is many orders of magnitude above
the identity's round-off. The operators below are the 7-point stencils
written out for interior nodes, independent of ``oracle.mac``; N^n and
N^{n-1} are the oracle's own advection terms (pinned elsewhere), phi is
recovered from the stored divergence by the (dense-LU-pinned) Poisson solve.
"""
import numpy as np
import pytest

from oracle import poisson
from oracle.solver import OracleSolver
from paper_2103_08246_gb300 import inputs


def _d2(a, axis, h):
    """Second difference along an axis; y, z periodic (np.roll), x interior
    values only (the caller discards the wrapped x ends)."""
    return (np.roll(a, -1, axis) - 2.0 * a + np.roll(a, 1, axis)) / (h * h)


def _grad_p(p, h, nxp1):
    """G p on the u, v, w lattices (shape (nx+1, ny, nz) each; u faces 1..nx-1
    and v, w planes 0..nx-1 filled)."""
    nx = p.shape[0]
    gu = np.zeros((nxp1,) + p.shape[1:])
    gu[1:nx] = (p[1:] - p[:-1]) / h
    gv = np.zeros_like(gu)
    gv[:nx] = (p - np.roll(p, 1, 1)) / h
    gw = np.zeros_like(gu)
    gw[:nx] = (p - np.roll(p, 1, 2)) / h
    return gu, gv, gw


def _step_with_history(wl, noise, nsteps):
    ora = OracleSolver(wl, noise)
    ora.run(nsteps - 1)
    before = dict(u=[q.copy() for q in (ora.u, ora.v, ora.w)], p=ora.p.copy(),
                  n_prev=[q.copy() for q in ora.n_prev], dt_old=ora.dt_old)
    dt = ora.step()
    return ora, before, dt


def _balance(ora, before, dt, p1):
    """Per component: (residual + E du/dt, scale) on the interior nodes."""
    wl, h, nu = ora.wl, ora.h, ora.nu
    nx = wl.nx
    a = 0.5 * nu * dt
    alpha = 1.0 + dt / (2.0 * before["dt_old"])
    beta = -dt / (2.0 * before["dt_old"])
    phi = poisson.solve(ora.last_D, h)
    G1 = _grad_p(p1, h, nx + 1)
    Gphi = _grad_p(phi, h, nx + 1)
    out = []
    for c, (u0, u1) in enumerate(zip(before["u"], (ora.u, ora.v, ora.w))):
        lap = lambda q: _d2(q, 0, h) + _d2(q, 1, h) + _d2(q, 2, h)  # noqa: E731
        nstar = alpha * ora.n_prev[c] + beta * before["n_prev"][c]
        R = (u1 - u0) / dt + nstar - 0.5 * nu * lap(u1 + u0) + G1[c]
        du = u1 - u0 + dt * Gphi[c]
        Lx, Ly, Lz = (lambda q, ax=ax: _d2(q, ax, h) for ax in range(3))
        E = (a * a * (Lx(Ly(du)) + Ly(Lz(du)) + Lz(Lx(du)))
             - a ** 3 * Lx(Ly(Lz(du))))
        # u faces 2..nx-2, v/w planes 1..nx-2: every stencil stays on
        # unknowns of the x factor, and L G = G L there
        sl = slice(2, nx - 1) if c == 0 else slice(1, nx - 1)
        res = (R + E / dt)[sl]
        scale = max(np.abs(((u1 - u0) / dt)[sl]).max(), np.abs(G1[c][sl]).max(),
                    np.abs(nstar[sl]).max())
        out.append((np.abs(res).max(), scale))
    return out


@pytest.fixture(scope="module")
def stepped():
    # viscous enough that (nu dt / 2) L phi is not small (r = nu dt / 2h^2 = 0.16),
    # a strong perturbation so that the pressure changes quickly
    wl = inputs.small(24, 8, 8, re=1.0, dt=0.02, bars_on=False, flag_on=False)
    noise = inputs.initial_noise(wl, amp=0.4)
    return _step_with_history(wl, noise, 4)


def test_step_is_crank_nicolson_momentum_balance(stepped):
    ora, before, dt = stepped
    for err, scale in _balance(ora, before, dt, ora.p):
        assert err <= 1e-11 * scale, (err, scale)


def test_pressure_without_correction_breaks_the_balance(stepped):
    """The planted omission p1 = p0 + phi (and the flipped sign) miss the
    balance by far more than its round-off."""
    ora, before, dt = stepped
    h, nu = ora.h, ora.nu
    phi = poisson.solve(ora.last_D, h)
    corr = 0.5 * nu * dt * (_d2(phi, 1, h) + _d2(phi, 2, h))
    # the x part of L phi with Neumann ends, written out
    lx = np.zeros_like(phi)
    lx[1:-1] = (phi[2:] - 2.0 * phi[1:-1] + phi[:-2]) / (h * h)
    lx[0] = (phi[1] - phi[0]) / (h * h)
    lx[-1] = (phi[-2] - phi[-1]) / (h * h)
    corr = corr + 0.5 * nu * dt * lx
    good = _balance(ora, before, dt, ora.p)
    for planted in (ora.p + corr, ora.p + 2.0 * corr):
        bad = _balance(ora, before, dt, planted)
        worst = max(e / s for e, s in bad)
        best = max(e / s for e, s in good)
        assert worst > 1e4 * max(best, 1e-16) and worst > 1e-6, (worst, best)
