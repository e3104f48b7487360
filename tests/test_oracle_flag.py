"""Pins for the oracle's spring-network flag (Sec. II.B structural model;
Sec. II.A hinged-at-the-leading-edge flag with free other edges).

* lattice bookkeeping: spring / hinge counts, lumped areas sum to the sheet
  area, masses are mass_ratio * area;
* the energy of an isometric cylindrical bend is k_e (1 - cos psi) per
  turning hinge (closed form; stretching energy exactly zero), i.e.
  beta kappa^2 / 2 per area for any cell aspect ratio;
* the forces are minus the energy gradient (central differences);
* rigid motions produce no force;
* in vacuo, a small-amplitude first mode oscillates at the Euler--Bernoulli
  hinged-free frequency omega_1 = k_1^2 sqrt(beta / rho) within 2 % at the
  tiny workload's 17-vertex resolution (k_1 from
  tests/golden/euler_bernoulli_hinged_free.txt), converging with resolution.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import flag

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split("=")
            out[k.strip()] = float(v)
    return out


def _mesh(ns=9, nt=7, L=1.0, span=0.8, rho=1.3, ks=1000.0, kb=0.01):
    return flag.FlagMesh(ns, nt, L, span, rho, ks, kb)


def test_lattice_bookkeeping():
    ns, nt = 9, 7
    m = _mesh(ns, nt)
    assert len(m.springs) == (ns - 1) * nt + ns * (nt - 1) + 2 * (ns - 1) * (nt - 1)
    # each of the two triangulations has every interior lattice edge and
    # every cell diagonal as a hinge
    interior = (ns - 1) * (nt - 2) + (ns - 2) * (nt - 1) + (ns - 1) * (nt - 1)
    assert len(m.hinge_tris) == 2 * interior
    assert len(m.tris) == 4 * (ns - 1) * (nt - 1)
    assert abs(m.area.sum() - 1.0 * 0.8) < 1e-14
    np.testing.assert_allclose(m.mass, 1.3 * m.area)
    assert not m.free[:nt].any() and m.free[nt:].all()


def _flat(m, span):
    return m.initial_positions(0.0, 0.0, 0.5 * span, span, 0.0)


@pytest.mark.parametrize("axis", ["s", "t"])
def test_isometric_cylindrical_bend_energy(axis):
    ns, nt, span = 9, 7, 0.8
    m = _mesh(ns, nt, span=span)
    X0 = _flat(m, span)
    l0 = m.rest_lengths(X0)
    psi = 0.2
    X = X0.reshape(ns, nt, 3).copy()
    if axis == "s":
        # vertices on a circle with chord ds: every chord turns by psi
        R = m.ds / (2 * math.sin(psi / 2))
        ang = np.arange(ns) * psi
        X[:, :, 0] = (R * np.sin(ang))[:, None]
        X[:, :, 1] = (R * (1 - np.cos(ang)))[:, None]
        turning = (ns - 2) * (nt - 1)
        k_e = m.k_b * m.dt / m.ds            # beta |e|^2 / A for an edge along t (both splits)
    else:
        R = m.dt / (2 * math.sin(psi / 2))
        ang = np.arange(nt) * psi
        X[:, :, 2] = (R * np.sin(ang))[None, :]
        X[:, :, 1] = (R * (1 - np.cos(ang)))[None, :]
        turning = (ns - 1) * (nt - 2)
        k_e = m.k_b * m.ds / m.dt
    X = X.reshape(-1, 3)
    e = flag.energy(torch.tensor(X), m, l0).item()
    np.testing.assert_allclose(m.rest_lengths(X), l0, rtol=1e-13)
    assert abs(e - k_e * turning * (1 - math.cos(psi))) < 1e-12
    # energy per area -> beta kappa^2 / 2 with kappa = psi / (cell side across the hinge)
    side = m.ds if axis == "s" else m.dt
    bent_area = turning * m.ds * m.dt
    assert abs(e / bent_area - 0.5 * m.k_b * (psi / side) ** 2) < 0.01 * 0.5 * m.k_b * (psi / side) ** 2


def test_forces_are_minus_energy_gradient():
    m = _mesh(5, 4)
    X0 = _flat(m, 0.8)
    l0 = m.rest_lengths(X0)
    rng = np.random.default_rng(0)
    X = X0 + 0.02 * rng.standard_normal(X0.shape)
    F = flag.elastic_forces(X, m, l0)
    eps = 1e-6
    for v in (5, 9, 17):
        for c in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, c] += eps
            Xm[v, c] -= eps
            ep = flag.energy(torch.tensor(Xp), m, l0).item()
            em = flag.energy(torch.tensor(Xm), m, l0).item()
            assert abs(F[v, c] + (ep - em) / (2 * eps)) < 1e-6 * max(1.0, abs(F[v, c]))


def test_rigid_motion_gives_no_force():
    m = _mesh(6, 5)
    X0 = _flat(m, 0.8)
    l0 = m.rest_lengths(X0)
    a = 0.7
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(0.3), -math.sin(0.3)], [0, math.sin(0.3), math.cos(0.3)]])
    X = X0 @ (Rz @ Rx).T + np.array([1.0, -2.0, 0.5])
    assert np.abs(flag.elastic_forces(X, m, l0)).max() < 1e-10


def _first_mode_frequency(ns, beta=0.01, rho=1.0):
    k1 = _golden("euler_bernoulli_hinged_free.txt")["k1"]
    nt, span = 3, 1.0
    m = flag.FlagMesh(ns, nt, 1.0, span, rho, 1000.0, beta)
    X0 = _flat(m, span)
    l0 = m.rest_lengths(X0)
    s = np.repeat(np.arange(ns) * m.ds, nt)
    shape = np.sin(k1 * s) + math.sin(k1) / math.sinh(k1) * np.sinh(k1 * s)
    eps = 1e-4
    X = X0.copy()
    X[:, 1] += eps * shape
    V = np.zeros_like(X)
    F0 = np.zeros_like(X)
    omega_th = k1 ** 2 * math.sqrt(beta / rho)
    T = 2 * math.pi / omega_th
    dt = 0.01
    tip = []
    t = 0.0
    while t < 1.3 * T:
        X, V = flag.advance(X, V, F0, dt, m, l0)
        t += dt
        tip.append((t, X[-1, 1]))
    tip = np.array(tip)
    # zero crossings by linear interpolation; consecutive crossings are T/2 apart
    y = tip[:, 1]
    idx = np.where(np.sign(y[:-1]) != np.sign(y[1:]))[0]
    cross = [tip[i, 0] - y[i] * (tip[i + 1, 0] - tip[i, 0]) / (y[i + 1] - y[i]) for i in idx]
    assert len(cross) >= 2
    period = 2 * (cross[1] - cross[0])
    return 2 * math.pi / period, omega_th


def test_euler_bernoulli_first_mode_frequency():
    w17, w_th = _first_mode_frequency(17)
    err17 = abs(w17 - w_th) / w_th
    assert err17 < 0.02, (w17, w_th)
    w9, _ = _first_mode_frequency(9)
    assert abs(w9 - w_th) / w_th > err17      # converges with resolution


def _hessian_omega(m, X0, l0):
    """Largest eigenfrequency of M^-1 K on the free vertices (exact, by eigh)."""
    Xt = torch.tensor(X0, dtype=torch.float64)
    H = torch.autograd.functional.hessian(lambda x: flag.energy(x.reshape(-1, 3), m, l0),
                                          Xt.reshape(-1)).numpy()
    free = np.repeat(m.free, 3)
    minv = 1.0 / np.sqrt(np.repeat(m.mass, 3)[free])
    Hf = H[np.ix_(free, free)] * minv[:, None] * minv[None, :]
    return math.sqrt(max(np.linalg.eigvalsh(Hf).max(), 0.0))


def test_substeps_respect_the_verlet_stability_limit():
    """Gershgorin bounds the true spectrum, so dt_s * omega_true <= 1.8 < 2;
    energy stays bounded over many sub-steps there, while a step 15 % past
    the stability limit 2 / omega_true blows up (the bound is not vacuous)."""
    m = _mesh(5, 4, ks=400.0, kb=0.5)
    X0 = _flat(m, 0.8)
    l0 = m.rest_lengths(X0)
    rng = np.random.default_rng(3)
    Xp = X0 + np.where(m.free[:, None], 1e-3 * rng.standard_normal(X0.shape), 0.0)
    w_true = _hessian_omega(m, Xp, l0)
    w_bound = m.omega_max()
    assert w_true <= w_bound

    def total_energy(X, V):
        Xt = torch.tensor(X, dtype=torch.float64)
        return float(flag.energy(Xt, m, l0)) + 0.5 * float((m.mass[:, None] * V * V).sum())

    dt = 0.05
    n_sub = m.substeps(dt)
    assert dt / n_sub * w_bound <= 1.8 + 1e-12
    X, V = Xp.copy(), np.zeros_like(Xp)
    e0 = total_energy(X, V)
    for _ in range(40):
        X, V = flag.advance(X, V, np.zeros_like(X), dt, m, l0)
    assert total_energy(X, V) < 1.5 * e0

    h_bad = 2.3 / w_true
    X, V = Xp.copy(), np.zeros_like(Xp)
    for _ in range(40):
        X, V = flag.advance(X, V, np.zeros_like(X), h_bad, m, l0, n_sub=1)
    assert not np.isfinite(total_energy(X, V)) or total_energy(X, V) > 1e3 * e0
