"""Pins for the oracle's staggered-grid operators (Sec. II.B: second-order
centred differences on a staggered mesh; Sec. II.A boundary conditions).

Each check ties the oracle to mathematics, not to itself:
* advection converges at second order to the analytic (u . grad) u of a
  divergence-free field that satisfies the inflow condition;
* the Laplacian reproduces the exact discrete eigenvalue of trigonometric
  modes, including the inflow reflection ghost;
* div(G p) equals the Neumann cell Laplacian (the Poisson operator);
* a velocity built as the discrete curl of a potential has zero discrete
  divergence to round-off.
"""
import math

import numpy as np
import pytest

from oracle import mac

sympy = pytest.importorskip("sympy")


def _analytic_field(lx, ly, lz):
    x, y, z = sympy.symbols("x y z")
    a = sympy.cos(sympy.pi * x / lx)
    b = sympy.sin(2 * sympy.pi * y / ly)
    c = 0.5 * sympy.cos(sympy.pi * x / lx)
    d = sympy.cos(2 * sympy.pi * z / lz)
    u = 1 + a * sympy.diff(b, y) - c * sympy.diff(d, z)
    v = -sympy.diff(a, x) * b
    w = sympy.diff(c, x) * d
    assert sympy.simplify(sympy.diff(u, x) + sympy.diff(v, y) + sympy.diff(w, z)) == 0
    conv = [sympy.simplify(u * sympy.diff(q, x) + v * sympy.diff(q, y) + w * sympy.diff(q, z))
            for q in (u, v, w)]
    f = [sympy.lambdify((x, y, z), e, "numpy") for e in (u, v, w)]
    g = [sympy.lambdify((x, y, z), e, "numpy") for e in conv]
    return f, g


def _sample(f, nx, ny, nz, h, comp):
    off = [(0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0)][comp]
    i = np.arange(nx + 1)[:, None, None]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[None, None, :]
    val = f((i + off[0]) * h, (j + off[1]) * h, (k + off[2]) * h)
    return np.broadcast_to(val, (nx + 1, ny, nz)).astype(float).copy()


def test_advection_second_order_against_analytic():
    lx, ly, lz = 2.0, 1.0, 1.0
    f, g = _analytic_field(lx, ly, lz)
    errs = []
    for n in (16, 32, 64):
        nx, ny, nz = 2 * n, n, n
        h = lx / nx
        u, v, w = (_sample(f[c], nx, ny, nz, h, c) for c in range(3))
        N = mac.advection(u, v, w, h)
        e = 0.0
        for c in range(3):
            exact = _sample(g[c], nx, ny, nz, h, c)
            sl = slice(1, nx) if c == 0 else slice(0, nx)
            e = max(e, np.abs(N[c][sl] - exact[sl]).max())
        errs.append(e)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.9, (errs, orders)


def test_laplacian_exact_discrete_eigenvalues():
    nx, ny, nz = 12, 8, 6
    h = 0.25
    ky, kz, kx = 2 * math.pi / (ny * h), 2 * 2 * math.pi / (nz * h), 0.7
    lam = lambda k: (2 * math.cos(k * h) - 2) / h ** 2
    i = np.arange(nx + 1)[:, None, None]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[None, None, :]
    # u: linear in x (exact zero second difference), trigonometric in y, z
    u = (1.0 + 0.3 * i * h) * np.cos(ky * (j + 0.5) * h) * np.sin(kz * (k + 0.5) * h)
    # v, w: sin(kx x) in x is odd about x = 0, so the reflection ghost is exact
    v = np.sin(kx * (i + 0.5) * h) * np.cos(ky * j * h) * np.cos(kz * (k + 0.5) * h)
    w = np.sin(kx * (i + 0.5) * h) * np.sin(ky * (j + 0.5) * h) * np.cos(kz * k * h)
    lu, lv, lw = mac.laplacian(u, v, w, h)
    np.testing.assert_allclose(lu[1:nx], (lam(ky) + lam(kz)) * u[1:nx], atol=1e-11)
    lv_exact = (lam(kx) + lam(ky) + lam(kz)) * v[:nx]
    np.testing.assert_allclose(lv[:nx], lv_exact, atol=1e-11)
    np.testing.assert_allclose(lw[:nx], (lam(kx) + lam(ky) + lam(kz)) * w[:nx], atol=1e-11)
    assert np.all(lu[0] == 0) and np.all(lu[nx] == 0) and np.all(lv[nx] == 0)


def test_div_grad_is_neumann_cell_laplacian():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((7, 6, 5))
    h = 0.3
    gu, gv, gw = mac.pressure_gradient(p, h)
    np.testing.assert_allclose(mac.divergence(gu, gv, gw, h),
                               mac.cell_laplacian_neumann(p, h), atol=1e-12)


def test_discrete_curl_is_divergence_free():
    # u = d(psi)/dy, v = -d(psi)/dx with psi on xy-edges: exactly solenoidal
    rng = np.random.default_rng(4)
    nx, ny, nz, h = 6, 5, 4, 0.5
    psi = rng.standard_normal((nx + 1, ny, nz))
    u = (np.roll(psi, -1, axis=1) - psi) / h
    v = np.zeros_like(u)
    v[:nx] = -(psi[1:] - psi[:-1]) / h
    w = np.zeros_like(u)
    assert np.abs(mac.divergence(u, v, w, h)).max() < 1e-12


def test_uniform_flow_has_no_advection():
    nx, ny, nz = 6, 4, 4
    u = np.ones((nx + 1, ny, nz))
    v = np.zeros_like(u)
    w = np.zeros_like(u)
    for q in mac.advection(u, v, w, 0.25):
        assert np.abs(q).max() == 0.0


def test_convective_outflow_is_upwind_transport():
    nx, ny, nz, h, dt = 5, 2, 2, 0.5, 0.1
    u = np.zeros((nx + 1, ny, nz))
    u[nx - 1], u[nx] = 2.0, 1.0
    v = u.copy()
    w = u.copy()
    un, vn, wn = mac.outflow_convective(u, v, w, dt, h, uc=1.0)
    expect = 1.0 - dt / h * (1.0 - 2.0)
    for q in (un, vn, wn):
        np.testing.assert_allclose(q, expect)
