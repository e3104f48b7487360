"""Pins for the oracle's implicit diffusion (approximate factorisation) and
pressure Poisson solve (Sec. II.B).

* AF: separable trigonometric modes that satisfy each line's boundary rows are
  eigenvectors of every factor, so (1 - aL_x)(1 - aL_y)(1 - aL_z) du = RHS has
  the closed-form solution RHS / prod_d (1 + r mu_d), mu = 2 - 2 cos(theta).
  The outflow- and inflow-increment rows are pinned by closed-form sinh
  profiles.
* Poisson: the DFT + Thomas solution equals a dense direct solve of the
  assembled operator (Neumann in x, periodic in y, z, mean-zero gauge),
  on grids with unequal sides so that a transposed axis fails.
"""
import math

import numpy as np
import pytest

from oracle import af, mac, poisson


def _modes(nx, ny, nz, mx, my, mz):
    i = np.arange(nx + 1)[:, None, None]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[None, None, :]
    ty, tz = 2 * math.pi * my / ny, 2 * math.pi * mz / nz
    yz = np.cos(ty * j + 0.3) * np.sin(tz * k + 0.1)
    tu = math.pi * mx / nx                       # u: zero on faces 0 and nx
    mode_u = np.sin(tu * i) * yz
    tv = math.pi * mx / (nx + 0.5)               # v: odd about i = -1/2, zero at i = nx
    mode_v = np.sin(tv * (i + 0.5)) * yz
    mu = lambda t: 2.0 - 2.0 * math.cos(t)
    return mode_u, mode_v, mu(tu), mu(tv), mu(ty), mu(tz)


@pytest.mark.parametrize("mx,my,mz", [(1, 1, 1), (3, 2, 0), (5, 0, 3)])
def test_af_closed_form_modes(mx, my, mz):
    nx, ny, nz = 10, 8, 6
    r = 0.37
    mode_u, mode_v, mux_u, mux_v, muy, muz = _modes(nx, ny, nz, mx, my, mz)
    zero = np.zeros((ny, nz))
    du, dv, dw = af.af_solve(mode_u, mode_v, mode_v, r, zero, zero, zero)
    fac = (1 + r * muy) * (1 + r * muz)
    np.testing.assert_allclose(du[1:nx], mode_u[1:nx] / ((1 + r * mux_u) * fac), atol=1e-13)
    np.testing.assert_allclose(dv[:nx], mode_v[:nx] / ((1 + r * mux_v) * fac), atol=1e-13)
    np.testing.assert_allclose(dw[:nx], mode_v[:nx] / ((1 + r * mux_v) * fac), atol=1e-13)


def test_af_outflow_increment_profile():
    # zero RHS, du_nx = c: the x-line solution is c sinh(theta i) / sinh(theta nx)
    nx, ny, nz, r, c = 9, 4, 4, 0.8, 0.25
    rhs = np.zeros((nx + 1, ny, nz))
    out = np.full((ny, nz), c)
    du, dv, _ = af.af_solve(rhs, rhs, rhs, r, out, out, out)
    theta = math.acosh((1 + 2 * r) / (2 * r))
    i = np.arange(1, nx)
    expect_u = c * np.sinh(theta * i) / math.sinh(theta * nx)
    np.testing.assert_allclose(du[1:nx, 0, 0], expect_u, rtol=1e-12)
    # v: ghost reflection about i = -1/2 -> cosh-free odd profile sinh(theta (i + 1/2))
    iv = np.arange(nx)
    expect_v = c * np.sinh(theta * (iv + 0.5)) / math.sinh(theta * (nx + 0.5))
    np.testing.assert_allclose(dv[:nx, 0, 0], expect_v, rtol=1e-12)


def test_af_inflow_increment_profile():
    # zero RHS and outflow increments, inflow increment c: u (Dirichlet face
    # value c at i = 0, zero at i = nx) follows c sinh(theta (nx - i)) / sinh(theta nx);
    # v, w (ghost 2c - q_0, so the inflow-plane value (q_-1 + q_0) / 2 is c):
    # A sinh(theta (nx - i)) with A (sinh(theta (nx + 1)) + sinh(theta nx)) / 2 = c
    nx, ny, nz, r, c = 9, 4, 4, 0.8, 0.25
    rhs = np.zeros((nx + 1, ny, nz))
    zero = np.zeros((ny, nz))
    inc = np.full((ny, nz), c)
    du, dv, dw = af.af_solve(rhs, rhs, rhs, r, zero, zero, zero, inc, inc, inc)
    theta = math.acosh((1 + 2 * r) / (2 * r))
    i = np.arange(1, nx)
    np.testing.assert_allclose(du[1:nx, 0, 0], c * np.sinh(theta * (nx - i)) / math.sinh(theta * nx),
                               rtol=1e-12)
    iv = np.arange(nx)
    A = 2 * c / (math.sinh(theta * (nx + 1)) + math.sinh(theta * nx))
    np.testing.assert_allclose(dv[:nx, 1, 2], A * np.sinh(theta * (nx - iv)), rtol=1e-12)
    np.testing.assert_allclose(dw[:nx, 3, 0], A * np.sinh(theta * (nx - iv)), rtol=1e-12)


def _assembled_operator(nx, ny, nz, h):
    n = nx * ny * nz
    A = np.zeros((n, n))
    idx = lambda i, j, k: (i * ny + j) * nz + k
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                row = idx(i, j, k)
                for (di, dj, dk) in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    ii = i + di
                    if ii < 0 or ii >= nx:          # Neumann: no flux through x ends
                        continue
                    col = idx(ii, (j + dj) % ny, (k + dk) % nz)
                    A[row, col] += 1.0 / h ** 2
                    A[row, row] -= 1.0 / h ** 2
    return A


@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 6, 4), (5, 4, 6)])
def test_poisson_matches_dense_direct_solve(shape):
    nx, ny, nz = shape
    h = 0.4
    rng = np.random.default_rng(11)
    D = rng.standard_normal(shape)
    D -= D.mean()                               # compatibility
    A = _assembled_operator(nx, ny, nz, h)
    n = A.shape[0]
    bordered = np.zeros((n + 1, n + 1))
    bordered[:n, :n] = A
    bordered[:n, n] = 1.0
    bordered[n, :n] = 1.0
    sol = np.linalg.solve(bordered, np.concatenate([D.reshape(-1), [0.0]]))
    ref = sol[:n].reshape(shape)
    phi = poisson.solve(D, h)
    scale = np.abs(ref).max()
    assert np.abs(phi - ref).max() <= 1e-12 * scale
    assert abs(phi.mean()) < 1e-13 * scale
    # and the residual with the oracle's own operator
    assert np.abs(mac.cell_laplacian_neumann(phi, h) - D).max() < 1e-11 * np.abs(D).max()


def test_dft_matrix_is_the_fft():
    # the plain DFT matches the FFT library routine (sign and normalisation)
    x = np.random.default_rng(2).standard_normal(12)
    np.testing.assert_allclose(poisson.dft_matrix(12, -1) @ x, np.fft.fft(x), atol=1e-12)


def test_thomas_matches_banded_solver():
    from scipy.linalg import solve_banded
    rng = np.random.default_rng(5)
    n = 9
    lo, up = rng.uniform(0.1, 1, n), rng.uniform(0.1, 1, n)
    lo[0] = up[-1] = 0.0
    dg = 3.0 + rng.uniform(0, 1, n)
    b = rng.standard_normal(n)
    x = poisson.thomas(lo, dg, up, b[:, None])[:, 0]
    ab = np.zeros((3, n))
    ab[0, 1:] = up[:-1]
    ab[1] = dg
    ab[2, :-1] = lo[1:]
    np.testing.assert_allclose(x, solve_banded((1, 1), ab, b), rtol=1e-13)
