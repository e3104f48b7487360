"""Staggered (MAC) grid operators, plain numpy FP64.

Sec. II.B: the equations are discretised with second-order centred finite
differences on a regular staggered mesh; Sec. II.A: uniform inflow (U, 0, 0)
at x = 0, convective (non-reflecting) outflow at x = Lx, periodic y and z.

Array conventions (x slowest, z fastest; h is the uniform spacing):

* ``u`` shape (nx+1, ny, nz): u[i, j, k] at (i h, (j+1/2) h, (k+1/2) h).
  Face i = 0 is the inflow (u = U), face i = nx the outflow.
* ``v`` shape (nx+1, ny, nz): v[i, j, k] at ((i+1/2) h, j h, (k+1/2) h) for
  i < nx; v[nx] is the ghost value just outside the outflow, advanced by the
  convective condition. The inflow ghost is v_{-1} = -v_0 (v = 0 on the
  inflow plane).
* ``w`` likewise with w[i, j, k] at ((i+1/2) h, (j+1/2) h, k h).
* ``p``, divergence and phi shape (nx, ny, nz) at cell centres.

Readings where the paper is silent: advection in flux (divergence) form with
arithmetic-mean interpolation; the inflow ghost reflection for v, w; the
convective velocity U_c = U in the outflow condition.
"""
from __future__ import annotations

import numpy as np


def _yp(a):
    """a[:, j+1, :] (periodic)."""
    return np.roll(a, -1, axis=1)


def _ym(a):
    """a[:, j-1, :] (periodic)."""
    return np.roll(a, 1, axis=1)


def _zp(a):
    return np.roll(a, -1, axis=2)


def _zm(a):
    return np.roll(a, 1, axis=2)


def with_x_ghosts(q, q_in=None):
    """v or w with the inflow ghost prepended: index m holds q_{m-1}, m = 0..nx+1.

    The inflow ghost is q_{-1} = 2 q_in - q_0, so that the linear interpolant
    equals the prescribed inflow value q_in on the inflow plane x = 0; with
    the uniform inflow (U, 0, 0) of Sec. II.A, q_in = 0 and q_{-1} = -q_0.
    """
    ghost = -q[:1] if q_in is None else 2.0 * q_in[None] - q[:1]
    return np.concatenate([ghost, q], axis=0)


def advection(u, v, w, h, v_in=None, w_in=None):
    """Nonlinear term N = div(u u) in flux form on the MAC grid (Sec. II.B).

    Returns (Nu, Nv, Nw) with the shapes of (u, v, w); entries that are not
    unknowns (u faces 0 and nx, the v/w ghost plane nx) are zero. v_in, w_in:
    prescribed transverse inflow planes (None: zero).
    """
    nx = u.shape[0] - 1
    vg = with_x_ghosts(v, v_in)    # vg[i+1] = v_i for i = -1..nx
    wg = with_x_ghosts(w, w_in)

    # normal fluxes at cell centres
    uc = 0.5 * (u[1:] + u[:-1])                    # (i+1/2): shape (nx, ny, nz)
    fxx = uc * uc
    vc = 0.5 * (v[:nx] + _yp(v[:nx]))              # (j+1/2)
    fyy = vc * vc
    wc = 0.5 * (w[:nx] + _zp(w[:nx]))              # (k+1/2)
    fzz = wc * wc

    # cross fluxes on cell edges
    # xy-edge (x = i h, y = j h), i = 0..nx
    fxy = (0.5 * (u + _ym(u))) * (0.5 * (vg[:-1] + vg[1:]))
    # xz-edge (x = i h, z = k h), i = 0..nx
    fxz = (0.5 * (u + _zm(u))) * (0.5 * (wg[:-1] + wg[1:]))
    # yz-edge (y = j h, z = k h) at x = (i+1/2) h, i = 0..nx-1
    fyz = (0.5 * (v[:nx] + _zm(v[:nx]))) * (0.5 * (w[:nx] + _ym(w[:nx])))

    nu = np.zeros_like(u)
    nu[1:nx] = ((fxx[1:] - fxx[:-1])
                + (_yp(fxy) - fxy)[1:nx]
                + (_zp(fxz) - fxz)[1:nx]) / h
    nv = np.zeros_like(v)
    nv[:nx] = ((fxy[1:] - fxy[:-1])
               + (fyy - _ym(fyy))
               + (_zp(fyz) - fyz)) / h
    nw = np.zeros_like(w)
    nw[:nx] = ((fxz[1:] - fxz[:-1])
               + (_yp(fyz) - fyz)
               + (fzz - _zm(fzz))) / h
    return nu, nv, nw


def laplacian(u, v, w, h, v_in=None, w_in=None):
    """7-point Laplacian of each velocity component on its own lattice
    (v_in, w_in: prescribed transverse inflow planes, None: zero)."""
    nx = u.shape[0] - 1
    inv = 1.0 / (h * h)
    lu = np.zeros_like(u)
    lu[1:nx] = (u[2:] - 2.0 * u[1:nx] + u[:-2]
                + _yp(u)[1:nx] - 2.0 * u[1:nx] + _ym(u)[1:nx]
                + _zp(u)[1:nx] - 2.0 * u[1:nx] + _zm(u)[1:nx]) * inv
    out = [lu]
    for q, q_in in ((v, v_in), (w, w_in)):
        g = with_x_ghosts(q, q_in)
        lq = np.zeros_like(q)
        c = q[:nx]
        lq[:nx] = (g[2:] - 2.0 * c + g[:nx]
                   + _yp(c) - 2.0 * c + _ym(c)
                   + _zp(c) - 2.0 * c + _zm(c)) * inv
        out.append(lq)
    return tuple(out)


def pressure_gradient(p, h):
    """G p on the interior faces (zero on the u boundary faces and v/w ghosts)."""
    nx = p.shape[0]
    shape = (nx + 1,) + p.shape[1:]
    gu = np.zeros(shape)
    gu[1:nx] = (p[1:] - p[:-1]) / h
    gv = np.zeros(shape)
    gv[:nx] = (p - _ym(p)) / h
    gw = np.zeros(shape)
    gw[:nx] = (p - _zm(p)) / h
    return gu, gv, gw


def divergence(u, v, w, h):
    """Discrete divergence at cell centres."""
    nx = u.shape[0] - 1
    return ((u[1:] - u[:-1]) + (_yp(v[:nx]) - v[:nx]) + (_zp(w[:nx]) - w[:nx])) / h


def cell_laplacian_neumann(phi, h):
    """Laplacian of a cell-centred field with dphi/dx = 0 at both x ends, periodic y, z.

    This is div(G phi) when G acts on interior faces only, i.e. the operator
    of the pressure Poisson equation.
    """
    g = np.concatenate([phi[:1], phi, phi[-1:]], axis=0)
    return (g[2:] - 2.0 * phi + g[:-2]
            + _yp(phi) - 2.0 * phi + _ym(phi)
            + _zp(phi) - 2.0 * phi + _zm(phi)) / (h * h)


def outflow_convective(u, v, w, dt, h, uc=1.0):
    """Convective outflow dq/dt + U_c dq/dx = 0 at x = Lx, first-order upwind in x.

    Returns the new outflow planes (u_nx, v_nx, w_nx) at time n+1 from the
    values at time n (Sec. II.A non-reflecting outlet).
    """
    nx = u.shape[0] - 1
    c = uc * dt / h
    un = u[nx] - c * (u[nx] - u[nx - 1])
    vn = v[nx] - c * (v[nx] - v[nx - 1])
    wn = w[nx] - c * (w[nx] - w[nx - 1])
    return un, vn, wn


def cfl_speed(u, v, w):
    """max over cells of |u_c| + |v_c| + |w_c| with centre-averaged components."""
    nx = u.shape[0] - 1
    uc = 0.5 * (u[1:] + u[:-1])
    vc = 0.5 * (v[:nx] + _yp(v[:nx]))
    wc = 0.5 * (w[:nx] + _zp(w[:nx]))
    return float(np.max(np.abs(uc) + np.abs(vc) + np.abs(wc)))
