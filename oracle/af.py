"""Crank--Nicolson diffusion by approximate factorisation (Sec. II.B).

The provisional velocity solves, per component,

    (1 - a L_x)(1 - a L_y)(1 - a L_z) du = RHS,   a = nu dt / 2,

with L_d the one-dimensional second difference along d, and u* = u^n + du.
Each factor is one tridiagonal solve per grid line: x lines carry the
inflow/outflow conditions, y and z lines are periodic (cyclic). The factors
commute mathematically; the oracle applies them in the order x, y, z.

Boundary rows along x (readings of the boundary conditions of Sec. II.A):

* u: unknowns are faces 1..nx-1; the inflow-face increment
  du_0 = u_0^{n+1} - u_0^n (zero for a steady inflow) and the outflow-face
  increment du_nx = u_nx^{n+1} - u_nx^n move to the RHS.
* v, w: unknowns are i = 0..nx-1; the inflow ghost follows
  dq_{-1} = 2 dq_in - dq_0 (dq_in: increment of the prescribed inflow value,
  zero for a steady inflow), the outflow ghost increment moves to the RHS.

Library primitives: ``scipy.linalg.solve_banded`` for the x lines and
``scipy.linalg.solve_circulant`` for the periodic lines.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded, solve_circulant


def solve_x_u(rhs_inner, r, du_out, du_in=None):
    """Tridiagonal solve along x for u on faces 1..nx-1.

    rhs_inner: shape (nx-1, ny, nz); r = a / h^2; du_out, du_in: (ny, nz)
    outflow / inflow face increments (du_in None: zero).
    """
    m = rhs_inner.shape[0]
    ab = np.zeros((3, m))
    ab[0, 1:] = -r
    ab[1, :] = 1.0 + 2.0 * r
    ab[2, :-1] = -r
    b = rhs_inner.reshape(m, -1).copy()
    b[-1] += r * du_out.reshape(-1)
    if du_in is not None:
        b[0] += r * du_in.reshape(-1)
    return solve_banded((1, 1), ab, b).reshape(rhs_inner.shape)


def solve_x_vw(rhs, r, dq_out, dq_in=None):
    """Tridiagonal solve along x for v or w on i = 0..nx-1 (inflow ghost
    dq_{-1} = 2 dq_in - dq_0; dq_in None: zero)."""
    m = rhs.shape[0]
    ab = np.zeros((3, m))
    ab[0, 1:] = -r
    ab[1, :] = 1.0 + 2.0 * r
    ab[1, 0] = 1.0 + 3.0 * r       # the -dq_0 of the ghost folded into the first row
    ab[2, :-1] = -r
    b = rhs.reshape(m, -1).copy()
    b[-1] += r * dq_out.reshape(-1)
    if dq_in is not None:
        b[0] += 2.0 * r * dq_in.reshape(-1)
    return solve_banded((1, 1), ab, b).reshape(rhs.shape)


def solve_periodic(rhs, r, axis):
    """Cyclic tridiagonal (-r, 1 + 2 r, -r) solve along a periodic axis."""
    n = rhs.shape[axis]
    c = np.zeros(n)
    c[0] = 1.0 + 2.0 * r
    c[1] = -r
    c[-1] = -r
    if n == 2:
        c[1] = -2.0 * r
    moved = np.moveaxis(rhs, axis, 0)
    sol = solve_circulant(c, moved.reshape(n, -1), baxis=0, outaxis=0)
    return np.moveaxis(np.real(sol).reshape(moved.shape), 0, axis)


def af_solve(rhs_u, rhs_v, rhs_w, r, du_out, dv_out, dw_out, du_in=None, dv_in=None,
             dw_in=None):
    """Apply (1 - aL_x)^-1, then (1 - aL_y)^-1, then (1 - aL_z)^-1 to each RHS.

    rhs_*: full-shape arrays (nx+1, ny, nz); only unknown entries are used.
    d*_out / d*_in: outflow / inflow boundary increments (inflow None: zero).
    Returns increments du, dv, dw with zeros outside the unknowns.
    """
    nx = rhs_u.shape[0] - 1
    du = np.zeros_like(rhs_u)
    du[1:nx] = solve_x_u(rhs_u[1:nx], r, du_out, du_in)
    du[1:nx] = solve_periodic(du[1:nx], r, axis=1)
    du[1:nx] = solve_periodic(du[1:nx], r, axis=2)
    out = [du]
    for rhs, dq_out, dq_in in ((rhs_v, dv_out, dv_in), (rhs_w, dw_out, dw_in)):
        dq = np.zeros_like(rhs)
        dq[:nx] = solve_x_vw(rhs[:nx], r, dq_out, dq_in)
        dq[:nx] = solve_periodic(dq[:nx], r, axis=1)
        dq[:nx] = solve_periodic(dq[:nx], r, axis=2)
        out.append(dq)
    return tuple(out)
