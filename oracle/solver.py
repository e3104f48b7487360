"""One fractional step of the immersed-boundary Navier--Stokes solver (Sec. II.B).

Order of one step (n -> n+1), following the paper's description: provisional
velocity by AB2 + Crank--Nicolson with approximate factorisation, then the
immersed-boundary forcing, then the Poisson equation and the projection.

  A0  dt: fixed, or CFL * h / max_cells(|u|+|v|+|w|); AB2 weights
      alpha = 1 + dt / (2 dt_old), beta = -dt / (2 dt_old) (Euler on step 1)
  A1  convective outflow values at n+1 (Sec. II.A)
  A2  RHS = dt [ -(alpha N^n + beta N^{n-1}) - G p^n + nu L u^n ]
  A3  (1 - aL_x)(1 - aL_y)(1 - aL_z) du = RHS, a = nu dt / 2; u* = u^n + du
  A4  U*_l = I u* at every marker (flag and bars)
  A5  F_l = (U_l - U*_l) / dt with U_l = V^n_l (flag), 0 (bars);
      u** = u* + dt S F. With Eulerian bar forcing (bar_forcing "eulerian")
      the bars carry no markers: first u* <- (1 - alpha) u* at every velocity
      node, alpha the node cell's solid fraction, then the flag markers.
  A6  flag: fluid force -F_l dV_l, velocity Verlet sub-steps -> X^{n+1}, V^{n+1}
  A7  mass fix: (Q_in - Q_out) / (Ly Lz) added to u on the outflow face;
      D = div(u**) / dt
  A8  L_h phi = D (mean(phi) = 0)
  A9  u^{n+1} = u** - dt G phi;  p^{n+1} = p^n + phi - (nu dt / 2) L_h phi

The AB2 weights (A0) are pinned by the step's second-order temporal
convergence on a non-uniform step sequence, and the pressure by its
second-order convergence at the half step. The pressure update of A9,
including its correction term -(nu dt / 2) L_h phi, is pinned by the
momentum balance the three sub-steps must reproduce: away from the x
boundaries, (u1 - u0)/dt + N* - (nu/2) L (u1 + u0) + G p1 equals minus the
factorisation's splitting term, to round-off, only with that term present.

Readings (the paper does not state them): nu = 1 / Re with U = L = 1;
fluid density 1; the initial state is u = U plus the given perturbation,
made divergence-free by one projection at t = 0 with p = 0.

Prescribed (time-dependent) inflow, optional: ``set_inflow`` gives the inflow
planes (u_in, v_in, w_in) of the next step's new time level. The step uses
the current planes for the explicit terms (v, w ghosts q_{-1} = 2 q_in - q_0),
shifts u_in by a constant so that its mean is U (Q_in = U Ly Lz exactly), and
carries the boundary increments (u_in^{n+1} - u_0^n, v_in^{n+1} - v_in^n, ...)
into the x factor of A3; the new u_in becomes face 0 of u^{n+1}. Without a
call the inflow stays uniform (U, 0, 0).
"""
from __future__ import annotations

import math

import numpy as np

from . import af, flag, ib, mac, poisson


class OracleSolver:
    """The full time step of Sec. II.B in FP64 (steps A0-A9 of the module
    header) on the domain of Sec. II.A, with the bar grid and the flag;
    state: u, v, w, p, the flag's X, V, and the AB2 history."""

    U_IN = 1.0

    def __init__(self, wl, noise=None):
        self.wl = wl
        nx, ny, nz = wl.nx, wl.ny, wl.nz
        h = wl.lx / nx
        if not (math.isclose(h, wl.ly / ny) and math.isclose(h, wl.lz / nz)):
            raise ValueError("the grid spacing must be the same in x, y and z")
        self.h = h
        self.nu = 1.0 / wl.re
        shape = (nx + 1, ny, nz)
        self.u = np.full(shape, self.U_IN)
        self.v = np.zeros(shape)
        self.w = np.zeros(shape)
        if noise is not None:
            self.u += noise[0]
            self.v += noise[1]
            self.w += noise[2]
        self.p = np.zeros((nx, ny, nz))
        self.v_in = np.zeros((ny, nz))     # current transverse inflow planes
        self.w_in = np.zeros((ny, nz))
        self.pending_inflow = None
        self.n_prev = None
        self.dt_old = None
        self.t = 0.0
        self.nstep = 0

        # markers: flag vertices first, then the bar grid
        self.mesh = None
        self.nf = 0
        xs, dvs = [], []
        if wl.flag_on:
            self.mesh = flag.FlagMesh(wl.flag_ns, wl.flag_nt, wl.flag_len, wl.flag_span,
                                      wl.mass_ratio, wl.stretch, wl.bending)
            self.X = self.mesh.initial_positions(wl.flag_x_le, 0.5 * wl.ly, 0.5 * wl.lz,
                                                 wl.flag_span, wl.pitch0)
            self.V = np.zeros_like(self.X)
            self.l0 = self.mesh.rest_lengths(self.X)
            self.nf = self.mesh.nv
            self.flag_dv = self.mesh.area * h
            self.F_flag = np.zeros_like(self.X)
        self.bar_alpha = None
        if wl.bars_on and wl.bar_forcing == "eulerian":
            self.bar_alpha = [ib.bar_volume_fraction(wl, c, h) for c in range(3)]
            self.Xb = np.zeros((0, 3))
            self.bar_dv = np.zeros(0)
        elif wl.bars_on:
            self.Xb, dvb = ib.bar_markers(wl, h)
            self.bar_dv = np.full(self.Xb.shape[0], dvb)
        else:
            self.Xb = np.zeros((0, 3))
            self.bar_dv = np.zeros(0)

        # initial projection (time-step factor absorbed in phi)
        D = mac.divergence(self.u, self.v, self.w, h)
        phi = poisson.solve(D, h)
        self._project(phi, 1.0)

    # ------------------------------------------------------------------ helpers
    def _project(self, phi, dt):
        gu, gv, gw = mac.pressure_gradient(phi, self.h)
        self.u -= dt * gu
        self.v -= dt * gv
        self.w -= dt * gw

    def markers(self):
        """Lagrangian points forced this step: flag vertices then bar markers
        (Sec. II.B: both bodies are immersed boundaries)."""
        if self.nf:
            return np.concatenate([self.X, self.Xb], axis=0)
        return self.Xb

    def set_inflow(self, u_in, v_in, w_in):
        """Inflow planes (ny, nz) for the new time level of the following steps."""
        self.pending_inflow = tuple(np.array(a, dtype=np.float64) for a in (u_in, v_in, w_in))

    def next_dt(self):
        """A0: the fixed step, or CFL h / max over cells of (|u|+|v|+|w|)."""
        if self.wl.dt > 0:
            return self.wl.dt
        return self.wl.cfl * self.h / mac.cfl_speed(self.u, self.v, self.w)

    # ------------------------------------------------------------------ step
    def step(self, dt=None):
        """One time step A0-A9 (Sec. II.B order); returns the step size."""
        wl, h, nu = self.wl, self.h, self.nu
        nx = wl.nx
        u, v, w = self.u, self.v, self.w
        dt = self.next_dt() if dt is None else dt                        # A0
        if self.n_prev is None:
            alpha, beta = 1.0, 0.0
        else:
            alpha = 1.0 + dt / (2.0 * self.dt_old)
            beta = -dt / (2.0 * self.dt_old)

        un, vn, wn = mac.outflow_convective(u, v, w, dt, h, self.U_IN)  # A1
        du_out, dv_out, dw_out = un - u[nx], vn - v[nx], wn - w[nx]

        N = mac.advection(u, v, w, h, self.v_in, self.w_in)              # A2
        L = mac.laplacian(u, v, w, h, self.v_in, self.w_in)
        G = mac.pressure_gradient(self.p, h)
        rhs = []
        for c in range(3):
            nl = alpha * N[c]
            if self.n_prev is not None:
                nl = nl + beta * self.n_prev[c]
            rhs.append(dt * (-nl - G[c] + nu * L[c]))

        r = nu * dt / (2.0 * h * h)                                      # A3
        du_in = dv_in = dw_in = None
        if self.pending_inflow is not None:
            pu, pv, pw = self.pending_inflow
            u_new = pu - pu.mean() + self.U_IN          # Q_in = U Ly Lz
            du_in, dv_in, dw_in = u_new - u[0], pv - self.v_in, pw - self.w_in
        du, dv, dw = af.af_solve(rhs[0], rhs[1], rhs[2], r, du_out, dv_out, dw_out,
                                 du_in, dv_in, dw_in)
        us = u + du
        vs = v + dv
        ws = w + dw
        us[nx], vs[nx], ws[nx] = un, vn, wn
        if self.pending_inflow is not None:
            us[0] = u_new
            self.v_in, self.w_in = self.pending_inflow[1].copy(), self.pending_inflow[2].copy()

        if self.bar_alpha is not None:                                   # A4-A5, Eulerian bars
            us *= 1.0 - self.bar_alpha[0]
            vs *= 1.0 - self.bar_alpha[1]
            ws *= 1.0 - self.bar_alpha[2]
        Xm = self.markers()                                              # A4
        if Xm.shape[0]:
            Ustar = ib.interpolate((us, vs, ws), Xm, h, nx)
            target = np.zeros_like(Ustar)
            dv_m = self.bar_dv
            if self.nf:
                target[:self.nf] = self.V
                dv_m = np.concatenate([self.flag_dv, self.bar_dv])
            coef = (dv_m / h ** 3)[:, None] * (target - Ustar)           # A5
            ib.spread((us, vs, ws), Xm, coef, h, nx)
            if self.nf:                                                  # A6
                F = (target[:self.nf] - Ustar[:self.nf]) / dt
                self.F_flag = -F * self.flag_dv[:, None]
                self.X, self.V = flag.advance(self.X, self.V, self.F_flag, dt,
                                              self.mesh, self.l0)
            self.last_slip = Ustar - target

        q_in = us[0].sum() * h * h                                       # A7
        q_out = us[nx].sum() * h * h
        us[nx] += (q_in - q_out) / (wl.ly * wl.lz)
        D = mac.divergence(us, vs, ws, h) / dt

        phi = poisson.solve(D, h)                                        # A8

        self.u, self.v, self.w = us, vs, ws                              # A9
        self._project(phi, dt)
        self.p = self.p + phi - 0.5 * nu * dt * mac.cell_laplacian_neumann(phi, h)

        self.n_prev = N
        self.dt_old = dt
        self.t += dt
        self.nstep += 1
        self.last_dt = dt
        self.last_D = D
        return dt

    def run(self, nsteps, dt=None):
        """nsteps calls of ``step``."""
        for _ in range(nsteps):
            self.step(dt)

    def fields(self):
        """(u, v, w, p) in the array conventions of ``oracle.mac``."""
        return self.u, self.v, self.w, self.p
