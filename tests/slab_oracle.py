"""Test helper: the x-slab phase protocol of include/ibm.h carried out on the
host in FP64 with the oracle's operators, one slab window per rank.

It follows the library's phases and buffer layouts (sizes from the library's
host-only ``ibm_slab_plan``) so that the package's driver and communicators
(``paper_2103_08246_gb300.slab``) can run real multi-process exchanges on CPU
ranks, and so that the decomposition itself (overlap width, duplicated
forcing near the cuts, owned flag forces, end fluxes, the partition method of
the pressure equation's x solve) can be checked against the single-domain
oracle. Pressure transforms here are separable Hartley transforms computed
with numpy's FFT; the partition-method algebra is written out per line.
"""
from __future__ import annotations

import numpy as np

from oracle import af, flag, ib, mac
from paper_2103_08246_gb300 import binding as B
from paper_2103_08246_gb300.slab import window


def dht(a, axis):
    """Unnormalised Hartley transform along one axis: Re F - Im F."""
    f = np.fft.fft(a, axis=axis)
    return f.real - f.imag


def dht2(a):
    return dht(dht(a, 1), 2)


def idht2(a):
    return dht(dht(a, 2), 1)


def _pivots(lam, n, first_phys, last_phys, pinned):
    """Inverse pivots and upper factors of the slab rows (h^2 units)."""
    inv = np.empty((n,) + lam.shape)
    cp = np.zeros(lam.shape)
    for i in range(n):
        diag = -2.0 + lam
        if (i == 0 and first_phys) or (i == n - 1 and last_phys):
            diag = -1.0 + lam
        if i == 0:
            diag = np.where(pinned, 1.0, diag)
        lower = 0.0 if i == 0 else 1.0
        prev = np.where(pinned, 0.0, cp) if i == 1 else cp
        inv[i] = 1.0 / (diag - lower * prev)
        cp = inv[i]
    upper = inv.copy()
    upper[0] = np.where(pinned, 0.0, inv[0])
    return inv, upper


def _thomas(inv, upper, rhs):
    n = rhs.shape[0]
    d = np.empty_like(rhs)
    y = np.zeros(rhs.shape[1:])
    for i in range(n):
        y = (rhs[i] - y) * inv[i]
        d[i] = y
    x = np.empty_like(rhs)
    x[n - 1] = d[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = d[i] - upper[i] * x[i + 1]
    return x


class OracleSlab:
    """One slab of a case on the host (FP64), with ``phase`` and ``plan`` as
    ``paper_2103_08246_gb300.slab.SlabState`` has them (torch CPU tensors)."""

    U_IN = 1.0

    def __init__(self, wl, slab, noise=None):
        self.wl, self.slab = wl, slab
        self.h = wl.lx / wl.nx
        self.nu = 1.0 / wl.re
        self.x0, self.nxw = window(slab)
        self.gL = slab.ghosts if slab.rank > 0 else 0
        self.gR = slab.ghosts if slab.rank < slab.nranks - 1 else 0
        self.n = slab.x_end - slab.x_begin
        self.first = slab.rank == 0
        self.last = slab.rank == slab.nranks - 1
        shape = (self.nxw + 1, wl.ny, wl.nz)
        cut = slice(self.x0, self.x0 + self.nxw + 1)
        self.u = np.full(shape, self.U_IN) + (noise[0][cut] if noise is not None else 0.0)
        self.v = np.zeros(shape) + (noise[1][cut] if noise is not None else 0.0)
        self.w = np.zeros(shape) + (noise[2][cut] if noise is not None else 0.0)
        self.p = np.zeros((self.nxw, wl.ny, wl.nz))
        self.N = [np.zeros(shape) for _ in range(3)]
        self.have_n = False
        self.dt_old = None
        self.nf = 0
        if wl.flag_on:
            self.mesh = flag.FlagMesh(wl.flag_ns, wl.flag_nt, wl.flag_len, wl.flag_span,
                                      wl.mass_ratio, wl.stretch, wl.bending)
            self.X = self.mesh.initial_positions(wl.flag_x_le, 0.5 * wl.ly, 0.5 * wl.lz,
                                                 wl.flag_span, wl.pitch0)
            self.V = np.zeros_like(self.X)
            self.l0 = self.mesh.rest_lengths(self.X)
            self.nf = self.mesh.nv
            self.flag_dv = self.mesh.area * self.h
        Xb, dvb = (ib.bar_markers(wl, self.h) if wl.bars_on else (np.zeros((0, 3)), 0.0))
        cx = np.floor(Xb[:, 0] / self.h).astype(np.int64)
        keep = (cx >= self.x0 - 3) & (cx <= self.x0 + self.nxw + 2)
        self.Xb = Xb[keep] - np.array([self.x0 * self.h, 0.0, 0.0])
        self.bar_dv = np.full(self.Xb.shape[0], dvb)
        grid = B.ibm_grid(wl.nx, wl.ny, wl.nz)
        self._plans = {ph: B.ibm_slab_plan(grid, self.nf, slab, ph) for ph in range(6)}
        ly, lz = wl.ny, wl.nz
        jy = np.arange(ly)[:, None]
        kz = np.arange(lz)[None, :]
        self.lam = (2.0 * np.cos(2.0 * np.pi * jy / ly) - 2.0) + (2.0 * np.cos(2.0 * np.pi * kz / lz) - 2.0)
        pinned = np.zeros((ly, lz), dtype=bool)
        pinned[0, 0] = self.first
        self.pinned = pinned
        self.inv, self.upper = _pivots(self.lam, self.n, self.first, self.last, pinned)
        e = np.zeros((self.n, ly, lz))
        e[0] = 1.0
        self.g1 = _thomas(self.inv, self.upper, e)
        e = np.zeros((self.n, ly, lz))
        e[-1] = 1.0
        self.g2 = _thomas(self.inv, self.upper, e)
        self.initial = False

    def plan(self, phase):
        return self._plans[phase]

    # ----------------------------------------------------------- pressure
    def _rhs(self):
        own = slice(self.gL, self.gL + self.n)
        scale = self.h * self.h / (self.wl.ny * self.wl.nz)
        rhs = self.phi_hat[own] * scale
        rhs[0] = np.where(self.pinned, 0.0, rhs[0])
        return rhs

    def _local(self, D):
        self.phi_hat = dht2(D)
        y = _thomas(self.inv, self.upper, self._rhs())
        g1, g2 = self.g1, self.g2
        out = np.stack([y[0], y[-1], y.sum(0), g1[0], g1[-1], g2[0], g2[-1], g1.sum(0), g2.sum(0)], axis=-1)
        return out.ravel()

    def _reduce(self, gath):
        R = self.slab.nranks
        ny, nz = self.wl.ny, self.wl.nz
        e = np.asarray(gath).reshape(R, ny, nz, 9)
        M = 2 * (R - 1)
        left = np.zeros((ny, nz))
        right = np.zeros((ny, nz))
        if M:
            A = np.zeros((ny, nz, M, M))
            b = np.zeros((ny, nz, M))
            for k in range(R):
                if k >= 1:
                    row = 2 * k - 1
                    A[..., row, row] = 1.0
                    A[..., row, 2 * (k - 1)] += e[k, ..., 3]
                    if k <= R - 2:
                        A[..., row, 2 * k + 1] += e[k, ..., 5]
                    b[..., row] = e[k, ..., 0]
                if k <= R - 2:
                    row = 2 * k
                    A[..., row, row] = 1.0
                    if k >= 1:
                        A[..., row, 2 * (k - 1)] += e[k, ..., 4]
                    A[..., row, 2 * k + 1] += e[k, ..., 6]
                    b[..., row] = e[k, ..., 1]
            sol = np.linalg.solve(A, b[..., None])[..., 0]
            r = self.slab.rank
            if r >= 1:
                left = sol[..., 2 * (r - 1)]
            if r <= R - 2:
                right = sol[..., 2 * r + 1]
        else:
            sol = np.zeros((ny, nz, 0))
        tot = 0.0
        for k in range(R):
            tot += e[k, 0, 0, 2]
            if k >= 1:
                tot -= sol[0, 0, 2 * (k - 1)] * e[k, 0, 0, 7]
            if k <= R - 2:
                tot -= sol[0, 0, 2 * k + 1] * e[k, 0, 0, 8]
        mean = tot / self.wl.nx
        rhs = self._rhs()
        rhs[0] -= left
        rhs[-1] -= right
        x = _thomas(self.inv, self.upper, rhs)
        x[:, 0, 0] -= mean
        ph = np.zeros_like(self.phi_hat)
        ph[self.gL:self.gL + self.n] = x
        self.phi = idht2(ph)

    # ----------------------------------------------------------- phases
    def phase(self, phase, dt, recv):
        import torch
        recv = recv.numpy() if recv is not None else None
        wl, h, nu = self.wl, self.h, self.nu
        nxw, P = self.nxw, wl.ny * wl.nz
        send = None
        if phase == B.IBM_SLAB_INIT:
            send = self._local(mac.divergence(self.u, self.v, self.w, h))
            self.initial = True
        elif phase == B.IBM_SLAB_FORCE:
            u, v, w = self.u, self.v, self.w
            if not self.have_n:
                alpha, beta = 1.0, 0.0
            else:
                alpha, beta = 1.0 + dt / (2.0 * self.dt_old), -dt / (2.0 * self.dt_old)
            un, vn, wn = mac.outflow_convective(u, v, w, dt, h, self.U_IN)
            outs = (un - u[nxw], vn - v[nxw], wn - w[nxw])
            N = mac.advection(u, v, w, h)
            L = mac.laplacian(u, v, w, h)
            G = mac.pressure_gradient(self.p, h)
            rhs = [dt * (-(alpha * N[c] + beta * self.N[c]) - G[c] + nu * L[c]) for c in range(3)]
            r = nu * dt / (2.0 * h * h)
            du, dv, dw = af.af_solve(rhs[0], rhs[1], rhs[2], r, *outs)
            us, vs, ws = u + du, v + dv, w + dw
            us[nxw], vs[nxw], ws[nxw] = un, vn, wn
            shift = np.array([self.x0 * h, 0.0, 0.0])
            parts = [self.X - shift] if self.nf else []
            Xm = np.concatenate(parts + [self.Xb], axis=0)
            F = np.zeros((self.nf, 3))
            if Xm.shape[0]:
                Ustar = ib.interpolate((us, vs, ws), Xm, h, nxw)
                target = np.zeros_like(Ustar)
                dvm = self.bar_dv
                if self.nf:
                    target[:self.nf] = self.V
                    dvm = np.concatenate([self.flag_dv, self.bar_dv])
                coef = (dvm / h ** 3)[:, None] * (target - Ustar)
                ib.spread((us, vs, ws), Xm, coef, h, nxw)
                if self.nf:
                    F = -(target[:self.nf] - Ustar[:self.nf]) / dt * self.flag_dv[:, None]
            if self.nf:
                x = self.X[:, 0]
                own = ((self.first | (x >= self.slab.x_begin * h)) & (self.last | (x < self.slab.x_end * h)))
                F = np.where(own[:, None], F, 0.0)
            q = [us[0].sum() if self.first else 0.0, us[nxw].sum() if self.last else 0.0]
            send = np.concatenate([F.ravel(), q])
            self.us, self.vs, self.ws, self.Nn, self.dt = us, vs, ws, N, dt
            self.initial = False
        elif phase == B.IBM_SLAB_SOLVE:
            nf = self.nf
            if nf:
                F = recv[:3 * nf].reshape(nf, 3)
                self.X, self.V = flag.advance(self.X, self.V, F, self.dt, self.mesh, self.l0)
            qi, qo = recv[3 * nf], recv[3 * nf + 1]
            self.us[nxw] += (qi - qo) * h * h / (wl.ly * wl.lz)
            send = self._local(mac.divergence(self.us, self.vs, self.ws, h) / self.dt)
        elif phase == B.IBM_SLAB_REDUCE:
            self._reduce(recv)
            g, n = self.gL, self.n
            send = np.concatenate([self.phi[g].ravel(), self.phi[g + n - 1].ravel()])
        elif phase == B.IBM_SLAB_PROJECT:
            g, n = self.gL, self.n
            if self.gL > 0:
                self.phi[g - 1] = recv[:P].reshape(wl.ny, wl.nz)
            if self.gR > 0:
                self.phi[g + n] = recv[P:2 * P].reshape(wl.ny, wl.nz)
            gu, gv, gw = mac.pressure_gradient(self.phi, h)
            if self.initial:
                self.u, self.v, self.w = self.u - gu, self.v - gv, self.w - gw
            else:
                dt = self.dt
                self.u, self.v, self.w = self.us - dt * gu, self.vs - dt * gv, self.ws - dt * gw
                self.p = self.p + self.phi - 0.5 * nu * dt * mac.cell_laplacian_neumann(self.phi, h)
                self.N = list(self.Nn)
                self.have_n = True
                self.dt_old = dt
            _, count, _ = self._plans[phase]
            send = np.zeros(count)
            half = count // 2
            gg = self.slab.ghosts
            arrs = [self.u, self.v, self.w, self.p]
            if self.gL > 0:
                pieces = [a[g:g + gg + 1] for a in arrs[:3]] + [self.p[g:g + gg]]
                flat = np.concatenate([q.ravel() for q in pieces])
                send[:flat.size] = flat
            if self.gR > 0:
                pieces = [a[g + n - gg:g + n] for a in arrs]
                flat = np.concatenate([q.ravel() for q in pieces])
                send[half:half + flat.size] = flat
            self.initial = False
        elif phase == B.IBM_SLAB_GHOSTS:
            half = recv.size // 2
            gg = self.slab.ghosts
            arrs = [self.u, self.v, self.w, self.p]
            if self.gL > 0:
                off = 0
                for a in arrs:
                    m = gg * P
                    a[:gg] = recv[off:off + m].reshape((gg,) + a.shape[1:])
                    off += m
            if self.gR > 0:
                off = half
                for i, a in enumerate(arrs):
                    planes = gg + 1 if i < 3 else gg
                    m = planes * P
                    a[a.shape[0] - planes:] = recv[off:off + m].reshape((planes,) + a.shape[1:])
                    off += m
        return torch.from_numpy(np.ascontiguousarray(send, dtype=np.float64)) if send is not None else None

    def owned(self):
        """Owned planes of (u, v, w, p), as ``SlabState.owned_field`` cuts them."""
        lo = self.slab.x_begin - self.x0
        hi = lo + self.n
        hv = hi + (1 if self.last else 0)
        return self.u[lo:hv], self.v[lo:hv], self.w[lo:hv], self.p[lo:hi]
