"""Pressure Poisson equation L_h phi = D (Sec. II.B, projection step).

L_h is div(G .) on cell centres: second differences with d phi/dx = 0 at both
x ends (the velocity on the inflow and outflow faces is not corrected) and
periodic in y and z. The solution is fixed by the gauge mean(phi) = 0.

Method (transforms in the periodic directions, a tridiagonal solve along x):

1. plain O(N^2) forward DFT along y, then along z (complex FP64, twiddles from
   cos/sin of 2 pi j m / N with j m reduced modulo N);
2. for each wavenumber pair (m, n) the x-line problem
       (phi_{i+1} - 2 phi_i + phi_{i-1}) / h^2 + (lam_y(m) + lam_z(n)) phi_i = D_i
   with phi_{-1} = phi_0 and phi_nx = phi_{nx-1}, where
       lam(m) = (2 cos(2 pi m / N) - 2) / h^2
   are the eigenvalues of the periodic second difference; solved by the
   Thomas algorithm (all modes at once, one x position at a time);
3. mode (0, 0) is singular: it is solved with phi_0 = 0 pinned (dense solve of
   the remaining rows), then its x-mean is removed, which sets mean(phi) = 0;
4. inverse DFTs along z and y; the imaginary part is round-off and dropped.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n, sign=-1):
    """W[j, m] = exp(sign * 2 pi i j m / n) with j m reduced modulo n."""
    jm = np.outer(np.arange(n), np.arange(n)) % n
    ang = 2.0 * np.pi * jm / n
    return np.cos(ang) + 1j * sign * np.sin(ang)


def eigenvalues(n, h):
    """Eigenvalues (2 cos(2 pi m / n) - 2) / h^2, m = 0 .. n-1, of the periodic
    second difference that the transverse transforms diagonalise (Sec. II.B:
    transforms in the periodic directions, Sec. II.A: periodic y and z)."""
    m = np.arange(n)
    return (2.0 * np.cos(2.0 * np.pi * m / n) - 2.0) / (h * h)


def thomas(lower, diag, upper, rhs):
    """Thomas algorithm along axis 0, vectorised over the remaining axes.

    lower[i] multiplies x[i-1], upper[i] multiplies x[i+1]; diag may vary per
    line (broadcast against rhs).
    """
    n = rhs.shape[0]
    diag = np.asarray(diag)
    if diag.ndim == 1:
        diag = diag.reshape((n,) + (1,) * (rhs.ndim - 1))
    diag = np.broadcast_to(diag, rhs.shape)
    cp = np.empty(rhs.shape, dtype=float)
    dp = np.empty(rhs.shape, dtype=rhs.dtype)
    denom = diag[0]
    cp[0] = upper[0] / denom
    dp[0] = rhs[0] / denom
    for i in range(1, n):
        denom = diag[i] - lower[i] * cp[i - 1]
        cp[i] = upper[i] / denom
        dp[i] = (rhs[i] - lower[i] * dp[i - 1]) / denom
    x = np.empty_like(dp)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def solve(D, h):
    """Solve L_h phi = D; D has shape (nx, ny, nz). Returns phi (real)."""
    nx, ny, nz = D.shape
    wy = dft_matrix(ny, -1)
    wz = dft_matrix(nz, -1)
    dh = np.einsum("mj,ijk->imk", wy, D.astype(complex), optimize=True)
    dh = np.einsum("nk,imk->imn", wz, dh, optimize=True)

    lam = eigenvalues(ny, h)[:, None] + eigenvalues(nz, h)[None, :]
    inv_h2 = 1.0 / (h * h)
    lower = np.full(nx, inv_h2)
    upper = np.full(nx, inv_h2)
    lower[0] = 0.0
    upper[-1] = 0.0
    base = np.full(nx, -2.0 * inv_h2)
    base[0] = base[-1] = -inv_h2
    if nx == 1:
        base[0] = 0.0
    diag = base[:, None, None] + lam[None, :, :]
    # the singular (0, 0) mode is handled separately below; give its line a
    # harmless diagonal so that the vectorised sweep does not divide by zero
    diag = diag.copy()
    diag[:, 0, 0] = 1.0
    ph = thomas(lower, diag, upper, dh)

    # mode (0, 0): pin phi_0 = 0, solve rows 1..nx-1 densely, remove the mean
    line = dh[:, 0, 0]
    a = np.zeros((nx, nx))
    for i in range(nx):
        a[i, i] = base[i]
        if i > 0:
            a[i, i - 1] = inv_h2
        if i < nx - 1:
            a[i, i + 1] = inv_h2
    a[0, :] = 0.0
    a[0, 0] = 1.0
    b = line.copy()
    b[0] = 0.0
    sol = np.linalg.solve(a, b)
    ph[:, 0, 0] = sol - sol.mean()

    wyi = dft_matrix(ny, +1)
    wzi = dft_matrix(nz, +1)
    out = np.einsum("kn,imn->imk", wzi, ph, optimize=True)
    out = np.einsum("jm,imk->ijk", wyi, out, optimize=True)
    return np.real(out) / (ny * nz)
