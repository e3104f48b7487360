"""Immersed-boundary direct forcing with a regularised delta kernel (Sec. II.B).

The paper forces the flag with a Lagrangian direct-forcing method based on
moving-least-squares (MLS) interpolation. With a linear MLS basis and weights
w_i = delta_h(x_i - X) h^3, the discrete moment conditions of the kernel
(sum w_i = 1, sum w_i (x_i - X) = 0) make the MLS moment matrix the identity
in its constant block, and the MLS shape functions reduce to w_i exactly: on
a uniform grid the MLS interpolation IS delta-kernel interpolation. The bar
grid is forced the same way (markers filling the bars).

Kernel: the three-point kernel of Roma, Peskin and Berger (1999),
    phi(r) = (1 + sqrt(1 - 3 r^2)) / 3                    |r| <= 1/2
    phi(r) = (5 - 3|r| - sqrt(1 - 3 (1 - |r|)^2)) / 6     1/2 <= |r| <= 3/2
    phi(r) = 0                                             otherwise,
delta_h(x) = phi(x/h) phi(y/h) phi(z/h) / h^3.

Forcing (one direct-forcing pass, all markers together):
    U*_l = sum_nodes phi phi phi  u*(node)              (interpolation)
    F_l  = (U_l - U*_l) / dt                             (direct forcing)
    u**  = u* + dt sum_l delta_h(x - X_l) F_l dV_l       (spreading)
Spreading is the adjoint of interpolation in the inner products
<a, b>_grid = h^3 sum a b and <A, B>_markers = sum dV_l A_l B_l.

Readings: nodes outside the unknowns along x (u faces 0 and nx, the v/w ghost
planes) take no part in interpolation or spreading; y and z wrap periodically.
"""
from __future__ import annotations

import math

import numpy as np

# staggered offsets of the u, v, w lattices in units of h
OFFSETS = ((0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))


def roma_phi(r):
    """Three-point regularised delta kernel (one dimension, unit spacing)."""
    a = np.abs(np.asarray(r, dtype=float))
    out = np.zeros_like(a)
    inner = a <= 0.5
    outer = (a > 0.5) & (a < 1.5)
    out[inner] = (1.0 + np.sqrt(1.0 - 3.0 * a[inner] ** 2)) / 3.0
    ao = a[outer]
    out[outer] = (5.0 - 3.0 * ao - np.sqrt(np.maximum(0.0, 1.0 - 3.0 * (1.0 - ao) ** 2))) / 6.0
    return out


def _valid_x_range(comp, nx):
    return (1, nx - 1) if comp == 0 else (0, nx - 1)


def _stencil(X, comp, h, dims):
    """Yield (i, j, k, weight, valid) for the 4x4x4 candidate nodes of each marker."""
    nx, ny, nz = dims
    off = OFFSETS[comp]
    base = [np.floor(X[:, d] / h - off[d]).astype(np.int64) - 1 for d in range(3)]
    lo, hi = _valid_x_range(comp, nx)
    for a in range(4):
        i = base[0] + a
        wx = roma_phi(i + off[0] - X[:, 0] / h)
        for b in range(4):
            j = base[1] + b
            wy = roma_phi(j + off[1] - X[:, 1] / h)
            for c in range(4):
                k = base[2] + c
                wz = roma_phi(k + off[2] - X[:, 2] / h)
                valid = (i >= lo) & (i <= hi)
                yield i, np.mod(j, ny), np.mod(k, nz), wx * wy * wz, valid


def interpolate(fields, X, h, nx):
    """U*_l for all markers; fields = (u, v, w) full arrays. Returns (M, 3)."""
    M = X.shape[0]
    out = np.zeros((M, 3))
    dims = (nx, fields[0].shape[1], fields[0].shape[2])
    for comp in range(3):
        q = fields[comp]
        for i, j, k, wgt, valid in _stencil(X, comp, h, dims):
            ii = np.where(valid, i, 0)
            out[:, comp] += np.where(valid, wgt * q[ii, j, k], 0.0)
    return out


def spread(fields, X, coef, h, nx):
    """fields[c][node] += sum_l phi phi phi * coef[l, c] (in place).

    For the forcing step coef = dV_l / h^3 * (U_l - U*_l) (= dt F_l dV_l / h^3).
    """
    dims = (nx, fields[0].shape[1], fields[0].shape[2])
    for comp in range(3):
        q = fields[comp]
        for i, j, k, wgt, valid in _stencil(X, comp, h, dims):
            sel = valid
            np.add.at(q, (i[sel], j[sel], k[sel]), wgt[sel] * coef[sel, comp])


def bar_markers(wl, h):
    """Markers filling the passive grid of square bars (Sec. II.A geometry).

    Bars of side d lie in the plane x = bar_x: rods along y centred at
    z = (r + 1/2) M and rods along z centred at y = (r + 1/2) M. Each rod is
    filled with a lattice of n_w = ceil(d/h) + 1 points across each of its two
    short sides and n_along = ceil(L_along / h) points along it, at
    (m + 1/2) L_along / n_along. Points of the y-rods that fall inside a z-rod
    (the crossings) are dropped so that no volume is sampled twice. Every
    marker carries the same volume dV = (union volume of the bars) / count.

    Returns (X (M, 3), dV scalar).
    """
    d = wl.bar_width
    M = wl.bar_mesh
    ny_r = int(round(wl.ly / M))
    nz_r = int(round(wl.lz / M))
    n_w = int(math.ceil(d / h - 1e-12)) + 1
    across = d * (np.arange(n_w) / (n_w - 1) - 0.5)
    xs = wl.bar_x + across
    yc = (np.arange(ny_r) + 0.5) * M          # centres of rods along z
    zc = (np.arange(nz_r) + 0.5) * M          # centres of rods along y
    n_ay = int(math.ceil(wl.ly / h - 1e-12))
    n_az = int(math.ceil(wl.lz / h - 1e-12))
    ya = (np.arange(n_ay) + 0.5) * wl.ly / n_ay
    za = (np.arange(n_az) + 0.5) * wl.lz / n_az

    pts = []
    # rods along y (centred in z at zc), minus the crossings with rods along z
    for z0 in zc:
        for x in xs:
            for z in z0 + across:
                for y in ya:
                    dy = np.abs(((y - yc) + 0.5 * wl.ly) % wl.ly - 0.5 * wl.ly)
                    if np.any(dy <= 0.5 * d + 1e-12):
                        continue
                    pts.append((x, y, z))
    # rods along z (centred in y at yc), complete
    for y0 in yc:
        for x in xs:
            for y in y0 + across:
                for z in za:
                    pts.append((x, y, z))
    X = np.array(pts, dtype=float)
    volume = d * d * (ny_r * wl.lz + nz_r * wl.ly) - ny_r * nz_r * d ** 3
    return X, volume / X.shape[0]


def bar_volume_fraction(wl, comp, h):
    """Eulerian forcing of the bar grid (Sec. II.B: the fixed grid is forced
    on Eulerian nodes, after Fadlun et al.), read as a volume-fraction direct
    forcing: each velocity node of component `comp` carries the fraction
    alpha of its cell [x - h/2, x + h/2]^3 that lies inside the bars, and the
    forcing sets u** = (1 - alpha) u* (zero inside the solid).

    The solid is the union of the rods of the bar_markers geometry: square
    rods of side d in the slab |x - bar_x| <= d/2, along y centred at
    z = (r + 1/2) M and along z centred at y = (r + 1/2) M (periodic in y, z).
    With ox, oy, oz the overlaps of the cell with the slab and with the rods
    across y and z, |cell and (Y-rods or Z-rods)| = ox (h oz + oy h - oy oz).

    Returns alpha with the shape of the component's field, (nx + 1, ny, nz),
    zero on the planes that are not unknowns (u faces 0 and nx, v/w plane nx).
    """
    nx, ny, nz = wl.nx, wl.ny, wl.nz
    d, M = wl.bar_width, wl.bar_mesh

    def overlap(c, lo, hi):
        return np.clip(np.minimum(c + 0.5 * h, hi) - np.maximum(c - 0.5 * h, lo), 0.0, None)

    def rods(c, centres, period):
        o = np.zeros_like(c)
        for c0 in centres:
            for img in (-period, 0.0, period):
                o += overlap(c, c0 + img - 0.5 * d, c0 + img + 0.5 * d)
        return o

    i = np.arange(nx + 1)
    x = i * h if comp == 0 else (i + 0.5) * h
    y = np.arange(ny) * h if comp == 1 else (np.arange(ny) + 0.5) * h
    z = np.arange(nz) * h if comp == 2 else (np.arange(nz) + 0.5) * h
    ox = overlap(x, wl.bar_x - 0.5 * d, wl.bar_x + 0.5 * d)
    oy = rods(y, (np.arange(int(round(wl.ly / M))) + 0.5) * M, wl.ly)
    oz = rods(z, (np.arange(int(round(wl.lz / M))) + 0.5) * M, wl.lz)
    alpha = ox[:, None, None] * (h * oz[None, None, :] + oy[None, :, None] * h
                                 - oy[None, :, None] * oz[None, None, :]) / h ** 3
    lo, hi = _valid_x_range(comp, nx)
    alpha[:lo] = 0.0
    alpha[hi + 1:] = 0.0
    return alpha
