"""Pins for the oracle's immersed-boundary kernel, interpolation, spreading
and marker geometry (Sec. II.B; the geometry of Sec. II.A).

* the three-point kernel satisfies its defining moment conditions
  (sum phi = 1, sum r phi = 0, sum phi^2 = 1/2 for every shift; fixture
  tests/golden/roma_kernel_moments.txt);
* with those moments the linear-basis MLS shape functions equal the kernel
  weights (the reading that makes the paper's MLS forcing delta-kernel
  forcing);
* interpolation reproduces linear fields exactly on each staggered lattice
  (a wrong staggering offset fails);
* spreading is the adjoint of interpolation:
  h^3 <u, S F> = sum dV <I u, F> to 1e-13 relative;
* bar markers: count, containment, no duplicates, volume.
"""
import math
import os

import numpy as np

from oracle import ib
from paper_2103_08246_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def test_kernel_moment_conditions():
    g = _read_golden("roma_kernel_moments.txt")
    rng = np.random.default_rng(0)
    for r in rng.uniform(-3, 3, 200):
        j = np.arange(math.floor(r) - 3, math.floor(r) + 4)
        ph = ib.roma_phi(r - j)
        assert abs(ph.sum() - g["sum_phi"]) < 1e-14
        assert abs(((r - j) * ph).sum() - g["sum_r_phi"]) < 1e-14
        assert abs((ph ** 2).sum() - g["sum_phi_squared"]) < 1e-14
    assert ib.roma_phi(np.array([1.5]))[0] == 0.0
    assert abs(ib.roma_phi(np.array([0.0]))[0] - 2.0 / 3.0) < 1e-15


def test_mls_linear_basis_reduces_to_kernel_weights():
    # MLS with basis p = [1, dx, dy, dz] and weights w_i = phi phi phi:
    # shape_i = p(X)^T A^{-1} w_i p(x_i) with A = sum w_i p(x_i) p(x_i)^T
    rng = np.random.default_rng(1)
    for _ in range(20):
        X = rng.uniform(3, 5, 3)
        base = np.floor(X) - 1
        nodes = np.array([[base[0] + a, base[1] + b, base[2] + c]
                          for a in range(4) for b in range(4) for c in range(4)], float)
        w = np.prod([ib.roma_phi(nodes[:, d] - X[d]) for d in range(3)], axis=0)
        P = np.concatenate([np.ones((len(nodes), 1)), nodes - X], axis=1)
        A = (w[:, None, None] * P[:, :, None] * P[:, None, :]).sum(axis=0)
        pX = np.array([1.0, 0, 0, 0])
        shape = (P @ np.linalg.solve(A, pX)) * w
        np.testing.assert_allclose(shape, w, atol=1e-14)


def _grid(nx=12, ny=10, nz=8, h=0.5):
    return nx, ny, nz, h


def test_interpolation_exact_for_linear_fields():
    nx, ny, nz, h = _grid()
    coef = np.array([0.3, -0.7, 0.45, 1.1])
    rng = np.random.default_rng(2)
    # keep markers away from the periodic seam (linear fields are not periodic)
    X = np.stack([rng.uniform(3 * h, (nx - 3) * h, 50),
                  rng.uniform(3 * h, (ny - 3) * h, 50),
                  rng.uniform(3 * h, (nz - 3) * h, 50)], axis=1)
    fields = []
    for comp in range(3):
        off = ib.OFFSETS[comp]
        i = np.arange(nx + 1)[:, None, None]
        j = np.arange(ny)[None, :, None]
        k = np.arange(nz)[None, None, :]
        f = coef[0] + coef[1] * (i + off[0]) * h + coef[2] * (j + off[1]) * h + coef[3] * (k + off[2]) * h
        fields.append(np.broadcast_to(f, (nx + 1, ny, nz)).copy() * (comp + 1))
    U = ib.interpolate(fields, X, h, nx)
    exact = coef[0] + X @ coef[1:]
    for comp in range(3):
        np.testing.assert_allclose(U[:, comp], exact * (comp + 1), atol=1e-12)


def test_spreading_is_adjoint_of_interpolation():
    nx, ny, nz, h = _grid()
    rng = np.random.default_rng(3)
    M = 40
    # include markers that wrap through the periodic y, z seams
    X = np.stack([rng.uniform(2 * h, (nx - 2) * h, M),
                  rng.uniform(0, ny * h, M), rng.uniform(0, nz * h, M)], axis=1)
    dV = rng.uniform(0.5, 2.0, M) * h ** 3
    u = [rng.standard_normal((nx + 1, ny, nz)) for _ in range(3)]
    F = rng.standard_normal((M, 3))
    SF = [np.zeros((nx + 1, ny, nz)) for _ in range(3)]
    ib.spread(SF, X, (dV / h ** 3)[:, None] * F, h, nx)
    lhs = h ** 3 * sum((u[c] * SF[c]).sum() for c in range(3))
    rhs = (dV[:, None] * ib.interpolate(u, X, h, nx) * F).sum()
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_spreading_conserves_total_force():
    nx, ny, nz, h = _grid()
    rng = np.random.default_rng(4)
    X = np.stack([rng.uniform(3 * h, (nx - 3) * h, 30),
                  rng.uniform(0, ny * h, 30), rng.uniform(0, nz * h, 30)], axis=1)
    coef = rng.standard_normal((30, 3))
    SF = [np.zeros((nx + 1, ny, nz)) for _ in range(3)]
    ib.spread(SF, X, coef, h, nx)
    for c in range(3):
        assert abs(SF[c].sum() - coef[:, c].sum()) < 1e-12


def test_bar_markers_geometry():
    wl = inputs.TINY
    h = wl.lx / wl.nx
    X, dv = ib.bar_markers(wl, h)
    d, M = wl.bar_width, wl.bar_mesh
    n_w = math.ceil(d / h) + 1                   # 3 at h = 1/16, d = 0.1
    n_rod = round(wl.ly / M)
    along = wl.ny
    # crossings drop the y-rod points with |y - yc| <= d/2 (2 per crossing at this spacing)
    ya = (np.arange(along) + 0.5) * wl.ly / along
    drop = int(np.sum(np.abs(ya - 0.25) <= d / 2 + 1e-12))
    expected = 2 * n_rod * n_w * n_w * along - n_rod * n_rod * n_w * n_w * drop
    assert X.shape == (expected, 3)
    assert len({tuple(np.round(p, 12)) for p in X}) == X.shape[0]
    assert np.all(np.abs(X[:, 0] - wl.bar_x) <= d / 2 + 1e-12)
    # every marker lies inside a rod along y or a rod along z
    centres = (np.arange(n_rod) + 0.5) * M
    in_y_rod = np.min(np.abs(X[:, 2][:, None] - centres[None]), axis=1) <= d / 2 + 1e-12
    in_z_rod = np.min(np.abs(X[:, 1][:, None] - centres[None]), axis=1) <= d / 2 + 1e-12
    assert np.all(in_y_rod | in_z_rod)
    volume = d * d * n_rod * (wl.ly + wl.lz) - n_rod * n_rod * d ** 3
    assert abs(dv * X.shape[0] - volume) < 1e-12


def test_bar_volume_fraction():
    """Eulerian bar forcing: the fractions sum to the exact solid volume of
    the bars (union of the rods), lie in [0, 1], are 1 at the rod centre
    lines and 0 away from the grid, and respect the rods' symmetry."""
    from oracle import ib as oib
    from paper_2103_08246_gb300 import inputs
    for h, d in ((0.125, 0.1), (0.0625, 0.1), (0.0625, 0.25)):
        wl = inputs.small(32, 16, 16, bars_on=True, bar_x=1.0, bar_width=d).replace(
            lx=32 * h, ly=16 * h, lz=16 * h)
        M = wl.bar_mesh
        nr_y, nr_z = int(round(wl.ly / M)), int(round(wl.lz / M))
        exact = d * d * (nr_y * wl.lz + nr_z * wl.ly) - nr_y * nr_z * d ** 3
        for comp in range(3):
            a = oib.bar_volume_fraction(wl, comp, h)
            assert a.shape == (wl.nx + 1, wl.ny, wl.nz)
            assert a.min() >= 0.0 and a.max() <= 1.0 + 1e-12
            assert abs(a.sum() * h ** 3 - exact) < 1e-12 * max(exact, 1.0)
    # a node on a rod's centre line inside the slab is fully solid, one far away empty
    h = 1.0 / 64
    wl = inputs.small(128, 64, 64, bars_on=True, bar_x=1.0).replace(lx=2.0, ly=1.0, lz=1.0)
    a = oib.bar_volume_fraction(wl, 1, h)      # v at ((i + 1/2) h, j h, (k + 1/2) h)
    i = int(round(1.0 / h - 0.5))              # x = 1 - h/2 ... inside the slab of width 0.1
    k = int(round(0.25 / h - 0.5))             # z = 0.25 - h/2 near the centre of a y-rod
    assert a[i, 5, k] == 1.0
    assert a[i - 20, 5, k] == 0.0
    # z-rods and y-rods are the same solid turned by 90 degrees
    au, av, aw = (oib.bar_volume_fraction(wl, c, h) for c in range(3))
    assert np.allclose(av, np.transpose(aw, (0, 2, 1)), atol=0)
