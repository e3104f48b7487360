"""Laminar flag validation helpers (CPU): the oscillation analysis against a
synthetic trailing-edge signal and the workloads' geometry."""
import numpy as np

from paper_2103_08246_gb300 import inputs, validation


def test_flag_oscillation_of_a_synthetic_signal():
    t = np.linspace(0.0, 30.0, 6000)
    te = np.stack([3.0 + 0.01 * np.sin(t), 2.0 + 0.01 * t * 0, 2.0 + 0.3 * np.sin(2 * np.pi * 0.25 * t)], axis=1)
    out = validation.flag_oscillation(t, te)
    assert out["component"] == 2
    assert abs(out["strouhal"] - 0.25) < 0.003
    assert abs(out["period"] - 4.0) < 0.05
    assert abs(out["amplitude"] - 0.3) < 1e-3


def test_laminar_workloads():
    fine = validation.laminar_workload(64)
    coarse = validation.laminar_workload(32)
    p = inputs.PRODUCTION
    assert (fine.nx, fine.ny, fine.nz) == (p.nx, p.ny, p.nz) and not fine.bars_on and fine.flag_on
    assert (coarse.nx, coarse.ny, coarse.nz) == (256, 128, 128)
    for wl, n in ((fine, 64), (coarse, 32)):
        assert abs(wl.lx / wl.nx - 1.0 / n) < 1e-12 and abs(wl.ly / wl.ny - 1.0 / n) < 1e-12
        assert wl.flag_ns == wl.flag_nt == n + 1


def test_inside_rods_mask():
    wl = inputs.PRODUCTION
    h = wl.lx / wl.nx
    i = int(round(wl.bar_x / h))            # u face at x = bar_x, mid-slab
    m = validation._inside_rods(wl, 0, i)
    # rods of width 0.1 = 6.4 cells, centred at (r + 1/2) M between cell
    # centres: 6 whole cells across each rod, 8 rods per direction
    full = 6 * 8 / 256
    assert abs(m.mean() - (2 * full - full * full)) < 1e-12
    assert m[int(0.25 / h), :].all() and m[:, int(0.25 / h)].all()
    assert not validation._inside_rods(wl, 0, i + 10).any()


def test_cycle_statistics_of_a_synthetic_signal():
    """Zero-crossing period and per-cycle amplitude of a sampled sine with an
    offset: exact to the interpolation error of the crossings, far below a
    periodogram bin (1 / record length = 0.025 here)."""
    t = np.linspace(0.0, 40.0, 2001)
    y = 0.05 + 0.2 * np.sin(2 * np.pi * t / 4.5 + 0.7)
    out = validation.cycle_statistics(t, y)
    assert out["cycles"] == 7
    assert abs(out["period"] - 4.5) < 1e-4
    assert abs(out["amplitude"] - 0.2) < 1e-3
    # a growing oscillation: the mean per-cycle amplitude, not the largest
    g = np.sin(2 * np.pi * t / 4.0) * (1.0 + 0.01 * t)
    out = validation.cycle_statistics(t, g)
    assert abs(out["period"] - 4.0) < 2e-3 and out["amplitude_std"] > 0


def test_cycle_statistics_ignores_harmonics():
    """A second harmonic strong enough to add zero crossings of its own
    leaves the period and the cycle count unchanged."""
    t = np.linspace(0.0, 45.0, 9001)
    y = np.sin(2 * np.pi * t / 4.5) + 0.8 * np.sin(2 * np.pi * 2 * t / 4.5)
    naive = np.count_nonzero((y[:-1] < 0) & (y[1:] >= 0))
    out = validation.cycle_statistics(t, y)
    assert naive >= 19
    assert out["cycles"] == 8 and abs(out["period"] - 4.5) < 1e-3
