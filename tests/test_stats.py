"""Grid-turbulence statistics from probe histories (CPU): closed forms on
frozen sinusoidal turbulence, the integral scale of an exponentially
correlated signal, the decay fit, and the probe layout."""
import numpy as np

from paper_2103_08246_gb300 import inputs, stats


def test_frozen_sinusoid_statistics():
    rng = np.random.default_rng(0)
    U, a, kap, nu = 1.2, 0.05, 8.0, 1e-3
    t = np.cumsum(rng.uniform(0.9, 1.1, 20000)) * 2e-3
    ph = rng.uniform(0, 2 * np.pi, 5)
    u = U + a * np.sin(kap * (0.0 - U * t[:, None]) + ph[None, :])
    v = 0.5 * a * np.cos(kap * U * t[:, None] + ph[None, :])
    w = np.zeros_like(v)
    st = stats.station_statistics(t, u, v, w, nu)
    assert abs(st["U"] - U) < 1e-3
    assert abs(st["u_rms"] - a / np.sqrt(2)) < 1e-3 * a
    assert abs(st["lambda_f"] - np.sqrt(2) / kap) < 2e-3 * (np.sqrt(2) / kap)
    assert abs(st["eps"] - 15 * nu * a * a * kap * kap / 2) < 5e-3 * (15 * nu * a * a * kap * kap / 2)
    assert abs(st["k"] - 0.5 * (a * a / 2 + a * a / 8)) < 1e-3 * st["k"]


def test_integral_scale_of_an_exponential_correlation():
    rng = np.random.default_rng(1)
    dt, tau, n = 0.01, 0.5, 400000
    phi = np.exp(-dt / tau)
    x = np.zeros(n)
    e = rng.standard_normal(n) * np.sqrt(1 - phi * phi)
    for i in range(1, n):
        x[i] = phi * x[i - 1] + e[i]
    t = np.arange(n) * dt
    U = 2.0
    st = stats.station_statistics(t, (U + 0.1 * x)[:, None], np.zeros((n, 1)), np.zeros((n, 1)), 1e-3)
    assert abs(st["L"] - U * tau) < 0.1 * U * tau


def test_decay_fit():
    x = np.linspace(3.0, 8.0, 20)
    n, A = stats.decay_fit(x, 0.7 * (x - 0.5) ** -1.4, 0.5, 3.0)
    assert abs(n - 1.4) < 1e-10 and abs(A - 0.7) < 1e-10


def test_probe_layout():
    wl = inputs.PRODUCTION
    cells, x = stats.probe_cells(wl)
    h = wl.lx / wl.nx
    assert cells.shape[1] == 3 and cells.shape[0] == 9 * len(x)
    assert cells[:, 0].min() * h > wl.bar_x + wl.bar_width and cells[:, 0].max() < wl.nx
    assert len(set(map(tuple, cells[:9, 1:]))) == 9
