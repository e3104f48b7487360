"""Host statistics of the learned-inflow campaign (CPU): the z spectrum, the
decay-exponent fit, the Strouhal estimate and the station accumulators
against closed forms, the bounds logic, and the driven domain's geometry."""
import numpy as np

from paper_2103_08246_gb300 import inflow, inputs


def test_spectrum_of_a_cosine_and_parseval():
    nz = 64
    z = np.arange(nz)
    plane = np.tile(2.0 + 0.5 * np.cos(2 * np.pi * 5 * z / nz + 0.3), (4, 1))
    e = inflow.spectrum_z(plane)
    assert e.shape == (nz // 2 + 1,)
    assert abs(e[5] - 0.125) < 1e-12 and np.abs(np.delete(e, 5)).max() < 1e-12
    a = np.random.default_rng(0).standard_normal((6, nz))
    assert abs(inflow.spectrum_z(a).sum() - ((a - a.mean()) ** 2).mean()) < 1e-12 * 10


def test_decay_exponent_recovers_a_power_law():
    x = np.array([1.5, 2.0, 2.5, 2.9])
    assert abs(inflow.decay_exponent(x, 3.0 * (x - 0.5) ** -1.3, 0.5) - 1.3) < 1e-12


def test_strouhal_of_a_sinusoid_on_uneven_times():
    rng = np.random.default_rng(1)
    t = np.cumsum(rng.uniform(0.8, 1.2, 4000)) * 0.01
    y = 0.3 + np.sin(2 * np.pi * 0.2 * t)
    st, rms = inflow.strouhal(t, y, length=1.0, speed=1.0)
    assert abs(st - 0.2) < 0.002
    assert abs(rms - np.sqrt(0.5)) < 0.01


def test_station_stats_turbulence_intensity():
    rng = np.random.default_rng(2)
    st = inflow.StationStats(2, 16)
    for _ in range(400):
        u = 1.0 + 0.1 * rng.standard_normal((8, 16))
        st.add([(u, 0.1 * rng.standard_normal((8, 16)), 0.1 * rng.standard_normal((8, 16))),
                (np.ones((8, 16)), np.zeros((8, 16)), np.zeros((8, 16)))])
    tu = st.tu()
    assert abs(tu[0] - 0.1) < 0.005 and tu[1] == 0.0


def test_compare_and_bounds():
    R = {"tu": [0.1, 0.08, 0.07], "spectrum_u": list(np.linspace(1, 0.01, 40)), "strouhal": 0.2, "y_rms": 0.1}
    G = {"tu": [0.1, 0.079, 0.072], "spectrum_u": list(np.linspace(1, 0.01, 40) * 1.1), "strouhal": 0.21,
         "y_rms": 0.11}
    U = {"tu": [1e-6, 1e-6, 1e-6], "spectrum_u": list(np.full(40, 1e-12)), "strouhal": 0.3, "y_rms": 0.3}
    out = inflow.compare({"R": R, "G": G, "U": U}, [2.03, 2.5, 2.89], 0.5)
    assert all(out["G_within_bounds"].values())
    assert out["G_better_than"]["tu_flag_station_vs_U"] and out["G_better_than"]["y_rms_vs_U"]


def test_driven_domain_geometry():
    d = inflow.driven_workload(inputs.PRODUCTION)
    p = inputs.PRODUCTION
    assert (d.nx, d.ny, d.nz) == (384, 256, 256)
    assert abs(d.lx - 6.0) < 1e-12 and not d.bars_on and d.flag_on
    assert abs(d.flag_x_le - 1.0) < 1e-12
    assert abs((p.lx - p.flag_x_le) - (d.lx - d.flag_x_le)) < 1e-12
