"""Taylor-Green decay through the oracle's full time step (Sec. II.B).

The inflow/outflow domain admits no 3-D Taylor-Green vortex, but the
transverse plane is periodic (Sec. II.A): a Taylor-Green vortex in y-z,
uniform in x, on top of the uniform inflow, with its inflow plane prescribed
from the same pattern, is an exact solution of the discrete step away from
the outflow. Its velocity comes from a discrete stream function
psi = A sin(k y) sin(k z) on the x-parallel cell edges (v = d psi/dz,
w = -d psi/dy by differences), so it is divergence-free on the MAC grid; at
A = 1e-9 the nonlinear terms are below round-off relative to the decay.
Each step multiplies the mode by the factor of the approximately factorised
Crank-Nicolson step,
    g = 1 - 2 r (ly + lz) / ((1 + r ly)(1 + r lz)),   r = nu dt / 2,
    ly = lz = (4 / h^2) sin^2(k h / 2)   (the discrete Laplacian's eigenvalue).
After 20 steps the amplitude upstream of the outflow equals g^20 to 1e-9;
the test resolves the alternatives (unfactorised Crank-Nicolson, explicit
diffusion, the continuum rate exp(-2 nu k^2 dt)), which differ by more.
"""
import numpy as np

from oracle.solver import OracleSolver
from paper_2103_08246_gb300 import inputs

NX, NY, NZ = 32, 8, 8
A0 = 1e-9
DT = 0.01
STEPS = 20


def _setup():
    wl = inputs.small(NX, NY, NZ, re=100.0)     # h = 1/4, ly = lz = 2
    h = wl.lx / NX
    k = 2 * np.pi / wl.ly
    yf = np.arange(NY) * h
    zf = np.arange(NZ) * h
    yc, zc = yf + h / 2, zf + h / 2
    s2 = 2 * np.sin(k * h / 2) / h
    pv = A0 * s2 * np.sin(k * yf)[:, None] * np.cos(k * zc)[None, :]
    pw = -A0 * s2 * np.cos(k * yc)[:, None] * np.sin(k * zf)[None, :]
    shape = (NX + 1, NY, NZ)
    v = np.broadcast_to(pv, shape).copy()
    w = np.broadcast_to(pw, shape).copy()
    return wl, h, k, pv, pw, v, w


def _factors(wl, h, k):
    nu = 1.0 / wl.re
    lam = (4 / h ** 2) * np.sin(k * h / 2) ** 2
    r = nu * DT / 2
    g = 1 - 2 * r * (2 * lam) / ((1 + r * lam) ** 2)
    alternatives = {
        "unfactorised Crank-Nicolson": (1 - r * 2 * lam) / (1 + r * 2 * lam),
        "explicit diffusion": 1 - 2 * r * 2 * lam,
        "continuum rate": np.exp(-2 * nu * k * k * DT),
    }
    return g, alternatives


def test_taylor_green_decays_at_the_discrete_rate():
    wl, h, k, pv, pw, v, w = _setup()
    s = OracleSolver(wl, [np.zeros_like(v), v, w])
    # the initial projection leaves the discretely divergence-free field alone
    assert np.abs(s.v - v).max() < 1e-14 * A0 and np.abs(s.w - w).max() < 1e-14 * A0
    s.v_in, s.w_in = pv.copy(), pw.copy()      # the inflow plane carries the pattern
    g, alternatives = _factors(wl, h, k)
    ones = np.ones((NY, NZ))
    for n in range(1, STEPS + 1):
        s.set_inflow(ones, pv * g ** n, pw * g ** n)
        s.step(DT)
    pred = g ** STEPS
    up = slice(2, 12)                            # x in (0.5, 3); the outflow is at x = 8
    amp_v = (s.v[up] * pv).sum() / (pv * pv).sum() / 10
    amp_w = (s.w[up] * pw).sum() / (pw * pw).sum() / 10
    assert abs(amp_v - pred) < 1e-9 * pred and abs(amp_w - pred) < 1e-9 * pred, (amp_v, amp_w, pred)
    # the field keeps its shape
    scale = A0 * 2 * np.sin(k * h / 2) / h * pred
    assert np.abs(s.v[up] - pred * pv).max() < 1e-8 * scale
    assert np.abs(s.w[up] - pred * pw).max() < 1e-8 * scale
    # the uniform inflow velocity is untouched
    assert np.abs(s.u[1:NX] - 1.0).max() < 1e-12
    # each alternative rate would miss the measured amplitude by far more
    for name, ga in alternatives.items():
        assert abs(ga ** STEPS - amp_v) > 5e-9 * pred, name
