"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64: relative max-norm error <= 1e-9 per field (u, v, w, gauge-fixed p) and
for the flag positions/velocities, after up to 100 steps, including the tiny
workload (64 x 32 x 32, bars + flag, dt = 2e-3) for 100 steps. Only rounding
order differs between the two (atomic spreading order, FFT vs plain DFT,
closed-form vs recursive pivots), so 1e-9 leaves a wide margin over the
~1e-13 seen per step.

FP32: the same workloads, errors measured against the natural scales
(velocity U = 1, pressure U^2 = 1, flag positions L = 1, flag velocity U)
because the noise-driven pressure and flag velocity are themselves near
zero. Derivation of the bound: each field operation rounds to
eps = 2^-24 ~ 6e-8; the divergence of O(U) face values carries an error
~eps U / h, so D = div / dt carries eps U / (h dt) and phi (~h^2 D / 6 for the
high modes that white rounding noise excites) eps U h / (6 dt) per step,
~1.3e-6 U^2 at h = 1/4, dt = 2e-3; p accumulates phi over the steps. Velocity
errors stay near eps times the number of operations per step. Bounds used:
2e-5 for velocities and flag quantities, 2e-4 for p, after 10-20 steps
(about 10x above the measured values).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def _rel(g, o):
    return np.abs(g - o).max() / max(np.abs(o).max(), 1e-300)


def _compare(gpu, ora, tol, flag=True, floor=None):
    """Max-norm error of each quantity divided by max(|oracle|, floor[q]).

    tol: a number, or a dict per quantity. floor None: pure relative error."""
    floor = floor or {}
    errs = {}
    for name, g, o in zip("uvwp", gpu.fields(), ora.fields()):
        if name == "p":
            g, o = g - g.mean(), o - o.mean()
        errs[name] = np.abs(g - o).max() / max(np.abs(o).max(), floor.get(name, 1e-300))
    if flag and ora.nf:
        X, V, F = gpu.flag()
        errs["X"] = np.abs(X - ora.X).max() / max(np.abs(ora.X).max(), floor.get("X", 1e-300))
        errs["V"] = np.abs(V - ora.V).max() / max(np.abs(ora.V).max(), floor.get("V", 1e-30))
        errs["F"] = np.abs(F - ora.F_flag).max() / max(np.abs(ora.F_flag).max(), 1e-30)
    tols = tol if isinstance(tol, dict) else {k: tol for k in errs}
    bad = {k: v for k, v in errs.items() if not v <= tols[k]}
    assert not bad, (errs, tols)
    return errs


FP32_FLOOR = {"u": 1.0, "v": 1.0, "w": 1.0, "p": 1.0, "X": 1.0, "V": 1.0}
FP32_TOL = {"u": 2e-5, "v": 2e-5, "w": 2e-5, "p": 2e-4, "X": 2e-5, "V": 2e-5, "F": 2e-4}


def _run(wl, precision, nsteps, amp=0.05, dt=None):
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import binding, inputs
    noise = inputs.initial_noise(wl, amp=amp)
    gpu = binding.Solver(wl, precision, noise=noise)
    ora = OracleSolver(wl, noise)
    gpu.step(nsteps, dt)
    ora.run(nsteps, dt if dt is not None and dt > 0 else None)
    return gpu, ora


def _small(**kw):
    from paper_2103_08246_gb300 import inputs
    nx, ny, nz = kw.pop("shape", (16, 8, 8))
    return inputs.small(nx, ny, nz, **kw)


FLAG = dict(flag_on=True, flag_x_le=2.0, flag_ns=5, flag_nt=5, flag_len=1.0, flag_span=1.0)


@pytest.mark.parametrize("case", ["plain", "ragged", "bars", "flag", "bars_flag"])
def test_fp64_small_cases(lib, case):
    from paper_2103_08246_gb300 import binding
    kw = {"plain": {}, "ragged": dict(shape=(20, 8, 16)), "bars": dict(bars_on=True, bar_x=1.0),
          "flag": dict(FLAG), "bars_flag": dict(bars_on=True, bar_x=1.0, **FLAG)}[case]
    wl = _small(**kw)
    gpu, ora = _run(wl, binding.IBM_FP64, 10)
    _compare(gpu, ora, 1e-9)
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_wide_transverse_grid(lib, precision):
    """256 x 256 transverse planes (the size the register-resident and
    cluster transforms, the tensor-core (tcgen05) transform GEMMs and the
    streamed kernels are specialised for), 16 x-planes, 3 steps."""
    from paper_2103_08246_gb300 import binding
    prec = {"fp64": binding.IBM_FP64, "fp32": binding.IBM_FP32, "mixed": binding.IBM_MIXED}[precision]
    wl = _small(shape=(16, 256, 256))
    gpu, ora = _run(wl, prec, 3)
    if prec == binding.IBM_FP64:
        _compare(gpu, ora, 1e-9)
    else:
        _compare(gpu, ora, FP32_TOL, floor=FP32_FLOOR)
    gpu.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_eulerian_bar_forcing(lib, precision):
    """The bars forced on the Eulerian nodes (solid volume fraction) instead of
    markers, with the flag's markers: FP64 to 1e-9, FP32 to its bounds; the
    Eulerian forcing costs a fraction of the markers' (no gathers, no
    atomics)."""
    from paper_2103_08246_gb300 import binding
    prec = {"fp64": binding.IBM_FP64, "fp32": binding.IBM_FP32, "mixed": binding.IBM_MIXED}[precision]
    wl = _small(shape=(24, 16, 16), bars_on=True, bar_x=1.5, bar_forcing="eulerian", **FLAG)
    gpu, ora = _run(wl, prec, 10)
    if prec == binding.IBM_FP64:
        _compare(gpu, ora, 1e-9)
    else:
        _compare(gpu, ora, FP32_TOL, floor=FP32_FLOOR)
    assert gpu.markers().shape[0] == wl.flag_ns * wl.flag_nt
    gpu.close()


def test_fp64_single_step_each_stage(lib):
    from paper_2103_08246_gb300 import binding
    wl = _small(bars_on=True, bar_x=1.0, **FLAG)
    gpu, ora = _run(wl, binding.IBM_FP64, 1)
    errs = _compare(gpu, ora, 1e-11)
    assert errs["u"] < 1e-11
    gpu.close()


def test_fp64_cfl_mode(lib):
    from paper_2103_08246_gb300 import binding
    wl = _small(dt=-1.0, cfl=0.3, bars_on=True, bar_x=1.0)
    gpu, ora = _run(wl, binding.IBM_FP64, 8)
    st = gpu.stats()
    assert abs(st["dt"] - ora.last_dt) <= 1e-12 * ora.last_dt
    assert abs(st["t"] - ora.t) <= 1e-12 * ora.t
    _compare(gpu, ora, 1e-9)
    gpu.close()


def test_fp64_tiny_workload_100_steps(lib):
    """The tiny workload of the paper's setup (bars + 17x17 flag), 100 steps."""
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.TINY
    gpu, ora = _run(wl, binding.IBM_FP64, wl.steps, amp=wl.noise_amp)
    errs = _compare(gpu, ora, 1e-9)
    st = gpu.stats()
    assert st["step"] == wl.steps and st["n_markers"] == ora.nf + ora.Xb.shape[0]
    assert st["max_div"] < 1e-9
    gpu.close()
    print("tiny workload FP64 errors:", errs)


@pytest.mark.parametrize("case", ["plain", "bars_flag"])
def test_fp32_small_cases(lib, case):
    from paper_2103_08246_gb300 import binding
    kw = {"plain": {}, "bars_flag": dict(bars_on=True, bar_x=1.0, **FLAG)}[case]
    wl = _small(**kw)
    gpu, ora = _run(wl, binding.IBM_FP32, 10)
    errs = _compare(gpu, ora, FP32_TOL, floor=FP32_FLOOR)
    gpu.close()
    print(case, "FP32 errors:", errs)


def test_fp32_tiny_workload(lib):
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.TINY
    gpu, ora = _run(wl, binding.IBM_FP32, 20, amp=wl.noise_amp)
    errs = _compare(gpu, ora, FP32_TOL, floor=FP32_FLOOR)
    gpu.close()
    print("tiny workload FP32 errors:", errs)


def test_markers_match_oracle_geometry(lib):
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.TINY
    gpu = binding.Solver(wl, binding.IBM_FP64)
    ora = OracleSolver(wl)
    Xg = gpu.markers()
    Xo = ora.markers()
    assert Xg.shape == Xo.shape
    # same set of points (order may differ)
    kg = np.lexsort(Xg.T)
    ko = np.lexsort(Xo.T)
    np.testing.assert_allclose(Xg[kg], Xo[ko], atol=1e-12)
    gpu.close()


def test_uniform_flow_stays_uniform(lib):
    from paper_2103_08246_gb300 import binding
    wl = _small()
    gpu = binding.Solver(wl, binding.IBM_FP64)
    gpu.step(20)
    u, v, w, p = gpu.fields()
    assert np.abs(u - 1).max() < 1e-13 and np.abs(v).max() < 1e-13 and np.abs(p).max() < 1e-11
    gpu.close()


def test_production_size_properties_fp32(lib):
    """512 x 256 x 256 with bars and the 65x65 flag, CFL 0.3, in FP32: the
    properties that hold at any size (projection leaves a divergence-free
    field to FP32 rounding, fluxes balance, everything finite)."""
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.PRODUCTION
    gpu = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl))
    gpu.step(3)
    st = gpu.stats()
    assert st["step"] == 3 and np.isfinite(st["ke"])
    assert abs(st["q_in"] - st["q_out"]) < 1e-4 * st["q_in"]
    # |div u| relative to the velocity scale / h
    assert st["max_div"] * (wl.lx / wl.nx) < 1e-4
    assert 0 < st["cfl"] <= 0.5
    X, V, F = gpu.flag()
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(V))
    gpu.close()


# ---------------------------------------------------------------- mixed precision
# FP32 fields with the Poisson transforms as split-TF32 tensor-core GEMMs and
# one refinement sweep on a double-single (FP64-class) residual: errors
# against the FP64 oracle are held
# to the FP32 bounds above (the split products keep ~FP32 accuracy and the
# refinement removes the amplification of the transform rounding by the
# Poisson conditioning).
@pytest.mark.parametrize("case", ["plain", "ragged", "bars_flag"])
def test_mixed_small_cases(lib, case):
    """ragged: 8 x 16 planes (not square) take the mma.sync transform GEMMs."""
    from paper_2103_08246_gb300 import binding
    kw = {"plain": {}, "ragged": dict(shape=(20, 8, 16)),
          "bars_flag": dict(bars_on=True, bar_x=1.0, **FLAG)}[case]
    wl = _small(**kw)
    gpu, ora = _run(wl, binding.IBM_MIXED, 10)
    errs = _compare(gpu, ora, FP32_TOL, floor=FP32_FLOOR)
    gpu.close()
    print(case, "mixed errors:", errs)


@pytest.mark.parametrize("shape", [(7, 32, 32), (21, 64, 64), (13, 128, 128)])
def test_mixed_tensor_core_plane_sizes(lib, shape):
    """Square planes of 32, 64 and 128 take the tcgen05 transform GEMMs too;
    7 x 32 and 21 x 64 rows leave the last 128-row tile partly empty."""
    from paper_2103_08246_gb300 import binding
    wl = _small(shape=shape, bars_on=True, bar_x=1.0)
    gpu, ora = _run(wl, binding.IBM_MIXED, 5)
    errs = _compare(gpu, ora, FP32_TOL, flag=False, floor=FP32_FLOOR)
    gpu.close()
    print(shape, "mixed errors:", errs)


def test_mixed_tiny_workload(lib):
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.TINY
    gpu, ora = _run(wl, binding.IBM_MIXED, 20, amp=wl.noise_amp)
    errs = _compare(gpu, ora, FP32_TOL, floor=FP32_FLOOR)
    st = gpu.stats()
    assert st["max_div"] * (wl.lx / wl.nx) < 1e-5
    gpu.close()
    print("tiny workload mixed errors:", errs, "max_div", st["max_div"])
