"""Parity with the CPU oracle on the paths that only large or long grids take.

* The x factor of the implicit step (Sec. II.B, approximate factorisation)
  runs in segments of x planes that start their LU recursions a warm-up of
  H planes early (exact to rho^H). With nx = 200 every segment length the
  library offers (16 and 24 planes in registers, 32 and 64 staged in shared
  memory) runs 4 to 13 segments, with a ragged last one; the inflow
  increment enters the first segment; FP64 to 1e-9 after 10 steps.
* The same at an implicit diffusion number r = nu dt / 2h^2 = 0.24, where
  the FP64 warm-up (22 planes) is close to its 24-plane limit; beyond the
  limit the step refuses to run (IBM_EINVAL) instead of losing accuracy.
* The production transverse shape (256 x 256 planes at h = 1/64) with the
  bar grid and the 65 x 65 flag, CFL 0.3, 3 steps: FP64 to 1e-9, FP32 and
  mixed precision to the FP32 bounds of ``test_gpu_parity``.
* The 65 x 65 flag (the production flag, whose structural update runs as
  one 16-CTA cluster) in a 1.5 x 1 x 2 box at h = 1/64, 10 steps: flag positions,
  velocities and forces to 1e-9 (FP64).
* A mixed-precision ensemble of uneven members (32^2 and 64^2 planes on the
  tcgen05 transform GEMMs, an 8 x 16 plane on the warp-level one, stepped as
  concurrent branches of one graph): every member against the oracle
  within the FP32 bounds, and equal to the member stepped alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_parity import FLAG, FP32_FLOOR, FP32_TOL, _compare  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def _solver_pair(wl, prec, amp=0.05, tiles=None, inflow=False):
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import binding, inputs
    noise = inputs.initial_noise(wl, amp=amp)
    return (binding.Solver(wl, prec, noise=noise, tiles=tiles, inflow=inflow),
            OracleSolver(wl, noise))


@pytest.mark.parametrize("afx_planes", [16, 24, 32, 64])
def test_fp64_x_factor_segments(lib, afx_planes):
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.small(200, 16, 16, bars_on=True, bar_x=1.0, **FLAG)
    gpu, ora = _solver_pair(wl, binding.IBM_FP64, tiles={"afx_planes": afx_planes})
    gpu.step(10)
    ora.run(10)
    _compare(gpu, ora, 1e-9)
    gpu.close()


@pytest.mark.parametrize("afx_planes", [16, 64])
def test_fp64_x_factor_segments_with_inflow(lib, afx_planes):
    """Prescribed inflow planes: the boundary increments enter the first
    row of the first segment."""
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.small(200, 16, 16, bars_on=True, bar_x=1.0)
    gpu, ora = _solver_pair(wl, binding.IBM_FP64, tiles={"afx_planes": afx_planes}, inflow=True)
    rng = np.random.default_rng(7)
    for _ in range(6):
        planes = (1.2 + 0.2 * rng.standard_normal((16, 16)), 0.1 * rng.standard_normal((16, 16)),
                  0.1 * rng.standard_normal((16, 16)))
        gpu.set_inflow(*planes)
        ora.set_inflow(*planes)
        gpu.step(1)
        ora.step()
    _compare(gpu, ora, 1e-9, flag=False)
    gpu.close()


@pytest.mark.parametrize("afx_planes", [16, 64])
def test_fp64_x_factor_near_warmup_limit(lib, afx_planes):
    """Re = 1, h = 1/4, dt = 0.03: r = 0.24, rho = 0.166, warm-up 22 planes."""
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.small(200, 16, 16, re=1.0, dt=0.03, bars_on=True, bar_x=1.0)
    gpu, ora = _solver_pair(wl, binding.IBM_FP64, tiles={"afx_planes": afx_planes})
    gpu.step(10)
    ora.run(10)
    _compare(gpu, ora, 1e-9, flag=False)
    gpu.close()


def test_x_factor_beyond_warmup_limit_is_refused(lib):
    """r = 0.4 needs a 28-plane FP64 warm-up (more than the 24 the segments
    carry): the step returns IBM_EINVAL."""
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.small(64, 8, 8, re=1.0, dt=0.05)
    gpu = binding.Solver(wl, binding.IBM_FP64, noise=inputs.initial_noise(wl, amp=0.05))
    rc = binding.ibm_step(gpu.state, 0.05, 1)
    assert rc == binding.IBM_EINVAL
    gpu.close()


def _production_slab():
    """The production workload's spacing, transverse planes, bodies and CFL
    on a shorter domain: 128 x 256 x 256 at h = 1/64 (2 x 4 x 4), bars at
    x = 0.5, the 65 x 65 flag with its leading edge at x = 0.8."""
    from paper_2103_08246_gb300 import inputs
    return inputs.PRODUCTION.replace(name="production-slab-128x256x256", nx=128, lx=2.0,
                                     flag_x_le=0.8, steps=3)


@pytest.fixture(scope="module")
def production_oracle():
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import inputs
    wl = _production_slab()
    noise = inputs.initial_noise(wl)
    ora = OracleSolver(wl, noise)
    ora.run(wl.steps)
    return wl, noise, ora


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed", "mixed_tc"])
def test_production_transverse_shape(lib, production_oracle, precision):
    """mixed: FP32 FFT predictor + single-TF32 tensor-core correction (the
    default at 256 x 256 planes); mixed_tc: both solves on the tensor cores."""
    from paper_2103_08246_gb300 import binding
    wl, noise, ora = production_oracle
    prec = {"fp64": binding.IBM_FP64, "fp32": binding.IBM_FP32, "mixed": binding.IBM_MIXED,
            "mixed_tc": binding.IBM_MIXED}[precision]
    gpu = binding.Solver(wl, prec, noise=noise, tc_predictor=precision == "mixed_tc")
    gpu.step(wl.steps)
    st = gpu.stats()
    assert st["step"] == wl.steps and abs(st["t"] - ora.t) <= 1e-6 * ora.t
    if prec == binding.IBM_FP64:
        errs = _compare(gpu, ora, 1e-9)
        assert abs(st["dt"] - ora.last_dt) <= 1e-12 * ora.last_dt
    else:
        errs = _compare(gpu, ora, FP32_TOL, floor=FP32_FLOOR)
    gpu.close()
    print(precision, "production-shape errors:", errs, "max_div", st["max_div"])


def test_fp64_production_flag_65x65(lib):
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.small(96, 64, 128, lx=1.5, ly=1.0, lz=2.0, re=200.0, flag_on=True,
                      flag_x_le=0.25, flag_ns=65, flag_nt=65, bending=0.005, dt=2e-3)
    gpu, ora = _solver_pair(wl, binding.IBM_FP64)
    gpu.step(10)
    ora.run(10)
    errs = _compare(gpu, ora, 1e-9)
    assert gpu.stats()["n_sub"] > 1
    assert np.abs(ora.V).max() > 1e-3      # the flag moves
    gpu.close()
    print("65x65 flag errors:", errs)


def _ensemble_members():
    from paper_2103_08246_gb300 import inputs
    return [inputs.small(24, 32, 32, bars_on=True, bar_x=1.0, **FLAG),
            inputs.small(20, 64, 64, bars_on=True, bar_x=1.0, seed=3),
            inputs.small(16, 8, 16, **FLAG, seed=5)]


def test_mixed_ensemble_members_match_oracle(lib):
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import binding, inputs
    cases = _ensemble_members()
    noises = [inputs.initial_noise(wl, amp=0.05) for wl in cases]
    team = [binding.Solver(wl, binding.IBM_MIXED, noise=n) for wl, n in zip(cases, noises)]
    ens = binding.Ensemble(team)
    ens.step(5, dt=2e-3)
    for wl, n, g in zip(cases, noises, team):
        ora = OracleSolver(wl, n)
        ora.run(5, 2e-3)
        _compare(g, ora, FP32_TOL, floor=FP32_FLOOR)
        solo = binding.Solver(wl, binding.IBM_MIXED, noise=n)
        solo.step(5, dt=2e-3)
        for a, b in zip(solo.fields(), g.fields()):
            assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1.0)
        solo.close()
    ens.close()
    for s in team:
        s.close()
