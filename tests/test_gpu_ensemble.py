"""Ensembles and tile parameters (GPU).

* stepping members together (one graph launch per step, every member a
  branch) gives the same fields as stepping each member on its own;
* a member of an FP64 ensemble still matches the CPU oracle to 1e-9;
* results do not depend on the tile parameters the autotuner chooses.
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


def _cases():
    from paper_2103_08246_gb300 import inputs
    flag = dict(flag_on=True, flag_x_le=2.0, flag_ns=5, flag_nt=5, flag_len=1.0, flag_span=1.0)
    return [inputs.small(16, 8, 8, bars_on=True, bar_x=1.0, **flag),
            inputs.small(20, 8, 16, **flag, seed=3),
            inputs.small(24, 16, 16, bars_on=True, bar_x=1.0, seed=5)]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ensemble_equals_individual_steps(lib, precision):
    from paper_2103_08246_gb300 import binding, inputs
    prec = binding.IBM_FP64 if precision == "fp64" else binding.IBM_FP32
    cases = _cases()
    solo = [binding.Solver(wl, prec, noise=inputs.initial_noise(wl, amp=0.05)) for wl in cases]
    team = [binding.Solver(wl, prec, noise=inputs.initial_noise(wl, amp=0.05)) for wl in cases]
    for s in solo:
        s.step(6, dt=2e-3)
    ens = binding.Ensemble(team)
    ens.step(6, dt=2e-3)
    tol = 1e-12 if prec == binding.IBM_FP64 else 1e-5
    for a, b in zip(solo, team):
        for fa, fb in zip(a.fields(), b.fields()):
            assert _rel(fb, fa) < tol
        if a.nf:
            assert np.abs(a.flag()[0] - b.flag()[0]).max() < tol
    ens.close()
    for s in solo + team:
        s.close()


def test_ensemble_member_matches_oracle(lib):
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import binding, inputs
    cases = _cases()
    team = [binding.Solver(wl, binding.IBM_FP64, noise=inputs.initial_noise(wl, amp=0.05))
            for wl in cases]
    ens = binding.Ensemble(team)
    ens.step(5, dt=2e-3)
    ora = OracleSolver(cases[1], inputs.initial_noise(cases[1], amp=0.05))
    ora.run(5, 2e-3)
    for g, o in zip(team[1].fields()[:3], ora.fields()[:3]):
        assert _rel(g, o) < 1e-9
    ens.close()
    for s in team:
        s.close()


def test_tiles_do_not_change_results(lib):
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.small(40, 16, 16, bars_on=True, bar_x=1.0)
    out = []
    for tiles in ({"rhs_planes": 8, "afx_planes": 32}, {"rhs_planes": 64, "afx_planes": 128}):
        s = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl, amp=0.05),
                           tiles=tiles)
        s.step(4)
        out.append(s.fields())
        s.close()
    # only the order of the atomic spreading sums differs: FP32 rounding of
    # O(U) values
    for a, b in zip(*out):
        assert np.abs(a - b).max() < 1e-6 * max(np.abs(b).max(), 1.0)


def test_autotuner_returns_candidates(lib, tmp_path):
    from paper_2103_08246_gb300 import autotune, binding, inputs
    wl = inputs.small(40, 16, 16)
    tiles = autotune.tune(wl, binding.IBM_FP32, cache_path=str(tmp_path / "c.json"), reps=2)
    assert tiles["rhs_planes"] in autotune.CANDIDATES["rhs_planes"]
    assert tiles["afx_planes"] in autotune.CANDIDATES["afx_planes"]
    again = autotune.tune(wl, binding.IBM_FP32, cache_path=str(tmp_path / "c.json"))
    assert again == tiles


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_batched_explicit_stage_equals_graph_ensemble(lib, precision):
    """The ensemble with every member's explicit stage in one persistent
    case-table launch steps like the graph-of-graphs ensemble (FP64 to
    1e-12 relative: the generic explicit-stage kernel differs from the
    specialised ones only in rounding order; FP32 and mixed to 1e-5), and an
    FP64 member still matches the oracle to 1e-9."""
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import binding, inputs
    prec = {"fp64": binding.IBM_FP64, "fp32": binding.IBM_FP32, "mixed": binding.IBM_MIXED}[precision]
    cases = _cases() + [inputs.small(16, 32, 32, bars_on=True, bar_x=1.0, seed=7)]
    mk = lambda: [binding.Solver(wl, prec, noise=inputs.initial_noise(wl, amp=0.05)) for wl in cases]  # noqa: E731
    ref, bat = mk(), mk()
    e_ref = binding.Ensemble(ref)
    e_bat = binding.Ensemble(bat, batched=True)
    e_ref.step(5, dt=2e-3)
    e_bat.step(5, dt=2e-3)
    tol = 1e-12 if prec == binding.IBM_FP64 else 1e-5
    for a, b in zip(ref, bat):
        for fa, fb in zip(a.fields(), b.fields()):
            assert np.abs(fb - fa).max() <= tol * max(np.abs(fa).max(), 1.0)
        if a.nf:
            assert np.abs(a.flag()[0] - b.flag()[0]).max() < tol
    if prec == binding.IBM_FP64:
        ora = OracleSolver(cases[0], inputs.initial_noise(cases[0], amp=0.05))
        ora.run(5, 2e-3)
        for g, o in zip(bat[0].fields()[:3], ora.fields()[:3]):
            assert _rel(g, o) < 1e-9
    # an odd number of steps, then more: the parities of the two graphs stay in step
    e_ref.step(3, dt=2e-3)
    e_bat.step(3, dt=2e-3)
    for a, b in zip(ref, bat):
        assert np.abs(b.fields()[0] - a.fields()[0]).max() <= tol * 2.0
    for e in (e_ref, e_bat):
        e.close()
    for s in ref + bat:
        s.close()
