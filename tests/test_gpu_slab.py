"""x-slab decomposition of one case on the GPU (Sec. II.B: slabs of whole
y-z planes along x, one per GPU): the library's slab states and phases,
with 1 (the whole line: the degenerate partition), 2 and 3 ranks emulated
in one process on one device (exchanges as device copies between phases;
no kernel waits on another rank).

* bars + flag, 64x16x16 at h = 1/16 (the transforms of general planes): the
  assembled fields and the flag after the initial projection and 8 steps
  equal the single-domain oracle to 1e-9 (the FP64 parity bound), with the
  flag across a cut and the bars in the first slab;
* the production transverse plane, 96x256x256 at h = 1/64 (the 2-D cluster
  transform of 256 x 256 planes): 3 slabs equal the single-domain GPU solver
  (itself oracle-checked) to 1e-9 after 3 steps;
* the production workload in four slabs (the paper's own split), against the
  single-domain solver;
* phases out of order, a step too long for the overlap, and ibm_step, step
  timing and ensembles on a slab state are refused with IBM_EINVAL.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _small():
    from paper_2103_08246_gb300 import inputs
    return inputs.small(64, 16, 16, lx=4.0, ly=1.0, lz=1.0, re=100.0, bars_on=True, bar_x=0.5,
                        bar_mesh=0.5, bar_width=0.1, flag_on=True, flag_x_le=1.8, flag_len=1.0,
                        flag_span=0.5, flag_ns=5, flag_nt=5, dt=2e-3)


def _run_slabs(wl, nranks, nsteps, noise):
    from paper_2103_08246_gb300 import slab as S
    ranks = S.make_ranks(wl, nranks, wl.dt, noise)
    comm = S.LoopbackComm()
    S.run_phases(ranks, comm, S.INIT_SEQUENCE)
    for _ in range(nsteps):
        S.run_phases(ranks, comm, S.STEP_SEQUENCE, wl.dt)
    return ranks, S.gather_fields(ranks)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


@pytest.mark.parametrize("nranks", [1, 2, 3])
def test_slabs_match_oracle(nranks):
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import inputs
    wl = _small()
    noise = inputs.initial_noise(wl, amp=0.05)
    nsteps = 8
    ranks, got = _run_slabs(wl, nranks, nsteps, noise)
    ora = OracleSolver(wl, noise)
    ora.run(nsteps)
    for name, g, o in zip("uvwp", got, ora.fields()):
        assert g.shape == o.shape, name
        if name == "p":
            g, o = g - g.mean(), o - o.mean()
        assert _rel(g, o) < 1e-9, (name, _rel(g, o))
    X0, V0 = ranks[0].flag()
    for r in ranks[1:]:
        X, V = r.flag()
        assert np.abs(X - X0).max() < 1e-13 and np.abs(V - V0).max() < 1e-13
    assert np.abs(X0 - ora.X).max() < 1e-9 and np.abs(V0 - ora.V).max() < 1e-9
    cuts = np.array([r.slab.x_end for r in ranks[:-1]]) * wl.lx / wl.nx
    assert nranks == 1 or any(ora.X[:, 0].min() < c < ora.X[:, 0].max() for c in cuts)
    assert ranks[0].nf == 25
    for r in ranks:
        r.close()


def test_slabs_at_the_production_plane_match_single_domain():
    from paper_2103_08246_gb300 import binding as B
    from paper_2103_08246_gb300 import inputs
    wl = inputs.small(96, 256, 256, lx=1.5, ly=4.0, lz=4.0, re=200.0, bars_on=True, bar_x=0.25,
                      bar_mesh=0.5, bar_width=0.1, flag_on=True, flag_x_le=0.55, flag_len=0.6,
                      flag_span=1.0, flag_ns=17, flag_nt=17, bending=0.005, dt=2e-3)
    noise = inputs.initial_noise(wl, amp=0.05)
    nsteps = 3
    ranks, got = _run_slabs(wl, 3, nsteps, noise)
    one = B.Solver(wl, B.IBM_FP64, noise=noise)
    one.step(nsteps)
    for name, g, o in zip("uvwp", got, one.fields()):
        if name == "p":
            g, o = g - g.mean(), o - o.mean()
        assert _rel(g, o) < 1e-9, (name, _rel(g, o))
    X, V = ranks[1].flag()
    X1, V1, _ = one.flag()
    assert np.abs(X - X1).max() < 1e-9 and np.abs(V - V1).max() < 1e-9
    for r in ranks:
        r.close()


def test_four_slabs_of_the_production_workload_match_single_domain():
    """The paper's own configuration (four x slabs, Sec. II.B) on the
    production grid, 512x256x256 with the bar grid and the 65x65 flag, FP64
    at a fixed step: four slabs equal the single-domain solver to 1e-9 after
    the initial projection and 2 steps."""
    from paper_2103_08246_gb300 import binding as B
    from paper_2103_08246_gb300 import inputs
    wl = inputs.PRODUCTION.replace(dt=2e-3)
    noise = inputs.initial_noise(wl)
    ranks, got = _run_slabs(wl, 4, 2, noise)
    assert all(r.slab.x_end - r.slab.x_begin == 128 for r in ranks)
    one = B.Solver(wl, B.IBM_FP64, noise=noise)
    one.step(2)
    for name, g, o in zip("uvwp", got, one.fields()):
        if name == "p":
            g, o = g - g.mean(), o - o.mean()
        assert _rel(g, o) < 1e-9, (name, _rel(g, o))
    X, V = ranks[3].flag()
    X1, V1, _ = one.flag()
    assert np.abs(X - X1).max() < 1e-9 and np.abs(V - V1).max() < 1e-9
    one.close()
    for r in ranks:
        r.close()


def test_phase_order_and_overlap_are_enforced():
    import ctypes

    import torch

    from paper_2103_08246_gb300 import binding as B
    from paper_2103_08246_gb300 import slab as S
    wl = _small()
    ranks = S.make_ranks(wl, 2, wl.dt)
    st = ranks[0]
    buf = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    # before the initial sequence only INIT or FORCE may run
    for ph in (B.IBM_SLAB_SOLVE, B.IBM_SLAB_REDUCE, B.IBM_SLAB_PROJECT, B.IBM_SLAB_GHOSTS):
        assert B.ibm_slab_phase(st.state, ph, wl.dt, p, p) == B.IBM_EINVAL
    # a step whose implicit decay length exceeds the overlap
    assert B.ibm_slab_phase(st.state, B.IBM_SLAB_FORCE, 50 * wl.dt, None, p) == B.IBM_EINVAL
    assert B.ibm_step(st.state, wl.dt, 1) == B.IBM_EINVAL
    with pytest.raises(B.IBMError):   # no captured step to time or to join an ensemble
        B.ibm_time_stage(st.state, B.STAGES["step"], 1)
    with pytest.raises(B.IBMError):
        B.ibm_ensemble_create([st.state])
    # the full sequences still run afterwards
    S.run_phases(ranks, S.LoopbackComm(), S.INIT_SEQUENCE)
    S.run_phases(ranks, S.LoopbackComm(), S.STEP_SEQUENCE, wl.dt)
    for r in ranks:
        r.close()
