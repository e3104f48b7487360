"""Checkpoint / restart through the C ABI (GPU).

* saving after n steps and loading into a fresh state gives, after m more
  steps, the fields, pressure, flag and diagnostics of an uninterrupted
  n + m step run (FP64 and FP32; only the order of the forcing's atomic
  additions may differ, so the bound is a few ulps grown over m steps);
* save -> load -> save reproduces the file byte for byte;
* a missing, truncated or foreign file is refused (IBM_EIO), a checkpoint of
  another problem is refused (IBM_EINVAL), and a refused load leaves the
  state as it was.
"""
import os

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


def _case(**kw):
    from paper_2103_08246_gb300 import inputs
    return inputs.small(24, 16, 16, bars_on=True, bar_x=1.0, flag_on=True, flag_x_le=2.0,
                        flag_ns=5, flag_nt=5, flag_len=1.0, flag_span=1.0, **kw)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_restart_continues_the_run(lib, tmp_path, precision):
    from paper_2103_08246_gb300 import binding, inputs
    prec = binding.IBM_FP64 if precision == "fp64" else binding.IBM_FP32
    wl = _case()
    noise = inputs.initial_noise(wl, amp=0.05)
    path = str(tmp_path / "state.ckpt")
    a = binding.Solver(wl, prec, noise=noise)
    a.step(8, dt=-1.0)            # CFL mode: dt and dt_old travel in the checkpoint
    a.save(path)
    a.step(7, dt=-1.0)
    b = binding.Solver(wl, prec, noise=inputs.initial_noise(wl, amp=0.0))
    b.load(path)
    b.step(7, dt=-1.0)
    tol = 1e-11 if prec == binding.IBM_FP64 else 2e-5
    for fa, fb in zip(a.fields(), b.fields()):
        assert _rel(fb, fa) < tol
    Xa, Va, _ = a.flag()
    Xb, Vb, _ = b.flag()
    assert np.abs(Xa - Xb).max() < tol
    assert np.abs(Va - Vb).max() < tol * max(np.abs(Va).max(), 1.0)
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"] == 15
    assert abs(sa["t"] - sb["t"]) <= tol * sa["t"]
    a.close()
    b.close()


def test_save_load_save_is_byte_identical(lib, tmp_path):
    from paper_2103_08246_gb300 import binding, inputs
    wl = _case()
    p1, p2 = str(tmp_path / "a.ckpt"), str(tmp_path / "b.ckpt")
    a = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl, amp=0.05))
    a.step(5, dt=2e-3)
    a.save(p1)
    b = binding.Solver(wl, binding.IBM_FP32)
    b.load(p1)
    b.save(p2)
    assert open(p1, "rb").read() == open(p2, "rb").read()
    a.close()
    b.close()


def test_bad_checkpoints_are_refused(lib, tmp_path):
    from paper_2103_08246_gb300 import binding, inputs
    wl = _case()
    good = str(tmp_path / "good.ckpt")
    a = binding.Solver(wl, binding.IBM_FP64, noise=inputs.initial_noise(wl, amp=0.05))
    a.step(3, dt=2e-3)
    a.save(good)
    before = a.fields()

    def code(path, state):
        return binding.load().ibm_load(state, os.fsencode(path))

    assert code(str(tmp_path / "missing.ckpt"), a.state) == binding.IBM_EIO
    blob = open(good, "rb").read()
    short = str(tmp_path / "short.ckpt")
    open(short, "wb").write(blob[: len(blob) // 2])
    assert code(short, a.state) == binding.IBM_EIO
    longer = str(tmp_path / "long.ckpt")
    open(longer, "wb").write(blob + b"\0")
    assert code(longer, a.state) == binding.IBM_EIO
    junk = str(tmp_path / "junk.ckpt")
    open(junk, "wb").write(b"\0" * len(blob))
    assert code(junk, a.state) == binding.IBM_EIO
    # same file, other problems: precision, grid, bodies
    b32 = binding.Solver(wl, binding.IBM_FP32)
    assert code(good, b32.state) == binding.IBM_EINVAL
    other = binding.Solver(_case().replace(re=123.0), binding.IBM_FP64)
    assert code(good, other.state) == binding.IBM_EINVAL
    for fa, fb in zip(before, a.fields()):
        assert np.array_equal(fa, fb)
    for s in (a, b32, other):
        s.close()
