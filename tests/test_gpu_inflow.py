"""Prescribed time-dependent inflow through the C ABI (GPU).

* a fresh random inflow plane every step (u with a mean other than U, v, w):
  FP64 matches the CPU oracle to 1e-9 (on the vector kernels' shape and on
  a small shape served by the fallback kernels), FP32 to the FP32 bounds;
* the inflow face carries the pending u shifted to mean U, so the inflow
  flux is U ly lz exactly and the mass fix balances the outflow;
* writing the pending planes in device memory (ibm_inflow_planes) gives the
  same result as passing host planes (ibm_set_inflow);
* the inflow planes travel in checkpoints;
* plane access (ibm_get_plane, ibm_plane_device) returns the x-planes of the
  current velocity, so a run can feed its own planes back as inflow.
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


def _planes(wl, seed):
    rng = np.random.default_rng(seed)
    shape = (wl.ny, wl.nz)
    return (1.0 + 0.2 * rng.standard_normal(shape) + 0.3, 0.1 * rng.standard_normal(shape),
            0.1 * rng.standard_normal(shape))


def _case(shape):
    from paper_2103_08246_gb300 import inputs
    nx, ny, nz = shape
    return inputs.small(nx, ny, nz, bars_on=True, bar_x=1.0)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1.0)


@pytest.mark.parametrize("shape,precision", [((20, 32, 32), "fp64"), ((16, 8, 8), "fp64"),
                                             ((20, 32, 32), "fp32"), ((16, 8, 8), "fp32"),
                                             ((20, 32, 32), "mixed"), ((12, 256, 256), "mixed")])
def test_inflow_matches_oracle(lib, shape, precision):
    """mixed at 32 x 32 planes: both solves on the tensor cores; at 256 x 256:
    the FFT predictor with the bfloat16 correction."""
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import binding, inputs
    prec = {"fp64": binding.IBM_FP64, "fp32": binding.IBM_FP32, "mixed": binding.IBM_MIXED}[precision]
    wl = _case(shape)
    noise = inputs.initial_noise(wl, amp=0.05)
    gpu = binding.Solver(wl, prec, noise=noise, inflow=True)
    ora = OracleSolver(wl, noise=noise)
    for step in range(6):
        planes = _planes(wl, 100 + step)
        gpu.set_inflow(*planes)
        ora.set_inflow(*planes)
        gpu.step(1)
        ora.step()
    tol = 1e-9 if prec == binding.IBM_FP64 else 2e-4
    u, v, w, p = gpu.fields()
    for g, o in ((u, ora.u), (v, ora.v), (w, ora.w)):
        assert _rel(g, o) < tol
    assert _rel(p - p.mean(), ora.p - ora.p.mean()) < (tol if prec == binding.IBM_FP64 else 2e-3)
    st = gpu.stats()
    h = wl.lx / wl.nx
    # fluxes relative to the inflow area (FP32 planes of up to 65536 values)
    area = wl.ly * wl.lz
    assert abs(st["q_in"] - area) < (1e-13 if prec == binding.IBM_FP64 else 1e-6) * area
    assert abs(st["q_out"] - st["q_in"]) < (1e-12 if prec == binding.IBM_FP64 else 1e-5) * area
    pu = planes[0]
    assert np.abs(u[0] - (pu - pu.mean() + 1.0)).max() < (1e-14 if prec == binding.IBM_FP64 else 1e-6)
    gpu.close()


class _DeviceArray:
    """A raw device pointer as a CUDA array (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


def test_device_planes_equal_host_planes(lib, tmp_path):
    from paper_2103_08246_gb300 import binding, inputs
    wl = _case((20, 32, 32))
    noise = inputs.initial_noise(wl, amp=0.05)
    # deterministic forcing: equal inputs must give bitwise equal fields
    a = binding.Solver(wl, binding.IBM_FP32, noise=noise, inflow=True, deterministic=True)
    b = binding.Solver(wl, binding.IBM_FP32, noise=noise, inflow=True, deterministic=True)
    for step in range(4):
        planes = _planes(wl, 7 + step)
        a.set_inflow(*planes)
        torch.cuda.synchronize()
        for ptr, q in zip(binding.ibm_inflow_planes(b.state), planes):
            dev = torch.as_tensor(_DeviceArray(ptr, (wl.ny, wl.nz), "<f4"), device="cuda")
            dev.copy_(torch.as_tensor(q, dtype=torch.float32))
        torch.cuda.synchronize()
        a.step(1)
        b.step(1)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    # checkpoint with inflow planes: continue identically after a reload
    path = str(tmp_path / "inflow.ckpt")
    a.save(path)
    c = binding.Solver(wl, binding.IBM_FP32, inflow=True, deterministic=True)
    c.load(path)
    a.step(2)
    c.step(2)
    for x, y in zip(a.fields(), c.fields()):
        assert np.array_equal(x, y)
    plain = binding.Solver(wl, binding.IBM_FP32)
    assert binding.load().ibm_load(plain.state, path.encode()) == binding.IBM_EINVAL
    with pytest.raises(binding.IBMError):
        plain.set_inflow(*_planes(wl, 1))
    for s in (a, b, c, plain):
        s.close()


def test_plane_access_and_feedback(lib):
    from paper_2103_08246_gb300 import binding, inputs
    wl = _case((20, 32, 32))
    s = binding.Solver(wl, binding.IBM_FP64, noise=inputs.initial_noise(wl, amp=0.05), inflow=True)
    s.step(2)
    u, v, w, _ = s.fields()
    for i in (0, 7, wl.nx):
        pu, pv, pw = s.plane(i)
        assert np.array_equal(pu, u[i]) and np.array_equal(pv, v[i]) and np.array_equal(pw, w[i])
    ptrs = binding.ibm_plane_device(s.state, 7)
    dev = torch.as_tensor(_DeviceArray(ptrs[1], (wl.ny, wl.nz), "<f8"), device="cuda")
    assert np.array_equal(dev.cpu().numpy(), v[7])
    # recycle plane 7 as the next inflow (a precursor-style feedback)
    s.set_inflow(*s.plane(7))
    s.step(1)
    pu = u[7]
    assert np.abs(s.field(binding.IBM_FIELD_U)[0] - (pu - pu.mean() + 1.0)).max() < 1e-14
    s.close()
