"""Failure reporting on the GPU, without a fault: the library returns a
status and the CUDA context stays usable.

* a step whose CFL number (U dt / h summed over components) exceeds the
  state's limit returns IBM_EDIVERGED; the state still answers ibm_stats and
  a fresh state steps normally;
* the bounded-wait self-test waits on an mbarrier that nothing completes and
  returns IBM_ETIMEOUT after its iteration limit; work on the device runs
  normally afterwards;
* a non-finite value injected on the host (ibm_set_field uploads a velocity
  field with one NaN) is reported as IBM_EDIVERGED by the next step, in every
  precision, and the device stays usable.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def _small():
    from paper_2103_08246_gb300 import inputs
    return inputs.small(16, 8, 8)      # h = 1/4, Re 100, no bodies


def test_cfl_above_limit_is_reported(lib):
    from paper_2103_08246_gb300 import binding, inputs
    wl = _small()
    s = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl))
    with pytest.raises(binding.IBMError) as e:
        s.step(1, dt=0.6)              # U dt / h = 2.4 > the default limit 2
    assert e.value.code == binding.IBM_EDIVERGED
    st = s.stats()
    assert st["cfl"] > 2.0 and np.isfinite(st["ke"])
    s.close()
    t = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl))
    t.step(5)
    assert t.stats()["cfl"] < 0.5
    t.close()


def test_bounded_wait_times_out_and_the_context_survives(lib):
    import torch
    from paper_2103_08246_gb300 import binding, inputs
    assert binding.ibm_check_bounded_wait(1000) == binding.IBM_ETIMEOUT
    x = torch.arange(1024, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 1023 * 1024 / 2
    wl = _small()
    s = binding.Solver(wl, binding.IBM_FP32, noise=inputs.initial_noise(wl))
    s.step(3)
    assert np.isfinite(s.stats()["ke"])
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_injected_nan_is_reported(lib, precision):
    import torch
    from paper_2103_08246_gb300 import binding, inputs
    prec = {"fp64": binding.IBM_FP64, "fp32": binding.IBM_FP32, "mixed": binding.IBM_MIXED}[precision]
    wl = inputs.small(16, 32, 32)
    s = binding.Solver(wl, prec, noise=inputs.initial_noise(wl))
    s.step(2)
    u = s.fields()[0].copy()
    u[5, 3, 7] = np.nan
    binding.ibm_set_field(s.state, binding.IBM_FIELD_U, u)
    with pytest.raises(binding.IBMError) as e:
        s.step(1)
    assert e.value.code == binding.IBM_EDIVERGED
    s.close()
    x = torch.ones(4096, device="cuda")
    assert float(x.sum()) == 4096.0
