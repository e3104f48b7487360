"""Virtual probes through the C ABI (GPU): the gathered samples are the
cell-centred velocities of the fields; out-of-range cells are refused."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_probes_are_cell_centred_velocities(lib, precision):
    from paper_2103_08246_gb300 import binding, inputs
    prec = binding.IBM_FP64 if precision == "fp64" else binding.IBM_FP32
    wl = inputs.small(20, 8, 16, bars_on=True, bar_x=1.0)
    s = binding.Solver(wl, prec, noise=inputs.initial_noise(wl, amp=0.05))
    s.step(3)
    rng = np.random.default_rng(0)
    cells = np.stack([rng.integers(0, wl.nx, 50), rng.integers(0, wl.ny, 50), rng.integers(0, wl.nz, 50)], axis=1)
    cells[0] = (wl.nx - 1, wl.ny - 1, wl.nz - 1)      # the periodic wrap in y and z
    s.set_probes(cells)
    buf = torch.zeros((len(cells), 3), dtype=torch.float64 if prec == binding.IBM_FP64 else torch.float32,
                      device="cuda")
    torch.cuda.synchronize()
    s.probe_sample(buf.data_ptr())
    s.stream.synchronize()
    got = buf.double().cpu().numpy()
    u, v, w, _ = s.fields()
    i, j, k = cells.T
    ref = np.stack([0.5 * (u[i, j, k] + u[i + 1, j, k]),
                    0.5 * (v[i, j, k] + v[i, (j + 1) % wl.ny, k]),
                    0.5 * (w[i, j, k] + w[i, j, (k + 1) % wl.nz])], axis=1)
    tol = 1e-15 if prec == binding.IBM_FP64 else 1e-6
    assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max())
    with pytest.raises(binding.IBMError):
        s.set_probes(np.array([[wl.nx, 0, 0]]))
    s.close()
