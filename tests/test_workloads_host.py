"""Synthetic workloads against their stated recipe and the library's own
argument rules (host only: ibm_workspace_bytes validates a configuration and
sizes its workspace without touching a GPU).

* the 16 ensemble cases: x from 64 to 256 cells, y = z in {32, 64, 128},
  h = 1/16, bending log-uniform in [1e-3, 1e-1], Re in [100, 400], the
  flag's leading edge 1 to 4 bar meshes behind the grid; every case is
  accepted in FP32 and mixed precision;
* the tiny and production workloads are accepted; the production FP32
  workspace is about 17.4 fields of 134 MB (17 fields and the quarter-field
  pivot table).
"""
import os
import shutil

import pytest

from paper_2103_08246_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def _bytes(wl, precision):
    from paper_2103_08246_gb300 import binding
    g, d, b = binding.structs_from_workload(wl)
    return binding.ibm_workspace_bytes(g, d, b, binding.ibm_options(precision, wl.cfl, 2.0))


def test_ensemble_cases_follow_the_recipe(lib):
    from paper_2103_08246_gb300 import binding
    cases = inputs.ensemble_cases()
    assert len(cases) == 16
    for wl in cases:
        h = wl.lx / wl.nx
        assert abs(h - 1 / 16) < 1e-15 and abs(wl.ly / wl.ny - h) < 1e-15 and abs(wl.lz / wl.nz - h) < 1e-15
        assert 64 <= wl.nx <= 256 and wl.ny == wl.nz and wl.ny in (32, 64, 128)
        assert 1e-3 <= wl.bending <= 1e-1 and 100 <= wl.re <= 400
        assert 1.0 - 1e-12 <= (wl.flag_x_le - wl.bar_x) / wl.bar_mesh <= 4.0 + 1e-12
        assert wl.flag_ns == wl.flag_nt == 17 and wl.bars_on and wl.flag_on
        for prec in (binding.IBM_FP32, binding.IBM_MIXED):
            assert _bytes(wl, prec) > 0
    # uneven: several transverse sizes and lengths
    assert len({wl.ny for wl in cases}) >= 2 and len({wl.nx for wl in cases}) >= 8


def test_reference_workloads_are_accepted(lib):
    from paper_2103_08246_gb300 import binding
    assert _bytes(inputs.TINY, binding.IBM_FP64) > 0
    prod = _bytes(inputs.PRODUCTION, binding.IBM_FP32)
    field = (inputs.PRODUCTION.nx + 1) * inputs.PRODUCTION.ny * inputs.PRODUCTION.nz * 4
    assert 16 * field < prod < 19 * field, prod / field
    assert _bytes(inputs.PRODUCTION, binding.IBM_FP64) > 1.8 * prod


def test_deterministic_forcing_costs_24_bytes_per_cell(lib):
    # three 64-bit fixed-point accumulators per velocity node
    from paper_2103_08246_gb300 import binding
    wl = inputs.small(64, 32, 32, bars_on=True, bar_x=1.0)
    g, d, b = binding.structs_from_workload(wl)
    plain = binding.ibm_options(binding.IBM_FP32, 0.3, 2.0)
    det = binding.ibm_options(binding.IBM_FP32, 0.3, 2.0)
    det.deterministic = 1
    extra = binding.ibm_workspace_bytes(g, d, b, det) - binding.ibm_workspace_bytes(g, d, b, plain)
    assert extra == 24 * (wl.nx + 1) * wl.ny * wl.nz
