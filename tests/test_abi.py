"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/ibm.h declares; host-only entry points validate arguments."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ibm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2103_08246_gb300 import binding
    declared = _declared()
    assert declared, "no declarations found"
    assert sorted(binding.SYMBOLS) == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_names_every_code(lib):
    for code in range(0, -7, -1):
        assert lib.ibm_strerror(code).decode() not in ("", "unknown status")
    assert lib.ibm_strerror(-99).decode() == "unknown status"


def test_workspace_bytes_and_argument_checks(lib):
    from paper_2103_08246_gb300 import binding, inputs
    wl = inputs.TINY
    g, d, b = binding.structs_from_workload(wl)
    n64 = binding.ibm_workspace_bytes(g, d, b, binding.ibm_options(binding.IBM_FP64, 0.3, 2.0))
    n32 = binding.ibm_workspace_bytes(g, d, b, binding.ibm_options(binding.IBM_FP32, 0.3, 2.0))
    cells = (wl.nx + 1) * wl.ny * wl.nz
    assert n64 > 15 * cells * 8 and n32 > 15 * cells * 4 and n32 < n64
    # non-uniform spacing, non power-of-two transverse size, bad precision
    bad = [binding.ibm_grid(wl.nx, wl.ny, wl.nz * 2), binding.ibm_grid(wl.nx, 24, 24)]
    for gb in bad:
        with pytest.raises(binding.IBMError) as e:
            binding.ibm_workspace_bytes(gb, d, b, None)
        assert e.value.code == binding.IBM_EINVAL
    with pytest.raises(binding.IBMError):
        binding.ibm_workspace_bytes(g, d, b, binding.ibm_options(7, 0.3, 2.0))
    # bar mesh that does not tile the transverse period
    b2 = binding.ibm_bodies.from_buffer_copy(b)
    b2.bar_mesh = 0.3
    with pytest.raises(binding.IBMError):
        binding.ibm_workspace_bytes(g, d, b2, None)


def test_create_rejects_null_output_without_gpu(lib):
    from paper_2103_08246_gb300 import binding, inputs
    g, d, b = binding.structs_from_workload(inputs.TINY)
    rc = lib.ibm_create(ctypes.byref(g), ctypes.byref(d), 100.0, ctypes.byref(b), None, None, 0, None)
    assert rc == binding.IBM_EINVAL


def test_bounded_wait_selftest_checks_its_argument(lib):
    # refused before any CUDA call, so this runs without a GPU
    assert lib.ibm_check_bounded_wait(0) == -1
    assert lib.ibm_check_bounded_wait((1 << 24) + 1) == -1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # no fallback: without the built library the binding refuses to work
    from paper_2103_08246_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        binding.load(str(tmp_path / "absent.so"))
