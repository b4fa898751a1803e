"""The C-ABI library builds, loads and exports every function include/ctm.h declares (no GPU)."""
import ctypes
import shutil

import pytest

from paper_2509_05090_gb300 import binding


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not binding.os.path.exists(binding.LIB_PATH):
        pytest.skip("no nvcc and no prebuilt libctm.so")
    from paper_2509_05090_gb300 import build
    build.build()
    return binding.load()


def test_exports_every_declared_symbol(lib):
    names = binding.header_functions()
    assert "ctm_init" in names and "ctm_step" in names and "ctm_energy" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing


def test_status_strings_and_bad_arguments(lib):
    assert binding.status_str(0) == "CTM_OK"
    assert "invalid" in binding.status_str(1)
    bad = binding.make_config(2, 0, 8)
    assert binding.ctm_workspace_bytes(bad) == 0
    out = ctypes.c_void_p()
    # null pointers are rejected before any CUDA call
    assert lib.ctm_init(ctypes.byref(binding.make_config(2, 2, 8)), None, None, 0, None, ctypes.byref(out)) == 1
    assert lib.ctm_step(None, 1, None) == 1
    assert lib.ctm_energy(None, None, None, None, None) == 1


def test_workspace_grows_with_chi(lib):
    small = binding.ctm_workspace_bytes(binding.make_config(2, 2, 8))
    big = binding.ctm_workspace_bytes(binding.make_config(2, 6, 72))
    assert 0 < small < big
    # two n x n FP64 intermediates at least
    n = 72 * 36
    assert big >= 2 * 8 * n * n


def test_configuration_limits(lib):
    """The size limits include/ctm.h states, checked by the host-side workspace query (no
    device work): real chi <= 512 with n = chi D^2 <= 20000, complex chi <= 256 with
    n <= 12000."""
    ws = binding.ctm_workspace_bytes
    assert ws(binding.make_config(2, 3, 512)) > 0
    assert ws(binding.make_config(2, 3, 513)) == 0
    assert ws(binding.make_config(2, 6, 512)) > 0          # n = 18432
    assert ws(binding.make_config(2, 7, 409)) == 0         # n = 20041
    zws = lib.ctm_complex_workspace_bytes
    E = 1
    assert zws(ctypes.byref(binding.make_config(2, 2, 256)), E) > 0
    assert zws(ctypes.byref(binding.make_config(2, 2, 257)), E) == 0
    assert zws(ctypes.byref(binding.make_config(2, 7, 245)), E) == 0   # n = 12005
