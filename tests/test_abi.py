"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gpulsm.h declares (no GPU needed, no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "gpulsm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsm_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lsm_lib):
    lib = ctypes.CDLL(lsm_lib.LIB_PATH)
    names = declared_entry_points()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(lsm_lib.EXPORTED)


def test_host_only_calls_without_gpu(lsm_lib):
    assert lsm_lib.lsm_status_str(0) == "LSM_OK"
    assert lsm_lib.lsm_status_str(6) == "LSM_ERR_CAPACITY"
    lib = lsm_lib._lib
    assert lib.lsm_stats(None, None, None, None, None) == lsm_lib.LSM_ERR_ARG
    assert lib.lsm_capacity(None) == 0
    h = ctypes.c_void_p()
    assert lib.lsm_create(ctypes.byref(h), 0, 100, 0) == lsm_lib.LSM_ERR_ARG      # b = 0
    assert lib.lsm_create(None, 16, 100, 0) == lsm_lib.LSM_ERR_ARG                # no handle slot
    assert lib.lsm_create(ctypes.byref(h), 1 << 27, 100, 0) == lsm_lib.LSM_ERR_ARG  # b too large


def test_built_for_sm_103a():
    from paper_1707_05354_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_library_resolves_its_own_symbols(lsm_lib):
    """Every internal (gpulsm::) function the library calls is defined in it:
    a declaration left without a definition would only fail when loaded."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "-C", "--undefined-only", lsm_lib.LIB_PATH], capture_output=True, text=True)
    missing = [ln for ln in out.stdout.splitlines() if "gpulsm::" in ln]
    assert not missing, missing
