"""The C ABI library builds, loads without a GPU and exports every function ``include/wipes.h`` declares."""
import ctypes
import os
import subprocess

import pytest

from paper_2508_12615_gb300 import _abi, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.lib()


def test_header_declares_the_boundary():
    names = _abi.header_functions()
    for required in ["wipes_create", "wipes_destroy", "wipes_state_create", "wipes_state_destroy", "wipes_render2d",
                     "wipes_render3d", "wipes_render_backward", "wipes_deform6d", "wipes_deform6d_backward",
                     "wipes_l2_loss", "wipes_status_string", "wipes_last_error", "wipes_sync_status"]:
        assert required in names


def test_every_declared_function_is_exported(lib):
    exported = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True,
                              check=True).stdout
    syms = {line.split()[-1] for line in exported.splitlines() if line.strip()}
    missing = [n for n in _abi.header_functions() if n not in syms]
    assert not missing, missing
    for n in _abi.header_functions():
        assert hasattr(lib, n)
        assert n in _abi._SIGNATURES, f"{n} has no ctypes signature"


def test_no_cuda_needed_for_host_helpers(lib):
    o = _abi.default_opts(3)
    assert o.cutoff_sigma == 3.0 and abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.dilation - 0.3) < 1e-7
    o2 = _abi.default_opts(2)
    assert o2.dilation == 0.0
    assert lib.wipes_status_string(2) == b"capacity exceeded"
    assert lib.wipes_last_error() is not None


def test_struct_layouts_match_header():
    assert ctypes.sizeof(_abi.Camera) == 17 * 4
    assert ctypes.sizeof(_abi.Opts) == 11 * 4
    assert ctypes.sizeof(_abi.StateInfo) == 5 * 4 + 4 + 3 * 8  # int32 x5, padding, int64 x3


def test_invalid_arguments_rejected_before_any_device_work(lib):
    # NULL context/state pointers are rejected on the host with WIPES_ERR_INVALID
    st = lib.wipes_render2d(None, None, None, 0, 16, 16, None, None, None)
    assert st == 1
    assert b"null" in lib.wipes_last_error()
    assert lib.wipes_state_get_info(None, None) == 1


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
