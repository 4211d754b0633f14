"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU).

Only calls that return before touching a device run here: argument checks and the
version / error strings.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1210_6412_gb300 as R
from paper_1210_6412_gb300 import _build


@pytest.fixture(scope="module")
def so():
    return R.lib()


def test_library_is_sm103a_build(so):
    assert _build.up_to_date()
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_exports_every_header_symbol(so):
    names = R.header_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(so, name), name


def test_version_string(so):
    assert "sm_103a" in R.reach_version()


def test_argument_checks_need_no_device(so):
    ctx = C.c_void_p()
    rp = np.array([0, 1], np.int64)
    col = np.array([0], np.int32)
    val = np.array([1.0])
    goal = np.array([1], np.uint8)
    # NULL out pointer
    assert so.reach_create(None, 1, 1, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                           goal.ctypes.data, 0, None) == R.REACH_EINVAL
    # n < 1
    assert so.reach_create(C.byref(ctx), 0, 1, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                           goal.ctypes.data, 0, None) == R.REACH_EINVAL
    assert "n must be" in R.reach_last_error()
    # unknown pointer kind
    assert so.reach_create(C.byref(ctx), 1, 1, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                           goal.ctypes.data, 7, None) == R.REACH_EINVAL
    # NULL context everywhere
    assert so.reach_precompute(None, 0) == R.REACH_EINVAL
    assert so.reach_solve(None, 0, 1e-9, 10, 0, None, None, 0, None) == R.REACH_EINVAL
    assert so.reach_grad(None, 0, 1e-9, 10, None, 0, None) == R.REACH_EINVAL
    assert so.reach_grad_method(None, R.REACH_BICGSTAB_FP64, 0, 1e-9, 10, None, 0, None) == R.REACH_EINVAL
    assert so.reach_get_classes(None, None, 0) == R.REACH_EINVAL
    so.reach_destroy(None)
    assert ctx.value is None


def test_batch_entry_points_reject_null_batch(so):
    off = np.array([0, 1], np.int64)
    assert so.reach_batch_set_chains(None, 1, off.ctypes.data) == R.REACH_EINVAL
    assert so.reach_batch_chain_info(None, None, None) == R.REACH_EINVAL
    assert so.reach_batch_solve(None, 1e-9, 10, 0, None, 0, None) == R.REACH_EINVAL


def test_param_entry_points_reject_bad_arguments(so):
    assert so.reach_param_probs(0, 0, None, None, None, None, 0, None, None) == R.REACH_EINVAL
    assert so.reach_param_grad_theta(1, 1, None, None, None, None, 5000, None, None) == R.REACH_EINVAL
