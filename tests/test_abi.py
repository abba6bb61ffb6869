"""The C-ABI library loads and exports what include/tsk.h declares (CPU)."""
import ctypes as C
import os

import pytest

import paper_2209_14637_gb300 as tsk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tsk.LIB_PATH):
        from paper_2209_14637_gb300 import build
        build.build()
    return tsk.load_library()


def test_header_declares_the_boundary():
    names = tsk.header_functions()
    for required in ("tsk_train_sketch", "tsk_approx_batch", "tsk_error",
                     "tsk_create", "tsk_destroy", "tsk_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = C.CDLL(tsk.LIB_PATH)
    names = tsk.header_functions()
    # names with digits are read too (the FP8 entry points)
    assert "tsk_quantize_e4m3" in names and "tsk_gram_e4m3" in names
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.tsk_destroy(None) == 1            # TSK_EINVAL
    assert lib.tsk_plan_execute(None, None) == 1
    assert lib.tsk_plan_destroy(None) == 1
    assert lib.tsk_sync_status(None, None) == 1
    assert lib.tsk_approx_batch(None, 1, None, 1, None, None, None, None) == 1
    assert lib.tsk_create(None, None) == 1
    assert isinstance(lib.tsk_last_error(None), bytes)


def test_default_options(lib):
    o = tsk.default_options()
    assert o.kernel == tsk.KERNEL_AUTO and o.refine_q == tsk.REFINE_AUTO
    assert o.max_iter == 300 and o.spin_limit == 1 << 24
    assert o.small_fp64 == 0 and o.gram_tile == 0


def test_create_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.tsk_create(C.byref(h), None)
    assert st == 3  # TSK_ECUDA
    assert b"device" in lib.tsk_last_error(None).lower()


def test_struct_layouts_match_header():
    # tsk_mat_desc: 2 pointers, 3 int64, 2 int32; tsk_mat_out: 3 pointers
    assert C.sizeof(tsk.MatDesc) == 2 * 8 + 3 * 8 + 2 * 4
    assert C.sizeof(tsk.MatOut) == 3 * 8
    # tsk_mat2_desc: 3 pointers, 3 int64, 4 int32
    assert C.sizeof(tsk.Mat2Desc) == 3 * 8 + 3 * 8 + 4 * 4
    assert C.sizeof(tsk.Options) == 4 * 4 + 8 + 8 + 2 * 4


def test_environment_overrides_the_default_options(lib, monkeypatch):
    """tsk_default_options: TSK_* variables with valid values replace the
    defaults; unset, unparsable or out-of-range ones leave them (no GPU)."""
    names = ["TSK_KERNEL", "TSK_REFINE_Q", "TSK_MAX_ITER", "TSK_ERR_MODE", "TSK_EIG_TOL",
             "TSK_SPIN_LIMIT", "TSK_SMALL_FP64", "TSK_GRAM_TILE"]
    for n in names:
        monkeypatch.delenv(n, raising=False)
    d = tsk.default_options()
    assert (d.kernel, d.refine_q, d.max_iter, d.err_mode, d.eig_tol, d.spin_limit,
            d.small_fp64, d.gram_tile) == (0, 2, 300, 0, 0.0, 1 << 24, 0, 0)
    for n, v in zip(names, ["1", "0", "50", "2", "1e-9", "4096", "1", "1"]):
        monkeypatch.setenv(n, v)
    o = tsk.default_options()
    assert (o.kernel, o.refine_q, o.max_iter, o.err_mode, o.eig_tol, o.spin_limit,
            o.small_fp64, o.gram_tile) == (1, 0, 50, 2, 1e-9, 4096, 1, 1)
    for n, v in zip(names, ["3", "x", "0", "-1", "2.5", "12q", "7", ""]):
        monkeypatch.setenv(n, v)
    o = tsk.default_options()
    assert (o.kernel, o.refine_q, o.max_iter, o.err_mode, o.eig_tol, o.spin_limit,
            o.small_fp64, o.gram_tile) == (0, 2, 300, 0, 0.0, 1 << 24, 0, 0)
