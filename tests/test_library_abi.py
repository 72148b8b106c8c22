"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol that include/hpx.h declares; argument checks that precede any CUDA call
report their error codes (no compute call is made here)."""

import os
import re

import pytest

from helpers import ROOT

HEADER = os.path.join(ROOT, "include", "hpx.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hpx_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def hp():
    import paper_1904_10514_gb300 as hp
    if not os.path.exists(hp.LIB_PATH):
        hp.build()
    return hp


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["hpx_plan", "hpx_plan_ex", "hpx_set_stream", "hpx_analyze", "hpx_synthesize",
              "hpx_cl", "hpx_sync", "hpx_destroy", "hpx_last_error", "hpx_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(hp):
    import ctypes
    L = ctypes.CDLL(hp.LIB_PATH)
    for n in _declared():
        assert hasattr(L, n), n
    assert sorted(hp.EXPORTS) == _declared()


def test_invalid_arguments_rejected_before_any_cuda_call(hp):
    assert not hp.hpx_plan(3, -1, 1)
    assert hp.hpx_last_error() == hp.HPX_ERR_NSIDE
    assert not hp.hpx_plan(1, -1, 1)
    assert hp.hpx_last_error() == hp.HPX_ERR_NSIDE
    assert not hp.hpx_plan(4096, -1, 1)
    assert hp.hpx_last_error() == hp.HPX_ERR_NSIDE
    assert not hp.hpx_plan_ex(2048, -1, 1, hp.HPX_FP64)
    assert hp.hpx_last_error() == hp.HPX_ERR_NSIDE
    assert not hp.hpx_plan(8, 17, 1)
    assert hp.hpx_last_error() == hp.HPX_ERR_LMAX
    assert not hp.hpx_plan(8, -1, 0)
    assert hp.hpx_last_error() == hp.HPX_ERR_ARG
    assert not hp.hpx_plan_ex(8, -1, 1, 7)
    assert hp.hpx_last_error() == hp.HPX_ERR_ARG
    assert hp.hpx_analyze(None, None, None) == hp.HPX_ERR_ARG
    assert hp.hpx_cl(None, None, None) == hp.HPX_ERR_ARG
    assert hp.hpx_sync(None) == hp.HPX_ERR_ARG
    assert "nside" in hp.strerror(hp.HPX_ERR_NSIDE)


def test_descriptor_fields_rejected_before_any_cuda_call(hp):
    assert not hp.hpx_plan_ex(8, -1, 1, hp.HPX_FP32, 1 << 10)             # unknown flag
    assert hp.hpx_last_error() == hp.HPX_ERR_ARG
    assert not hp.hpx_plan_ex(8, -1, 2, hp.HPX_FP32, 0, None, [16, 17])   # lmax_1 > 2 nside
    assert hp.hpx_last_error() == hp.HPX_ERR_LMAX
    assert not hp.hpx_plan_ex(8, -1, 2, hp.HPX_FP32, 0, None, [-2, 4])    # lmax_0 < -1
    assert hp.hpx_last_error() == hp.HPX_ERR_LMAX
    assert not hp.hpx_plan_ex(0, -1, 2, hp.HPX_FP32, 0, [8, 4], [16, 9])  # lmax_1 > 2 nside_1
    assert hp.hpx_last_error() == hp.HPX_ERR_LMAX
    assert not hp.hpx_plan_ex(0, -1, 2, hp.HPX_FP32, 0, [8, 12], None)    # nside not a power of two
    assert hp.hpx_last_error() == hp.HPX_ERR_NSIDE


def test_service_calls_reject_null_plans(hp):
    """The plan queries and the tuning calls check their arguments on the host."""
    import ctypes
    L = hp.lib()
    v = [ctypes.c_int(0) for _ in range(5)]
    assert L.hpx_plan_tuning(None, *[ctypes.byref(x) for x in v]) == hp.HPX_ERR_ARG
    assert L.hpx_plan_set_tuning(None, 16, 16, 0, 0, 0) == hp.HPX_ERR_ARG
    assert L.hpx_plan_launches(None) == -1
    assert L.hpx_plan_flags(None) == -1
    assert L.hpx_plan_lmax(None) == -1
