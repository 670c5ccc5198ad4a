"""Allocation failure injected on the host (fw_selftest_fail_alloc), without a GPU.

The hook fails the armed allocation before the CUDA allocator is reached, so on a machine
without a GPU the first allocation of a create call can still be made to fail: the call must
return FW_ENOMEM with a NULL handle, and the hook must disarm after that one failure. The GPU
test (test_alloc_failure_gpu.py) moves the failure across every allocation of every create call.
"""
import ctypes

import numpy as np
import pytest

from paper_1312_4188_gb300 import build as B
from paper_1312_4188_gb300 import fw, workload as W


@pytest.fixture(scope="module")
def L():
    B.build()
    lib = fw.lib()
    yield lib
    lib.fw_selftest_fail_alloc(-1)


def _rules():
    r = np.ascontiguousarray(W.gen_rules(200, 1))
    return r, r.ctypes.data_as(ctypes.c_void_p)


def test_ruleset_first_allocation_fails_then_disarms(L):
    r, ptr = _rules()
    out = ctypes.c_void_p()
    assert L.fw_selftest_fail_alloc(0) == fw.FW_OK
    assert L.fw_ruleset_create_ex(ptr, len(r), ctypes.byref(out)) == fw.FW_ENOMEM
    assert out.value is None
    # the hook fired once: the next create reaches the real allocator (a GPU: OK; none: a CUDA error)
    s = L.fw_ruleset_create_ex(ptr, len(r), ctypes.byref(out))
    assert s in (fw.FW_OK, fw.FW_ECUDA)
    if s == fw.FW_OK:
        L.fw_ruleset_destroy(out)


def test_short_form_reports_enomem_in_last_status(L):
    r, ptr = _rules()
    L.fw_selftest_fail_alloc(0)
    assert L.fw_ruleset_create(ptr, len(r)) is None
    assert L.fw_last_status() == fw.FW_ENOMEM


def test_negative_disarms(L):
    r, ptr = _rules()
    out = ctypes.c_void_p()
    L.fw_selftest_fail_alloc(0)
    L.fw_selftest_fail_alloc(-1)
    s = L.fw_ruleset_create_ex(ptr, len(r), ctypes.byref(out))
    assert s in (fw.FW_OK, fw.FW_ECUDA)
    if s == fw.FW_OK:
        L.fw_ruleset_destroy(out)


def test_learned_index_and_plan_first_allocation(L):
    r, ptr = _rules()
    out = ctypes.c_void_p()
    L.fw_selftest_fail_alloc(0)
    assert L.fw_lindex_create(ptr, len(r), None, ctypes.byref(out)) == fw.FW_ENOMEM and out.value is None
    L.fw_selftest_fail_alloc(0)
    assert L.fw_plan_create(None, 0, None, ctypes.byref(out)) == fw.FW_ENOMEM and out.value is None
    L.fw_selftest_fail_alloc(-1)


def test_argument_errors_come_before_the_hook(L):
    """A call rejected for its arguments allocates nothing, so it does not consume the armed failure."""
    r, ptr = _rules()
    out = ctypes.c_void_p()
    L.fw_selftest_fail_alloc(0)
    assert L.fw_ruleset_create_ex(None, 5, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_ruleset_create_ex(ptr, len(r), ctypes.byref(out)) == fw.FW_ENOMEM
    L.fw_selftest_fail_alloc(-1)
