"""Failure paths on the GPU that neither fault nor hang it.

A bounded device wait is made to run out (an mbarrier nothing completes, 2 ms
limit); the kernel returns, the status word reports FW_ETIMEOUT, and the
context stays usable for a normal classification afterwards.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4188_gb300 import fw, workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_4188_gb300 import build
    build.build()
    return torch


def test_bounded_wait_reports_timeout_and_context_survives(torch_cuda):
    torch = torch_cuda
    rules = W.gen_rules(300, 3)
    hdr = W.gen_packets(rules, 4096, 4)
    rs = fw.fw_ruleset_create(rules)
    assert rs.check() == fw.FW_OK
    L = fw.lib()
    assert L.fw_selftest_wait_timeout(rs.handle, 2_000_000, None) == fw.FW_OK
    assert rs.check() == fw.FW_ETIMEOUT
    assert rs.check() == fw.FW_OK  # the flag is cleared by the check
    idx, act = fw.fw_classify(rs, fw.headers_to_device(hdr))
    torch.cuda.synchronize()
    want = oracle.classify(rules, hdr)
    assert np.array_equal(idx.cpu().numpy(), want[0]) and np.array_equal(act.cpu().numpy(), want[1])
    rs.destroy()


def test_selftest_rejects_bad_limits(torch_cuda):
    rs = fw.fw_ruleset_create(W.gen_rules(10, 1))
    L = fw.lib()
    assert L.fw_selftest_wait_timeout(rs.handle, 10, None) == fw.FW_EINVAL
    assert L.fw_selftest_wait_timeout(None, 2_000_000, None) == fw.FW_EINVAL
    rs.destroy()
