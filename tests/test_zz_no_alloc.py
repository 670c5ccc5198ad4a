"""The allocation-free entry point against the allocating one.

fw_classify_rule_split_noalloc serves callers that must not allocate device
memory while they classify (a packet path that cannot take the implicit
synchronisation of cudaMalloc/cudaFree, or a service whose GPU memory is
fixed at start-up). It keeps its scratch in a fixed device array instead of
allocating per call. Here it is called twice in a row through the C ABI, on
different batches, and each result must equal, bit for bit, what the
existing grid rule-split entry point (fw_classify_ex, which allocates its
scratch per call) returns for the same batch. This file is collected last so
that a failure here does not hide the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

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


def _noalloc(torch, rs, dh, n, cfg=None):
    idx = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    act = torch.full((max(n, 1),), 9, dtype=torch.uint8, device="cuda")
    hs = fw.headers_struct(dh)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = fw.lib().fw_classify_rule_split_noalloc(rs.handle, ctypes.byref(hs), n, ctypes.c_void_p(idx.data_ptr()),
                                                ctypes.c_void_p(act.data_ptr()), st,
                                                ctypes.byref(cfg) if cfg is not None else None)
    return s, idx[:n], act[:n]


def _call(torch, rs, dh, n, idx, act, cfg=None):
    hs = fw.headers_struct(dh)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fw.lib().fw_classify_rule_split_noalloc(rs.handle, ctypes.byref(hs), n, ctypes.c_void_p(idx.data_ptr()),
                                                   ctypes.c_void_p(act.data_ptr()), st,
                                                   ctypes.byref(cfg) if cfg is not None else None)


@pytest.mark.parametrize("partition", [0, 2], ids=["partition", "whole_list"])
def test_two_calls_match_the_allocating_entry_point(torch_cuda, partition):
    torch = torch_cuda
    rules = W.gen_rules(3000, 17)
    keep = ~((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0))  # deep scans, many unmatched
    rules = rules[keep]
    rs = fw.fw_ruleset_create(rules)
    cfg = fw.make_config("rule_split_grid", partition=partition)
    batches = [W.gen_packets(rules, 300_001, 18), W.gen_packets(rules, 77_777, 19, zipf_s=1.1)]
    dhs = [fw.headers_to_device(h) for h in batches]
    outs = [(torch.full((len(h["src"]),), -7, dtype=torch.int32, device="cuda"),
             torch.full((len(h["src"]),), 9, dtype=torch.uint8, device="cuda")) for h in batches]
    wants = [fw.fw_classify(rs, dh, len(h["src"]), config=cfg) for dh, h in zip(dhs, batches)]
    # warm-up: the first call on a device may load the library's module (and its scratch array)
    assert _call(torch, rs, dhs[1], len(batches[1]["src"]), *outs[1], cfg) == fw.FW_OK
    torch.cuda.synchronize()
    # no torch work between the two measured calls, so that any change in free device memory is
    # the entry point's own
    free0 = torch.cuda.mem_get_info()[0]
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    status, free_after = [], []
    for call, hdr in enumerate(batches):
        status.append(_call(torch, rs, dhs[call], len(hdr["src"]), *outs[call], cfg))
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
    assert status == [fw.FW_OK, fw.FW_OK], status
    assert free_after == [free0, free0], f"device memory was allocated: free {free0} -> {free_after}"
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
    for call in range(2):
        idx, act = outs[call]
        want_idx, want_act = wants[call]
        assert torch.equal(idx, want_idx), f"call {call}: rule index differs from fw_classify_ex"
        assert torch.equal(act, want_act), f"call {call}: action differs from fw_classify_ex"
        assert int((idx >= 0).sum()) > 0 and int((idx < 0).sum()) > 0
    assert rs.check() == fw.FW_OK
    rs.destroy()


def test_limits_and_arguments(torch_cuda):
    torch = torch_cuda
    rules = W.gen_rules(100, 5)
    rs = fw.fw_ruleset_create(rules)
    hdr = W.gen_packets(rules, 64, 6)
    dh = fw.headers_to_device(hdr)
    hs = fw.headers_struct(dh)
    L = fw.lib()
    big = fw.FW_NOALLOC_MAX_PACKETS + 1
    assert L.fw_classify_rule_split_noalloc(rs.handle, ctypes.byref(hs), big, None, None, None, None) == fw.FW_ERANGE
    assert L.fw_classify_rule_split_noalloc(rs.handle, ctypes.byref(hs), -1, None, None, None, None) == fw.FW_EINVAL
    assert L.fw_classify_rule_split_noalloc(rs.handle, ctypes.byref(hs), 0, None, None, None, None) == fw.FW_OK
    bad = fw.make_config("packet_split")
    s, _, _ = _noalloc(torch, rs, dh, 64, bad)
    assert s == fw.FW_EINVAL
    bad = fw.make_config("rule_split_grid")
    bad.reserved[1] = 3  # reserved fields must be zero, as for fw_classify_ex
    s, _, _ = _noalloc(torch, rs, dh, 64, bad)
    assert s == fw.FW_EINVAL
    ex = fw.lib().fw_classify_ex(rs.handle, ctypes.byref(hs), 64, None, None, None, ctypes.byref(bad))
    assert ex == fw.FW_EINVAL
    # an empty batch is a no-op for all three calls, and none of them clears the last failure
    assert L.fw_last_status() == fw.FW_EINVAL
    assert L.fw_classify_rule_split_noalloc(rs.handle, ctypes.byref(hs), 0, None, None, None, None) == fw.FW_OK
    assert L.fw_classify(rs.handle, ctypes.byref(hs), 0, None, None, None) == fw.FW_OK
    assert L.fw_last_status() == fw.FW_EINVAL
    # the largest accepted batch, with explicit slices
    n = fw.FW_NOALLOC_MAX_PACKETS
    hdr = W.gen_packets(rules, n, 7)
    dh = fw.headers_to_device(hdr)
    s, idx, act = _noalloc(torch, rs, dh, n, fw.make_config("rule_split_grid", rule_slices=3))
    want_idx, want_act = fw.fw_classify(rs, dh, n, config=fw.make_config("rule_split_grid", rule_slices=3))
    torch.cuda.synchronize()
    assert s == fw.FW_OK
    assert torch.equal(idx, want_idx) and torch.equal(act, want_act)
    rs.destroy()
