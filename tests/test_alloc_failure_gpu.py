"""Allocation failure injected on the host (fw_selftest_fail_alloc), walked across every allocation.

For each create call the armed failure moves from the call's first allocation to its last:
every failing call must raise FW_ENOMEM, hand back no object, and free what it held (checked
through the device's free memory for the rule set). The call then succeeds, and the objects it
builds, and the context, still classify correctly. No GPU fault is involved: the failure is
taken on the host before the CUDA allocator is reached. This file is collected last, so that a
failure here does not hide the other GPU tests.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1312_4188_gb300 import fw, workload as W

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_4188_gb300 import build
    build.build()
    yield torch
    fw.lib().fw_selftest_fail_alloc(-1)


def walk(create, limit=400):
    """Fail allocation k = 0, 1, ... of ``create()`` until it succeeds; every failure must be
    FW_ENOMEM. Returns (allocations the call makes, what the successful call returned)."""
    lib = fw.lib()
    try:
        for k in range(limit):
            lib.fw_selftest_fail_alloc(k)
            try:
                obj = create()
            except fw.FwError as e:
                assert e.status == fw.FW_ENOMEM, (k, e.status)
                continue
            return k, obj
    finally:
        lib.fw_selftest_fail_alloc(-1)
    raise AssertionError(f"no success within {limit} allocations")


def check(torch, idx, act, rules, hdr):
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert np.array_equal(idx.cpu().numpy(), want[0]) and np.array_equal(act.cpu().numpy(), want[1])


def test_ruleset(torch_cuda):
    torch = torch_cuda
    rules = W.gen_rules(100_000, 5)  # ~20 MB of device arrays: a leak per failure would show
    fw.fw_ruleset_create(rules).destroy()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    m, rs = walk(lambda: fw.fw_ruleset_create(rules))
    rs.destroy()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert m >= 10
    assert abs(free1 - free0) <= 64 << 20, f"free memory {free0} before the walk, {free1} after"
    rs = fw.fw_ruleset_create(rules)
    hdr = W.gen_packets(rules, 100_000, 6)
    idx, act = fw.fw_classify(rs, fw.headers_to_device(hdr))
    torch.cuda.synchronize()
    check(torch, idx, act, rules, hdr)
    rs.destroy()


def test_learned_index(torch_cuda):
    torch = torch_cuda
    rules = W.without_catch_alls(W.gen_rules(3000, 7))
    m, li = walk(lambda: fw.fw_lindex_create(rules, truncate=2))
    assert m >= 10
    hdr = W.gen_packets(rules, 50_000, 8)
    idx, act = fw.fw_lindex_classify(li, fw.headers_to_device(hdr))
    torch.cuda.synchronize()
    check(torch, idx, act, rules, hdr)
    li.destroy()


def test_plan(torch_cuda):
    torch = torch_cuda
    jobs, data = [], []
    for j in range(3):
        rules = W.gen_rules(500 * (j + 1), 10 + j)
        hdr = W.gen_packets(rules, 20_000 + 7 * j, 20 + j)
        dh = fw.headers_to_device(hdr)
        oi = torch.empty(len(hdr["src"]), dtype=torch.int32, device="cuda")
        oa = torch.empty(len(hdr["src"]), dtype=torch.uint8, device="cuda")
        jobs.append((fw.fw_ruleset_create(rules), dh, oi, oa))
        data.append((rules, hdr))
    m, plan = walk(lambda: fw.fw_plan_create(jobs))
    assert m >= 1
    plan.launch()
    torch.cuda.synchronize()
    for (rs, _, oi, oa), (rules, hdr) in zip(jobs, data):
        check(torch, oi, oa, rules, hdr)
        rs.destroy()
    plan.destroy()


def test_server(torch_cuda):
    torch = torch_cuda
    rules = W.gen_rules(1000, 30)
    rs = fw.fw_ruleset_create(rules)
    m, sv = walk(lambda: fw.Server([rs], slots=2, max_group_requests=8))
    assert m >= 5  # the staging arena and each slot's work lists
    hdr = W.gen_packets(rules, 10_000, 31)
    h = fw.pinned_headers(hdr)  # copy mode (the default) stages pinned host buffers
    oi = torch.empty(10_000, dtype=torch.int32).pin_memory()
    oa = torch.empty(10_000, dtype=torch.uint8).pin_memory()
    st, _ = sv.wait(sv.submit(0, h, oi, oa), timeout_us=30_000_000)
    assert st == fw.FW_OK
    check(torch, oi, oa, rules, hdr)
    sv.destroy()
    rs.destroy()


def test_host_pipeline(torch_cuda):
    torch = torch_cuda
    m, pl = walk(lambda: fw.fw_host_pipeline_create(1 << 16, 2))
    assert m == 14  # seven staging arrays per stream
    rules = W.gen_rules(1000, 40)
    rs = fw.fw_ruleset_create(rules)
    hdr = W.gen_packets(rules, 200_003, 41)  # several 65,536-packet chunks and a ragged tail
    h = fw.pinned_headers(hdr)
    oi = torch.empty(200_003, dtype=torch.int32).pin_memory()
    oa = torch.empty(200_003, dtype=torch.uint8).pin_memory()
    fw.fw_classify_host(pl, rs, h, oi, oa)
    check(torch, oi, oa, rules, hdr)
    pl.destroy()
    rs.destroy()
