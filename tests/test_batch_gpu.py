"""Batched persistent plans against fw_classify and the CPU oracle (bit-exact per job)."""
import os

import numpy as np
import pytest

import oracle
from paper_1312_4188_gb300 import autotune, fw, workload as W

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_4188_gb300 import build
    build.build()
    return torch


def no_catch_all(rules):
    return rules[~((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0))]


def many_protocols(rules):
    # exact protocols beyond TCP, UDP and ICMP share the "other" class: no bucket filter
    rules = rules.copy()
    rules["proto_any"] = 0
    rules["proto"] = np.arange(len(rules)) % 12
    return rules


def make_jobs(torch, specs, misalign=()):
    jobs, host = [], []
    for i, (nr, npk, drop) in enumerate(specs):
        rules = W.gen_rules(nr, 500 + i)
        if drop == "protos":
            rules = many_protocols(rules)
        elif drop:
            rules = no_catch_all(rules)
        hdr = W.gen_packets(rules, npk, 600 + i)
        rs = fw.fw_ruleset_create(rules)
        if i in misalign:
            pad = {f: np.concatenate([np.zeros(1, hdr[f].dtype), hdr[f]]) for f in W.HEADER_FIELDS}
            dh = {f: t[1:] for f, t in fw.headers_to_device(pad).items()}
        else:
            dh = fw.headers_to_device(hdr)
        oi = torch.full((npk,), -9, dtype=torch.int32, device="cuda")
        oa = torch.full((npk,), 7, dtype=torch.uint8, device="cuda")
        jobs.append((rs, dh, oi, oa))
        host.append((rules, hdr))
    return jobs, host


# every rule set here has a bucket filter ...
FILTER_SPECS = [(0, 10, False), (1, 1, False), (33, 5, True), (300, 1000, True), (5000, 50_000, True),
                (2000, 0, False), (64, 4099, False), (700, 30_000, False), (12_000, 20_000, True), (3, 129, True),
                (40, 2, False), (200, 3, True)]
# ... and two here have none (their items take the general kernel's scan path)
SPECS = FILTER_SPECS[:10] + [(300, 5000, "protos"), (60, 1001, "protos")]


@pytest.mark.parametrize("cfg,threads", [(None, 0), ([(256, 128, 8), (4096, 256, 16), (0, 384, 32)], 0),
                                         ([(100, 4096, 4)], 64)],
                         ids=["default", "three_classes", "big_items"])
@pytest.mark.parametrize("graph", [False, True], ids=["direct", "graph"])
def test_plan_matches_scan_and_oracle(torch_cuda, cfg, threads, graph):
    torch = torch_cuda
    jobs, host = make_jobs(torch, SPECS, misalign=(3, 7, 11))
    assert [j[0].filter()["words"] == 0 for j in jobs].count(True) == 2
    plan = fw.fw_plan_create(jobs, fw.make_plan_config(cfg, block_threads=threads) if cfg else None)
    assert plan.kernel() == 0  # the general kernel: two jobs have no filter
    plan.launch(graph=graph)
    plan.launch(graph=graph)  # a relaunch rewrites the same outputs
    torch.cuda.synchronize()
    for (rs, dh, oi, oa), (rules, hdr) in zip(jobs, host):
        n = len(hdr["src"])
        if n == 0:
            continue
        si, sa = fw.fw_classify(rs, dh, n)
        torch.cuda.synchronize()
        assert torch.equal(oi, si) and torch.equal(oa, sa)
        want = oracle.classify(rules, hdr, threads=THREADS)
        assert np.array_equal(oi.cpu().numpy(), want[0]) and np.array_equal(oa.cpu().numpy(), want[1])
    plan.destroy()
    for j in jobs:
        j[0].destroy()


@pytest.mark.parametrize("per_sm", [0, 3], ids=["two_blocks", "three_blocks"])
@pytest.mark.parametrize("graph", [False, True], ids=["direct", "graph"])
def test_filter_only_plan(torch_cuda, per_sm, graph):
    """Every job has a bucket filter: the filter-only kernel (four packets a lane; ragged and
    misaligned jobs take its scalar loads and stores) must equal fw_classify and the oracle."""
    torch = torch_cuda
    jobs, host = make_jobs(torch, FILTER_SPECS, misalign=(2, 7, 10))
    assert all(j[0].filter()["words"] > 0 for j in jobs)
    plan = fw.fw_plan_create(jobs, fw.make_plan_config(None, blocks_per_sm=per_sm))
    assert plan.kernel() == (3 if per_sm == 3 else 2)
    plan.launch(graph=graph)
    torch.cuda.synchronize()
    for (rs, dh, oi, oa), (rules, hdr) in zip(jobs, host):
        n = len(hdr["src"])
        if n == 0:
            continue
        si, sa = fw.fw_classify(rs, dh, n)
        torch.cuda.synchronize()
        assert torch.equal(oi, si) and torch.equal(oa, sa)
        want = oracle.classify(rules, hdr, threads=THREADS)
        assert np.array_equal(oi.cpu().numpy(), want[0]) and np.array_equal(oa.cpu().numpy(), want[1])
    plan.destroy()
    for j in jobs:
        j[0].destroy()


def test_graph_replay_sees_new_headers(torch_cuda):
    torch = torch_cuda
    jobs, host = make_jobs(torch, [(500, 3000, True), (40, 777, False)])
    plan = fw.fw_plan_create(jobs)
    plan.launch(graph=True)
    torch.cuda.synchronize()
    # overwrite the first job's headers in place (same addresses), replay the graph
    rules = host[0][0]
    new = W.gen_packets(rules, 3000, 4242)
    for f, t in fw.headers_to_device(new).items():
        jobs[0][1][f].copy_(t)
    plan.launch(graph=True)
    torch.cuda.synchronize()
    want = oracle.classify(rules, new)
    assert np.array_equal(jobs[0][2].cpu().numpy(), want[0])
    plan.destroy()


def test_batched_256_sets_scaled(torch_cuda):
    """256 independent sets (log-uniform 64..4096 rules, 1K..16K packets): every verdict vs the oracle."""
    torch = torch_cuda
    data = W.gen_batched(256, seed=3, rules_range=(64, 4096), packets_range=(1024, 16384))
    jobs = []
    for rules, hdr in data:
        n = len(hdr["src"])
        jobs.append((fw.fw_ruleset_create(rules), fw.headers_to_device(hdr),
                     torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda")))
    classes, table = autotune.tune_plan_classes(jobs, reps=2)
    plan = fw.fw_plan_create(jobs, fw.make_plan_config(classes))
    plan.launch(graph=True)
    torch.cuda.synchronize()
    for (rs, dh, oi, oa), (rules, hdr) in zip(jobs, data):
        want = oracle.classify(rules, hdr, threads=THREADS)
        assert np.array_equal(oi.cpu().numpy(), want[0]) and np.array_equal(oa.cpu().numpy(), want[1])
    plan.destroy()


def test_plan_rejects_bad_config(torch_cuda):
    torch = torch_cuda
    jobs, _ = make_jobs(torch, [(10, 10, False)])
    with pytest.raises(fw.FwError):
        fw.fw_plan_create(jobs, fw.make_plan_config([(0, 100, 16)]))  # not a multiple of 128
    with pytest.raises(fw.FwError):
        fw.fw_plan_create(jobs, fw.make_plan_config([(0, 4096, 16)], block_threads=1024))  # shared memory too big
