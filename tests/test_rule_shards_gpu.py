"""Rule split across ranks, exercised on one GPU as virtual shards.

Each virtual rank's rule range is its own CUDA rule set, classified by fw_classify; the ranks'
global first matches combine by an elementwise minimum (what all_reduce MIN does across GPUs)
and the action comes from the whole list's table. The result must equal the whole-list
classification bit for bit, and the oracle on a fixed sample. This file is collected after the
other GPU tests, so that a failure here does not hide them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1312_4188_gb300 import fw, rule_shards as S, workload as W

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


CASES = [  # (rules seed, rules, packets, Zipf, drop catch-alls)
    (3, 10_000, 1 << 20, 1.1, False),
    (1, 1000, 100_000, None, False),
    (4, 500, 30_001, None, True),
]


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_virtual_shards_equal_the_whole_list(torch_cuda, world):
    torch = torch_cuda
    for seed, n_rules, n, zipf, drop in CASES:
        rules = W.gen_rules(n_rules, seed)
        if drop:
            rules = W.without_catch_alls(rules)
        hdr = W.gen_packets(rules, n, seed + 1, zipf_s=zipf)
        dh = fw.headers_to_device(hdr)
        g = None
        for r in range(world):
            lo, hi = S.shard_range(len(rules), world, r)
            rs = fw.fw_ruleset_create(rules[lo:hi])
            local, _ = fw.fw_classify(rs, dh)
            part = S.to_global(local, lo)
            g = part if g is None else torch.minimum(g, part)
            torch.cuda.synchronize()
            rs.destroy()
        actions = torch.as_tensor(rules["action"].astype(np.uint8), device="cuda")
        idx, act = S.finalize(g, actions)
        rs = fw.fw_ruleset_create(rules)
        w_idx, w_act = fw.fw_classify(rs, dh)
        torch.cuda.synchronize()
        rs.destroy()
        assert torch.equal(idx, w_idx) and torch.equal(act, w_act), f"world {world}, {n_rules} rules"
        pos = W.sample_positions(n, 50_000, seed=7)
        want = oracle.classify(rules, W.take(hdr, pos), threads=THREADS)
        pt = torch.from_numpy(pos).cuda()
        assert np.array_equal(idx[pt].cpu().numpy(), want[0]) and np.array_equal(act[pt].cpu().numpy(), want[1])


def test_rule_shard_alone_is_the_whole_list(torch_cuda):
    """One rank, no process group: the combine is the identity and RuleShard is fw_classify."""
    torch = torch_cuda
    rules = W.gen_rules(2000, 9)
    hdr = W.gen_packets(rules, 200_000, 10)
    dh = fw.headers_to_device(hdr)
    sh = S.RuleShard(rules, 1, 0)
    idx, act = sh.classify(dh)
    torch.cuda.synchronize()
    sh.destroy()
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert np.array_equal(idx.cpu().numpy(), want[0]) and np.array_equal(act.cpu().numpy(), want[1])


@pytest.mark.parametrize("world", [4, 9])
def test_more_ranks_than_rules(torch_cuda, world):
    """RuleShard on ranks whose range is empty (more ranks than rules): an empty CUDA rule set
    answers no match for every packet, and the minimum over ranks equals the oracle, DROP for
    every packet that no rule matches."""
    torch = torch_cuda
    for seed, rules in ((21, W.gen_rules(3, 21)), (22, W.without_catch_alls(W.gen_rules(2, 22))),
                        (23, W.empty_rules(0))):
        src = rules if len(rules) else W.gen_rules(40, 24)
        hdr = W.gen_packets(src, 20_000, seed + 5)
        dh = fw.headers_to_device(hdr)
        g = None
        for r in range(world):
            sh = S.RuleShard(rules, world, r)
            local, _ = fw.fw_classify(sh.rs, dh)
            part = S.to_global(local, sh.lo)
            g = part if g is None else torch.minimum(g, part)
            torch.cuda.synchronize()
            sh.destroy()
        actions = torch.as_tensor(rules["action"].astype(np.uint8), device="cuda")
        idx, act = S.finalize(g, actions)
        want = oracle.classify(rules, hdr, threads=THREADS)
        got_i, got_a = idx.cpu().numpy(), act.cpu().numpy()
        assert np.array_equal(got_i, want[0]) and np.array_equal(got_a, want[1]), f"{len(rules)} rules"
        assert np.all(got_a[want[0] < 0] == fw.FW_DROP)
