"""Learned-index decomposition classifier against the CPU oracle and the linear scan.

Bit-exact rule index and action. The linear scan (fw_classify) stays the
judge at full size: 100,000 rules x 67,108,864 packets are compared
element by element with it, and a fixed 1M-packet sample with the oracle.
No verified search window may fail (fallbacks == 0).
"""
import os

import numpy as np
import pytest

import oracle
import partition_ref as R
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
    return torch


def no_catch_all(rules):
    return rules[~((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0))]


def run_li(torch, rules, hdr, **kw):
    li = fw.fw_lindex_create(rules, **kw)
    idx, act = fw.fw_lindex_classify(li, fw.headers_to_device(hdr))
    torch.cuda.synchronize()
    st = li.stats()
    li.destroy()
    return idx.cpu().numpy(), act.cpu().numpy(), st


@pytest.mark.parametrize("kw", [{}, {"truncate": 2}, {"segments": 1}, {"segments": 16, "truncate": 2},
                                {"segments": 65536}], ids=["default", "full", "seg1", "seg16full", "seg64k"])
@pytest.mark.parametrize("n_rules,n_pkts,drop_ca", [(0, 50, False), (1, 1, False), (33, 1000, True),
                                                    (255, 4097, True), (1000, 20_000, False), (4000, 30_001, True)])
def test_parity_vs_oracle(torch_cuda, kw, n_rules, n_pkts, drop_ca):
    rules = W.gen_rules(n_rules, 300 + n_rules)
    if drop_ca:
        rules = no_catch_all(rules)
    hdr = W.gen_packets(rules, n_pkts, 17 + n_pkts)
    want = oracle.classify(rules, hdr, threads=THREADS)
    gi, ga, st = run_li(torch_cuda, rules, hdr, **kw)
    assert np.array_equal(gi, want[0]) and np.array_equal(ga, want[1])
    assert st["fallbacks"] == 0


def test_golden_and_tiny_domain(torch_cuda):
    import oracle_pins as P
    rules, h, expect = P.parse_golden()
    gi, ga, _ = run_li(torch_cuda, rules, h)
    assert [(int(a), int(b)) for a, b in zip(gi, ga)] == expect
    rng = np.random.default_rng(5)
    dom = P.headers_from_tuples(P.tiny_domain())
    for _ in range(20):
        rules = P.random_tiny_rules(rng, int(rng.integers(1, 5)))
        want = oracle.classify(rules, dom)
        gi, ga, st = run_li(torch_cuda, rules, dom, truncate=2)
        assert np.array_equal(gi, want[0]) and np.array_equal(ga, want[1])
        assert st["fallbacks"] == 0


def test_stats_shape(torch_cuda):
    rules = no_catch_all(W.gen_rules(2000, 8))
    li = fw.fw_lindex_create(rules, truncate=2)
    st = li.stats()
    assert st["rules_indexed"] == len(rules)
    assert all(1 <= m <= 2 * len(rules) + 1 for m in st["intervals"])
    assert st["intervals"][4] <= 257
    # the scan's partition, keyed by what a packet here reads: whole 128-rule row words (at least
    # one), the key with the lowest mean (partition_ref's definition; fw_partition_plan agrees)
    words = R.best_key(rules, 128)
    assert (st["key_field"], st["key_bits"]) == words
    plan = fw.fw_partition_plan(rules, 128)
    assert (plan["key_field"], plan["key_bits"], plan["classes"]) == (*words, st["classes"])
    # the scan reads rules one at a time: its key minimises the mean length (here another key)
    rs = fw.fw_ruleset_create(rules)
    part = rs.partition()
    rs.destroy()
    length = R.best_key(rules, 1)
    assert (part["key_field"], part["key_bits"]) == length != words
    lists = R.class_sublists(rules, *words)
    assert len(lists) == st["classes"]
    wpr = [max(4, -(-len(x) // 128) * 4) for x in lists]
    assert st["words_per_row"] == max(wpr)
    # one set of rows per class over the four address and port fields (three exact
    # protocols here, so no class mixes protocols and none has protocol rows)
    assert len(set(rules["proto"][rules["proto_any"] == 0].tolist())) <= 7
    rows = sum(st["intervals"][:4])
    assert st["bitmap_bytes"] == rows * 4 * sum(wpr)
    li.destroy()


def test_full_size_against_scan_and_oracle(torch_cuda):
    torch = torch_cuda
    rules, hdr = W.make_workload("lindex_100k_x_64m")
    n = len(hdr["src"])
    dh = fw.headers_to_device(hdr)
    rs = fw.fw_ruleset_create(rules)
    s_idx, s_act = fw.fw_classify(rs, dh, n)
    li = fw.fw_lindex_create(rules, truncate=2)  # the full 100K-rule structure
    l_idx, l_act = fw.fw_lindex_classify(li, dh, n)
    torch.cuda.synchronize()
    st = li.stats()
    assert st["rules_indexed"] == 100_000 and st["fallbacks"] == 0
    assert torch.equal(l_idx, s_idx) and torch.equal(l_act, s_act), "learned index differs from the linear scan"
    pos = W.sample_positions(n, 1 << 20, seed=99)
    want = oracle.classify(rules, W.take(hdr, pos), threads=THREADS)
    pt = torch.from_numpy(pos).cuda()
    assert np.array_equal(l_idx[pt].cpu().numpy(), want[0]) and np.array_equal(l_act[pt].cpu().numpy(), want[1])
    li.destroy()
    rs.destroy()


@pytest.mark.parametrize("truncate", [1, 2])
def test_many_protocols_other_class(torch_cuda, truncate):
    """More exact protocols than classes: the "other" class then also holds exact-protocol rules
    (its rows must keep them, in list order, with the protocol-any rules)."""
    rng = np.random.default_rng(11)
    rules = no_catch_all(W.gen_rules(3000, 12))
    rules["proto_any"] = (rng.random(len(rules)) < 0.1).astype(np.uint8)
    rules["proto"] = rng.integers(0, 256, size=len(rules))
    hdr = W.gen_packets(rules, 40_000, 13)
    # half the packets get a random protocol, many of them without a class of their own
    flip = rng.random(len(hdr["proto"])) < 0.5
    hdr["proto"] = np.where(flip, rng.integers(0, 256, size=len(flip)), hdr["proto"]).astype(np.uint8)
    want = oracle.classify(rules, hdr, threads=THREADS)
    gi, ga, st = run_li(torch_cuda, rules, hdr, truncate=truncate)
    assert st["classes"] == 8 and st["fallbacks"] == 0
    assert np.array_equal(gi, want[0]) and np.array_equal(ga, want[1])
    assert (want[0] >= 0).mean() > 0.2  # the case is not all default deny (here a third match)
