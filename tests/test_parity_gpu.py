"""CUDA path against the CPU oracle, element by element (bit-exact rule index and action).

Every call goes through the C ABI (libfw.so). Sizes span several rule
chunks / thread quads and ragged tails; the full-size scan (10,000 rules x
16,777,216 packets, Zipf traffic) is checked on a fixed 1M-packet sample.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1312_4188_gb300 import fw, workload as W

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1

CONFIGS = [
    ("packet_split", {}),
    ("packet_split", {"partition": 2}),
    ("packet_split", {"compact": 2, "partition": 1}),
    ("packet_split", {"compact": 1, "partition": 1, "lane_packets": 1}),
    ("packet_split", {"compact": 1, "partition": 1, "lane_packets": 1, "smem_rules": 256, "segment_rules": 4,
                      "block_threads": 256}),
    ("packet_split", {"compact": 1, "partition": 1, "block_threads": 768, "blocks_per_sm": 2, "smem_rules": 256}),
    ("packet_split", {"compact": 1, "partition": 1, "lane_packets": 2, "block_threads": 1024, "blocks_per_sm": 1}),
    ("packet_split", {"compact": 1, "partition": 1, "lane_packets": 2, "block_threads": 256, "blocks_per_sm": 1,
                      "segment_rules": 4, "smem_rules": -1}),
    ("packet_split", {"compact": 1, "partition": 2, "block_threads": 512, "blocks_per_sm": 2, "segment_rules": 8}),
    ("packet_split", {"predicate": fw.FW_PRED_CMP}),
    ("packet_split", {"predicate": fw.FW_PRED_CLAMP}),
    ("packet_split", {"predicate": fw.FW_PRED_RANGE}),
    ("packet_split", {"predicate": fw.FW_PRED_RANGE, "compact": 2}),
    ("packet_split", {"smem_rules": -1, "segment_rules": 8}),
    ("packet_split", {"smem_rules": 256, "segment_rules": 4, "packets_per_group": 256, "block_threads": 512,
                      "blocks_per_sm": 2}),
    ("packet_split", {"compact": 2}),
    ("packet_split", {"compact": 2, "predicate": fw.FW_PRED_CLAMP}),
    ("packet_split", {"compact": 2, "smem_rules": -1, "predicate": fw.FW_PRED_CMP}),
    ("packet_split", {"compact": 2, "block_threads": 96, "blocks_per_sm": 1, "smem_rules": 512}),
    ("packet_split", {"filter": 2}),
    ("rule_split_warp", {}),
    ("rule_split_warp", {"block_threads": 64, "blocks_per_sm": 8}),
    ("rule_split_warp", {"segment_rules": 2}),
    ("rule_split_warp", {"segment_rules": 8}),
    ("rule_split_warp", {"segment_rules": 16, "block_threads": 96}),
    ("rule_split_warp", {"partition": 2}),
    ("rule_split_warp", {"partition": 2, "packets_per_group": 32, "block_threads": 64}),
    ("rule_split_block", {}),
    ("rule_split_block", {"block_threads": 160}),
    ("rule_split_block", {"block_threads": 32}),
    ("rule_split_block", {"partition": 2}),
    ("rule_split_block", {"partition": 2, "block_threads": 64, "packets_per_group": 96}),
    ("rule_split_block", {"partition": 2, "block_threads": 160}),
    ("rule_split_block", {"partition": 2, "block_threads": 512, "packets_per_group": 128}),
    ("rule_split_grid", {}),
    ("rule_split_grid", {"rule_slices": 3}),
    ("rule_split_grid", {"rule_slices": 2, "block_threads": 96}),
    ("rule_split_grid", {"partition": 2}),
    ("rule_split_grid", {"partition": 2, "rule_slices": 3}),
    ("rule_split_grid", {"partition": 2, "rule_slices": 64, "packets_per_group": 32}),
]
CFG_IDS = [f"{m}-{'-'.join(f'{k}{v}' for k, v in kw.items()) or 'default'}" for m, kw in CONFIGS]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_4188_gb300 import build
    build.build()
    return torch


def run_gpu(torch, rules, hdr, mode, kw, rs=None, offset=0):
    own = rs is None
    if own:
        rs = fw.fw_ruleset_create(rules)
    n = len(hdr["src"])
    if offset:
        # misaligned views: the same packets starting `offset` elements into each buffer
        pad = {f: np.concatenate([np.zeros(offset, hdr[f].dtype), hdr[f]]) for f in W.HEADER_FIELDS}
        dh = {f: t[offset:] for f, t in fw.headers_to_device(pad).items()}
    else:
        dh = fw.headers_to_device(hdr)
    idx, act = fw.fw_classify(rs, dh, n, config=fw.make_config(mode, **kw))
    torch.cuda.synchronize()
    assert rs.check() == fw.FW_OK
    out = idx.cpu().numpy(), act.cpu().numpy()
    if own:
        rs.destroy()
    return out


def assert_same(got, want, what=""):
    gi, ga = got
    wi, wa = want[0], want[1]
    bad = np.nonzero((gi != wi) | (ga != wa))[0]
    assert bad.size == 0, (f"{what}: {bad.size} mismatches, first at {bad[0]}: got ({gi[bad[0]]},{ga[bad[0]]}) "
                           f"want ({wi[bad[0]]},{wa[bad[0]]})")


def no_catch_all(rules):
    keep = ~((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0))
    return rules[keep]


@pytest.mark.parametrize("mode,kw", CONFIGS, ids=CFG_IDS)
def test_plain_1k_x_100k(torch_cuda, mode, kw):
    rules, hdr = W.make_workload("plain_1k_x_100k")
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert_same(run_gpu(torch_cuda, rules, hdr, mode, kw), want, mode)


@pytest.mark.parametrize("mode,kw", CONFIGS, ids=CFG_IDS)
@pytest.mark.parametrize("n_rules,n_pkts", [(0, 100), (1, 1), (1, 37), (31, 64), (32, 4), (33, 5), (255, 1023),
                                            (256, 4097), (257, 3), (1000, 17), (4000, 20_011)])
def test_sizes_no_catch_all(torch_cuda, mode, kw, n_rules, n_pkts):
    # without catch-alls every unmatched packet scans the whole list: tails of
    # the rule chunks, the shared-memory prefix and the global tail all matter
    rules = no_catch_all(W.gen_rules(n_rules, 100 + n_rules))
    hdr = W.gen_packets(rules, n_pkts, 7 + n_pkts)
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert_same(run_gpu(torch_cuda, rules, hdr, mode, kw), want, f"{mode} {n_rules}x{n_pkts}")


@pytest.mark.parametrize("mode,kw", [("packet_split", {}), ("packet_split", {"compact": 2}), ("rule_split_warp", {}),
                                     ("rule_split_grid", {})], ids=["ps", "ps_lockstep", "rsw", "rsg"])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_misaligned_buffers(torch_cuda, mode, kw, offset):
    rules = no_catch_all(W.gen_rules(700, 5))
    hdr = W.gen_packets(rules, 5003, 6)
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert_same(run_gpu(torch_cuda, rules, hdr, mode, kw, offset=offset), want, f"{mode} offset {offset}")


@pytest.mark.parametrize("mode,kw", CONFIGS, ids=CFG_IDS)
def test_golden_policy_on_gpu(torch_cuda, mode, kw):
    import oracle_pins as P
    rules, h, expect = P.parse_golden()
    gi, ga = run_gpu(torch_cuda, rules, h, mode, kw)
    assert [(int(a), int(b)) for a, b in zip(gi, ga)] == expect


@pytest.mark.parametrize("mode,kw", [("packet_split", {}), ("packet_split", {"compact": 2, "predicate": 2}),
                                     ("packet_split", {"compact": 2}), ("packet_split", {"partition": 2}),
                                     ("packet_split", {"compact": 1, "packets_per_group": 128}),
                                     ("rule_split_warp", {}), ("rule_split_block", {}), ("rule_split_grid", {})],
                         ids=["ps", "ps_lockstep_cmp", "ps_lockstep_part", "ps_nopart", "ps_compact_part",
                              "rsw", "rsb", "rsg"])
def test_special_rule_sets(torch_cuda, mode, kw):
    import oracle_pins as P
    rng = np.random.default_rng(3)
    many = no_catch_all(W.gen_rules(2000, 6))
    many["proto_any"] = (rng.random(len(many)) < 0.1).astype(np.uint8)
    many["proto"] = rng.integers(0, 256, size=len(many))  # far more exact protocols than classes
    cases = {
        "many_protocols": many,
        "catch_all_first": np.concatenate([P.catch_all(W.DROP), W.gen_rules(100, 1)]).astype(W.RULE_DTYPE),
        "catch_all_last": np.concatenate([no_catch_all(W.gen_rules(600, 2)), P.catch_all(W.ACCEPT)]).astype(
            W.RULE_DTYPE),
        "tiny_domain": P.random_tiny_rules(rng, 4),
        "exact_only": W.gen_rules(300, 4),
        "any_protocol_only": W.gen_rules(500, 5),  # one protocol class
    }
    cases["any_protocol_only"]["proto_any"] = 1
    cases["any_protocol_only"]["proto"] = 0
    ex = cases["exact_only"]
    ex["src_prefix"] = ex["dst_prefix"] = 32
    ex["sport_hi"] = ex["sport_lo"]
    ex["dport_hi"] = ex["dport_lo"]
    ex["proto_any"] = 0
    for name, rules in cases.items():
        if name == "tiny_domain":
            hdr = P.headers_from_tuples(P.tiny_domain())
        else:
            hdr = W.gen_packets(rules, 6000, 9)
        want = oracle.classify(rules, hdr, threads=THREADS)
        assert_same(run_gpu(torch_cuda, rules, hdr, mode, kw), want, f"{mode} {name}")


def test_result_independent_of_batch_split(torch_cuda):
    rules, hdr = W.make_workload("plain_1k_x_100k", 30_000)
    rs = fw.fw_ruleset_create(rules)
    whole = run_gpu(torch_cuda, rules, hdr, "packet_split", {}, rs=rs)
    parts = [run_gpu(torch_cuda, rules, {f: hdr[f][a:b] for f in W.HEADER_FIELDS}, "packet_split", {}, rs=rs)
             for a, b in [(0, 1), (1, 4099), (4099, 30_000)]]
    assert np.array_equal(whole[0], np.concatenate([p[0] for p in parts]))
    assert np.array_equal(whole[1], np.concatenate([p[1] for p in parts]))
    rs.destroy()


@pytest.fixture(scope="module")
def big(torch_cuda):
    rules, hdr = W.make_workload("scan_10k_x_16m_zipf")
    n = len(hdr["src"])
    pos = W.sample_positions(n, 1 << 20, seed=99)
    want = oracle.classify(rules, W.take(hdr, pos), threads=THREADS)
    return rules, hdr, fw.headers_to_device(hdr), want, pos


@pytest.mark.parametrize("mode,kw", [("packet_split", {}), ("packet_split", {"compact": 2}),
                                     ("packet_split", {"partition": 2}),
                                     ("packet_split", {"compact": 2, "predicate": fw.FW_PRED_CLAMP}),
                                     ("packet_split", {"predicate": fw.FW_PRED_RANGE}),
                                     ("rule_split_warp", {}), ("rule_split_block", {}), ("rule_split_grid", {})],
                         ids=["ps", "ps_lockstep", "ps_nopart", "ps_lockstep_clamp", "ps_range", "rsw", "rsb", "rsg"])
def test_scan_10k_x_16m_sampled(torch_cuda, big, mode, kw):
    torch = torch_cuda
    rules, hdr, dh, want, pos = big
    n = len(hdr["src"])
    rs = fw.fw_ruleset_create(rules)
    idx, act = fw.fw_classify(rs, dh, n, config=fw.make_config(mode, **kw))
    torch.cuda.synchronize()
    assert rs.check() == fw.FW_OK
    pos_t = torch.from_numpy(pos).to(idx.device)
    got = idx[pos_t].cpu().numpy(), act[pos_t].cpu().numpy()
    assert_same(got, want, mode)
    # properties that hold at every position: indices in range, action consistent with the rule
    gi = idx.cpu().numpy()
    assert gi.min() >= -1 and gi.max() < len(rules)
    ga = act.cpu().numpy()
    assert np.array_equal(ga, np.where(gi >= 0, rules["action"][np.maximum(gi, 0)], W.DROP))
    rs.destroy()


@pytest.mark.parametrize("n_pkts", [98_303, 98_304, 200_003, 1_048_576, 4_194_304, 4_194_305])
@pytest.mark.parametrize("catch_all", [True, False], ids=["plain", "no_catch_all"])
def test_default_shapes_around_size_thresholds(torch_cuda, n_pkts, catch_all):
    """AUTO switches lockstep -> two-packet scan in 128-thread blocks at 98,304 packets and to
    1,024-thread blocks above 2^22: every side of both switches against the oracle."""
    rules = W.gen_rules(1000, 21)
    if not catch_all:
        rules = no_catch_all(rules)
    hdr = W.gen_packets(rules, n_pkts, 23)
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert_same(run_gpu(torch_cuda, rules, hdr, "packet_split", {}), want, f"auto {n_pkts}")


def test_partition_key_on_destination(torch_cuda):
    """With every source prefix a wildcard the rule set must key its partition on the destination
    address; every partitioned kernel then agrees with the oracle."""
    rules = W.gen_rules(2000, 31)
    rules["src_prefix"] = 0
    rules = no_catch_all(rules)
    rs = fw.fw_ruleset_create(rules)
    part = rs.partition()
    assert part["key_field"] == 2 and 1 <= part["key_bits"] <= 3 and part["classes"] <= 8
    plan = fw.fw_partition_plan(rules, 1)  # the host-only plan of the same rules
    assert (plan["classes"], plan["key_field"], plan["key_bits"]) == (part["classes"], part["key_field"],
                                                                      part["key_bits"])
    hdr = W.gen_packets(rules, 300_000, 32)
    want = oracle.classify(rules, hdr, threads=THREADS)
    for kw in ({}, {"compact": 1}, {"compact": 1, "lane_packets": 1}, {"compact": 2, "partition": 1},
               {"compact": 1, "block_threads": 256, "segment_rules": 8}):
        assert_same(run_gpu(torch_cuda, rules, hdr, "packet_split", kw, rs=rs), want, f"dst key {kw}")
    rs.destroy()


def test_partition_matches_host_plan_up_to_first_catch_all(torch_cuda):
    """A rule set partitions its rules up to and including the first catch-all (no packet gets
    past it): the plan of exactly those rules."""
    rules = W.gen_rules(10_000, 3)
    rs = fw.fw_ruleset_create(rules)
    part = rs.partition()
    ca = rs.first_catch_all
    assert ca >= 0
    plan = fw.fw_partition_plan(rules[:ca + 1], 1)
    rs.destroy()
    assert (plan["classes"], plan["key_field"], plan["key_bits"]) == (part["classes"], part["key_field"],
                                                                      part["key_bits"])
