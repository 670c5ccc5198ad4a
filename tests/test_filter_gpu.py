"""The bucket-filter packet split against the CPU oracle, element by element.

Every call goes through the C ABI. The rule sets are built so that the filter
applies and so that they reach the cases its exactness rests on: address
prefixes of every length 0..32 (lengths 1..7 cover several address buckets, 8
and below are decided by the bucket alone), port ranges that cross or line up
with the 4,096-port bucket edges, exact ports on those edges, rules that need
no exact test (whole buckets on every field), one- and two-word bitmaps, wider
ones, ones of 32 words or more (read through row summaries), the partition's
address key, and
packets that no rule of their class matches (default deny). Edge packets sit
just inside and just outside every rule's prefix and port range.
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
    return torch


def edge_rules(n, seed, whole_share=0.15):
    """n rules with prefixes over 0..32, port ranges on and across 4,096 edges, some whole-bucket rules."""
    rng = np.random.default_rng(seed)
    r = W.gen_rules(n, seed)
    r["src_prefix"] = rng.integers(0, 33, n)
    r["dst_prefix"] = rng.integers(0, 33, n)
    for lo_f, hi_f in (("sport_lo", "sport_hi"), ("dport_lo", "dport_hi")):
        kind = rng.integers(0, 6, n)
        lo = rng.integers(0, 65536, n)
        width = rng.integers(1, 9000, n)
        edge = rng.integers(0, 16, n) * 4096
        lo_v = np.where(kind == 0, 0, np.where(kind == 1, lo, np.where(kind == 2, edge, np.where(kind == 3, edge - 1, np.where(kind == 4, np.maximum(edge - width // 2, 0), edge)))))
        lo_v = np.clip(lo_v, 0, 65535)
        hi_v = np.where(kind == 0, 65535, np.where(kind == 1, lo_v, np.where(kind == 5, np.minimum(lo_v + 4095, 65535), np.minimum(lo_v + width, 65535))))
        r[lo_f] = lo_v
        r[hi_f] = hi_v
    u = rng.random(n)
    whole = u < whole_share
    # nearly whole: every field on bucket edges but one port end a little inside its bucket
    near = (u >= whole_share) & (u < 2 * whole_share)
    wn = whole | near
    r["src_prefix"][wn] = rng.integers(0, 9, wn.sum())
    r["dst_prefix"][wn] = rng.integers(0, 9, wn.sum())
    for lo_f, hi_f in (("sport_lo", "sport_hi"), ("dport_lo", "dport_hi")):
        a = rng.integers(0, 16, wn.sum())
        b = np.minimum(a + rng.integers(0, 4, wn.sum()), 15)
        r[lo_f][wn] = a * 4096
        r[hi_f][wn] = b * 4096 + 4095
    k = np.nonzero(near)[0]
    which = rng.integers(0, 4, k.size)  # sport lo / sport hi / dport lo / dport hi moved inside
    step = rng.integers(1, 200, k.size)
    for f, w in (("sport_lo", 0), ("sport_hi", 1), ("dport_lo", 2), ("dport_hi", 3)):
        sel = k[which == w]
        v = r[f][sel].astype(np.int64) + (step[which == w] if w % 2 == 0 else -step[which == w])
        r[f][sel] = v
    return r


def edge_packets(rules, seed, per_rule=8):
    """Packets on the edges of every rule: just inside / just outside its prefixes and port ranges."""
    rng = np.random.default_rng(seed)
    n = len(rules) * per_rule
    k = np.repeat(np.arange(len(rules)), per_rule)
    r = rules[k]
    h = {}
    for f, pf in (("src", "src_prefix"), ("dst", "dst_prefix")):
        a = r[f + "_addr"].astype(np.int64)
        plen = r[pf].astype(np.int64)
        low = rng.integers(0, 1 << 32, n, dtype=np.int64)
        span = np.left_shift(np.int64(1), 32 - plen)
        inside = (a - a % span) + low % span
        # flip the lowest prefix bit: just outside (for prefix >= 1)
        outside = inside ^ np.where(plen > 0, np.left_shift(np.int64(1), np.maximum(32 - plen, 0)), 0)
        pick = rng.random(n) < 0.25
        h[f] = np.where(pick, outside, inside).astype(np.uint32)
    for f, lo_f, hi_f in (("sport", "sport_lo", "sport_hi"), ("dport", "dport_lo", "dport_hi")):
        lo = r[lo_f].astype(np.int64)
        hi = r[hi_f].astype(np.int64)
        c = rng.integers(0, 6, n)
        v = np.where(c == 0, lo, np.where(c == 1, hi, np.where(c == 2, lo - 1, np.where(c == 3, hi + 1,
                     lo + rng.integers(0, 1 << 16, n) % (hi - lo + 1)))))
        h[f] = np.clip(v, 0, 65535).astype(np.uint16)
    pr = np.where(r["proto_any"] != 0, rng.integers(0, 256, n), r["proto"].astype(np.int64))
    h["proto"] = np.where(rng.random(n) < 0.1, rng.integers(0, 256, n), pr).astype(np.uint8)
    return h


def mixed_packets(rules, n, seed):
    a = W.gen_packets(rules, n, seed)
    b = edge_packets(rules, seed + 1)
    return {f: np.concatenate([a[f], b[f]]) for f in W.HEADER_FIELDS}


def classify(torch, rs, hdr, cfg, offset=0):
    n = len(hdr["src"])
    if offset:
        pad = {f: np.concatenate([np.zeros(offset, hdr[f].dtype), hdr[f]]) for f in W.HEADER_FIELDS}
        dh = {f: t[offset:] for f, t in fw.headers_to_device(pad).items()}
    else:
        dh = fw.headers_to_device(hdr)
    idx, act = fw.fw_classify(rs, dh, n, config=cfg)
    torch.cuda.synchronize()
    assert rs.check() == fw.FW_OK
    return idx.cpu().numpy(), act.cpu().numpy()


def assert_same(got, want, what=""):
    gi, ga = got
    wi, wa = want[0], want[1]
    bad = np.nonzero((gi != wi) | (ga != wa))[0]
    assert bad.size == 0, (f"{what}: {bad.size} mismatches, first at {bad[0]}: got ({gi[bad[0]]},{ga[bad[0]]}) "
                           f"want ({wi[bad[0]]},{wa[bad[0]]})")


# one- and two-word rows, wider rows, and rows of 32 words or more (with row summaries)
CASES = [(12, 1), (30, 2), (45, 3), (70, 4), (100, 5), (160, 6), (400, 7), (900, 8), (2000, 9), (6000, 11)]


@pytest.mark.parametrize("n_rules,seed", CASES)
@pytest.mark.parametrize("cfg", [{"filter": 1}, {}, {"filter": 1, "block_threads": 64, "blocks_per_sm": 1},
                                 {"filter": 1, "lane_packets": 2}],
                         ids=["forced", "auto", "small_blocks", "pairs"])
def test_edges_against_oracle(torch_cuda, n_rules, seed, cfg):
    rules = edge_rules(n_rules, 900 + seed)
    rs = fw.fw_ruleset_create(rules)
    if rs.filter()["words"] == 0:
        rs.destroy()
        pytest.skip("this rule set has no filter")
    hdr = mixed_packets(rules, 6000, 40 + seed)
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert_same(classify(torch_cuda, rs, hdr, fw.make_config("packet_split", **cfg)), want, f"{n_rules} rules")
    rs.destroy()


def test_all_bitmap_widths_are_exercised(torch_cuda):
    """One- and two-word rows (staged in shared memory), wider rows (read from global memory) and
    rows of 32 words or more (read through their summaries)."""
    widths = set()
    for n_rules, seed in CASES:
        rs = fw.fw_ruleset_create(edge_rules(n_rules, 900 + seed))
        widths.add(rs.filter()["words"])
        rs.destroy()
    assert {1, 2} <= widths and any(2 < w < 32 for w in widths) and max(widths) >= 32, widths


@pytest.mark.parametrize("n_pkts", [1, 3, 4, 5, 63, 1023, 4097, 100_003])
@pytest.mark.parametrize("offset", [0, 1, 3])
@pytest.mark.parametrize("lane_packets", [0, 2])
def test_sizes_and_misaligned_views(torch_cuda, n_pkts, offset, lane_packets):
    rules = edge_rules(40, 77)
    rs = fw.fw_ruleset_create(rules)
    assert rs.filter()["words"] > 0
    full = mixed_packets(rules, max(n_pkts, 16), 5)
    hdr = {f: full[f][-n_pkts:] for f in W.HEADER_FIELDS}
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert_same(classify(torch_cuda, rs, hdr, fw.make_config("packet_split", filter=1, lane_packets=lane_packets),
                         offset), want, f"n={n_pkts} offset={offset} lane_packets={lane_packets}")
    rs.destroy()


def test_catch_all_truncation_and_address_key(torch_cuda):
    """A long list whose first catch-all comes early: only the reachable rules are filtered."""
    rules = W.gen_rules(5000, 31)
    ca = np.zeros(1, dtype=W.RULE_DTYPE)
    ca["sport_hi"] = ca["dport_hi"] = 65535
    ca["proto_any"] = 1
    rules = np.concatenate([rules[:50], ca, rules[50:]]).astype(W.RULE_DTYPE)
    rs = fw.fw_ruleset_create(rules)
    assert rs.first_catch_all <= 50 and rs.filter()["words"] > 0
    hdr = mixed_packets(rules[:60], 50_000, 8)
    want = oracle.classify(rules, hdr, threads=THREADS)
    assert_same(classify(torch_cuda, rs, hdr, fw.make_config("packet_split", filter=1)), want, "truncated")
    part = rs.partition()
    rs.destroy()
    assert part["classes"] >= 4


def test_default_deny_and_empty_rule_set(torch_cuda):
    for rules in (W.empty_rules(0), edge_rules(20, 3)[:0], W.gen_rules(3, 4)):
        rs = fw.fw_ruleset_create(rules)
        assert rs.filter()["words"] > 0
        hdr = W.gen_packets(W.gen_rules(50, 9), 3000, 10)  # packets drawn from unrelated rules
        want = oracle.classify(rules, hdr, threads=THREADS)
        got = classify(torch_cuda, rs, hdr, fw.make_config("packet_split", filter=1))
        assert_same(got, want, f"{len(rules)} rules")
        if len(rules) == 0:
            assert np.all(got[0] == -1) and np.all(got[1] == fw.FW_DROP)
        rs.destroy()


def test_filter_refused_when_the_rule_set_has_none(torch_cuda):
    long_list = W.gen_rules(40_000, 12)
    long_list = long_list[~((long_list["src_prefix"] == 0) & (long_list["dst_prefix"] == 0))]
    many_protos = W.gen_rules(60, 13)
    many_protos["proto_any"] = 0
    many_protos["proto"] = np.arange(60) % 12  # 12 exact protocols: the "other" class mixes them
    for rules in (long_list, many_protos):
        rs = fw.fw_ruleset_create(rules)
        assert rs.filter()["words"] == 0
        dh = fw.headers_to_device(W.gen_packets(rules, 100, 1))
        with pytest.raises(fw.FwError) as e:
            fw.fw_classify(rs, dh, 100, config=fw.make_config("packet_split", filter=1))
        assert e.value.status == fw.FW_EINVAL
        # the default still classifies (the scan kernels), and matches the oracle
        hdr = W.gen_packets(rules, 5000, 2)
        assert_same(classify(torch_cuda, rs, hdr, fw.make_config("packet_split")),
                    oracle.classify(rules, hdr, threads=THREADS), "no filter")
        rs.destroy()


def test_filter_off_and_headline_rule_set(torch_cuda):
    rules = W.gen_rules(10_000, 3)
    rs = fw.fw_ruleset_create(rules)
    f = rs.filter()
    assert f["words"] in (1, 2) and 0 < f["bytes"] <= 227 * 1024
    hdr = W.gen_packets(rules, 300_000, 4, zipf_s=1.1)
    want = oracle.classify(rules, hdr, threads=THREADS)
    for cfg in (fw.make_config("packet_split", filter=2), fw.make_config("packet_split", filter=1), None):
        got = classify(torch_cuda, rs, hdr, cfg if cfg is not None else fw.make_config("auto"))
        assert_same(got, want, str(cfg))
    rs.destroy()
