"""The bucket filter's host-built tables and exact-test records against the oracle (CPU only).

fw_filter_plan returns the filter block a rule set would stage into shared
memory. Here the block is decoded by its documented layout and used to
classify packets the way the filter kernel does: AND the packet's three bucket
rows in its class, take the candidates in increasing record order, and accept
the first one whose exact-mask bit is set or whose exact-test record accepts
the packet. The verdict word of that record must equal the oracle's first
match and action for every packet (random and edge packets, many rule sets).
Two properties are checked on their own as well: the oracle's first match
always has all three bucket bits set (the rows never drop a matching rule),
and a record marked exact contains every packet whose bucket bits it has.
"""
import numpy as np
import pytest

import oracle
import partition_ref as R
from paper_1312_4188_gb300 import fw, workload as W
from test_filter_gpu import edge_packets, edge_rules


def up16(b):
    return (b + 15) // 16 * 16


def decode(plan, n_classes):
    """Arrays of the filter block (documented layout): rows [table][class][bucket][word] (uint32),
    exact masks [class][word], records [record][8], verdict words, protocol classes, class offsets."""
    blk, w = plan["block"], plan["words"]
    recs_n = int(plan["class_off"][-1] + plan["class_len"][-1])
    tab_bytes = n_classes * 3 * 256 * w * 4
    cls_off = up16(tab_bytes)
    ex_off = cls_off + n_classes * 16
    recs_off = up16(ex_off + n_classes * w * 4)
    vw_off = recs_off + recs_n * 32
    pc_off = up16(vw_off + recs_n * 4)
    rows = blk[:tab_bytes].view(np.uint32).reshape(n_classes, 3, 256, w).transpose(1, 0, 2, 3)
    ci = blk[cls_off:cls_off + n_classes * 16].view(np.uint32).reshape(n_classes, 4)
    exact = blk[ex_off:ex_off + n_classes * w * 4].view(np.uint32).reshape(n_classes, w)
    assert np.array_equal(ci[:, 1], exact[:, 0]) and (w == 1 or np.array_equal(ci[:, 2], exact[:, 1]))
    class_off = ci[:, 0].astype(np.int32)
    recs = blk[recs_off:recs_off + recs_n * 32].view(np.uint32).reshape(recs_n, 8)
    vw = blk[vw_off:vw_off + recs_n * 4].view(np.uint32)
    proto_class = blk[pc_off:pc_off + 256]
    return rows, exact, recs, vw, proto_class, class_off


def candidates(rows, c, hdr):
    """[packet][word] AND of the packet's three bucket rows."""
    s8 = hdr["src"].astype(np.int64) >> 24
    d8 = hdr["dst"].astype(np.int64) >> 24
    pb = ((hdr["sport"].astype(np.int64) >> 12) << 4) | (hdr["dport"].astype(np.int64) >> 12)
    return rows[0, c, s8] & rows[1, c, d8] & rows[2, c, pb]


def bit(words, j):
    return ((words[:, j // 32] >> np.uint32(j % 32)) & np.uint32(1)).astype(bool)


def reachable(rules):
    ca = np.nonzero((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0) & (rules["sport_lo"] == 0) &
                    (rules["sport_hi"] == 65535) & (rules["dport_lo"] == 0) & (rules["dport_hi"] == 65535) &
                    (rules["proto_any"] != 0))[0]
    return rules[:int(ca[0]) + 1] if len(ca) else rules


def exact_test(rec, h):
    """The record's exact test: masked address equality, port offsets within their widths (mod 2^32)."""
    r = rec.astype(np.int64)
    s, d = h["src"].astype(np.int64), h["dst"].astype(np.int64)
    sp, dp = h["sport"].astype(np.int64), h["dport"].astype(np.int64)
    m32 = 0xFFFFFFFF
    ok = ((s ^ r[:, 0]) & r[:, 1]) == 0
    ok &= ((d ^ r[:, 2]) & r[:, 3]) == 0
    ok &= ((sp + r[:, 4]) & m32) <= r[:, 5]
    ok &= ((dp + r[:, 6]) & m32) <= r[:, 7]
    return ok


def filter_classify(rules, hdr):
    """Verdicts of the filter built for `rules`, decoded and applied as the kernel applies it."""
    plan = fw.fw_filter_plan(rules)
    if plan["words"] == 0:
        return None
    part = fw.fw_partition_plan(reachable(rules))
    nc, kf, kb = part["classes"], part["key_field"], part["key_bits"]
    rows, exact, recs, vw, proto_class, class_off = decode(plan, nc)
    assert np.array_equal(proto_class, part["proto_class"])
    assert np.array_equal(class_off, plan["class_off"][:nc])
    c = R.packet_class(hdr, part["proto_class"], kf, kb).astype(np.int64)
    m = candidates(rows, c, hdr)
    off = class_off[c].astype(np.int64)
    n = len(c)
    idx = np.full(n, -1, dtype=np.int64)
    act = np.zeros(n, dtype=np.uint8)
    done = np.zeros(n, dtype=bool)
    for j in range(32 * plan["words"]):
        cand = bit(m, j) & ~done
        if not cand.any():
            continue
        at = off + j
        sel = np.nonzero(cand)[0]
        ex = bit(exact[c[sel]], j)
        ok = ex | exact_test(recs[at[sel]], {f: hdr[f][sel] for f in W.HEADER_FIELDS})
        hit = sel[ok]
        v = vw[at[hit]]
        idx[hit] = v & 0x7FFFFFFF
        act[hit] = v >> 31
        done[hit] = True
    return plan, (c, m, off, rows, exact, recs, vw), idx.astype(np.int32), act


RULE_SETS = [("edge", 12, 1), ("edge", 30, 2), ("edge", 45, 3), ("edge", 70, 4), ("edge", 100, 5), ("edge", 160, 6),
             ("edge", 400, 7), ("edge", 900, 8), ("gen", 3, 7), ("gen", 40, 8), ("gen", 10_000, 3),
             ("gen", 1000, 1), ("gen", 10_000, 40), ("gen", 1000, 41)]


def rule_set(kind, n, seed):
    return edge_rules(n, 900 + seed) if kind == "edge" else W.gen_rules(n, seed)


@pytest.mark.parametrize("kind,n,seed", RULE_SETS)
def test_filter_block_classifies_like_the_oracle(kind, n, seed):
    rules = rule_set(kind, n, seed)
    a = W.gen_packets(rules, 20_000, 60 + seed)
    b = edge_packets(reachable(rules), 61 + seed)
    hdr = {f: np.concatenate([a[f], b[f]]) for f in W.HEADER_FIELDS}
    got = filter_classify(rules, hdr)
    if got is None:
        pytest.skip("no filter for this rule set")
    _, (c, m, off, rows, exact, recs, vw), idx, act = got
    o_idx, o_act, _ = oracle.classify(rules, hdr)
    bad = np.nonzero((idx != o_idx) | (act != o_act))[0]
    assert bad.size == 0, f"{bad.size} packets differ from the oracle, first {bad[0]}"
    # the first match always survives the bucket rows
    matched = np.nonzero(o_idx >= 0)[0]
    orig = (vw & 0x7FFFFFFF).astype(np.int64)
    width = 32 * got[0]["words"]
    for i in matched[:3000]:
        pos = np.nonzero(orig[off[i]:off[i] + width] == o_idx[i])[0]
        assert pos.size >= 1, f"packet {i}: its first match is not in its class sub-list"
        j = int(pos[0])
        assert (int(m[i, j // 32]) >> (j % 32)) & 1, f"packet {i}: its first match is not a candidate"


def test_exact_records_contain_every_packet_of_their_buckets():
    for kind, n, seed in RULE_SETS:
        rules = rule_set(kind, n, seed)
        plan = fw.fw_filter_plan(rules)
        if plan["words"] == 0:
            continue
        part = fw.fw_partition_plan(reachable(rules))
        rows, exact, recs, vw, _, class_off = decode(plan, part["classes"])
        hdr = W.gen_packets(rules, 20_000, 70 + seed)
        c = R.packet_class(hdr, part["proto_class"], part["key_field"], part["key_bits"]).astype(np.int64)
        m = candidates(rows, c, hdr) & exact[c]
        for j in range(32 * plan["words"]):
            sel = np.nonzero(bit(m, j))[0]
            if sel.size == 0:
                continue
            rule = int(vw[class_off[c[sel[0]]] + j] & 0x7FFFFFFF)
            same = sel[(vw[class_off[c[sel]] + j] & 0x7FFFFFFF) == rule]
            one = rules[rule:rule + 1]
            o_idx, _, _ = oracle.classify(one, {f: hdr[f][same] for f in W.HEADER_FIELDS})
            assert np.all(o_idx == 0), f"exact record {j} (rule {rule}) misses packets of its buckets"


def no_catch_all(n, seed):
    r = W.gen_rules(n, seed)
    return r[~((r["src_prefix"] == 0) & (r["dst_prefix"] == 0))]


def test_wide_row_summaries_mark_nonzero_words():
    """Rows of 32 words or more carry summaries after the protocol class table: bit w of a row's
    summary is set exactly when word w of the row is not zero (so the AND of a packet's three
    summaries holds every word where the AND of its rows is not zero); narrower blocks end there."""
    seen_wide = False
    cases = [rule_set(k, n, s) for k, n, s in RULE_SETS] + [no_catch_all(3000, 12), no_catch_all(4000, 12),
                                                             no_catch_all(6000, 5)]
    for rules in cases:
        plan = fw.fw_filter_plan(rules)
        w = plan["words"]
        if w == 0:
            continue
        nc = fw.fw_partition_plan(reachable(rules))["classes"]
        rows = decode(plan, nc)[0]  # [table][class][bucket][word]
        recs_n = int(plan["class_off"][-1] + plan["class_len"][-1])
        tab_bytes = nc * 3 * 256 * w * 4
        ex_off = up16(tab_bytes) + nc * 16
        pc_off = up16(up16(ex_off + nc * w * 4) + recs_n * 32 + recs_n * 4)
        summ_off = up16(pc_off + 256)
        blk = plan["block"]
        if w < 32:
            assert blk.size == summ_off
            continue
        seen_wide = True
        sw = (w + 31) // 32
        assert blk.size == summ_off + nc * 3 * 256 * sw * 4
        summ = blk[summ_off:].view(np.uint32).reshape(nc, 3, 256, sw).transpose(1, 0, 2, 3)
        for word in range(w):
            marked = ((summ[..., word // 32] >> np.uint32(word % 32)) & np.uint32(1)).astype(bool)
            assert np.array_equal(marked, rows[..., word] != 0), (w, word)
        assert not np.any(summ[..., -1] >> np.uint32(w - 32 * (sw - 1))) if w % 32 else True
    assert seen_wide


def test_no_filter_cases_and_arguments():
    long_list = W.gen_rules(40_000, 12)
    long_list = long_list[~((long_list["src_prefix"] == 0) & (long_list["dst_prefix"] == 0))]
    assert fw.fw_filter_plan(long_list)["words"] == 0  # class sub-lists over FW_FILTER_MAX_RULES
    widths = {fw.fw_filter_plan(rule_set(k, n, s))["words"] for k, n, s in RULE_SETS}
    assert {1, 2} <= widths and max(widths) > 2, widths
    many = W.gen_rules(60, 13)
    many["proto_any"] = 0
    many["proto"] = np.arange(60) % 12
    assert fw.fw_filter_plan(many)["words"] == 0
    empty = fw.fw_filter_plan(W.empty_rules(0))
    assert empty["words"] == 1 and empty["block"].size > 0
    bad = W.gen_rules(5, 1)
    bad["src_prefix"][2] = 40
    with pytest.raises(fw.FwError):
        fw.fw_filter_plan(bad)
