"""The host-side partition of a rule list (fw_partition_plan), without a GPU.

Two links. The library's plan (key, class count, sub-list lengths, protocol
classes) equals the partition written out from its definition in
partition_ref.py, for the scan's granule (1) and the learned index's (128).
That definition is pinned by brute force with the oracle: on tiny domains,
for every candidate key, each packet's first match within its class's
sub-list is its first match in the whole list.
"""
import ctypes
import itertools

import numpy as np
import pytest

import oracle
import oracle_pins as P
import partition_ref as R
from paper_1312_4188_gb300 import build as B
from paper_1312_4188_gb300 import fw, workload as W


@pytest.fixture(scope="module")
def L():
    B.build()
    return fw.lib()


def no_catch_all(rules):
    return rules[~((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0))]


def many_protocol_rules(rng, n, protos):
    r = P.random_tiny_rules(rng, n)
    r["proto"] = rng.choice(protos, size=n)
    return r


def rule_sets():
    rng = np.random.default_rng(2024)
    sets = {
        "empty": W.gen_rules(0, 1),
        "one": W.gen_rules(1, 1),
        "gen300": W.gen_rules(300, 5),
        "gen2000_no_catch_all": no_catch_all(W.gen_rules(2000, 8)),
        "tiny40": P.random_tiny_rules(rng, 40),
        "tiny200": P.random_tiny_rules(rng, 200),
        "twelve_protocols": many_protocol_rules(rng, 300, np.arange(12)),
        "two_protocols": many_protocol_rules(rng, 300, np.array([6, 17])),
    }
    wild = W.gen_rules(200, 9)
    wild["src_prefix"] = 0
    wild["dst_prefix"] = 0
    sets["wildcard_addresses"] = wild  # no address key can shorten a sub-list
    dst_only = W.gen_rules(400, 10)
    dst_only["src_prefix"] = 0
    sets["dst_prefixes_only"] = dst_only  # only a destination key can
    return sets


SETS = rule_sets()


@pytest.mark.parametrize("granule", [1, 128, 16])
@pytest.mark.parametrize("name", sorted(SETS))
def test_plan_matches_definition(L, name, granule):
    rules = SETS[name]
    plan = fw.fw_partition_plan(rules, granule)
    want_key = R.best_key(rules, granule)
    assert (plan["key_field"], plan["key_bits"]) == want_key
    lists = R.class_sublists(rules, *want_key)
    assert plan["classes"] == len(lists) <= R.MAX_CLASSES
    assert plan["class_len"] == [len(x) for x in lists]
    assert np.array_equal(plan["proto_class"], R.protocol_classes(rules)[1])


def test_plan_special_cases(L):
    assert fw.fw_partition_plan(SETS["empty"])["classes"] == 1
    w = fw.fw_partition_plan(SETS["wildcard_addresses"])
    assert (w["key_field"], w["key_bits"]) == (0, 0)
    d = fw.fw_partition_plan(SETS["dst_prefixes_only"])
    assert d["key_field"] == 2 and d["key_bits"] >= 1
    t = fw.fw_partition_plan(SETS["twelve_protocols"])
    assert t["classes"] == 8 and t["key_field"] == 0  # 7 protocols + "other" fill the classes
    # two exact protocols leave room for two key bits (3 protocol classes x 2 = 6; x 4 = 12 > 8)
    two = fw.fw_partition_plan(SETS["two_protocols"])
    assert two["key_bits"] <= 1


def tiny_headers(protos):
    dom = list(itertools.product(P.ADDRS, P.ADDRS, [0, 3, 65535], [0, 2, 65534], protos))
    return P.headers_from_tuples(dom)


def check_first_match_within_sublists(rules, hdr):
    """Every candidate key: returns the keys checked."""
    want_idx, want_act, _ = oracle.classify(rules, hdr)
    _, proto_class = R.protocol_classes(rules)
    n_p = int(proto_class.max()) + 1
    keys = [(0, 0)] + [(f, b) for f in (1, 2) for b in (1, 2, 3) if n_p << b <= R.MAX_CLASSES]
    for kf, kb in keys:
        lists = R.class_sublists(rules, kf, kb)
        cls = R.packet_class(hdr, proto_class, kf, kb)
        assert cls.min() >= 0 and cls.max() < len(lists)
        for c, members in enumerate(lists):
            sel = np.nonzero(cls == c)[0]
            if len(sel) == 0:
                continue
            sub_hdr = {f: hdr[f][sel] for f in W.HEADER_FIELDS}
            got, act, _ = oracle.classify(rules[members], sub_hdr)
            mapped = np.where(got >= 0, members[np.maximum(got, 0)] if len(members) else -1, -1)
            assert np.array_equal(mapped, want_idx[sel]), f"key {(kf, kb)} class {c}"
            assert np.array_equal(act, want_act[sel])
    return set(keys)


def test_sublists_keep_every_first_match_brute_force():
    """0 to 3 exact protocols per set, so that keys of 1, 2 and 3 bits fit in the 8 classes."""
    rng = np.random.default_rng(77)
    hdr = tiny_headers(P.PROTOS)
    checked = set()
    for t in range(40):
        rules = P.random_tiny_rules(rng, int(rng.integers(1, 40)))
        protos = rng.choice(P.PROTOS, size=t % 4, replace=False)
        if len(protos) == 0:
            rules["proto_any"] = 1
        else:
            rules["proto"] = rng.choice(protos, size=len(rules))
        checked |= check_first_match_within_sublists(rules, hdr)
    assert {(f, b) for f in (1, 2) for b in (1, 2, 3)} <= checked


def test_sublists_keep_every_first_match_other_class():
    """More exact protocols than classes: "other" mixes several protocols (and packets of
    protocols no rule names fall into it too)."""
    rng = np.random.default_rng(78)
    hdr = tiny_headers(list(range(14)))
    for _ in range(10):
        check_first_match_within_sublists(many_protocol_rules(rng, int(rng.integers(8, 60)), np.arange(12)), hdr)


def test_plan_rejects_bad_arguments(L):
    out = [ctypes.c_int32() for _ in range(3)]
    refs = [ctypes.byref(o) for o in out]
    r = np.ascontiguousarray(W.gen_rules(10, 1))
    ptr = r.ctypes.data_as(ctypes.c_void_p)
    assert L.fw_partition_plan(None, -1, 1, *refs, None, None) == fw.FW_EINVAL
    assert L.fw_partition_plan(None, 5, 1, *refs, None, None) == fw.FW_EINVAL
    assert L.fw_partition_plan(ptr, 10, 0, *refs, None, None) == fw.FW_EINVAL
    assert L.fw_partition_plan(ptr, 10, 1, None, refs[1], refs[2], None, None) == fw.FW_EINVAL
    assert L.fw_partition_plan(ptr, 10, 1, *refs, None, None) == fw.FW_OK  # optional outputs may be NULL
    bad = r.copy()
    bad["src_prefix"][3] = 33
    assert L.fw_partition_plan(bad.ctypes.data_as(ctypes.c_void_p), 10, 1, *refs, None, None) == fw.FW_EINVAL


def random_rule_set(rng):
    """Small random lists that stress the partition's choices: 0 to 12 exact protocols (ties in
    their counts included), prefixes of 0 to 4 bits as often as long ones (shorter than a key
    of up to 3 bits), and sizes from empty up."""
    n = int(rng.integers(0, 60))
    r = W.empty_rules(n)
    protos = rng.choice(256, size=int(rng.integers(0, 13)), replace=False)
    for i in range(n):
        for f in ("src", "dst"):
            r[f + "_addr"][i] = rng.integers(0, 1 << 32, dtype=np.uint64)
            r[f + "_prefix"][i] = rng.integers(0, 5) if rng.random() < 0.5 else rng.integers(5, 33)
        for f in ("sport", "dport"):
            a, b = sorted(rng.integers(0, 65536, size=2))
            r[f + "_lo"][i], r[f + "_hi"][i] = a, b
        if len(protos) == 0 or rng.random() < 0.3:
            r["proto_any"][i] = 1
        else:
            r["proto"][i] = protos[rng.integers(len(protos))]
        r["action"][i] = rng.integers(2)
    return r


@pytest.mark.parametrize("seed", range(4))
def test_plan_matches_definition_on_random_lists(L, seed):
    rng = np.random.default_rng(500 + seed)
    keyed = 0
    for _ in range(60):
        rules = random_rule_set(rng)
        for granule in (1, 4, 128):
            plan = fw.fw_partition_plan(rules, granule)
            key = R.best_key(rules, granule)
            assert (plan["key_field"], plan["key_bits"]) == key
            lists = R.class_sublists(rules, *key)
            assert plan["class_len"] == [len(x) for x in lists]
            assert np.array_equal(plan["proto_class"], R.protocol_classes(rules)[1])
            keyed += key != (0, 0)
    assert keyed > 0  # the search reaches keyed partitions
