"""Checks that pin the CPU oracle to facts other than itself.

Each ``pin_*`` function takes a loaded oracle library (``oracle.load()`` or a
deliberately broken copy built by the mutation test) and raises
AssertionError when the oracle disagrees with:

* a hand-worked example (tests/golden/handworked_policy.txt), derived on paper
  from the first-match / default-deny policy (Sec. I) and the wildcard
  5-tuple rule model (Sec. IV);
* brute force over a tiny header domain, where every rule's set S_k is
  enumerated explicitly as address intervals (floor division, not shifts),
  port ranges and protocol sets, and idx(p) = min{k : p in S_k};
* invariants: a packet drawn inside rule k with no earlier rule overlapping k
  returns k; an unmatched packet gets -1 / DROP and no rule contains it;
  appending a catch-all changes only unmatched packets; permuting rules
  that pairwise do not overlap changes nothing but the index labels;
* closed forms: empty rule list, catch-all first, a single rule (per-field
  membership), all-exact rules (dictionary lookup of the first occurrence),
  and the scan-depth sum.
"""
from __future__ import annotations

import ipaddress
import itertools
import os

import numpy as np

import oracle
from paper_1312_4188_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "handworked_policy.txt")


def run(lib, rules, headers):
    return oracle.classify(rules, headers, threads=1, lib=lib)


def headers_from_tuples(tuples):
    h = W.empty_headers(len(tuples))
    for i, (s, d, sp, dp, pr) in enumerate(tuples):
        h["src"][i], h["dst"][i], h["sport"][i], h["dport"][i], h["proto"][i] = s, d, sp, dp, pr
    return h


# ---------------------------------------------------------------- set model
def addr_interval(addr: int, prefix: int):
    """[low, high] of the addresses sharing the top ``prefix`` bits of ``addr``."""
    block = 2 ** (32 - prefix)
    low = (addr // block) * block
    return low, low + block - 1


def rule_sets(r):
    """Per-field membership sets of one rule (intervals / explicit sets)."""
    return (
        addr_interval(int(r["src_addr"]), int(r["src_prefix"])),
        addr_interval(int(r["dst_addr"]), int(r["dst_prefix"])),
        (int(r["sport_lo"]), int(r["sport_hi"])),
        (int(r["dport_lo"]), int(r["dport_hi"])),
        None if r["proto_any"] else int(r["proto"]),
    )


def contains(sets, pkt):
    (s0, s1), (d0, d1), (a0, a1), (b0, b1), pr = sets
    s, d, sp, dp, p = pkt
    return s0 <= s <= s1 and d0 <= d <= d1 and a0 <= sp <= a1 and b0 <= dp <= b1 and (pr is None or pr == p)


def overlaps(a, b):
    """Exact test whether two rules' sets intersect."""
    for (lo1, hi1), (lo2, hi2) in zip(a[:4], b[:4]):
        if max(lo1, lo2) > min(hi1, hi2):
            return False
    return a[4] is None or b[4] is None or a[4] == b[4]


def catch_all(action=W.ACCEPT):
    r = W.empty_rules(1)
    r["sport_hi"] = 65535
    r["dport_hi"] = 65535
    r["proto_any"] = 1
    r["action"] = action
    return r


def sample_inside(rng, r, m):
    """``m`` packets drawn uniformly inside rule ``r``'s set."""
    sets = rule_sets(r)
    (s0, s1), (d0, d1), (a0, a1), (b0, b1), pr = sets
    h = W.empty_headers(m)
    h["src"][:] = rng.integers(s0, s1 + 1, size=m, dtype=np.uint64)
    h["dst"][:] = rng.integers(d0, d1 + 1, size=m, dtype=np.uint64)
    h["sport"][:] = rng.integers(a0, a1 + 1, size=m)
    h["dport"][:] = rng.integers(b0, b1 + 1, size=m)
    h["proto"][:] = rng.integers(0, 256, size=m) if pr is None else pr
    return h


# ---------------------------------------------------------------- golden
def parse_golden(path=GOLDEN):
    rules, pkts, expect = [], [], []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "R":
            assert int(tok[1]) == len(rules)
            s, sp_ = tok[3].split("/")
            d, dp_ = tok[4].split("/")
            a0, a1 = tok[5].split("-")
            b0, b1 = tok[6].split("-")
            rules.append(dict(
                action=W.ACCEPT if tok[2] == "ACCEPT" else W.DROP,
                src_addr=int(ipaddress.IPv4Address(s)), src_prefix=int(sp_),
                dst_addr=int(ipaddress.IPv4Address(d)), dst_prefix=int(dp_),
                sport_lo=int(a0), sport_hi=int(a1), dport_lo=int(b0), dport_hi=int(b1),
                proto=0 if tok[7] == "any" else int(tok[7]), proto_any=1 if tok[7] == "any" else 0))
        elif tok[0] == "P":
            arrow = tok.index("->")
            s, d, sp, dp, pr = tok[1:arrow]
            pkts.append((int(ipaddress.IPv4Address(s)), int(ipaddress.IPv4Address(d)), int(sp), int(dp), int(pr)))
            expect.append((int(tok[arrow + 1]), W.ACCEPT if tok[arrow + 2] == "ACCEPT" else W.DROP))
    r = W.empty_rules(len(rules))
    for i, d in enumerate(rules):
        for k, v in d.items():
            r[k][i] = v
    return r, headers_from_tuples(pkts), expect


def pin_golden(lib):
    rules, h, expect = parse_golden()
    idx, act, _ = run(lib, rules, h)
    for i, (ei, ea) in enumerate(expect):
        assert (int(idx[i]), int(act[i])) == (ei, ea), f"golden packet {i}: got {(idx[i], act[i])}, want {(ei, ea)}"


# ---------------------------------------------------------------- brute force
ADDRS = [0x00000000, 0x00000001, 0x00000002, 0x00000003, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF]
PREFIXES = [0, 1, 30, 31, 32]
PORTS = [0, 1, 2, 3, 65534, 65535]
PROTOS = [0, 1, 6, 17]


def tiny_domain():
    return list(itertools.product(ADDRS, ADDRS, PORTS, PORTS, PROTOS))


def random_tiny_rules(rng, n):
    r = W.empty_rules(n)
    for i in range(n):
        r["src_addr"][i] = ADDRS[rng.integers(len(ADDRS))]
        r["dst_addr"][i] = ADDRS[rng.integers(len(ADDRS))]
        r["src_prefix"][i] = PREFIXES[rng.integers(len(PREFIXES))]
        r["dst_prefix"][i] = PREFIXES[rng.integers(len(PREFIXES))]
        for f in ("sport", "dport"):
            a, b = sorted(rng.choice(PORTS, size=2))
            r[f + "_lo"][i], r[f + "_hi"][i] = a, b
        if rng.random() < 0.3:
            r["proto_any"][i] = 1
        else:
            r["proto"][i] = PROTOS[rng.integers(len(PROTOS))]
        r["action"][i] = rng.integers(2)
    return r


def pin_brute_force(lib, n_sets=150, seed=11):
    rng = np.random.default_rng(seed)
    dom = tiny_domain()
    h = headers_from_tuples(dom)
    for t in range(n_sets):
        rules = random_tiny_rules(rng, int(rng.integers(1, 5)))
        members = []
        for r in rules:
            sets = rule_sets(r)
            members.append({p for p in dom if contains(sets, p)})
        idx, act, depth = run(lib, rules, h)
        want_depth = 0
        for i, p in enumerate(dom):
            k = next((k for k, m in enumerate(members) if p in m), -1)
            a = int(rules["action"][k]) if k >= 0 else W.DROP
            assert (int(idx[i]), int(act[i])) == (k, a), f"set {t} packet {p}: got {(idx[i], act[i])}, want {(k, a)}"
            want_depth += (k + 1) if k >= 0 else len(rules)
        assert depth == want_depth, f"set {t}: depth sum {depth} != {want_depth}"


# ---------------------------------------------------------------- invariants
def pin_inside_no_earlier_overlap(lib, n_rules=300, seed=21, per_rule=20):
    rules = W.gen_rules(n_rules, seed)
    rng = np.random.default_rng(seed + 1)
    sets = [rule_sets(r) for r in rules]
    checked = 0
    for k in range(n_rules):
        if any(overlaps(sets[j], sets[k]) for j in range(k)):
            continue
        h = sample_inside(rng, rules[k], per_rule)
        idx, act, _ = run(lib, rules, h)
        assert np.all(idx == k), f"rule {k}: packets inside it returned {np.unique(idx)}"
        assert np.all(act == rules["action"][k])
        checked += 1
    assert checked >= 10, "too few rules without an earlier overlap to pin anything"


def pin_unmatched_default_deny(lib, seed=31):
    rules = W.gen_rules(200, seed)
    # drop catch-all-like rules so that many packets go unmatched
    keep = ~((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0))
    rules = rules[keep]
    h = W.gen_packets(rules, 3000, seed + 1)
    idx, act, depth = run(lib, rules, h)
    sets = [rule_sets(r) for r in rules]
    um = np.nonzero(idx < 0)[0]
    assert um.size > 100
    assert np.all(act[um] == W.DROP)
    for i in um[:400]:
        p = tuple(int(h[f][i]) for f in W.HEADER_FIELDS)
        assert not any(contains(s, p) for s in sets), f"packet {i} unmatched but a rule contains it"
    # every matched packet is in its rule and in no earlier one
    for i in np.nonzero(idx >= 0)[0][:400]:
        p = tuple(int(h[f][i]) for f in W.HEADER_FIELDS)
        k = int(idx[i])
        assert contains(sets[k], p)
        assert not any(contains(sets[j], p) for j in range(k))
        assert act[i] == rules["action"][k]


def pin_append_catch_all(lib, seed=41):
    rules = W.gen_rules(150, seed)
    keep = ~((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0))
    rules = rules[keep]
    h = W.gen_packets(rules, 4000, seed + 1)
    idx0, act0, _ = run(lib, rules, h)
    for action in (W.ACCEPT, W.DROP):
        ext = np.concatenate([rules, catch_all(action)])
        idx1, act1, _ = run(lib, ext, h)
        um = idx0 < 0
        assert um.any()
        assert np.array_equal(idx1[~um], idx0[~um]) and np.array_equal(act1[~um], act0[~um])
        assert np.all(idx1[um] == len(rules)) and np.all(act1[um] == action)


def non_overlapping_rules(n, seed):
    cand = W.gen_rules(8 * n, seed)
    chosen, sets = [], []
    for r in cand:
        s = rule_sets(r)
        if not any(overlaps(s, t) for t in sets):
            chosen.append(r)
            sets.append(s)
            if len(chosen) == n:
                break
    out = W.empty_rules(len(chosen))
    for i, r in enumerate(chosen):
        out[i] = r
    return out


def pin_permute_non_overlapping(lib, seed=51):
    rules = non_overlapping_rules(60, seed)
    assert len(rules) >= 20
    rng = np.random.default_rng(seed)
    # half the packets inside some rule, half uniform
    h = W.gen_packets(rules, 3000, seed + 2)
    idx0, act0, _ = run(lib, rules, h)
    assert (idx0 >= 0).sum() > 500
    for _ in range(3):
        perm = rng.permutation(len(rules))
        idx1, act1, _ = run(lib, rules[perm], h)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(len(perm))
        mapped = np.where(idx0 >= 0, inv[np.maximum(idx0, 0)], -1)
        assert np.array_equal(idx1, mapped)
        assert np.array_equal(act1, act0)


# ---------------------------------------------------------------- closed forms
def pin_empty_rules(lib):
    h = W.gen_packets(W.gen_rules(10, 1), 500, 2)
    idx, act, depth = run(lib, W.empty_rules(0), h)
    assert np.all(idx == -1) and np.all(act == W.DROP) and depth == 0


def pin_catch_all_first(lib):
    rules = np.concatenate([catch_all(W.DROP), W.gen_rules(50, 3)])
    h = W.gen_packets(rules, 1000, 4)
    idx, act, depth = run(lib, rules, h)
    assert np.all(idx == 0) and np.all(act == W.DROP) and depth == 1000


def pin_single_rule(lib, seed=61):
    rules = W.gen_rules(40, seed)
    rng = np.random.default_rng(seed)
    for k in range(len(rules)):
        one = rules[k:k + 1]
        h = W.gen_packets(one, 200, seed + k)
        # push some packets to the exact range ends
        s = rule_sets(one[0])
        h["sport"][:20] = [s[2][0], s[2][1]] * 10
        h["dport"][20:40] = [s[3][0], s[3][1]] * 10
        h["sport"][40:50] = np.clip(s[2][0] - 1, 0, 65535)
        h["dport"][50:60] = np.clip(s[3][1] + 1, 0, 65535)
        h["src"][60:70] = s[0][0]
        h["src"][70:80] = s[0][1]
        h["dst"][80:90] = (s[1][1] + 1) % (1 << 32)
        idx, act, _ = run(lib, one, h)
        for i in range(200):
            p = tuple(int(h[f][i]) for f in W.HEADER_FIELDS)
            want = 0 if contains(s, p) else -1
            assert idx[i] == want, f"rule {k} packet {p}: got {idx[i]}, want {want}"
            assert act[i] == (one["action"][0] if want == 0 else W.DROP)


def pin_exact_lookup(lib, seed=71):
    rng = np.random.default_rng(seed)
    n = 400
    rules = W.empty_rules(n)
    pool = rng.integers(0, 1 << 32, size=60, dtype=np.uint64)
    rules["src_addr"] = pool[rng.integers(0, 60, size=n)]
    rules["dst_addr"] = pool[rng.integers(0, 60, size=n)]
    rules["src_prefix"] = 32
    rules["dst_prefix"] = 32
    p = rng.integers(0, 4, size=n)
    rules["sport_lo"] = rules["sport_hi"] = p
    q = rng.integers(0, 4, size=n)
    rules["dport_lo"] = rules["dport_hi"] = q
    rules["proto"] = np.array([1, 6, 17])[rng.integers(0, 3, size=n)]
    rules["action"] = rng.integers(0, 2, size=n)
    table = {}
    for k, r in enumerate(rules):
        key = (int(r["src_addr"]), int(r["dst_addr"]), int(r["sport_lo"]), int(r["dport_lo"]), int(r["proto"]))
        table.setdefault(key, k)
    keys = list(table.keys())
    m = 3000
    tup = []
    for i in range(m):
        if i % 2 == 0:
            tup.append(keys[rng.integers(len(keys))])
        else:
            tup.append((int(pool[rng.integers(60)]), int(pool[rng.integers(60)]), int(rng.integers(0, 5)),
                        int(rng.integers(0, 5)), int(rng.choice([1, 6, 17, 0]))))
    h = headers_from_tuples(tup)
    idx, act, _ = run(lib, rules, h)
    for i, t in enumerate(tup):
        k = table.get(t, -1)
        assert idx[i] == k, f"exact packet {t}: got {idx[i]}, want {k}"
        assert act[i] == (rules["action"][k] if k >= 0 else W.DROP)


def pin_depth_sum(lib, seed=81):
    rules = W.gen_rules(300, seed)
    h = W.gen_packets(rules, 2000, seed + 1)
    idx, _, depth = run(lib, rules, h)
    want = int(np.where(idx >= 0, idx.astype(np.int64) + 1, len(rules)).sum())
    assert depth == want


def pin_threads_agree(lib, seed=91):
    rules = W.gen_rules(500, seed)
    h = W.gen_packets(rules, 20000, seed + 1)
    a = oracle.classify(rules, h, threads=1, lib=lib)
    b = oracle.classify(rules, h, threads=4, lib=lib)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


ALL_PINS = [
    pin_golden,
    pin_brute_force,
    pin_inside_no_earlier_overlap,
    pin_unmatched_default_deny,
    pin_append_catch_all,
    pin_permute_non_overlapping,
    pin_empty_rules,
    pin_catch_all_first,
    pin_single_rule,
    pin_exact_lookup,
    pin_depth_sum,
    pin_threads_agree,
]
