"""bench.py's partitioned-scan depth metric against an explicit construction of the sub-lists."""
import numpy as np

import bench
import oracle
from paper_1312_4188_gb300 import workload as W


def explicit_partition_depth(rules, idx, proto):
    r = rules
    ca = [k for k in range(len(r)) if r["src_prefix"][k] == 0 and r["dst_prefix"][k] == 0 and r["sport_lo"][k] == 0
          and r["sport_hi"][k] == 65535 and r["dport_lo"][k] == 0 and r["dport_hi"][k] == 65535 and r["proto_any"][k]]
    n_eff = ca[0] + 1 if ca else len(r)
    counts = {}
    for k in range(n_eff):
        if not r["proto_any"][k]:
            counts[int(r["proto"][k])] = counts.get(int(r["proto"][k]), 0) + 1
    chosen = sorted(counts, key=lambda p: (-counts[p], p))[:7]
    total = 0
    for i in range(len(idx)):
        p = int(proto[i])
        if p in chosen:
            lst = [k for k in range(n_eff) if r["proto_any"][k] or int(r["proto"][k]) == p]
        else:
            lst = [k for k in range(n_eff) if r["proto_any"][k] or int(r["proto"][k]) not in chosen]
        total += lst.index(int(idx[i])) + 1 if idx[i] >= 0 else len(lst)
    return total


def test_partition_depth_matches_explicit_sublists():
    for seed, n_rules in ((1, 300), (2, 60)):
        rules = W.gen_rules(n_rules, seed)
        rules["proto"][::7] = 47  # an exact protocol outside the usual three
        rules["proto_any"][::7] = 0
        h = W.gen_packets(rules, 1500, seed + 10)
        h["proto"][::5] = 47
        idx, _, _ = oracle.classify(rules, h)
        assert bench.partition_depth(rules, idx, h["proto"]) == explicit_partition_depth(rules, idx, h["proto"])
