"""bench.py's partitioned-scan depth metric against an explicit construction of the sub-lists."""
import numpy as np
import pytest

import bench
import oracle
from paper_1312_4188_gb300 import workload as W


def explicit_partition_depth(rules, idx, hdr, key_field, key_bits):
    """Sub-list of a packet: reachable rules whose protocol can match it and whose address range
    (field `key_field`) intersects the address range of the packet's top `key_bits` bits."""
    r = rules
    ca = [k for k in range(len(r)) if r["src_prefix"][k] == 0 and r["dst_prefix"][k] == 0 and r["sport_lo"][k] == 0
          and r["sport_hi"][k] == 65535 and r["dport_lo"][k] == 0 and r["dport_hi"][k] == 65535 and r["proto_any"][k]]
    n_eff = ca[0] + 1 if ca else len(r)
    counts = {}
    for k in range(n_eff):
        if not r["proto_any"][k]:
            counts[int(r["proto"][k])] = counts.get(int(r["proto"][k]), 0) + 1
    chosen = sorted(counts, key=lambda p: (-counts[p], p))[:7]
    fld = {1: "src", 2: "dst"}.get(key_field)

    def addr_range(k):
        plen = int(r[fld + "_prefix"][k])
        size = 1 << (32 - plen)
        lo = (int(r[fld + "_addr"][k]) // size) * size
        return lo, lo + size - 1

    total = 0
    for i in range(len(idx)):
        p = int(hdr["proto"][i])
        if p in chosen:
            lst = [k for k in range(n_eff) if r["proto_any"][k] or int(r["proto"][k]) == p]
        else:
            lst = [k for k in range(n_eff) if r["proto_any"][k] or int(r["proto"][k]) not in chosen]
        if fld:
            span = 1 << (32 - key_bits)
            klo = (int(hdr[fld][i]) // span) * span
            khi = klo + span - 1
            lst = [k for k in lst if addr_range(k)[0] <= khi and klo <= addr_range(k)[1]]
        total += lst.index(int(idx[i])) + 1 if idx[i] >= 0 else len(lst)
    return total


@pytest.mark.parametrize("key_field,key_bits", [(0, 0), (1, 1), (2, 2), (2, 3)])
def test_partition_depth_matches_explicit_sublists(key_field, key_bits):
    for seed, n_rules in ((1, 300), (2, 60)):
        rules = W.gen_rules(n_rules, seed)
        rules["proto"][::7] = 47  # an exact protocol outside the usual three
        rules["proto_any"][::7] = 0
        rules["dst_prefix"][::9] = 1  # prefixes shorter than the key
        h = W.gen_packets(rules, 1200, seed + 10)
        h["proto"][::5] = 47
        idx, _, _ = oracle.classify(rules, h)
        assert bench.partition_depth(rules, idx, h, key_field, key_bits) == \
            explicit_partition_depth(rules, idx, h, key_field, key_bits)
