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


def test_partition_depth_follows_the_library_plan():
    """For an unmatched packet the metric counts its whole sub-list: that length equals the class
    length in the library's own plan (fw_partition_plan) of the rules up to the first catch-all,
    for the key the library picks."""
    import partition_ref as R
    from paper_1312_4188_gb300 import fw
    keys = set()
    # five protocol classes leave no room for a key; four (the generator's protocols) leave one bit
    for seed, n_rules, extra_proto in ((1, 300, True), (4, 2000, False), (5, 1000, False)):
        rules = W.gen_rules(n_rules, seed)
        if extra_proto:
            rules["proto"][::7] = 47
            rules["proto_any"][::7] = 0
        ca = np.nonzero((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0) & (rules["sport_lo"] == 0)
                        & (rules["sport_hi"] == 65535) & (rules["dport_lo"] == 0) & (rules["dport_hi"] == 65535)
                        & (rules["proto_any"] != 0))[0]
        n_eff = int(ca[0]) + 1 if len(ca) else len(rules)
        plan = fw.fw_partition_plan(rules[:n_eff], 1)
        kf, kb = plan["key_field"], plan["key_bits"]
        keys.add((kf, kb))
        for proto in (0, 1, 6, 17, 47, 99, 255):
            for top in range(8):
                h = W.empty_headers(1)
                h["proto"][0] = proto
                h["src"][0] = (top << 29) | 12345
                h["dst"][0] = ((7 - top) << 29) | 678
                c = int(R.packet_class(h, plan["proto_class"], kf, kb)[0])
                got = bench.partition_depth(rules, np.array([-1], dtype=np.int32), h, kf, kb)
                assert got == plan["class_len"][c], (seed, proto, top)
    assert (0, 0) in keys and any(k != (0, 0) for k in keys)


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The committed ncu record applies while its kernel's sources are unchanged, and only to its
    own kernel and workload; a digest that no longer matches gives null."""
    import json
    rec = json.load(open(bench.TRAFFIC_FILE))
    got, note = bench.recorded_traffic(rec["kernel"], rec["workload"], rec["mode"])
    if rec["sources_sha"] == bench.sources_sha(rec["sources"]):
        assert got == rec["dram_bytes_per_launch"] and "ncu" in note
    else:
        assert got is None and "changed" in note
    assert bench.recorded_traffic("k_other", rec["workload"], rec["mode"])[0] is None
    stale = dict(rec, sources_sha="0" * 16)
    path = tmp_path / "dram_traffic.json"
    path.write_text(json.dumps(stale))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.recorded_traffic(rec["kernel"], rec["workload"], rec["mode"])[0] is None
