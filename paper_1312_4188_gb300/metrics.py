"""Workload metrics shared by bench.py and measure.py (host-side numpy, no GPU work)."""
import numpy as np


def partition_depth(rules, out_idx_np, hdr, key_field=0, key_bits=0):
    """Rules the partitioned scan examines per packet (position of the match in the packet's
    class sub-list, or the sub-list length when unmatched), summed. Mirrors how the library
    forms the classes: the 7 exact protocols most used by reachable rules, then "other", each
    split by the top ``key_bits`` bits of the source (``key_field`` 1) or destination (2)
    address (``Ruleset.partition()`` reports the key the library chose)."""
    r = rules
    ca = np.nonzero((r["src_prefix"] == 0) & (r["dst_prefix"] == 0) & (r["sport_lo"] == 0) &
                    (r["sport_hi"] == 65535) & (r["dport_lo"] == 0) & (r["dport_hi"] == 65535) &
                    (r["proto_any"] != 0))[0]
    n_eff = int(ca[0]) + 1 if len(ca) else len(r)
    r = r[:n_eff]
    exact = r["proto_any"] == 0
    cnt = np.bincount(r["proto"][exact].astype(np.int64), minlength=256)
    order = [int(p) for p in sorted(np.nonzero(cnt)[0], key=lambda p: (-cnt[p], p))][:7]
    n_p = len(order) + 1
    class_of = np.full(256, n_p - 1, dtype=np.int64)
    for c, p in enumerate(order):
        class_of[p] = c
    pc = class_of[hdr["proto"].astype(np.int64)]
    if key_field:
        fld = "src" if key_field == 1 else "dst"
        pkey = hdr[fld].astype(np.int64) >> (32 - key_bits)
        raddr = r[fld + "_addr"].astype(np.int64)
        rlen = r[fld + "_prefix"].astype(np.int64)
    else:
        pkey = np.zeros(len(pc), dtype=np.int64)
    total = 0
    for c in range(n_p):
        pmember = (~exact) | (exact & (class_of[r["proto"].astype(np.int64)] == c))
        for k in range(1 << key_bits if key_field else 1):
            member = pmember.copy()
            if key_field:
                long_ = rlen >= key_bits
                short = (rlen > 0) & ~long_
                top = np.where(long_, raddr >> (32 - key_bits), 0)
                cover = (rlen == 0) | (long_ & (top == k)) | (
                    short & ((k >> np.maximum(key_bits - rlen, 0)) == (raddr >> np.maximum(32 - rlen, 0))))
                member &= cover
            pos = np.cumsum(member)
            sel = (pc == c) & (pkey == k)
            idx = out_idx_np[sel]
            total += int(np.where(idx >= 0, pos[np.maximum(idx, 0)], member.sum()).sum())
    return total
