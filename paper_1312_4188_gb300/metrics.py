"""Workload metrics shared by bench.py and measure.py (host-side numpy, no GPU work)."""
import numpy as np


def partition_depth(rules, out_idx_np, proto_np):
    """Rules the protocol-partitioned scan examines per packet (position of the match in the
    packet's class sub-list, or the sub-list length when unmatched), summed. Mirrors how the
    library forms the classes: the 7 exact protocols most used by reachable rules, then "other"."""
    r = rules
    ca = np.nonzero((r["src_prefix"] == 0) & (r["dst_prefix"] == 0) & (r["sport_lo"] == 0) &
                    (r["sport_hi"] == 65535) & (r["dport_lo"] == 0) & (r["dport_hi"] == 65535) &
                    (r["proto_any"] != 0))[0]
    n_eff = int(ca[0]) + 1 if len(ca) else len(r)
    r = r[:n_eff]
    exact = r["proto_any"] == 0
    cnt = np.bincount(r["proto"][exact].astype(np.int64), minlength=256)
    order = [int(p) for p in sorted(np.nonzero(cnt)[0], key=lambda p: (-cnt[p], p))][:7]
    n_cls = len(order) + 1
    class_of = np.full(256, n_cls - 1, dtype=np.int64)
    for c, p in enumerate(order):
        class_of[p] = c
    total = 0
    pc = class_of[proto_np.astype(np.int64)]
    for c in range(n_cls):
        member = (~exact) | (exact & (class_of[r["proto"].astype(np.int64)] == c))
        pos = np.cumsum(member)
        sel = pc == c
        idx = out_idx_np[sel]
        total += int(np.where(idx >= 0, pos[np.maximum(idx, 0)], member.sum()).sum())
    return total
