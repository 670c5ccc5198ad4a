"""The rule-list partition written out from its definition, for tests.

Protocol classes: the up to 7 exact protocols used most by the rules (ties to
the lower value), then "other" for every remaining protocol value. Each class
is split by the top ``key_bits`` bits of one address (``key_field`` 1 = src,
2 = dst). A class's sub-list holds, in list order, every rule that can match
one of its packets: a rule whose protocol set meets the class's protocols and
whose address interval on the key field meets the class's key interval. A
packet's class is its protocol class << key_bits | its key.

The key is the one with the lowest mean per-class cost (the sub-list length,
or for a granule g > 1 ceil(length / g) and at least 1), candidates taken
source before destination, fewer bits first, a later one only if strictly
lower, at most 8 classes; no key when none is lower than the protocol classes
alone.
"""
import numpy as np

MAX_CLASSES = 8
FIELD = {1: "src", 2: "dst"}


def protocol_classes(rules):
    """(exact protocols with a class of their own, in class order; protocol value -> class)."""
    exact = rules["proto_any"] == 0
    cnt = np.bincount(rules["proto"][exact].astype(np.int64), minlength=256)
    order = sorted(np.nonzero(cnt)[0].tolist(), key=lambda p: (-int(cnt[p]), p))[:MAX_CLASSES - 1]
    proto_class = np.full(256, len(order), dtype=np.uint8)
    for c, p in enumerate(order):
        proto_class[p] = c
    return order, proto_class


def address_interval(addr, prefix):
    """[lo, hi] of the addresses a prefix rule accepts (prefix 0: all of them)."""
    if prefix == 0:
        return 0, 0xFFFFFFFF
    span = 1 << (32 - prefix)
    lo = (int(addr) // span) * span
    return lo, lo + span - 1


def class_sublists(rules, key_field, key_bits):
    """Per class, the indices of the rules that can match one of its packets, in list order."""
    order, proto_class = protocol_classes(rules)
    lists = []
    for pc in range(len(order) + 1):
        proto_ok = [bool(rules["proto_any"][j]) or int(proto_class[int(rules["proto"][j])]) == pc
                    for j in range(len(rules))]
        keys = range(1 << key_bits) if key_field else [None]
        for k in keys:
            members = []
            for j in range(len(rules)):
                if not proto_ok[j]:
                    continue
                if k is not None:
                    f = FIELD[key_field]
                    lo, hi = address_interval(rules[f + "_addr"][j], int(rules[f + "_prefix"][j]))
                    # the class's addresses are [k << (32 - b), ((k + 1) << (32 - b)) - 1]
                    k_lo, k_hi = k << (32 - key_bits), ((k + 1) << (32 - key_bits)) - 1
                    if hi < k_lo or lo > k_hi:
                        continue
                members.append(j)
            lists.append(np.array(members, dtype=np.int64))
    return lists


def cost(lists, granule):
    if granule <= 1:
        return float(np.mean([len(x) for x in lists]))
    return float(np.mean([max(1, -(-len(x) // granule)) for x in lists]))


def best_key(rules, granule=1):
    n_p = len(protocol_classes(rules)[0]) + 1
    key, best = (0, 0), cost(class_sublists(rules, 0, 0), granule)
    for f in (1, 2):
        for b in (1, 2, 3):
            if n_p << b <= MAX_CLASSES:
                c = cost(class_sublists(rules, f, b), granule)
                if c < best:
                    key, best = (f, b), c
    return key


def packet_class(hdr, proto_class, key_field, key_bits):
    c = proto_class[hdr["proto"].astype(np.int64)].astype(np.int64)
    if not key_field:
        return c
    a = hdr[FIELD[key_field]].astype(np.int64)
    return (c << key_bits) | (a >> (32 - key_bits))
