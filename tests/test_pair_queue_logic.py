"""CPU emulation of the two-packet scan's per-warp queue (run_batch_pairs).

The emulation follows the device routine step by step on queue positions:
the register counting sort (per-lane class counts, a warp-wide exclusive
scan, each lane writing its own packets), the even padding of every class
region, the pair layout (lane l of a 64-entry group holds sorted entries 2l
and 2l+1), the segment loop with its decisions, and the in-place re-sort of
undecided packets by per-class atomic counters, taken here in a random order
(any order the hardware may pick). Packets carry a class and the position of
their first match in that class's sub-list (or none), so the expected verdict
of every packet is known.

Invariants checked, each of which the device code relies on:
- a lane's first entry is never a pad, and its second is a pad or shares its class;
- no write of the re-sort lands in a group the warp has not read yet;
- the queue never holds more entries than its capacity;
- every packet is decided exactly once, with its expected result.
"""
import random

import pytest

NO_SLOT = None
MAX_CLASSES = 8


def pair_slot(pos):
    return (pos & ~63) + ((pos & 1) << 5) + ((pos >> 1) & 31)


def round4(x):
    return (x + 3) & ~3


def run_batch(cap, n_classes, cls, depth, class_len, seg0, rng):
    """Returns {packet: result}; result = match position in the class sub-list, or -1."""
    cnt = len(cls)
    assert cnt <= cap - round4(n_classes)
    Q = [None] * cap
    # register counting sort: lane l owns quads l, l + 32, ...; counts, exclusive scan, scatter
    quads = [list(range(q * 4, min(cnt, q * 4 + 4))) for q in range((cnt + 3) // 4)]
    own = [[0] * n_classes for _ in range(32)]
    for q, pk in enumerate(quads):
        for i in pk:
            own[q % 32][cls[i]] += 1
    total = [sum(own[l][c] for l in range(32)) for c in range(n_classes)]
    start, m = [], 0
    for c in range(n_classes):
        start.append(m)
        m += (total[c] + 1) & ~1
    assert m <= cap
    ex = [[sum(own[k][c] for k in range(l)) for c in range(n_classes)] for l in range(32)]
    for q, pk in enumerate(quads):
        lane = q % 32
        for i in pk:
            c = cls[i]
            pos = start[c] + ex[lane][c]
            ex[lane][c] += 1
            s = pair_slot(pos)
            assert pos < m and Q[s] is None
            Q[s] = (i, c)
    for c in range(n_classes):
        if total[c] & 1:
            s = pair_slot(start[c] + total[c])
            assert Q[s] is None
            Q[s] = (NO_SLOT, 0)

    out = {}
    max_len = max(class_len[:n_classes])
    s0, s1 = 0, seg0
    while m > 0:
        final = s1 >= max_len
        kept = [0] * n_classes
        for g0 in range(0, m, 64):
            for lane in range(32):
                if not g0 + 2 * lane < m:
                    continue
                e0, e1 = Q[g0 + lane], Q[g0 + 32 + lane]
                assert e0[0] is not NO_SLOT, "a pad or a decided packet in a lane's first entry"
                c = e0[1]
                assert e1[0] is NO_SLOT or e1[1] == c, "the two entries of a lane differ in class"
                length = class_len[c]
                last = s1 >= length
                for u, e in enumerate((e0, e1)):
                    if e[0] is NO_SLOT:
                        continue
                    d = depth[e[0]]
                    assert d is None or d >= s0, "a packet outlived its match"
                    r = d if d is not None and s0 <= d < min(s1, length) else -1
                    if r >= 0 or last:
                        assert e[0] not in out
                        out[e[0]] = r
                        if not final:
                            Q[g0 + 32 * u + lane] = (NO_SLOT, e[1])
                    elif not final:
                        kept[c] += 1
        if final:
            break
        m_old = m
        cur, m = [], 0
        for c in range(n_classes):
            cur.append(m)
            m += (kept[c] + 1) & ~1
        assert m <= m_old <= cap
        for g0 in range(0, m_old, 64):
            held = []
            for lane in range(32):  # every lane reads its two entries before any write
                if g0 + 2 * lane < m_old:
                    held += [Q[g0 + lane], Q[g0 + 32 + lane]]
            writes = [e for e in held if e[0] is not NO_SLOT]
            rng.shuffle(writes)  # the atomics' order is the hardware's choice
            for e in writes:
                pos = cur[e[1]]
                cur[e[1]] += 1
                assert pos < g0 + 64, "the re-sort overwrote an entry not read yet"
                Q[pair_slot(pos)] = e
        for c in range(n_classes):
            if kept[c] & 1:
                Q[pair_slot(cur[c])] = (NO_SLOT, 0)
        s0, s1 = s1, s1 * 2
    assert len(out) == cnt
    return out


def check(cap, n_classes, cnt, class_len, seg0, rng, one_class=False):
    cls = [0 if one_class else rng.randrange(n_classes) for _ in range(cnt)]
    depth = []
    for c in cls:  # the match position in the class sub-list, or None (no rule matches)
        d = rng.randrange(class_len[c] + 4) if class_len[c] else None
        depth.append(d if d is not None and d < class_len[c] else None)
    out = run_batch(cap, n_classes, cls, depth, class_len, seg0, rng)
    for i in range(cnt):
        assert out[i] == (depth[i] if depth[i] is not None else -1), i


@pytest.mark.parametrize("seed", range(6))
def test_random_batches(seed):
    rng = random.Random(seed)
    for _ in range(150):
        cap = rng.choice([128, 256, 512])
        n_classes = rng.randint(1, MAX_CLASSES)
        cnt = rng.randint(0, cap - round4(n_classes))
        class_len = [4 * rng.randint(0, 80) for _ in range(n_classes)]
        check(cap, n_classes, cnt, class_len, rng.choice([4, 8, 16, 32, 64, 512]), rng)


def test_edge_batches():
    rng = random.Random(99)
    for n_classes in (1, 2, 3, 7, 8):
        for cap in (128, 256):
            full = cap - round4(n_classes)
            for cnt in (0, 1, 2, 63, 64, 65, full - 1, full):
                for class_len in ([0] * n_classes, [4] * n_classes, [400] + [0] * (n_classes - 1)):
                    for seg0 in (4, 512):
                        check(cap, n_classes, cnt, class_len, seg0, rng)
    # every packet in one class, odd counts, deep sub-list: the most re-sorts per batch
    for cnt in (1, 3, 121, 247):
        check(256, 8, cnt, [1000] + [4] * 7, 4, rng, one_class=True)
