"""Seeded synthetic rule sets and packet batches.

This module only draws random inputs. It holds none of the classification
arithmetic: no match predicate, no first-match search, no packing. Both the
CUDA path (through the tests and the bench) and the CPU oracle consume what it
returns, so neither side can feed the other its expected values.

Rule model (Sec. IV, "Implementation on CUDA"): each rule carries a source and
destination IPv4 address, a source and destination port, a protocol and an
action; a field that is not specified matches every value of that field.
The concrete encoding used throughout this project:

* addresses: a host-order uint32 value plus a prefix length 0..32
  (0 = any address);
* ports: an inclusive range [lo, hi] (wildcard = [0, 65535], exact = [p, p]);
* protocol: a uint8 value plus a ``proto_any`` flag (proto 0 stays a legal value);
* action: DROP = 0, ACCEPT = 1.

Distributions (synthetic stand-in for the paper's hping3 traffic, Sec. IV
"Results and Analysis"):

* prefix length 0 with probability 0.2, otherwise uniform on 8..32 inclusive;
* each port: wildcard 0.5, exact 0.3 (uniform 0..65535), range 0.2 with width
  w uniform on 1..1024, lo uniform on 0..65536-w, hi = lo+w-1;
* protocol uniform over {6, 17, 1, any}; action ACCEPT/DROP 50/50;
* packets: 60 % drawn inside a chosen rule (every field uniform inside that
  rule's set; proto uniform 0..255 when the rule has proto any), 40 % uniform
  over the whole header space. The chosen rule is uniform over the rule list,
  or Zipf(s) over the rule index (P(k) proportional to (k+1)^-s).

Packet batches are generated in fixed blocks of ``BLOCK`` packets, each from
its own ``SeedSequence((seed, block))`` stream, so any slice of a large batch
can be regenerated without drawing the rest.
"""
from __future__ import annotations

import numpy as np

DROP = 0
ACCEPT = 1

# Layout of one rule as the C ABI sees it (struct fw_rule, 24 bytes).
RULE_DTYPE = np.dtype(
    {
        "names": [
            "src_addr", "dst_addr",
            "sport_lo", "sport_hi", "dport_lo", "dport_hi",
            "src_prefix", "dst_prefix", "proto", "proto_any", "action",
        ],
        "formats": [
            np.uint32, np.uint32,
            np.uint16, np.uint16, np.uint16, np.uint16,
            np.uint8, np.uint8, np.uint8, np.uint8, np.uint8,
        ],
        "offsets": [0, 4, 8, 10, 12, 14, 16, 17, 18, 19, 20],
        "itemsize": 24,
    }
)

HEADER_FIELDS = ("src", "dst", "sport", "dport", "proto")
HEADER_DTYPES = {
    "src": np.uint32,
    "dst": np.uint32,
    "sport": np.uint16,
    "dport": np.uint16,
    "proto": np.uint8,
}
HEADER_BYTES = 4 + 4 + 2 + 2 + 1

BLOCK = 1 << 20
PROTO_CHOICES = (6, 17, 1, -1)  # -1 = any


def empty_rules(n: int) -> np.ndarray:
    return np.zeros(n, dtype=RULE_DTYPE)


def empty_headers(n: int) -> dict:
    return {f: np.zeros(n, dtype=HEADER_DTYPES[f]) for f in HEADER_FIELDS}


def _port_rules(rng: np.random.Generator, n: int):
    kind = rng.random(n)
    lo = np.zeros(n, dtype=np.int64)
    hi = np.full(n, 65535, dtype=np.int64)
    exact = (kind >= 0.5) & (kind < 0.8)
    rng_ = kind >= 0.8
    p = rng.integers(0, 65536, size=n)
    lo[exact] = p[exact]
    hi[exact] = p[exact]
    w = rng.integers(1, 1025, size=n)
    start = (rng.random(n) * (65536 - w + 1)).astype(np.int64)
    lo[rng_] = start[rng_]
    hi[rng_] = start[rng_] + w[rng_] - 1
    return lo.astype(np.uint16), hi.astype(np.uint16)


def _prefix(rng: np.random.Generator, n: int) -> np.ndarray:
    any_ = rng.random(n) < 0.2
    plen = rng.integers(8, 33, size=n)
    plen[any_] = 0
    return plen.astype(np.uint8)


def gen_rules(n: int, seed: int) -> np.ndarray:
    """Draw ``n`` rules with the distributions listed in the module docstring."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence((int(seed), 0x52554C45))))
    r = empty_rules(n)
    r["src_addr"] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    r["dst_addr"] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    r["src_prefix"] = _prefix(rng, n)
    r["dst_prefix"] = _prefix(rng, n)
    r["sport_lo"], r["sport_hi"] = _port_rules(rng, n)
    r["dport_lo"], r["dport_hi"] = _port_rules(rng, n)
    pc = rng.integers(0, 4, size=n)
    proto = np.array(PROTO_CHOICES, dtype=np.int64)[pc]
    r["proto_any"] = (proto < 0).astype(np.uint8)
    r["proto"] = np.where(proto < 0, 0, proto).astype(np.uint8)
    r["action"] = (rng.random(n) < 0.5).astype(np.uint8)
    return r


def zipf_cdf(n_rules: int, s: float) -> np.ndarray:
    """Cumulative distribution of P(k) ~ (k+1)^-s over k = 0..n_rules-1 (float64)."""
    w = np.arange(1, n_rules + 1, dtype=np.float64) ** (-float(s))
    c = np.cumsum(w)
    return c / c[-1]


def _draw_rule_index(rng, m, n_rules, cdf):
    if cdf is None:
        return rng.integers(0, n_rules, size=m)
    u = rng.random(m)
    k = np.searchsorted(cdf, u, side="right")
    return np.minimum(k, n_rules - 1)


def _uniform_in(rng, lo, hi):
    """Uniform integer in the inclusive range [lo, hi], elementwise."""
    lo = lo.astype(np.int64)
    span = hi.astype(np.int64) - lo + 1
    return lo + (rng.random(lo.shape[0]) * span).astype(np.int64)


def _address_in(rng, addr, plen):
    """Uniform address sharing the top ``plen`` bits of ``addr`` (plen 0 = any)."""
    a = addr.astype(np.uint64)
    free_bits = 32 - plen.astype(np.uint64)
    low = rng.integers(0, 1 << 32, size=a.shape[0], dtype=np.uint64)
    span = np.left_shift(np.uint64(1), free_bits)  # 2^(32-plen), at most 2^32
    base = a - (a % span)
    return (base + (low % span)).astype(np.uint32)


def _gen_block(rules, n_rules, m, seed, block, in_rule_frac, cdf, rank_perm=None):
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence((int(seed), int(block), 0x504B54))))
    h = {
        "src": rng.integers(0, 1 << 32, size=m, dtype=np.uint64).astype(np.uint32),
        "dst": rng.integers(0, 1 << 32, size=m, dtype=np.uint64).astype(np.uint32),
        "sport": rng.integers(0, 65536, size=m).astype(np.uint16),
        "dport": rng.integers(0, 65536, size=m).astype(np.uint16),
        "proto": rng.integers(0, 256, size=m).astype(np.uint8),
    }
    if n_rules == 0 or in_rule_frac <= 0.0:
        return h
    inside = np.nonzero(rng.random(m) < in_rule_frac)[0]
    if inside.size == 0:
        return h
    k = _draw_rule_index(rng, inside.size, n_rules, cdf)
    if rank_perm is not None:  # the drawn rank names rule rank_perm[rank]
        k = rank_perm[k]
    rk = rules[k]
    h["src"][inside] = _address_in(rng, rk["src_addr"], rk["src_prefix"])
    h["dst"][inside] = _address_in(rng, rk["dst_addr"], rk["dst_prefix"])
    h["sport"][inside] = _uniform_in(rng, rk["sport_lo"], rk["sport_hi"]).astype(np.uint16)
    h["dport"][inside] = _uniform_in(rng, rk["dport_lo"], rk["dport_hi"]).astype(np.uint16)
    anyp = rk["proto_any"] != 0
    pr = np.where(anyp, rng.integers(0, 256, size=inside.size), rk["proto"].astype(np.int64))
    h["proto"][inside] = pr.astype(np.uint8)
    return h


def gen_packets(rules: np.ndarray, n: int, seed: int, in_rule_frac: float = 0.6,
                zipf_s: float | None = None, start: int = 0, rank_perm: np.ndarray | None = None,
                workers: int = 1) -> dict:
    """Draw packets ``start .. start+n-1`` of the batch defined by (rules, seed, ...).

    Returns SoA numpy arrays keyed by ``HEADER_FIELDS``. ``zipf_s=None`` picks the
    rule of an in-rule packet uniformly; otherwise Zipf(zipf_s) over the index, or,
    with ``rank_perm`` (a permutation of the rule indices), over the ranks, rank r
    naming rule ``rank_perm[r]`` (popular rules no longer sit at the top of the list).
    ``workers`` > 1 draws the blocks on that many threads (each block has its own
    generator, so the result does not depend on it).
    """
    n_rules = int(rules.shape[0])
    cdf = zipf_cdf(n_rules, zipf_s) if (zipf_s is not None and n_rules > 0) else None
    out = empty_headers(n)
    if n == 0:
        return out
    end = start + n
    b0, b1 = start // BLOCK, (end - 1) // BLOCK

    def one(b):
        bs = b * BLOCK
        blk = _gen_block(rules, n_rules, BLOCK, seed, b, in_rule_frac, cdf, rank_perm)
        lo = max(start, bs)
        hi = min(end, bs + BLOCK)
        for f in HEADER_FIELDS:
            out[f][lo - start:hi - start] = blk[f][lo - bs:hi - bs]

    if workers > 1 and b1 > b0:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(min(int(workers), b1 - b0 + 1)) as ex:
            list(ex.map(one, range(b0, b1 + 1)))
    else:
        for b in range(b0, b1 + 1):
            one(b)
    return out


def without_catch_alls(rules: np.ndarray) -> np.ndarray:
    """The rules minus every all-wildcard one (default deny then decides the unmatched packets)."""
    ca = ((rules["src_prefix"] == 0) & (rules["dst_prefix"] == 0) & (rules["sport_lo"] == 0) &
          (rules["sport_hi"] == 65535) & (rules["dport_lo"] == 0) & (rules["dport_hi"] == 65535) &
          (rules["proto_any"] != 0))
    return np.ascontiguousarray(rules[~ca])


def take(headers: dict, idx: np.ndarray) -> dict:
    return {f: np.ascontiguousarray(headers[f][idx]) for f in HEADER_FIELDS}


def sample_positions(n: int, m: int, seed: int) -> np.ndarray:
    """Fixed seeded sample of ``min(m, n)`` distinct positions in [0, n), sorted."""
    if m >= n:
        return np.arange(n, dtype=np.int64)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence((int(seed), 0x53414D))))
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)


# Named workloads. Sizes follow the plain first-match case (1,000 rules x
# 100,000 packets, uniform rule choice), the scan at scale (10,000 rules x
# 16,777,216 packets, Zipf(1.1) rule choice) and the learned-index case
# (100,000 rules x 67,108,864 packets, uniform rule choice).
WORKLOADS = {
    "plain_1k_x_100k": dict(n_rules=1000, n_packets=100_000, rules_seed=1, packets_seed=2, zipf_s=None),
    "scan_10k_x_16m_zipf": dict(n_rules=10_000, n_packets=1 << 24, rules_seed=3, packets_seed=4, zipf_s=1.1),
    "lindex_100k_x_64m": dict(n_rules=100_000, n_packets=1 << 26, rules_seed=5, packets_seed=6, zipf_s=None),
    # labelled variants of the scan workload: the Zipf rank order permuted over the rule list,
    # and every all-wildcard rule removed (deep scans, default deny for unmatched packets)
    "scan_10k_x_16m_zipf_permuted": dict(n_rules=10_000, n_packets=1 << 24, rules_seed=3, packets_seed=4,
                                         zipf_s=1.1, rank_perm_seed=0x5045524D),
    "scan_10k_x_16m_no_catch_all": dict(n_rules=10_000, n_packets=1 << 24, rules_seed=3, packets_seed=4,
                                        zipf_s=1.1, drop_catch_alls=True),
}


def make_workload(name: str, n_packets: int | None = None, workers: int = 1):
    w = WORKLOADS[name]
    rules = gen_rules(w["n_rules"], w["rules_seed"])
    if w.get("drop_catch_alls"):
        rules = without_catch_alls(rules)
    perm = None
    if "rank_perm_seed" in w:
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence((w["rules_seed"], w["rank_perm_seed"]))))
        perm = rng.permutation(len(rules))
    n = w["n_packets"] if n_packets is None else n_packets
    hdr = gen_packets(rules, n, w["packets_seed"], zipf_s=w["zipf_s"], rank_perm=perm, workers=workers)
    return rules, hdr


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int, size: int) -> np.ndarray:
    """Integers log-uniform on [lo, hi]."""
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=size))).astype(np.int64).clip(lo, hi)


def gen_batched(n_sets: int = 256, seed: int = 7, rules_range=(64, 65536), packets_range=(1024, 1 << 20),
                zipf_s: float | None = None, workers: int = 1):
    """``n_sets`` independent (rules, headers) jobs with log-uniform rule and packet counts.

    Every set is drawn with the rule generator above from its own seed, and its
    batch with the packet generator (same 60/40 in-rule / uniform mix).
    ``workers`` > 1 draws the sets on that many threads (same result).
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence((int(seed), 0x42415443))))
    nr = log_uniform_int(rng, rules_range[0], rules_range[1], n_sets)
    npk = log_uniform_int(rng, packets_range[0], packets_range[1], n_sets)

    def one(i):
        rules = gen_rules(int(nr[i]), 1_000_000 + 1000 * int(seed) + i)
        hdr = gen_packets(rules, int(npk[i]), 2_000_000 + 1000 * int(seed) + i, zipf_s=zipf_s)
        return rules, hdr

    if workers > 1 and n_sets > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(min(int(workers), n_sets)) as ex:
            return list(ex.map(one, range(n_sets)))
    return [one(i) for i in range(n_sets)]
