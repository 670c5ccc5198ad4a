"""The seeded generator draws what its recipe states (determinism, slices, in-rule packets, shares)."""
import numpy as np
import pytest

import oracle_pins as P
from paper_1312_4188_gb300 import workload as W


def test_rules_are_deterministic_and_valid():
    a, b = W.gen_rules(5000, 42), W.gen_rules(5000, 42)
    assert a.tobytes() == b.tobytes()
    assert a.tobytes() != W.gen_rules(5000, 43).tobytes()
    assert np.all(a["src_prefix"] <= 32) and np.all(a["dst_prefix"] <= 32)
    assert np.all(a["sport_lo"] <= a["sport_hi"]) and np.all(a["dport_lo"] <= a["dport_hi"])
    assert set(np.unique(a["action"])) <= {0, 1}


def test_rule_distribution_shares():
    r = W.gen_rules(200_000, 7)
    n = len(r)
    assert abs((r["src_prefix"] == 0).mean() - 0.2) < 0.01
    nz = r["src_prefix"][r["src_prefix"] > 0]
    assert nz.min() == 8 and nz.max() == 32
    wild = (r["sport_lo"] == 0) & (r["sport_hi"] == 65535)
    exact = r["sport_lo"] == r["sport_hi"]
    assert abs(wild.mean() - 0.5) < 0.01 and abs(exact.mean() - 0.3) < 0.01
    width = r["sport_hi"].astype(int) - r["sport_lo"].astype(int) + 1
    rng_ = ~wild & ~exact
    assert width[rng_].max() <= 1024
    assert abs(r["proto_any"].mean() - 0.25) < 0.01
    assert set(np.unique(r["proto"][r["proto_any"] == 0])) == {1, 6, 17}
    assert abs(r["action"].mean() - 0.5) < 0.01
    assert n == 200_000


def test_packet_slices_match_the_whole_batch():
    rules = W.gen_rules(300, 1)
    whole = W.gen_packets(rules, 3 * W.BLOCK // 2, 5, zipf_s=1.1)
    part = W.gen_packets(rules, 1000, 5, zipf_s=1.1, start=W.BLOCK - 400)
    for f in W.HEADER_FIELDS:
        assert np.array_equal(part[f], whole[f][W.BLOCK - 400:W.BLOCK + 600])


def test_in_rule_packets_lie_in_some_rule():
    rules = W.gen_rules(200, 3)
    h = W.gen_packets(rules, 20_000, 4, in_rule_frac=1.0)
    sets = [P.rule_sets(r) for r in rules]
    for i in range(0, 20_000, 97):
        p = tuple(int(h[f][i]) for f in W.HEADER_FIELDS)
        assert any(P.contains(s, p) for s in sets), f"packet {i} is in no rule"


def test_zipf_favours_early_rules():
    cdf = W.zipf_cdf(10_000, 1.1)
    assert cdf[-1] == pytest.approx(1.0) and np.all(np.diff(cdf) > 0)
    w = np.arange(1, 10_001, dtype=float) ** -1.1
    assert cdf[0] == pytest.approx(w[0] / w.sum())


def test_log_uniform_and_batched_shapes():
    rng = np.random.default_rng(0)
    x = W.log_uniform_int(rng, 64, 65536, 100_000)
    assert x.min() >= 64 and x.max() <= 65536
    # log-uniform: the median is near the geometric mean
    assert 1500 < np.median(x) < 2600
    jobs = W.gen_batched(4, seed=1, rules_range=(64, 128), packets_range=(1024, 2048))
    assert len(jobs) == 4 and all(64 <= len(r) <= 128 and 1024 <= len(h["src"]) <= 2048 for r, h in jobs)


def test_sample_positions():
    pos = W.sample_positions(1000, 100, 3)
    assert len(np.unique(pos)) == 100 and pos.min() >= 0 and pos.max() < 1000
    assert np.array_equal(pos, W.sample_positions(1000, 100, 3))
    assert np.array_equal(W.sample_positions(10, 100, 3), np.arange(10))


def test_permuted_zipf_ranks_name_the_permuted_rules():
    """With rank_perm the Zipf rank r draws rule rank_perm[r]. On pairwise non-overlapping rules a
    packet drawn inside a rule matches that rule alone, so the oracle's index recovers the draw."""
    import oracle
    rules = P.non_overlapping_rules(40, 12)
    n = len(rules)
    perm = np.random.default_rng(5).permutation(n)
    hdr = W.gen_packets(rules, 200_000, 6, in_rule_frac=1.0, zipf_s=1.1, rank_perm=perm)
    idx, _, _ = oracle.classify(rules, hdr)
    assert (idx >= 0).all()
    by_rank = np.bincount(idx, minlength=n)[perm]  # matches per Zipf rank
    p = np.arange(1, n + 1, dtype=float) ** -1.1
    p /= p.sum()
    # every rank's share within 5 standard deviations of its Zipf probability
    sd = np.sqrt(p * (1 - p) / len(idx))
    assert np.all(np.abs(by_rank / len(idx) - p) < 5 * sd + 1e-9)
    assert by_rank[0] == by_rank.max() and perm[0] != 0  # the top rank is not the first rule here


def test_without_catch_alls_removes_exactly_the_catch_alls():
    rules = W.gen_rules(5000, 3)
    ca = np.array([P.rule_sets(r) == P.rule_sets(P.catch_all()[0]) for r in rules])
    kept = W.without_catch_alls(rules)
    assert ca.sum() > 0 and len(kept) == len(rules) - ca.sum()
    assert np.array_equal(kept, rules[~ca])  # list order kept
    r2, _ = W.make_workload("scan_10k_x_16m_no_catch_all", 1000)
    assert not any(P.rule_sets(r) == P.rule_sets(P.catch_all()[0]) for r in r2)


def test_threaded_generation_gives_the_same_inputs():
    rules = W.gen_rules(300, 11)
    n = 3 * W.BLOCK + 12345
    a = W.gen_packets(rules, n, 12, zipf_s=1.1, start=777)
    b = W.gen_packets(rules, n, 12, zipf_s=1.1, start=777, workers=4)
    for f in W.HEADER_FIELDS:
        assert np.array_equal(a[f], b[f])
    s1 = W.gen_batched(6, seed=3, rules_range=(64, 512), packets_range=(1024, 4096))
    s4 = W.gen_batched(6, seed=3, rules_range=(64, 512), packets_range=(1024, 4096), workers=4)
    for (r1, h1), (r4, h4) in zip(s1, s4):
        assert np.array_equal(r1, r4)
        for f in W.HEADER_FIELDS:
            assert np.array_equal(h1[f], h4[f])
