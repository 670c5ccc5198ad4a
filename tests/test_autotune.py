"""Host side of the autotuner: choosing among timed candidates, the result cache, and the
candidate lists' launch shapes (the documented fw_config rules), all without a GPU."""
import json

import pytest

from paper_1312_4188_gb300 import autotune as A
from paper_1312_4188_gb300 import fw

INF = float("inf")


def test_pick_best_takes_the_fastest_candidate_with_equal_verdicts():
    res = [({"a": 1}, 2.0, True), ({"a": 2}, 1.5, True), ({"a": 3}, INF, "rejected: bad shape"),
           ({"a": 4}, 1.7, True)]
    assert A.pick_best(res) == {"a": 2}
    assert A.pick_best([({"a": 3}, INF, "rejected: x")]) is None
    assert A.pick_best([]) is None


def test_pick_best_refuses_differing_verdicts():
    res = [({"a": 1}, 2.0, True), ({"a": 2}, 0.5, False)]  # the fastest is wrong: a bug, not a winner
    with pytest.raises(RuntimeError):
        A.pick_best(res)


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "autotune.json"
    monkeypatch.setattr(A, "cache_path", lambda: str(path))
    assert A.load_cache() == {}
    A.store("dev|w|packet_split", {"mode": "packet_split", "block_threads": 512})
    A.store("dev|w|rule_split", {"mode": "rule_split_warp"})
    d = json.load(open(path))
    assert d == A.load_cache() and set(d) == {"dev|w|packet_split", "dev|w|rule_split"}


@pytest.mark.parametrize("c", A.PACKET_SPLIT_CANDIDATES + A.RULE_SPLIT_CANDIDATES, ids=str)
def test_candidates_are_valid_launch_shapes(c):
    cfg = A.config_of(c)
    assert cfg.mode in fw.MODES.values()
    bt = c.get("block_threads", 0)
    assert bt % 32 == 0 and bt <= (512 if c["mode"].startswith("rule_split") else 1024)
    if c["mode"] == "packet_split" and c.get("compact") == 1:
        assert c.get("packets_per_group", 0) % 128 == 0
        assert c.get("segment_rules", 0) % 4 == 0
        if c.get("lane_packets") == 2:  # the two-packet kernel: at most 1,024 threads per SM
            assert bt * c.get("blocks_per_sm", 1) <= 1024
    if c.get("filter") == 1:  # the bucket-filter kernel: at most 512 threads, at most 3 blocks of 512
        assert bt <= 512 and bt * c.get("blocks_per_sm", 3) <= 1536
    if c["mode"].startswith("rule_split") and c.get("partition", 0) != 2:
        # partitioned rule split: fixed groups, warp and grid mode in blocks of at most 256 threads
        assert c.get("packets_per_group", 0) == 0
        assert c["mode"] == "rule_split_block" or bt <= 256


def test_plan_candidates():
    for ppi, seg in A.PLAN_CANDIDATES:
        assert ppi % 128 == 0 and ppi <= 4096 and seg % 4 == 0
