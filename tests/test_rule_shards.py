"""Rule split across ranks (paper_1312_4188_gb300/rule_shards.py) on the CPU.

The oracle stands in for each rank's classification of its rule range, so these tests check
the exchange protocol itself: contiguous ranges, local-to-global indices, the elementwise
minimum (two real gloo ranks, and virtual ranks in one process), and the action lookup.
Every result must equal the oracle's whole-list first match.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1312_4188_gb300 import rule_shards as S, workload as W


def rule_set(seed, n):
    """Generated rules with a catch-all planted a third of the way down (when n >= 10): the range
    holding it stops there, and the ranges after it can only lose the minimum."""
    rules = W.gen_rules(n, seed)
    if n >= 10:
        k = n // 3
        rules[k] = (0, 0, 0, 65535, 0, 65535, 0, 0, 0, 1, W.ACCEPT)
    return rules


@pytest.mark.parametrize("n", [0, 1, 2, 7, 100, 1001])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_cover_the_list(n, world):
    ranges = [S.shard_range(n, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    sizes = [hi - lo for lo, hi in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        S.shard_range(n, world, world)


def local_first_match(rules, lo, hi, hdr):
    idx, _, _ = oracle.classify(rules[lo:hi], hdr)
    return torch.from_numpy(idx.astype(np.int32))


def test_to_global_and_finalize():
    local = torch.tensor([-1, 0, 3, -1], dtype=torch.int32)
    g = S.to_global(local, 10)
    assert g.tolist() == [S.NO_MATCH, 10, 13, S.NO_MATCH]
    actions = torch.zeros(20, dtype=torch.uint8)
    actions[10], actions[13] = 1, 0
    idx, act = S.finalize(g, actions)
    assert idx.tolist() == [-1, 10, 13, -1] and act.tolist() == [0, 1, 0, 0]
    idx, act = S.finalize(torch.full((3,), S.NO_MATCH, dtype=torch.int32), torch.zeros(0, dtype=torch.uint8))
    assert idx.tolist() == [-1, -1, -1] and act.tolist() == [0, 0, 0]
    assert S.combine(g) is g  # no process group: the identity


@pytest.mark.parametrize("world", [1, 2, 3, 5, 16])
def test_virtual_ranks_equal_the_whole_list(world):
    for seed, n in ((1, 400), (2, 60), (3, 7)):
        rules = rule_set(seed, n)
        hdr = W.gen_packets(rules, 3000, seed + 20)
        want_idx, want_act, _ = oracle.classify(rules, hdr)
        g = None
        for r in range(world):
            lo, hi = S.shard_range(len(rules), world, r)
            part = S.to_global(local_first_match(rules, lo, hi, hdr), lo)
            g = part if g is None else torch.minimum(g, part)
        idx, act = S.finalize(g, torch.from_numpy(rules["action"].astype(np.uint8)))
        assert np.array_equal(idx.numpy(), want_idx) and np.array_equal(act.numpy(), want_act)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rules = W.without_catch_alls(W.gen_rules(500, 4))  # deep scans: matches spread over both ranges
    hdr = W.gen_packets(rules, 4000, 5)  # the same headers on every rank
    lo, hi = S.shard_range(len(rules), world, rank)
    g = S.combine(S.to_global(local_first_match(rules, lo, hi, hdr), lo))
    idx, act = S.finalize(g, torch.from_numpy(rules["action"].astype(np.uint8)))
    q.put((rank, lo, hi, idx.numpy().tobytes(), act.numpy().tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_by_minimum():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rules = W.without_catch_alls(W.gen_rules(500, 4))
    hdr = W.gen_packets(rules, 4000, 5)
    want_idx, want_act, _ = oracle.classify(rules, hdr)
    (_, lo0, hi0, _, _), (_, lo1, hi1, _, _) = out
    assert (lo0, hi1) == (0, len(rules)) and hi0 == lo1
    # matches fall in both ranges, so the minimum does real work
    assert ((want_idx >= 0) & (want_idx < hi0)).any() and (want_idx >= lo1).any()
    for _, _, _, idx_b, act_b in out:  # every rank ends with the whole-list answer
        assert np.array_equal(np.frombuffer(idx_b, dtype=np.int32), want_idx)
        assert np.array_equal(np.frombuffer(act_b, dtype=np.uint8), want_act)


@pytest.mark.parametrize("world", [4, 9])
def test_more_ranks_than_rules(world):
    """Ranks beyond the rule count hold empty ranges: they report no match for every packet, and
    the minimum over ranks is still the whole list's first match (DROP where no rule matches)."""
    for rules in (rule_set(4, 3), W.without_catch_alls(rule_set(5, 2)), W.empty_rules(0)):
        src = rules if len(rules) else rule_set(6, 40)
        hdr = W.gen_packets(src, 4000, 26)
        want_idx, want_act, _ = oracle.classify(rules, hdr)
        g = None
        for r in range(world):
            lo, hi = S.shard_range(len(rules), world, r)
            part = S.to_global(local_first_match(rules, lo, hi, hdr), lo)
            g = part if g is None else torch.minimum(g, part)
        idx, act = S.finalize(g, torch.from_numpy(rules["action"].astype(np.uint8)))
        assert np.array_equal(idx.numpy(), want_idx) and np.array_equal(act.numpy(), want_act)
        assert np.all(act.numpy()[want_idx < 0] == 0)
