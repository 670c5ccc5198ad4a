"""The N>1 path (replicas) on CPU with two gloo ranks: per-rank batches and the max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_1312_4188_gb300 import replica, workload as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = replica.world()
    rules = W.gen_rules(50, 1)
    h = W.gen_packets(rules, 1000, replica.packets_seed(2, r))
    elapsed = 10.0 + r  # a slower rank 1
    m = replica.max_over_ranks(elapsed)
    rate = replica.job_rate(1000, 5, ws, m)
    q.put((r, ws, int(h["src"][:8].sum()), m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
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
    (r0, w0, s0, m0, rate0), (r1, w1, s1, m1, rate1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert s0 != s1, "ranks must classify different batches"
    assert m0 == m1 == 11.0, "elapsed time is the max over ranks"
    assert rate0 == rate1 == pytest.approx(2 * 1000 * 5 / 11e-3 / 1e6)


def test_single_process_defaults():
    from paper_1312_4188_gb300 import replica
    assert replica.packets_seed(4, 0) == 4
    assert replica.max_over_ranks(3.5) == 3.5
    assert replica.job_rate(100, 2, 1, 1.0) == pytest.approx(0.2)
