"""Device request queue: every request's result is the same alone and in the mix.

Requests of 1..65,536 packets (ragged sizes included) against four rule sets
(one without catch-alls, so its bucket filter has wide rows) are served one at
a time (submit, wait) and then all together, from device memory and from
pinned host memory; each result must equal, bit for bit, fw_classify's for the
same batch, and a sample is checked against the CPU oracle. Further tests make
the kernel's bounded waits run out (the idle limit and the time limit) and
check that the host launches it again, and check the argument errors.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1312_4188_gb300 import fw, workload as W

pytestmark = pytest.mark.gpu

POOL = 1 << 18
LIMIT = 10_000_000  # every wait of these tests gives up after 10 s


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_4188_gb300 import build
    build.build()
    sizes = [100, 1000, 3000, 10_000]
    rules = [W.gen_rules(n, 700 + i) for i, n in enumerate(sizes)]
    rules[2] = rules[2][~((rules[2]["src_prefix"] == 0) & (rules[2]["dst_prefix"] == 0))]
    sets = [fw.fw_ruleset_create(r) for r in rules]
    for rs in sets:
        assert rs.filter()["words"] > 0
    pools = [W.gen_packets(r, POOL, 70 + i, zipf_s=1.1 if i == 3 else None) for i, r in enumerate(rules)]
    dpools = [fw.headers_to_device(p) for p in pools]
    rng = np.random.default_rng(21)
    reqs = []
    for _ in range(300):
        s = int(rng.integers(0, 4))
        n = int(W.log_uniform_int(rng, 1, 65536, 1)[0])
        off = int(rng.integers(0, POOL - n + 1))
        reqs.append((s, off, n))
    reqs += [(0, 0, 1), (1, 3, 3), (2, 5, 65536), (3, 7, 257), (3, POOL - 65536, 65536)]
    total = sum(n for _, _, n in reqs)
    offs = np.concatenate([[0], np.cumsum([n for _, _, n in reqs])[:-1]]).astype(np.int64)
    ref_i = torch.empty(total, dtype=torch.int32, device="cuda")
    ref_a = torch.empty(total, dtype=torch.uint8, device="cuda")
    for (s, off, n), o in zip(reqs, offs):
        o = int(o)
        fw.fw_classify(sets[s], {f: t[off:off + n] for f, t in dpools[s].items()}, n, ref_i[o:o + n], ref_a[o:o + n])
    torch.cuda.synchronize()
    return torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a


def _queue(env, **cfg):
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q = fw.DeviceQueue(sets, **cfg)
    for p in dpools:
        for t in p.values():
            q.register(t)
    out_i = torch.full((total,), -9, dtype=torch.int32, device="cuda")
    out_a = torch.full((total,), 7, dtype=torch.uint8, device="cuda")
    q.register(out_i)
    q.register(out_a)
    return q, out_i, out_a


def _args(env, k, out_i, out_a):
    _, _, _, _, dpools, reqs, offs, _, _, _ = env
    s, off, n = reqs[k]
    o = int(offs[k])
    return s, {f: t[off:off + n] for f, t in dpools[s].items()}, out_i[o:o + n], out_a[o:o + n]


def test_alone_equals_mix(env):
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q, out_i, out_a = _queue(env)
    for k in range(len(reqs)):  # alone: one request on the device at a time
        st, lat = q.wait(q.submit(*_args(env, k, out_i, out_a)), timeout_us=LIMIT)
        assert st == fw.FW_OK and lat > 0
    torch.cuda.synchronize()
    assert torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a)
    out_i.fill_(-9)
    out_a.fill_(7)
    torch.cuda.synchronize()
    tickets = [q.submit(*_args(env, k, out_i, out_a)) for k in range(len(reqs))]  # the mix
    for t in tickets:
        assert q.wait(t, timeout_us=LIMIT)[0] == fw.FW_OK
    torch.cuda.synchronize()
    assert torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a)
    st = q.stats()
    assert st["completed"] == 2 * len(reqs) and st["fed_requests"] <= 2 * len(reqs)
    assert st["device_status"] == 0
    for k in range(0, len(reqs), 30):  # a sample against the oracle
        s, off, n = reqs[k]
        o = int(offs[k])
        want = oracle.classify(rules[s], {f: v[off:off + n] for f, v in pools[s].items()})
        assert np.array_equal(out_i[o:o + n].cpu().numpy(), want[0])
        assert np.array_equal(out_a[o:o + n].cpu().numpy(), want[1])
    q.destroy()


def test_pinned_host_buffers(env):
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q = fw.DeviceQueue(sets)
    ks = list(range(0, len(reqs), 7))
    bufs = []
    for k in ks:
        s, off, n = reqs[k]
        h = fw.pinned_headers({f: v[off:off + n] for f, v in pools[s].items()})
        oi = torch.full((n,), -3, dtype=torch.int32).pin_memory()
        oa = torch.full((n,), 5, dtype=torch.uint8).pin_memory()
        for t in list(h.values()) + [oi, oa]:
            q.register(t)
        bufs.append((s, h, oi, oa))
    tickets = [q.submit(s, h, oi, oa) for s, h, oi, oa in bufs]
    for t in tickets:
        assert q.wait(t, timeout_us=LIMIT)[0] == fw.FW_OK
    for k, (s, h, oi, oa) in zip(ks, bufs):
        o, n = int(offs[k]), reqs[k][2]
        assert np.array_equal(oi.numpy(), ref_i[o:o + n].cpu().numpy())
        assert np.array_equal(oa.numpy(), ref_a[o:o + n].cpu().numpy())
    q.destroy()


@pytest.mark.parametrize("load_gpps", [0.5, 20.0])
def test_poisson_replay(env, load_gpps):
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q, out_i, out_a = _queue(env, ring=64)  # a small ring: the replay must wait for entries to free up
    rng = np.random.default_rng(3)
    mean_n = total / len(reqs)
    arrivals = np.cumsum(rng.exponential(1e6 * mean_n / (load_gpps * 1e9), size=len(reqs)))
    specs = [(*_args(env, k, out_i, out_a), float(arrivals[k])) for k in range(len(reqs))]
    rc, status, lat = q.replay(specs, timeout_us=LIMIT)
    assert rc == fw.FW_OK and np.all(status == fw.FW_OK)
    assert np.all(lat > 0)
    torch.cuda.synchronize()
    assert torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a)
    assert q.stats()["device_status"] == 0
    q.destroy()


def test_replay_with_refused_requests(env):
    """Requests the queue refuses (a buffer outside the registered ranges, a request over the size
    limit) get their own status; every other request of the replay completes correctly."""
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q, out_i, out_a = _queue(env, max_request_packets=32768)
    loose = torch.empty(70_000, dtype=torch.int32, device="cuda")  # not registered
    specs, bad = [], {}
    for k in range(60):
        s, h, oi, oa = _args(env, k, out_i, out_a)
        if h["src"].shape[0] > 32768:  # checked before the buffers
            bad[k] = fw.FW_ERANGE
        elif k % 15 == 3:
            oi = loose[:oi.shape[0]]
            bad[k] = fw.FW_EINVAL
        specs.append((s, h, oi, oa, 2.0 * k))
    rc, status, lat = q.replay(specs, timeout_us=LIMIT)
    assert rc != fw.FW_OK and fw.FW_EINVAL in bad.values()
    for k in range(60):
        assert status[k] == bad.get(k, fw.FW_OK), (k, status[k])
    torch.cuda.synchronize()
    for k in range(60):
        if k in bad:
            continue
        o, n = int(offs[k]), reqs[k][2]
        assert torch.equal(out_i[o:o + n], ref_i[o:o + n]) and torch.equal(out_a[o:o + n], ref_a[o:o + n]), k
    q.destroy()


def test_idle_exit_and_relaunch(env):
    """The kernel's wait for new requests runs out (idle limit): it exits, and the next submit relaunches it."""
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q, out_i, out_a = _queue(env, idle_us=200)
    for rnd in range(3):
        ks = list(range(rnd, len(reqs), 40))
        tickets = [q.submit(*_args(env, k, out_i, out_a)) for k in ks]
        for t in tickets:
            assert q.wait(t, timeout_us=LIMIT)[0] == fw.FW_OK
        time.sleep(0.02)  # far past the idle limit
        st = q.stats()
        assert st["idle_exits"] >= rnd + 1, st
        assert st["launches"] == rnd + 1, st
    torch.cuda.synchronize()
    for k in range(0, len(reqs), 40):
        o, n = int(offs[k]), reqs[k][2]
        assert torch.equal(out_i[o:o + n], ref_i[o:o + n]) and torch.equal(out_a[o:o + n], ref_a[o:o + n])
    assert q.stats()["device_status"] == 0
    q.destroy()


def test_time_limit_relaunch(env):
    """A launch stops taking requests at its time limit; requests keep being served by the next launch."""
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q, out_i, out_a = _queue(env, life_ms=2, idle_us=1000)
    t_end = time.perf_counter() + 0.05
    k = 0
    while time.perf_counter() < t_end:
        st, _ = q.wait(q.submit(*_args(env, k % len(reqs), out_i, out_a)), timeout_us=LIMIT)
        assert st == fw.FW_OK
        k += 1
    st = q.stats()
    assert st["life_exits"] >= 1 and st["launches"] >= 2, st
    torch.cuda.synchronize()
    m = min(k, len(reqs))
    end = int(offs[m - 1]) + reqs[m - 1][2]
    assert torch.equal(out_i[:end], ref_i[:end]) and torch.equal(out_a[:end], ref_a[:end])
    assert st["device_status"] == 0
    q.destroy()


def test_register_refuses_a_range_across_allocations(env):
    """Device memory has one mapping everywhere, so a range whose two ends lie in two allocations
    passes a check of its ends although the addresses between them need not be mapped: the
    driver's record of the allocation decides. A range inside one allocation is taken."""
    import ctypes
    import os
    torch = env[0]
    if "expandable" in os.environ.get("PYTORCH_CUDA_ALLOC_CONF", ""):
        pytest.skip("the allocator maps its segments into reserved address ranges")
    q = fw.DeviceQueue(env[2])
    torch.cuda.empty_cache()
    size = 96 << 20
    a, b = (torch.empty(size, dtype=torch.uint8, device="cuda") for _ in range(2))
    dev = torch.cuda.current_device()
    segs = [(s["address"], s["total_size"]) for s in torch.cuda.memory_snapshot() if s["device"] == dev]

    def seg_of(t):
        return next((lo, n) for lo, n in segs if lo <= t.data_ptr() < lo + n)

    (lo1, n1), (lo2, n2) = sorted([seg_of(a), seg_of(b)])
    assert lo1 + n1 <= lo2  # two allocations
    reg = fw.lib().fw_dqueue_register_buffer
    assert reg(q.handle, ctypes.c_void_p(lo1), lo2 - lo1 + 1) == fw.FW_EINVAL
    assert reg(q.handle, ctypes.c_void_p(lo1 + n1 - 16), 32) == fw.FW_EINVAL
    assert reg(q.handle, ctypes.c_void_p(lo1), n1) == fw.FW_OK
    assert reg(q.handle, ctypes.c_void_p(a.data_ptr()), size) == fw.FW_OK
    q.destroy()
    del a, b


def test_argument_errors(env):
    torch, rules, sets, pools, dpools, reqs, offs, total, ref_i, ref_a = env
    q, out_i, out_a = _queue(env, ring=64, max_request_packets=4096)
    s, h, oi, oa = _args(env, 1, out_i, out_a)
    n = min(int(h["src"].shape[0]), 4096)
    h = {f: t[:n] for f, t in h.items()}
    loose = torch.empty(n, dtype=torch.int32, device="cuda")  # not registered
    with pytest.raises(fw.FwError) as e:
        q.submit(s, h, loose, oa[:n])
    assert e.value.status == fw.FW_EINVAL
    with pytest.raises(fw.FwError) as e:
        q.submit(4, h, oi[:n], oa[:n])
    assert e.value.status == fw.FW_EINVAL
    big = {f: t[:5000] for f, t in dpools[0].items()}
    with pytest.raises(fw.FwError) as e:
        q.submit(0, big, out_i[:5000], out_a[:5000])
    assert e.value.status == fw.FW_ERANGE
    assert q.wait(12345)[0] == fw.FW_EINVAL
    tickets = [q.submit(s, h, oi[:n], oa[:n]) for _ in range(64)]
    with pytest.raises(fw.FwError) as e:  # the ring is full until a ticket is released
        q.submit(s, h, oi[:n], oa[:n])
    assert e.value.status == fw.FW_EBUSY
    assert q.wait(tickets[0], timeout_us=LIMIT)[0] == fw.FW_OK
    tickets = tickets[1:] + [q.submit(s, h, oi[:n], oa[:n])]
    for t in tickets:
        assert q.wait(t, timeout_us=LIMIT)[0] == fw.FW_OK
    q.destroy()
    # a rule set without a bucket filter (exact protocols beyond the protocol classes) is refused
    r = W.gen_rules(16, 5)
    r["proto_any"] = 0
    r["proto"] = np.arange(100, 116)
    rs = fw.fw_ruleset_create(r)
    assert rs.filter()["words"] == 0
    with pytest.raises(fw.FwError) as e:
        fw.DeviceQueue([rs])
    assert e.value.status == fw.FW_EINVAL
    rs.destroy()
