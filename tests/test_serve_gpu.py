"""Serving with continuous batching: every request's result is the same alone and in the mix.

Requests (log-uniform 64..8192 packets) against four device-resident rule
sets are served one at a time (submit, wait) and then all together (a burst,
and an open-loop Poisson replay), in copy and zero-copy modes; each result
must equal, bit for bit, the alone result and fw_classify's, and a sample is
checked against the CPU oracle. Admission is bounded by a small arena.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4188_gb300 import fw, workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_4188_gb300 import build
    build.build()
    sizes = [100, 1000, 3000, 10_000]
    rules = [W.gen_rules(n, 900 + i) for i, n in enumerate(sizes)]
    rules[2] = rules[2][~((rules[2]["src_prefix"] == 0) & (rules[2]["dst_prefix"] == 0))]
    sets = [fw.fw_ruleset_create(r) for r in rules]
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(240):
        s = int(rng.integers(0, 4))
        n = int(W.log_uniform_int(rng, 64, 8192, 1)[0])
        hdr = W.gen_packets(rules[s], n, 10_000 + i, zipf_s=1.1 if s == 3 else None)
        reqs.append((s, hdr))
    # the plain scan is the reference for every request
    want = []
    for s, hdr in reqs:
        i, a = fw.fw_classify(sets[s], fw.headers_to_device(hdr))
        want.append((i.cpu().numpy(), a.cpu().numpy()))
    return torch, rules, sets, reqs, want


def buffers(torch, reqs, zerocopy):
    out = []
    for s, hdr in reqs:
        n = len(hdr["src"])
        h = fw.pinned_headers(hdr)
        oi = torch.full((n,), -5, dtype=torch.int32).pin_memory()
        oa = torch.full((n,), 9, dtype=torch.uint8).pin_memory()
        out.append((s, h, oi, oa))
    return out


@pytest.mark.parametrize("mode", [fw.FW_HOST_COPY, fw.FW_HOST_ZEROCOPY], ids=["copy", "zerocopy"])
def test_alone_equals_mix(env, mode):
    torch, rules, sets, reqs, want = env
    sv = fw.Server(sets, mode=mode, slots=4, max_group_requests=64)
    alone = buffers(torch, reqs, mode)
    for s, h, oi, oa in alone:
        st, lat = sv.wait(sv.submit(s, h, oi, oa))
        assert st == fw.FW_OK and lat > 0
    mix = buffers(torch, reqs, mode)
    tickets = [sv.submit(s, h, oi, oa) for s, h, oi, oa in mix]
    for t in tickets:
        assert sv.wait(t)[0] == fw.FW_OK
    st = sv.stats()
    assert st["completed"] == 2 * len(reqs) and st["failed"] == 0
    assert st["groups"] < 2 * len(reqs) and st["max_group_requests"] > 1, "requests were never batched together"
    for (a, b, w) in zip(alone, mix, want):
        assert np.array_equal(a[2].numpy(), w[0]) and np.array_equal(a[3].numpy(), w[1])
        assert np.array_equal(b[2].numpy(), w[0]) and np.array_equal(b[3].numpy(), w[1])
    for k in range(0, len(reqs), 40):  # a sample against the oracle
        s, hdr = reqs[k]
        o = oracle.classify(rules[s], hdr)
        assert np.array_equal(mix[k][2].numpy(), o[0]) and np.array_equal(mix[k][3].numpy(), o[1])
    sv.destroy()


def test_poisson_replay_and_memory_admission(env):
    torch, rules, sets, reqs, want = env
    # an arena that holds about three of the largest requests: admission must wait for memory
    arena = 3 * 8192 * 18 + 4096
    sv = fw.Server(sets, mode=fw.FW_HOST_COPY, slots=8, max_group_requests=16, arena_bytes=arena)
    bufs = buffers(torch, reqs, fw.FW_HOST_COPY)
    rng = np.random.default_rng(3)
    arrivals = np.cumsum(rng.exponential(20.0, size=len(bufs)))  # mean 20 us apart
    specs = [(s, h, oi, oa, float(t)) for (s, h, oi, oa), t in zip(bufs, arrivals)]
    rc, status, lat = sv.replay(specs)
    assert rc == fw.FW_OK and np.all(status == fw.FW_OK) and np.all(lat > 0)
    st = sv.stats()
    assert 0 < st["arena_high_water"] <= arena
    for b, w in zip(bufs, want):
        assert np.array_equal(b[2].numpy(), w[0]) and np.array_equal(b[3].numpy(), w[1])
    # a request that can never fit the arena is refused up front
    nbig = 30_000  # 18 bytes a packet: more than the arena holds
    big = W.gen_packets(rules[0], nbig, 1)
    h = fw.pinned_headers(big)
    oi = torch.empty(nbig, dtype=torch.int32).pin_memory()
    oa = torch.empty(nbig, dtype=torch.uint8).pin_memory()
    with pytest.raises(fw.FwError) as ei:
        sv.submit(0, h, oi, oa)
    assert ei.value.status == fw.FW_ERANGE
    sv.destroy()


def test_registered_buffers(env):
    torch, rules, sets, reqs, want = env
    sv = fw.Server(sets, mode=fw.FW_HOST_ZEROCOPY)
    bufs = buffers(torch, reqs[:50], fw.FW_HOST_ZEROCOPY)
    for s, h, oi, oa in bufs:
        for t in list(h.values()) + [oi, oa]:
            sv.register(t)
    tickets = [sv.submit(s, h, oi, oa) for s, h, oi, oa in bufs]
    assert all(sv.wait(t)[0] == fw.FW_OK for t in tickets)
    for b, w in zip(bufs, want):
        assert np.array_equal(b[2].numpy(), w[0]) and np.array_equal(b[3].numpy(), w[1])
    L = fw.lib()
    assert L.fw_server_unregister_buffer(sv.handle, ctypes_ptr(bufs[0][2])) == fw.FW_OK
    assert L.fw_server_unregister_buffer(sv.handle, ctypes_ptr(bufs[0][2])) == fw.FW_EINVAL
    pageable = torch.empty(100, dtype=torch.int32)
    with pytest.raises(fw.FwError):
        sv.register(pageable)
    sv.destroy()


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def test_bad_arguments(env):
    torch, rules, sets, reqs, want = env
    sv = fw.Server(sets)
    s, hdr = reqs[0]
    h = fw.pinned_headers(hdr)
    n = len(hdr["src"])
    oi = torch.empty(n, dtype=torch.int32).pin_memory()
    oa = torch.empty(n, dtype=torch.uint8).pin_memory()
    with pytest.raises(fw.FwError):
        sv.submit(7, h, oi, oa)  # no such rule set
    assert sv.wait(123456, 0)[0] == fw.FW_EINVAL  # unknown ticket
    sv.destroy()
    # zero-copy refuses pageable buffers (the device cannot reach them)
    sv = fw.Server(sets, mode=fw.FW_HOST_ZEROCOPY)
    pageable = {f: torch.from_numpy(np.ascontiguousarray(hdr[f]).view(
        {"src": np.int32, "dst": np.int32, "sport": np.int16, "dport": np.int16, "proto": np.uint8}[f]))
        for f in W.HEADER_FIELDS}
    with pytest.raises(fw.FwError):
        sv.submit(s, pageable, torch.empty(n, dtype=torch.int32), torch.empty(n, dtype=torch.uint8))
    sv.destroy()


def test_ticket_ring_reuse_and_limit(env):
    """Requests live in a ring of R entries (here R = 1,024): an unreleased ticket holds its entry, so
    the submit R tickets later is refused with FW_EBUSY until it is released, and the ring wraps
    around several times with every result still exact."""
    torch, rules, sets, reqs, want = env
    sv = fw.Server(sets, mode=fw.FW_HOST_ZEROCOPY, slots=1, max_group_requests=64, max_pending=512)
    s, hdr = 3, W.gen_packets(rules[3], 64 * 4096, 77, zipf_s=1.1)
    dh = fw.headers_to_device(hdr)
    ref_i, ref_a = fw.fw_classify(sets[s], dh)
    for t in dh.values():
        sv.register(t)
    out_i = torch.full((64 * 4096,), -3, dtype=torch.int32, device="cuda")
    out_a = torch.zeros(64 * 4096, dtype=torch.uint8, device="cuda")
    sv.register(out_i)
    sv.register(out_a)

    def sub(k):
        sl = slice(64 * k, 64 * (k + 1))
        return sv.submit(s, {f: t[sl] for f, t in dh.items()}, out_i[sl], out_a[sl], n=64)

    tickets = []
    for k in range(1024):  # 1,024 requests completed and not released: every ring entry is held
        tickets.append(sub(k))
        if len(tickets) % 256 == 0:
            assert sv.drain(10_000_000) == fw.FW_OK
    assert sv.drain(10_000_000) == fw.FW_OK
    with pytest.raises(fw.FwError) as ei:
        sub(1024)
    assert ei.value.status == fw.FW_EBUSY
    assert sv.wait(tickets[0])[0] == fw.FW_OK  # releasing the oldest ticket frees its entry
    tickets = tickets[1:] + [sub(1024)]
    assert all(sv.wait(t)[0] == fw.FW_OK for t in tickets)
    assert sv.wait(tickets[0])[0] == fw.FW_EINVAL  # already released
    # wrap around: windows of 256 submits, each window waited for
    for base in range(1025, 4096, 256):
        ts = [sub(k) for k in range(base, min(base + 256, 4096))]
        assert all(sv.wait(t)[0] == fw.FW_OK for t in ts)
    assert torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a)
    o = oracle.classify(rules[s], {f: v[:4096] for f, v in hdr.items()})
    assert np.array_equal(out_i[:4096].cpu().numpy(), o[0]) and np.array_equal(out_a[:4096].cpu().numpy(), o[1])
    st = sv.stats()
    assert st["completed"] == 4096 and st["failed"] == 0 and st["submit_ns"] > 0 and st["launch_ns"] > 0
    sv.destroy()
