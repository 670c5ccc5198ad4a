"""Measurements of the extended forms beside the plain GPU scan, on the same GPU.

  python -m paper_1312_4188_gb300.measure lindex   # learned index vs scan, 100K rules x 64M packets
  python -m paper_1312_4188_gb300.measure lindex_scan  # the same on 10K rules x 16M packets
  python -m paper_1312_4188_gb300.measure lindex_deep  # ... and on that list without catch-alls
  python -m paper_1312_4188_gb300.measure batched  # 256 rule sets in one persistent launch
  python -m paper_1312_4188_gb300.measure serving  # continuous batching, Poisson arrivals
  python -m paper_1312_4188_gb300.measure variants # the 10K x 16M scan: permuted Zipf ranks, no catch-all

Each prints JSON lines. Every form is compared bit for bit with the plain
scan on the same inputs before its time is reported. Times are CUDA-event
medians on one stream, after warm-up.
"""
from __future__ import annotations

import json
import statistics
import sys
import time

from . import build, fw, workload as W

BYTES_PER_PACKET = 18


def _events_ms(fn, reps=10, warmup=3):
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        ts.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(x.elapsed_time(y) for x, y in ts)


def lindex(args, workload="lindex_100k_x_64m", full=True):
    import torch
    rules, hdr = W.make_workload(workload)
    n = len(hdr["src"])
    dh = fw.headers_to_device(hdr)
    rs = fw.fw_ruleset_create(rules)
    s_idx = torch.empty(n, dtype=torch.int32, device="cuda")
    s_act = torch.empty(n, dtype=torch.uint8, device="cuda")
    t_scan = _events_ms(lambda: fw.fw_classify(rs, dh, n, s_idx, s_act))
    depth = torch.where(s_idx >= 0, s_idx.to(torch.int64) + 1, torch.full_like(s_idx, len(rules), dtype=torch.int64))
    depth_sum = int(depth.sum())
    out = [{"form": "scan", "workload": workload, "ms": t_scan, "mpackets_s": n / t_scan / 1e3,
            "mean_depth": depth_sum / n, "first_catch_all": rs.first_catch_all,
            "hbm_gbs": BYTES_PER_PACKET * n / t_scan / 1e6}]
    for label, kw in (("lindex_truncated", {}), ("lindex_full", {"truncate": 2}))[:2 if full else 1]:
        t0 = time.perf_counter()
        li = fw.fw_lindex_create(rules, **kw)
        torch.cuda.synchronize()
        create_s = time.perf_counter() - t0
        l_idx = torch.empty(n, dtype=torch.int32, device="cuda")
        l_act = torch.empty(n, dtype=torch.uint8, device="cuda")
        t = _events_ms(lambda: fw.fw_lindex_classify(li, dh, n, l_idx, l_act))
        st = li.stats()
        same = bool(torch.equal(l_idx, s_idx) and torch.equal(l_act, s_act))
        out.append({"form": label, "ms": t, "mpackets_s": n / t / 1e3, "speedup_vs_scan": t_scan / t,
                    "same_as_scan": same, "create_s": create_s, "hbm_gbs": BYTES_PER_PACKET * n / t / 1e6, **st})
        li.destroy()
    rs.destroy()
    return out


def batched(args):
    import torch

    from . import autotune
    data = W.gen_batched(256, seed=7)
    jobs = []
    for rules, hdr in data:
        n = len(hdr["src"])
        jobs.append((fw.fw_ruleset_create(rules), fw.headers_to_device(hdr),
                     torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda")))
    total = sum(len(h["src"]) for _, h in data)
    n_rules = sum(len(r) for r, _ in data)
    ref = [(torch.empty_like(j[2]), torch.empty_like(j[3])) for j in jobs]

    def sequential():
        for (rs, dh, _, _), (oi, oa) in zip(jobs, ref):
            fw.fw_classify(rs, dh, int(dh["src"].shape[0]), oi, oa)

    t_seq = _events_ms(sequential, reps=5, warmup=2)
    depth_sum = 0
    for (rs, _, _, _), (oi, _) in zip(jobs, ref):
        depth_sum += int(torch.where(oi >= 0, oi.to(torch.int64) + 1,
                                     torch.full_like(oi, rs.size(), dtype=torch.int64)).sum())
    out = [{"form": "sequential_fw_classify", "workload": "batched_256_sets", "sets": len(jobs), "packets": total,
            "rules": n_rules, "ms": t_seq, "mpackets_s": total / t_seq / 1e3, "rule_checks_per_s": depth_sum / t_seq * 1e3,
            "launches": len(jobs)}]
    t0 = time.perf_counter()
    classes, table = autotune.tune_plan_classes(jobs, reps=3)
    tune_s = time.perf_counter() - t0
    for label, cfg in (("plan_default_graph", None), ("plan_autotuned_graph", fw.make_plan_config(classes))):
        plan = fw.fw_plan_create(jobs, cfg)
        t = _events_ms(lambda: plan.launch(graph=True), reps=10, warmup=3)
        torch.cuda.synchronize()
        same = all(torch.equal(j[2], r[0]) and torch.equal(j[3], r[1]) for j, r in zip(jobs, ref))
        line = {"form": label, "ms": t, "mpackets_s": total / t / 1e3, "rule_checks_per_s": depth_sum / t * 1e3,
                "speedup_vs_sequential": t_seq / t, "same_as_sequential": same, "items": plan.items(),
                "graph_nodes": "memset + persistent kernel"}
        if cfg is not None:
            line["classes"] = classes
            line["tune_s"] = tune_s
            line["tune_table"] = table
        out.append(line)
        plan.destroy()
    for j in jobs:
        j[0].destroy()
    return out


def serving(args):
    """Poisson arrivals of log-uniform 64..65536-packet batches against 4 rule sets (1K/10K/50K/100K rules)."""
    import numpy as np
    import torch
    sizes = [1000, 10_000, 50_000, 100_000]
    rules = [W.gen_rules(n, 40 + i) for i, n in enumerate(sizes)]
    sets = [fw.fw_ruleset_create(r) for r in rules]
    pool_n = 1 << 20
    pools = [fw.pinned_headers(W.gen_packets(r, pool_n, 50 + i)) for i, r in enumerate(rules)]
    dpools = [{f: t.cuda() for f, t in p.items()} for p in pools]
    rng = np.random.default_rng(5)
    n_req = 4000
    req_set = rng.integers(0, 4, size=n_req)
    req_n = W.log_uniform_int(rng, 64, 65536, n_req)
    req_off = (rng.integers(0, pool_n - 65536, size=n_req) // 4) * 4
    total = int(req_n.sum())
    out_i = torch.empty(total, dtype=torch.int32).pin_memory()
    out_a = torch.empty(total, dtype=torch.uint8).pin_memory()
    offs = np.concatenate([[0], np.cumsum(req_n)[:-1]])
    # the plain scan of every request, for the check
    ref_i = torch.empty(total, dtype=torch.int32, device="cuda")
    ref_a = torch.empty(total, dtype=torch.uint8, device="cuda")
    for k in range(n_req):
        s, o, n, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
        fw.fw_classify(sets[s], {f: t[o:o + n] for f, t in dpools[s].items()}, n, ref_i[off:off + n], ref_a[off:off + n])
    torch.cuda.synchronize()
    # ceiling for this request mix: every request in one batched plan, device-resident buffers
    jobs = []
    for k in range(n_req):
        st_, o, n, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
        jobs.append((sets[st_], {f: t[o:o + n] for f, t in dpools[st_].items()}, ref_i[off:off + n].clone(),
                     ref_a[off:off + n].clone()))
    plan = fw.fw_plan_create(jobs)
    t_plan = _events_ms(lambda: plan.launch(graph=True), reps=5, warmup=2)
    plan.destroy()
    depth = 0
    for k in range(n_req):
        st_, off, n = int(req_set[k]), int(offs[k]), int(req_n[k])
        ii = ref_i[off:off + n]
        depth += int(torch.where(ii >= 0, ii.to(torch.int64) + 1, torch.full_like(ii, len(rules[st_]),
                                                                               dtype=torch.int64)).sum())
    ref_i, ref_a = ref_i.cpu(), ref_a.cpu()
    mean_n = float(req_n.mean())
    out = [{"form": "serve_mix_as_one_plan", "requests": n_req, "packets": total, "ms": t_plan,
            "mpackets_s": total / t_plan / 1e3, "mean_depth": depth / total,
            "first_catch_all": [r.first_catch_all for r in sets]}]
    dout_i = torch.empty(total, dtype=torch.int32, device="cuda")
    dout_a = torch.empty(total, dtype=torch.uint8, device="cuda")
    for mode, mname, slots in ((fw.FW_HOST_ZEROCOPY, "device_buffers", 4), (fw.FW_HOST_ZEROCOPY, "device_buffers", 8),
                               (fw.FW_HOST_ZEROCOPY, "zerocopy", 4), (fw.FW_HOST_ZEROCOPY, "zerocopy", 8),
                               (fw.FW_HOST_COPY, "copy", 4)):
        # "device_buffers": request headers and verdicts already in device memory (e.g. placed there
        # by the producer); the server reads and writes them in place
        on_dev = mname == "device_buffers"
        src_pools = dpools if on_dev else pools
        oi_all, oa_all = (dout_i, dout_a) if on_dev else (out_i, out_a)
        sv = fw.Server(sets, mode=mode, slots=slots, max_group_requests=256, arena_bytes=1 << 30)
        if mode == fw.FW_HOST_ZEROCOPY:
            for pool in src_pools:
                for t in pool.values():
                    sv.register(t)
            sv.register(oi_all)
            sv.register(oa_all)
        for load_gpps in (0.1, 0.25, 0.5, 1, 2, 4, 8, 16, 32):
            rate = load_gpps * 1e9 / mean_n  # requests per second
            arrivals = np.cumsum(rng.exponential(1e6 / rate, size=n_req))
            specs = []
            for k in range(n_req):
                s, o, n, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
                specs.append((s, {f: t[o:o + n] for f, t in src_pools[s].items()}, oi_all[off:off + n],
                              oa_all[off:off + n], float(arrivals[k])))
            oi_all.fill_(-7)
            st0 = sv.stats()
            t0 = time.perf_counter()
            rc, status, lat = sv.replay(specs)
            wall = time.perf_counter() - t0
            st1 = sv.stats()
            same = bool(torch.equal(oi_all.cpu(), ref_i) and torch.equal(oa_all.cpu(), ref_a))
            groups = st1["groups"] - st0["groups"]
            # makespan from the server's own completion times (scheduled arrival + latency), so the
            # replay's wait-and-collect loop after the last completion is not counted
            makespan_s = float(np.max(arrivals + lat)) * 1e-6
            out.append({"form": f"serve_{mname}_slots{slots}", "offered_gpackets_s": load_gpps, "requests": n_req,
                        "packets": total, "achieved_mpackets_s": total / makespan_s / 1e6, "makespan_s": makespan_s,
                        "wall_s": wall,
                        "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                        "mean_us": float(lat.mean()), "ok": bool(rc == fw.FW_OK and np.all(status == 0)),
                        "same_as_scan": same, "groups": groups, "requests_per_group": n_req / max(groups, 1),
                        "max_inflight_groups": st1["max_inflight_groups"], "arena_high_water": st1["arena_high_water"]})
        sv.destroy()
    for r in sets:
        r.destroy()
    return out


def variants(args):
    """The 10K-rule x 16M-packet scan under two labelled variants of its traffic: the Zipf rank
    order randomly permuted over the rule list (popular rules no longer at the top), and every
    all-wildcard rule removed (deep scans, many default-deny packets). Each is timed with the
    default configuration and checked bit for bit against the whole-list lockstep scan."""
    import numpy as np
    import torch

    from .metrics import partition_depth
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = []
    for name in ("scan_10k_x_16m_zipf_permuted", "scan_10k_x_16m_no_catch_all"):
        rules, hdr = W.make_workload(name)
        n = len(hdr["src"])
        dh = fw.headers_to_device(hdr)
        rs = fw.fw_ruleset_create(rules)
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        act = torch.empty(n, dtype=torch.uint8, device="cuda")
        t = _events_ms(lambda: fw.fw_classify(rs, dh, n, idx, act), reps=10, warmup=2)
        ref_i = torch.empty_like(idx)
        ref_a = torch.empty_like(act)
        fw.fw_classify(rs, dh, n, ref_i, ref_a, config=fw.make_config("packet_split", compact=2, partition=2))
        torch.cuda.synchronize()
        same = bool(torch.equal(idx, ref_i) and torch.equal(act, ref_a))
        idx_np = idx.cpu().numpy()
        depth = np.where(idx_np >= 0, idx_np.astype(np.int64) + 1, rs.size()).sum()
        part = rs.partition()
        scan = partition_depth(rules, idx_np, hdr, part["key_field"], part["key_bits"])
        checks_s = scan / (t * 1e-3)
        out.append({"form": "scan", "workload": name, "rules": int(len(rules)), "packets": n,
                    "ms": t, "mpackets_s": n / t / 1e3, "mean_depth": float(depth / n),
                    "mean_scan_depth": float(scan / n), "unmatched_frac": float((idx_np < 0).mean()),
                    "first_catch_all": rs.first_catch_all, "scan_checks_per_s": checks_s,
                    "int32_frac": checks_s * 8 / (sms * 128 * 2.07e9), "hbm_gbs": BYTES_PER_PACKET * n / t / 1e6,
                    "same_as_lockstep_whole_list": same})
        rs.destroy()
    return out


def lindex_scan_workload(args):
    """The learned index on the 10K-rule x 16M-packet scan workload (69 reachable rules)."""
    return lindex(args, "scan_10k_x_16m_zipf", full=False)


def lindex_deep(args):
    """The learned index on the 10K-rule x 16M-packet list without catch-alls (deep scans)."""
    return lindex(args, "scan_10k_x_16m_no_catch_all", full=False)


COMMANDS = {"lindex": lindex, "lindex_scan": lindex_scan_workload, "lindex_deep": lindex_deep, "batched": batched,
            "serving": serving, "variants": variants}


def main(argv=None):
    argv = list(sys.argv[1:] if argv is None else argv)
    build.build()
    import torch
    torch.cuda.set_device(0)
    names = argv or list(COMMANDS)
    for name in names:
        for line in COMMANDS[name](argv):
            line["device"] = torch.cuda.get_device_name()
            print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
