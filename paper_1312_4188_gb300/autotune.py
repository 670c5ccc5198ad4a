"""Launch-configuration autotuner for the classification kernels.

The paper studies how the launch configuration (threads per block, rules per
thread) moves packet delay (Sec. IV results, B). Here the knobs are the
fw_config fields: decomposition, predicate encoding, block size, resident
blocks per SM, shared-memory rule prefix, warp batch size and first rule
segment. ``sweep`` times each candidate with CUDA events on one stream and
checks that every candidate returns the same verdicts as the first one
(all forms compute the same function, so any difference is a bug).
Results can be cached per (device, workload) in a JSON file.
"""
from __future__ import annotations

import json
import os
import statistics
import sys

from . import fw

PACKET_SPLIT_CANDIDATES = (
    [dict(mode="packet_split", compact=c, partition=1, lane_packets=1, block_threads=bt, blocks_per_sm=bps,
          smem_rules=sr, packets_per_group=b, segment_rules=s0)
     for c in (1,) for (bt, bps, sr, b) in ((1024, 1, 2048, 256), (1024, 1, 2048, 128), (768, 1, 2048, 256),
                                           (512, 2, 1024, 256), (512, 1, 2048, 512))
     for s0 in (8, 16, 32, 64, 128)]
    + [dict(mode="packet_split", compact=1, partition=1, block_threads=768, blocks_per_sm=2, smem_rules=sr,
            packets_per_group=b, segment_rules=s0)
       for sr in (256, 1024) for b in (128, 256) for s0 in (32, 64)]
    + [dict(mode="packet_split", compact=1, partition=1, lane_packets=2, block_threads=1024, blocks_per_sm=1,
            smem_rules=sr, packets_per_group=b, segment_rules=s0)
       for (b, sr) in ((256, 2048), (384, 512)) for s0 in (32, 64, 128)]
    + [dict(mode="packet_split", compact=2, partition=1)]
    + [dict(mode="packet_split", compact=2, predicate=p, partition=2)
     for p in (fw.FW_PRED_CLAMP, fw.FW_PRED_CMP, fw.FW_PRED_ARITH, fw.FW_PRED_RANGE)]
    + [dict(mode="packet_split", compact=1, predicate=fw.FW_PRED_RANGE, block_threads=1024, blocks_per_sm=1,
            smem_rules=sr, packets_per_group=256, segment_rules=s0) for sr in (1024, 2048) for s0 in (16, 32)]
    + [dict(mode="packet_split", compact=1, predicate=fw.FW_PRED_ARITH, partition=2, block_threads=bt,
            blocks_per_sm=bps, smem_rules=sr, packets_per_group=b, segment_rules=s0)
       for (bt, bps, sr, b) in ((1024, 1, 2048, 256), (1024, 1, 2048, 128), (512, 2, 1024, 256), (768, 1, 2048, 256),
                                (768, 1, 3072, 256), (1024, 1, 1024, 256))
       for s0 in (8, 16, 32)]
    + [dict(mode="packet_split", compact=1, predicate=fw.FW_PRED_CLAMP, block_threads=1024, blocks_per_sm=1,
            smem_rules=3072, packets_per_group=256, segment_rules=16)]
)

# the bucket-filter packet split (rejected, and skipped, for a rule set without a filter)
PACKET_SPLIT_CANDIDATES += [dict(mode="packet_split", filter=1, block_threads=bt, blocks_per_sm=bps)
                            for (bt, bps) in ((512, 3), (512, 2), (256, 6), (384, 4), (128, 12))]

RULE_SPLIT_CANDIDATES = (
    [dict(mode="rule_split_warp", block_threads=bt, blocks_per_sm=bps, segment_rules=sr)
     for bt in (128, 256) for bps in (4, 8) for sr in (2, 4, 8, 16)]
    + [dict(mode="rule_split_block", block_threads=bt) for bt in (128, 256, 512)]
    + [dict(mode="rule_split_grid", rule_slices=s) for s in (1, 2, 4, 8)]
    + [dict(mode="rule_split_warp", partition=2, block_threads=bt, packets_per_group=g)
       for bt in (128, 256) for g in (32, 64, 128)]
    + [dict(mode="rule_split_block", partition=2, block_threads=bt, packets_per_group=g)
       for bt in (128, 256) for g in (128, 256)]
    + [dict(mode="rule_split_grid", partition=2, rule_slices=s, packets_per_group=g) for s in (2, 4, 8) for g in (32, 64)]
)


def config_of(c: dict) -> fw.fw_config:
    kw = dict(c)
    return fw.make_config(kw.pop("mode"), **kw)


def time_config(rs, dh, n, out_idx, out_act, cfg, reps=20, warmup=3, stream=None):
    """Median per-launch milliseconds of fw_classify_ex with ``cfg`` (CUDA events on ``stream``)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fw.fw_classify(rs, dh, n, out_idx, out_act, stream=stream, config=cfg)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fw.fw_classify(rs, dh, n, out_idx, out_act, stream=stream, config=cfg)
        b.record(stream)
        ts.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(x.elapsed_time(y) for x, y in ts)


def sweep(rs, dh, n, candidates, reps=20, warmup=3):
    """Time every candidate; returns [(candidate, ms, same_as_first)] sorted by time."""
    import torch
    dev = dh["src"].device
    ref_idx = ref_act = None
    out = []
    for c in candidates:
        idx = torch.empty(n, dtype=torch.int32, device=dev)
        act = torch.empty(n, dtype=torch.uint8, device=dev)
        try:
            ms = time_config(rs, dh, n, idx, act, config_of(c), reps=reps, warmup=warmup)
        except fw.FwError as e:
            out.append((c, float("inf"), f"rejected: {e}"))
            continue
        if ref_idx is None:
            ref_idx, ref_act, same = idx, act, True
        else:
            same = bool(torch.equal(idx, ref_idx) and torch.equal(act, ref_act))
        out.append((c, ms, same))
    out.sort(key=lambda t: t[1])
    return out


def pick_best(results):
    """The fastest candidate of a ``sweep`` whose verdicts equal the first candidate's (None when
    every candidate was rejected). Every candidate computes the same function, so a candidate
    whose verdicts differ is a bug: that raises instead of being ranked."""
    differ = [c for c, _, same in results if same is False]
    if differ:
        raise RuntimeError(f"{len(differ)} candidate(s) returned different verdicts, e.g. {differ[0]}")
    ok = [(ms, i) for i, (_, ms, same) in enumerate(results) if same is True and ms != float("inf")]
    return results[min(ok)[1]][0] if ok else None


PLAN_CANDIDATES = [(ppi, seg) for ppi in (128, 256) for seg in (16, 64, 256, 1024)]
CLASS_LIMITS = (256, 4096)  # reachable rules: <= 256, <= 4096, larger


def time_plan(plan, reps=10, warmup=3):
    """Median milliseconds of one graph launch of ``plan`` (CUDA events)."""
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.launch(s)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        plan.launch(s)
        b.record(s)
        ts.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(x.elapsed_time(y) for x, y in ts)


def tune_plan_classes(jobs, limits=CLASS_LIMITS, candidates=PLAN_CANDIDATES, reps=10):
    """Pick (packets_per_item, segment_rules) per rule-set size class by timing plans of each class alone.

    ``jobs``: list of (Ruleset, device headers, out_idx, out_act). Returns
    (classes for fw.make_plan_config, per-class timing table).
    """
    classes, table = [], []
    bounds = list(limits) + [1 << 30]
    lo = -1
    for c, hi in enumerate(bounds):
        sub = [j for j in jobs if lo < _reach(j[0]) <= hi]
        lo = hi
        if not sub:
            classes.append((hi, 256, 64))
            continue
        best = None
        for ppi, seg in candidates:
            plan = fw.fw_plan_create(sub, fw.make_plan_config([(hi, ppi, seg)]))
            ms = time_plan(plan, reps=reps)
            plan.destroy()
            table.append({"class": c, "max_rules": hi, "jobs": len(sub), "packets_per_item": ppi,
                          "segment_rules": seg, "ms": ms})
            if best is None or ms < best[0]:
                best = (ms, ppi, seg)
        classes.append((hi, best[1], best[2]))
    return classes, table


def _reach(rs) -> int:
    """Rules a scan of ``rs`` can reach (first catch-all + 1, else all)."""
    ca = rs.first_catch_all
    return ca + 1 if ca >= 0 else rs.size()


def cache_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def load_cache():
    p = cache_path()
    return json.load(open(p)) if os.path.exists(p) else {}


def store(key: str, best: dict):
    d = load_cache()
    d[key] = best
    os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
    json.dump(d, open(cache_path(), "w"), indent=1, sort_keys=True)


def main(argv=None):
    import argparse

    import torch

    from . import build, workload as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="scan_10k_x_16m_zipf", choices=sorted(W.WORKLOADS))
    ap.add_argument("--set", default="packet_split", choices=["packet_split", "rule_split", "all"])
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args(argv)
    build.build()
    rules, hdr = W.make_workload(a.workload)
    n = len(hdr["src"])
    rs = fw.fw_ruleset_create(rules)
    dh = fw.headers_to_device(hdr)
    cands = {"packet_split": PACKET_SPLIT_CANDIDATES, "rule_split": RULE_SPLIT_CANDIDATES,
             "all": PACKET_SPLIT_CANDIDATES + RULE_SPLIT_CANDIDATES}[a.set]
    res = sweep(rs, dh, n, cands, reps=a.reps)
    name = torch.cuda.get_device_name()
    for c, ms, same in res:
        print(json.dumps({"workload": a.workload, "device": name, "config": c, "ms": ms,
                          "mpackets_s": n / (ms * 1e-3) / 1e6 if ms != float("inf") else 0.0, "same": same}))
    try:
        best = pick_best(res)
    except RuntimeError as e:
        print(json.dumps({"workload": a.workload, "device": name, "error": str(e)}))
        rs.destroy()
        return 1
    if best is not None:
        store(f"{name}|{a.workload}|{a.set}", best)
    rs.destroy()
    return 0


if __name__ == "__main__":
    sys.exit(main())
