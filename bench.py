"""Benchmark of first-match packet classification on GB300.

One step = one fw_classify call over one batch of synthetic packet headers
already resident in device memory (the scan at scale: 10,000 rules x
16,777,216 packets, Zipf(1.1) rule choice for in-rule traffic). Prints one
JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Besides the headline step, a single-GPU run measures in the same process:
  - the integer throughput of this GPU (the INT32 roofline denominator);
  - the other workloads of the method, each as a record under "configs": the
    plain 1,000-rule x 100,000-packet case, the rule split (warp, block and
    grid minimum) beside the packet split on the headline batch, two labelled
    variants of the headline traffic (permuted Zipf ranks; no catch-all), 256 batched
    rule sets in one graph-replayed persistent launch, the learned index at
    100,000 rules x 67,108,864 packets, and serving (Poisson arrivals against
    four device-resident rule sets) at three offered loads.
Every record checks its verdicts element by element against the plain scan
and against the CPU oracle on a fixed sample (the oracle runs only in the
CPU-baseline leg, never on the timed path).

--impl reference times the CPU oracle (the sequential first-match loop) on
the host cores instead, each step a bounded sample of the same workload.
Under torchrun every rank classifies its own batch (weak scaling, no
data-path collective); the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1312_4188_gb300 import replica  # noqa: E402
from paper_1312_4188_gb300 import workload as W  # noqa: E402
from paper_1312_4188_gb300.metrics import partition_depth  # noqa: E402

METRIC = "Mpackets/s first-match at 10K rules; rule-checks/s vs INT32 peak; p99 latency"
UNIT = "Mpackets/s"
# Algorithmic work per rule check (the 5-field predicate: two masked address
# compares, two port-range tests, one masked protocol compare and their
# combination), about 10 INT32 operations. The same figure is used for the
# algorithmic count (first-match index + 1 per packet over the whole list) and
# for the checks a partitioned kernel executes; the arithmetic record form
# issues 8 instructions per executed check (see DESIGN).
OPS_PER_CHECK = 10
# Algorithmic bytes per packet: 13 B of header in + 4 B index + 1 B action out.
BYTES_PER_PACKET = 18
FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
# ncu record of the dominant kernel's DRAM traffic; it names the source files the kernel is
# compiled from and their digest, and is used only while those files are unchanged.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
COMPACT_MID_PACKETS = 98_304  # smallest batch the auto mode classifies with the compacting kernel
GEN_WORKERS = max(1, min(16, os.cpu_count() or 1))


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="scan_10k_x_16m_zipf", choices=sorted(W.WORKLOADS))
    ap.add_argument("--mode", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the per-config records (headline step only)")
    ap.add_argument("--only-side", default="", help="comma list of side records to run (default: all)")
    ap.add_argument("--modes", action="store_true", help="also time every record form of the packet split")
    ap.add_argument("--e2e-steps", type=int, default=10)
    return ap.parse_args()


def peaks():
    p = dict(FALLBACK)
    src = "fallback"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            m = json.load(open(path))
            p["hbm_gbs"] = float(m["hbm_gbs"])
            p["sm_max_mhz"] = float(m.get("sm_max_mhz", p["sm_max_mhz"]))
            src = "measured"
        except Exception:
            pass
    return p, src


def sources_sha(files) -> str:
    """Digest of the named source files (paths relative to the repository root), in the given order."""
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str, mode: str):
    """(DRAM bytes per launch, note) from the ncu record, or (None, why) when it does not apply."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, "no ncu record"
    try:
        rec = json.load(open(TRAFFIC_FILE))
        current = sources_sha(rec["sources"])
    except Exception as e:  # pragma: no cover
        return None, f"unreadable ncu record: {e}"
    if rec.get("sources_sha") != current:
        return None, "the kernel's sources changed since the ncu capture"
    if (rec.get("kernel"), rec.get("workload"), rec.get("mode")) != (kernel, workload, mode):
        return None, "ncu record is for another kernel or workload"
    return float(rec["dram_bytes_per_launch"]), f"ncu capture: {rec.get('command', '')}"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while a timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(mhz)}


def workload_config(name: str) -> dict:
    """The workload's identity: the same dict on both arms."""
    w = W.WORKLOADS[name]
    return {"workload": name, "rules": w["n_rules"], "packets": w["n_packets"], "zipf_s": w["zipf_s"],
            "rules_seed": w["rules_seed"], "packets_seed": w["packets_seed"]}


def run_reference(args, ws, rank):
    """The CPU oracle as the reference arm: each step classifies a bounded sample on all host cores."""
    if rank != 0:
        return
    import oracle
    cores = os.cpu_count() or 1
    w = W.WORKLOADS[args.workload]
    rules = W.gen_rules(w["n_rules"], w["rules_seed"])
    m = min(w["n_packets"], 1 << 18)
    pos = W.sample_positions(w["n_packets"], m, seed=99)
    full = W.gen_packets(rules, w["n_packets"], w["packets_seed"], zipf_s=w["zipf_s"], workers=GEN_WORKERS)
    sample = W.take(full, pos)
    del full
    for _ in range(max(args.warmup, 0)):
        oracle.classify(rules, sample, threads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.classify(rules, sample, threads=cores)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = m * args.steps / t / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(args.workload),
        "run": {"parallelism": f"CPU oracle on {cores} host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{m} packets at fixed seeded positions of the {w['n_packets']}-packet batch per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU helpers
def events_ms(fn, stream, reps, warmup=2, flush=None):
    """Per-call CUDA-event times (ms) of fn() on `stream`; flush() (outside the events) before each."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        ev = []
        for _ in range(reps):
            if flush is not None:
                flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((a, b))
    torch.cuda.synchronize()
    return sorted(a.elapsed_time(b) for a, b in ev)


def pct(sorted_ms, q):
    return sorted_ms[min(len(sorted_ms) - 1, int(q * len(sorted_ms)))]


def measure_int32_peak(stream, sms, gpu_id):
    """Integer instructions per second of this GPU (fw_int32_peak_launch), best of 5 launches per mix."""
    import torch

    from paper_1312_4188_gb300 import fw
    blocks, threads = sms * 4, 512
    sink = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    out = {}
    with ClockSampler(gpu_id) as clk:
        for name, kind in fw.INT32_PEAK_KINDS.items():
            iters = 1 << 12
            # size the launch to ~20 ms from a short probe
            t = events_ms(lambda: fw.fw_int32_peak_launch(kind, iters, blocks, threads, sink, stream), stream, 2, 1)
            iters = int(max(256, min(1 << 22, iters * 20.0 / max(t[0], 1e-3))))
            ops = [0]

            def go():
                ops[0] = fw.fw_int32_peak_launch(kind, iters, blocks, threads, sink, stream)
            ts = events_ms(go, stream, 5, 1)
            out[name] = ops[0] / (ts[0] * 1e-3)
    out["clocks"] = clk.summary()
    out["launch"] = f"{blocks} blocks x {threads} threads, 128 independent-chain instructions per loop trip"
    return out


def depth_sum_of(out_idx, n_rules):
    import torch
    d = torch.where(out_idx >= 0, out_idx.to(torch.int64) + 1, torch.full_like(out_idx, n_rules, dtype=torch.int64))
    return int(d.sum().item())


def oracle_leg(rules, sample, g_idx, g_act, threads=None):
    """CPU-baseline leg: the oracle on a sample, timed, and its verdicts compared with the GPU's."""
    import oracle
    cores = threads or (os.cpu_count() or 1)
    t0 = time.perf_counter()
    o_idx, o_act, o_depth = oracle.classify(rules, sample, threads=cores)
    t = time.perf_counter() - t0
    m = len(o_idx)
    return {"value": m / t / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle", "packets": m,
            "mean_depth": o_depth / max(m, 1),
            "parity_on_sample": bool(np.array_equal(np.asarray(g_idx), o_idx) and np.array_equal(np.asarray(g_act), o_act))}


def fractions(n, depth_sum, exec_checks, t_ms, int_peak, alu_peak, hbm_gbs):
    """Roofline fractions of one launch over n packets taking t_ms."""
    t = t_ms * 1e-3
    alg = depth_sum * OPS_PER_CHECK / t
    exe = exec_checks * OPS_PER_CHECK / t
    hbm = BYTES_PER_PACKET * n / t / 1e9
    return {"int32_algorithmic": {"achieved_tops": alg / 1e12, "frac": alg / int_peak,
                                  "frac_of_alu_pipe": alg / alu_peak},
            "int32_executed": {"achieved_tops": exe / 1e12, "frac": exe / int_peak,
                               "frac_of_alu_pipe": exe / alu_peak},
            "hbm": {"achieved_gbs": hbm, "frac": hbm / hbm_gbs}}


def measure_e2e(args, fw, rs, hdr, n, cfg, out_idx, out_act, ws):
    """Whole-job rate through fw_classify_host: pinned host headers in, host verdicts out, copies timed."""
    import torch
    pin = fw.pinned_headers(hdr)
    h_idx = torch.empty(n, dtype=torch.int32).pin_memory()
    h_act = torch.empty(n, dtype=torch.uint8).pin_memory()
    pl = fw.fw_host_pipeline_create(1 << 21, 4)
    e2e = {}
    for sname, strat in (("copy", fw.FW_HOST_COPY), ("zerocopy", fw.FW_HOST_ZEROCOPY)):
        fw.fw_classify_host(pl, rs, pin, h_idx, h_act, n, strategy=strat, config=cfg)
        ts = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            fw.fw_classify_host(pl, rs, pin, h_idx, h_act, n, strategy=strat, config=cfg)
            ts.append(time.perf_counter() - t0)
        ok = bool(torch.equal(h_idx, out_idx.cpu()) and torch.equal(h_act, out_act.cpu()))
        med_ms = replica.max_over_ranks(1e3 * statistics.median(ts), device="cuda")
        e2e[sname] = {"mpackets_s": replica.job_rate(n, 1, ws, med_ms), "same_as_device_path": ok}
    pl.destroy()
    best = max(e2e, key=lambda k: e2e[k]["mpackets_s"])
    return {"value": e2e[best]["mpackets_s"], "unit": UNIT, "h2d_bytes_per_step": 13 * n,
            "d2h_bytes_per_step": 5 * n, "strategy": best, "strategies": e2e,
            "api": "fw_classify_host (pinned host SoA headers in, host verdicts out)",
            "timing": "median host wall time per call, max over ranks"}


def roofline_object(kernel, fr, int_peak, hbm_gbs, hbm_src, peak_note, traffic, traffic_note):
    """The roofline of the dominant kernel. The filter kernel executes a few exact tests per
    packet, so the header stream (18 algorithmic bytes per packet) is its roof; the scan kernels
    execute rule checks, reported as the algorithmic INT32 rate against the measured peak."""
    if kernel == "k_packet_split_filter":
        return {"bound": "hbm", "achieved": fr["hbm"]["achieved_gbs"], "peak": hbm_gbs, "unit": "GB/s",
                "frac": fr["hbm"]["frac"], "traffic": traffic, "traffic_note": traffic_note, "kernel": kernel,
                "peak_source": f"{hbm_src}: MEASURED_PEAKS.json copy bandwidth (burst)",
                "definition": (f"algorithmic bytes ({BYTES_PER_PACKET} per packet: 13 header bytes in, 4 + 1 "
                               "verdict bytes out) x packets / mean launch time (CUDA events on the launching "
                               "stream), against the measured HBM copy bandwidth")}
    return {"bound": "alu", "achieved": fr["int32_algorithmic"]["achieved_tops"], "peak": int_peak / 1e12,
            "unit": "Tops/s", "frac": fr["int32_algorithmic"]["frac"], "traffic": traffic,
            "traffic_note": traffic_note, "kernel": kernel, "peak_source": peak_note,
            "definition": (f"algorithmic rule checks (first-match index + 1 per packet, N if unmatched, over "
                           f"the whole list) x {OPS_PER_CHECK} INT32 ops / mean launch time, against the "
                           "measured INT32 instruction peak; an effective rate: the partitioned scan "
                           "executes only the checks of each packet's class sub-list")}


# ------------------------------------------------------------------ side records (one per workload)
def side_plain(ctx):
    """1,000 rules x 100,000 packets: per-launch latency with L2 flushed before every launch."""
    import torch

    from paper_1312_4188_gb300 import fw
    name = "plain_1k_x_100k"
    w = W.WORKLOADS[name]
    rules = W.gen_rules(w["n_rules"], w["rules_seed"])
    hdr = W.gen_packets(rules, w["n_packets"], w["packets_seed"])
    n = w["n_packets"]
    rs = fw.fw_ruleset_create(rules)
    dh = fw.headers_to_device(hdr)
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    st = ctx["stream"]
    rec = {"config": workload_config(name), "l2": "flushed before every launch (outside the events)"}
    forms = {}
    with ClockSampler(ctx["gpu_id"]) as clk:
        for form, cfg in (("auto", None), ("rule_split_warp", fw.make_config("rule_split_warp")),
                          ("rule_split_block", fw.make_config("rule_split_block"))):
            ts = events_ms(lambda: fw.fw_classify(rs, dh, n, idx, act, stream=st, config=cfg), st, 200, 5,
                           flush=ctx["flush"])
            forms[form] = {"launch_p50_us": 1e3 * pct(ts, 0.5), "launch_p99_us": 1e3 * pct(ts, 0.99),
                           "mpackets_s": n / (1e-3 * statistics.mean(ts)) / 1e6}
            if form == "auto":
                a_idx, a_act = idx.clone(), act.clone()
                t_mean = statistics.mean(ts)
            else:
                forms[form]["same_as_auto"] = bool(torch.equal(idx, a_idx) and torch.equal(act, a_act))
    rec["clocks"] = clk.summary()
    depth = depth_sum_of(a_idx, n_rules=len(rules))
    part = rs.partition()
    scan = partition_depth(rules, a_idx.cpu().numpy(), hdr, part["key_field"], part["key_bits"])
    rec.update({"mpackets_s": forms["auto"]["mpackets_s"], "launch_p50_us": forms["auto"]["launch_p50_us"],
                "launch_p99_us": forms["auto"]["launch_p99_us"], "forms": forms,
                "roofline": fractions(n, depth, scan, t_mean, ctx["int_peak"], ctx["alu_peak"], ctx["hbm_gbs"]),
                "workload_stats": {"first_catch_all": rs.first_catch_all, "mean_depth": depth / n,
                                   "mean_scan_depth": scan / n}})
    if ctx["cpu"]:
        rec["cpu_baseline"] = oracle_leg(rules, hdr, a_idx.cpu().numpy(), a_act.cpu().numpy())
        rec["cpu_baseline"]["sample"] = "the whole 100,000-packet batch"
    rs.destroy()
    return rec


def side_rule_split(ctx):
    """The function-parallel decomposition (rule split + minimum) on the headline batch, beside the packet split."""
    import torch

    from paper_1312_4188_gb300 import fw
    m = ctx["main"]
    rs, dh, n, st = m["rs"], m["dh"], m["n"], ctx["stream"]
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    act = torch.empty(n, dtype=torch.uint8, device="cuda")
    rec = {"config": workload_config(m["workload"]), "packet_split_mpackets_s": m["value_1gpu"]}
    forms = {}
    with ClockSampler(ctx["gpu_id"]) as clk:
        for form in ("rule_split_warp", "rule_split_block", "rule_split_grid"):
            cfg = fw.make_config(form)
            ts = events_ms(lambda: fw.fw_classify(rs, dh, n, idx, act, stream=st, config=cfg), st, 10, 2)
            t = statistics.median(ts)
            forms[form] = {"ms": t, "mpackets_s": n / (1e-3 * t) / 1e6, "launch_p99_ms": pct(ts, 0.99),
                           "same_as_packet_split": bool(torch.equal(idx, m["out_idx"]) and torch.equal(act, m["out_act"])),
                           "rule_checks_per_s": m["depth_sum"] / (1e-3 * t),
                           "roofline": fractions(n, m["depth_sum"], m["depth_sum"], t, ctx["int_peak"],
                                                 ctx["alu_peak"], ctx["hbm_gbs"])}
            if m.get("oracle_sample") is not None:
                pt, o_idx, o_act = m["oracle_sample"]
                forms[form]["parity_on_oracle_sample"] = bool(np.array_equal(idx[pt].cpu().numpy(), o_idx)
                                                              and np.array_equal(act[pt].cpu().numpy(), o_act))
    rec["clocks"] = clk.summary()
    rec["forms"] = forms
    rec["note"] = ("rule_split_* scan the whole list (checks = first-match index + 1 per packet); the packet "
                   "split scans partition sub-lists")
    return rec


def side_variants(ctx):
    """Labelled variants of the headline traffic: Zipf ranks permuted over the rule list, and every
    all-wildcard rule removed (deep scans, a third of the packets default deny). AUTO beside the
    two-packet scan (filter = 2); both checked against the oracle on a 1M-packet sample."""
    import torch

    from paper_1312_4188_gb300 import fw
    st = ctx["stream"]
    out = {}
    for name in ("scan_10k_x_16m_zipf_permuted", "scan_10k_x_16m_no_catch_all"):
        rules, hdr = W.make_workload(name, workers=GEN_WORKERS)
        n = len(hdr["src"])
        dh = fw.headers_to_device(hdr)
        rs = fw.fw_ruleset_create(rules)
        idx = torch.empty(n, dtype=torch.int32, device="cuda")
        act = torch.empty(n, dtype=torch.uint8, device="cuda")
        rec = {"config": workload_config(name), "filter_words": rs.filter()["words"]}
        forms = {}
        ref = None
        with ClockSampler(ctx["gpu_id"]) as clk:
            for form, cfg in (("auto", None), ("scan_x2", fw.make_config("packet_split", filter=2))):
                ts = events_ms(lambda: fw.fw_classify(rs, dh, n, idx, act, stream=st, config=cfg), st, 5, 2)
                t = statistics.median(ts)
                forms[form] = {"ms": t, "mpackets_s": n / (1e-3 * t) / 1e6}
                if ref is None:
                    ref = (idx.clone(), act.clone())
                else:
                    forms[form]["same_as_auto"] = bool(torch.equal(idx, ref[0]) and torch.equal(act, ref[1]))
        rec["clocks"] = clk.summary()
        depth = depth_sum_of(ref[0], len(rules))
        rec.update({"forms": forms, "mpackets_s": forms["auto"]["mpackets_s"],
                    "workload_stats": {"first_catch_all": rs.first_catch_all, "mean_depth": depth / n,
                                       "unmatched_frac": float((ref[0] < 0).float().mean().item())},
                    "roofline": fractions(n, depth, depth, forms["auto"]["ms"], ctx["int_peak"], ctx["alu_peak"],
                                          ctx["hbm_gbs"])})
        rec["roofline"].pop("int32_executed")
        if ctx["cpu"]:
            pos = W.sample_positions(n, 1 << 20, seed=99)
            pt = torch.from_numpy(pos).cuda()
            rec["cpu_baseline"] = oracle_leg(rules, W.take(hdr, pos), ref[0][pt].cpu().numpy(), ref[1][pt].cpu().numpy())
            rec["cpu_baseline"]["sample"] = f"{len(pos)} packets at fixed seeded positions of the {n}-packet batch"
        rs.destroy()
        out[name] = rec
    return {"variants": out, "mpackets_s": {k: v["mpackets_s"] for k, v in out.items()}}


def side_batched(ctx):
    """256 rule sets (64..65,536 rules) with their own batches (1K..1M packets): one graph-replayed launch."""
    import torch

    from paper_1312_4188_gb300 import autotune, fw
    data = W.gen_batched(256, seed=7, workers=GEN_WORKERS)
    st = ctx["stream"]
    jobs = []
    for rules, hdr in data:
        n = len(hdr["src"])
        jobs.append((fw.fw_ruleset_create(rules), fw.headers_to_device(hdr),
                     torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda")))
    total = sum(len(h["src"]) for _, h in data)
    ref = [(torch.empty_like(j[2]), torch.empty_like(j[3])) for j in jobs]

    def sequential():
        for (rs, dh, _, _), (oi, oa) in zip(jobs, ref):
            fw.fw_classify(rs, dh, int(dh["src"].shape[0]), oi, oa, stream=st)

    rec = {"config": {"workload": "batched_256_sets", "sets": 256, "rules_range": [64, 65536],
                      "packets_range": [1024, 1 << 20], "seed": 7, "packets": total,
                      "rules": int(sum(len(r) for r, _ in data))}}
    with ClockSampler(ctx["gpu_id"]) as clk:
        t_seq = statistics.median(events_ms(sequential, st, 5, 2))
        t0 = time.perf_counter()
        with torch.cuda.stream(st):
            classes, _ = autotune.tune_plan_classes(jobs, reps=3)
        tune_s = time.perf_counter() - t0
        plans = {}
        for label, cfg in (("plan_default", None), ("plan_autotuned", fw.make_plan_config(classes))):
            plan = fw.fw_plan_create(jobs, cfg)
            ts = events_ms(lambda: plan.launch(stream=st, graph=True), st, 10, 3)
            t = statistics.median(ts)
            same = all(torch.equal(j[2], r[0]) and torch.equal(j[3], r[1]) for j, r in zip(jobs, ref))
            plans[label] = {"ms": t, "mpackets_s": total / (1e-3 * t) / 1e6, "launch_p99_ms": pct(ts, 0.99),
                            "speedup_vs_sequential": t_seq / t, "same_as_scan": same, "items": plan.items()}
            plan.destroy()
    rec["clocks"] = clk.summary()
    depth = sum(depth_sum_of(oi, rs.size()) for (rs, _, _, _), (oi, _) in zip(jobs, ref))
    best = min(plans, key=lambda k: plans[k]["ms"])
    rec.update({"sequential_fw_classify": {"ms": t_seq, "mpackets_s": total / (1e-3 * t_seq) / 1e6,
                                           "launches": len(jobs)},
                "plans": plans, "autotuned_classes": classes, "tune_s": tune_s, "best": best,
                "mpackets_s": plans[best]["mpackets_s"], "graph": "memset + persistent kernel, replayed",
                "rule_checks_per_s": depth / (1e-3 * plans[best]["ms"]),
                "roofline": fractions(total, depth, depth, plans[best]["ms"], ctx["int_peak"], ctx["alu_peak"],
                                      ctx["hbm_gbs"])})
    rec["roofline"].pop("int32_executed")
    if ctx["cpu"]:
        # oracle on the first 2,048 packets of every set
        g_i, g_a, o_ok, pk, t_all, d_all = [], [], True, 0, 0.0, 0
        import oracle
        cores = os.cpu_count() or 1
        for (rules, hdr), (rs, _, oi, oa) in zip(data, jobs):
            k = min(2048, len(hdr["src"]))
            s = {f: hdr[f][:k] for f in W.HEADER_FIELDS}
            t0 = time.perf_counter()
            o_idx, o_act, o_d = oracle.classify(rules, s, threads=cores)
            t_all += time.perf_counter() - t0
            d_all += o_d
            pk += k
            o_ok &= bool(np.array_equal(oi[:k].cpu().numpy(), o_idx) and np.array_equal(oa[:k].cpu().numpy(), o_act))
        rec["cpu_baseline"] = {"value": pk / t_all / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "the first 2,048 packets of every set", "packets": pk,
                               "mean_depth": d_all / pk, "parity_on_sample": o_ok}
    for j in jobs:
        j[0].destroy()
    return rec


def side_lindex(ctx):
    """Learned index at 100,000 rules x 67,108,864 packets: truncated at the first catch-all and over all rules."""
    import torch

    from paper_1312_4188_gb300 import fw
    name = "lindex_100k_x_64m"
    rules, hdr = W.make_workload(name, workers=GEN_WORKERS)
    n = len(hdr["src"])
    st = ctx["stream"]
    dh = fw.headers_to_device(hdr)
    rs = fw.fw_ruleset_create(rules)
    s_idx = torch.empty(n, dtype=torch.int32, device="cuda")
    s_act = torch.empty(n, dtype=torch.uint8, device="cuda")
    l_idx = torch.empty_like(s_idx)
    l_act = torch.empty_like(s_act)
    rec = {"config": workload_config(name)}
    forms = {}
    with ClockSampler(ctx["gpu_id"]) as clk:
        ts = events_ms(lambda: fw.fw_classify(rs, dh, n, s_idx, s_act, stream=st), st, 5, 2)
        t_scan = statistics.median(ts)
        depth = depth_sum_of(s_idx, len(rules))
        part = rs.partition()
        forms["scan"] = {"ms": t_scan, "mpackets_s": n / (1e-3 * t_scan) / 1e6,
                         "roofline": fractions(n, depth, partition_depth(rules, s_idx.cpu().numpy(), hdr,
                                                                          part["key_field"], part["key_bits"]),
                                               t_scan, ctx["int_peak"], ctx["alu_peak"], ctx["hbm_gbs"])}
        for label, kw in (("lindex_truncated", {}), ("lindex_full", {"truncate": 2})):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            li = fw.fw_lindex_create(rules, **kw)
            torch.cuda.synchronize()
            create_s = time.perf_counter() - t0
            ts = events_ms(lambda: fw.fw_lindex_classify(li, dh, n, l_idx, l_act, stream=st), st, 5, 2)
            t = statistics.median(ts)
            stats = li.stats()
            forms[label] = {"ms": t, "mpackets_s": n / (1e-3 * t) / 1e6, "speedup_vs_scan": t_scan / t,
                            "same_as_scan": bool(torch.equal(l_idx, s_idx) and torch.equal(l_act, s_act)),
                            "create_s": create_s, "rules_indexed": stats.get("rules_indexed"),
                            "intervals": stats.get("intervals"), "bitmap_bytes": stats.get("bitmap_bytes"),
                            "max_error": stats.get("max_error"), "fallbacks": stats.get("fallbacks"),
                            "segments": stats.get("segments"), "classes": stats.get("classes"),
                            "hbm": fractions(n, depth, 0, t, ctx["int_peak"], ctx["alu_peak"], ctx["hbm_gbs"])["hbm"]}
            li.destroy()
    rec["clocks"] = clk.summary()
    best = max(forms, key=lambda k: forms[k]["mpackets_s"])
    rec.update({"forms": forms, "best": best, "mpackets_s": forms[best]["mpackets_s"],
                "workload_stats": {"first_catch_all": rs.first_catch_all, "mean_depth": depth / n}})
    if ctx["cpu"]:
        pos = W.sample_positions(n, 1 << 20, seed=99)
        pt = torch.from_numpy(pos).cuda()
        rec["cpu_baseline"] = oracle_leg(rules, W.take(hdr, pos), s_idx[pt].cpu().numpy(), s_act[pt].cpu().numpy())
        rec["cpu_baseline"]["sample"] = f"{len(pos)} packets at fixed seeded positions of the {n}-packet batch"
        rec["cpu_baseline"]["compared"] = "scan verdicts (every learned-index form equals the scan element by element)"
    rs.destroy()
    del dh
    return rec


def serving_sustained(ctx, sets, dpools, pool_n, n_req=16_000, load=128.0):
    """Saturation over a long replay: n_req requests offered at `load` Gpackets/s to both serving forms,
    beside the same requests as one graph-replayed plan; every result checked against fw_classify."""
    import torch

    from paper_1312_4188_gb300 import fw
    rng = np.random.default_rng(17)
    req_set = rng.integers(0, len(sets), size=n_req)
    req_n = W.log_uniform_int(rng, 64, 65536, n_req)
    req_off = (rng.integers(0, pool_n - 65536, size=n_req) // 4) * 4
    total = int(req_n.sum())
    offs = np.concatenate([[0], np.cumsum(req_n)[:-1]])
    st = ctx["stream"]

    def views(k, oi, oa):
        s, o, m, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
        return s, {f: t[o:o + m] for f, t in dpools[s].items()}, oi[off:off + m], oa[off:off + m]

    ref_i = torch.empty(total, dtype=torch.int32, device="cuda")
    ref_a = torch.empty(total, dtype=torch.uint8, device="cuda")
    for k in range(n_req):
        s, h, oi, oa = views(k, ref_i, ref_a)
        fw.fw_classify(sets[s], h, int(req_n[k]), oi, oa, stream=st)
    out_i = torch.empty_like(ref_i)
    out_a = torch.empty_like(ref_a)
    plan = fw.fw_plan_create([(sets[s], h, oi, oa) for s, h, oi, oa in (views(k, out_i, out_a) for k in range(n_req))])
    t_plan = statistics.median(events_ms(lambda: plan.launch(stream=st, graph=True), st, 5, 2))
    ceiling = total / (1e-3 * t_plan) / 1e6
    rec = {"requests": n_req, "packets": total, "offered_gpackets_s": load,
           "one_plan_ceiling": {"ms": t_plan, "mpackets_s": ceiling,
                                "same_as_scan": bool(torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a))}}
    plan.destroy()
    arrivals = np.cumsum(rng.exponential(1e6 * float(req_n.mean()) / (load * 1e9), size=n_req))
    specs = [(*views(k, out_i, out_a), float(arrivals[k])) for k in range(n_req)]
    with ClockSampler(ctx["gpu_id"]) as clk:
        for form in ("host_scheduler", "device_queue"):
            if form == "host_scheduler":
                q = fw.Server(sets, mode=fw.FW_HOST_ZEROCOPY, slots=8, max_group_requests=4096,
                              max_group_packets=1 << 23, busy_groups=2, arena_bytes=1 << 30)
            else:
                q = fw.DeviceQueue(sets)
            for pool in dpools:
                for t in pool.values():
                    q.register(t)
            q.register(out_i)
            q.register(out_a)
            out_i.fill_(-7)
            torch.cuda.synchronize()
            rc, status, lat = q.replay(specs)
            torch.cuda.synchronize()
            q.destroy()
            rate = total / (float(np.max(arrivals + lat)) * 1e-6) / 1e6
            rec[form] = {"mpackets_s": rate, "frac_of_ceiling": rate / ceiling,
                         "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                         "ok": bool(rc == fw.FW_OK and np.all(status == 0)),
                         "same_as_scan": bool(torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a))}
    rec["clocks"] = clk.summary()
    return rec


def side_serving(ctx):
    """Continuous batching: Poisson arrivals of 64..65,536-packet requests against 1K/10K/50K/100K-rule sets."""
    import torch

    from paper_1312_4188_gb300 import fw
    sizes = [1000, 10_000, 50_000, 100_000]
    rules = [W.gen_rules(k, 40 + i) for i, k in enumerate(sizes)]
    sets = [fw.fw_ruleset_create(r) for r in rules]
    pool_n = 1 << 20
    host_pools = [W.gen_packets(r, pool_n, 50 + i, workers=GEN_WORKERS) for i, r in enumerate(rules)]
    dpools = [fw.headers_to_device(p) for p in host_pools]
    rng = np.random.default_rng(5)
    n_req = 4000
    req_set = rng.integers(0, 4, size=n_req)
    req_n = W.log_uniform_int(rng, 64, 65536, n_req)
    req_off = (rng.integers(0, pool_n - 65536, size=n_req) // 4) * 4
    total = int(req_n.sum())
    offs = np.concatenate([[0], np.cumsum(req_n)[:-1]])
    st = ctx["stream"]
    ref_i = torch.empty(total, dtype=torch.int32, device="cuda")
    ref_a = torch.empty(total, dtype=torch.uint8, device="cuda")
    for k in range(n_req):
        s, o, m, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
        fw.fw_classify(sets[s], {f: t[o:o + m] for f, t in dpools[s].items()}, m, ref_i[off:off + m],
                       ref_a[off:off + m], stream=st)
    torch.cuda.synchronize()
    # ceiling for this request mix: every request in one batched plan (graph-replayed)
    plan_i = torch.empty(total, dtype=torch.int32, device="cuda")
    plan_a = torch.empty(total, dtype=torch.uint8, device="cuda")
    jobs = []
    for k in range(n_req):
        s, o, m, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
        jobs.append((sets[s], {f: t[o:o + m] for f, t in dpools[s].items()}, plan_i[off:off + m], plan_a[off:off + m]))
    plan = fw.fw_plan_create(jobs)
    t_plan = statistics.median(events_ms(lambda: plan.launch(stream=st, graph=True), st, 10, 3))
    plan_same = bool(torch.equal(plan_i, ref_i) and torch.equal(plan_a, ref_a))
    plan.destroy()
    del jobs
    out_i = torch.empty(total, dtype=torch.int32, device="cuda")
    out_a = torch.empty(total, dtype=torch.uint8, device="cuda")
    mean_n = float(req_n.mean())
    rec = {"config": {"workload": "serving_4_sets", "sets_rules": sizes, "requests": n_req,
                      "request_packets": [64, 65536], "packets": total, "arrivals": "Poisson",
                      "buffers": "device-resident request headers and verdicts", "slots": 8,
                      "max_group_requests": 4096, "max_group_packets": 1 << 23, "busy_groups": 2}}
    loads = {}
    load_list = (1.0, 8.0, 128.0)
    arrivals_of = {load: np.cumsum(rng.exponential(1e6 * mean_n / (load * 1e9), size=n_req)) for load in load_list}
    sv = fw.Server(sets, mode=fw.FW_HOST_ZEROCOPY, slots=8, max_group_requests=4096, max_group_packets=1 << 23,
                   busy_groups=2, arena_bytes=1 << 30)
    for pool in dpools:
        for t in pool.values():
            sv.register(t)
    sv.register(out_i)
    sv.register(out_a)
    with ClockSampler(ctx["gpu_id"]) as clk:
        for load in load_list:
            arrivals = arrivals_of[load]
            specs = []
            for k in range(n_req):
                s, o, m, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
                specs.append((s, {f: t[o:o + m] for f, t in dpools[s].items()}, out_i[off:off + m],
                              out_a[off:off + m], float(arrivals[k])))
            out_i.fill_(-7)
            torch.cuda.synchronize()
            st0 = sv.stats()
            rc, status, lat = sv.replay(specs)
            st1 = sv.stats()
            makespan_s = float(np.max(arrivals + lat)) * 1e-6
            groups = st1["groups"] - st0["groups"]
            lag = sv.last_submit_lag_us
            loads[f"{load:g}"] = {
                "offered_gpackets_s": load, "achieved_mpackets_s": total / makespan_s / 1e6,
                "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                "submit_lag_p99_us": float(np.percentile(lag, 99)),
                "host_ns_per_request": {k: (st1[k + "_ns"] - st0[k + "_ns"]) / n_req for k in ("submit", "launch")},
                "ok": bool(rc == fw.FW_OK and np.all(status == 0)),
                "same_as_scan": bool(torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a)),
                "requests_per_group": n_req / max(groups, 1)}
    rec["clocks"] = clk.summary()
    sv.destroy()
    # the same requests and arrivals through the device request queue (one persistent kernel
    # takes requests from a host ring; no launch per group)
    dq_loads = {}
    dq = fw.DeviceQueue(sets)
    for pool in dpools:
        for t in pool.values():
            dq.register(t)
    dq.register(out_i)
    dq.register(out_a)
    with ClockSampler(ctx["gpu_id"]) as clk:
        for load in load_list:
            arrivals = arrivals_of[load]
            specs = []
            for k in range(n_req):
                s, o, m, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
                specs.append((s, {f: t[o:o + m] for f, t in dpools[s].items()}, out_i[off:off + m],
                              out_a[off:off + m], float(arrivals[k])))
            out_i.fill_(-7)
            torch.cuda.synchronize()
            st0 = dq.stats()
            rc, status, lat = dq.replay(specs)
            st1 = dq.stats()
            torch.cuda.synchronize()
            makespan_s = float(np.max(arrivals + lat)) * 1e-6
            lag = dq.last_submit_lag_us
            dq_loads[f"{load:g}"] = {
                "offered_gpackets_s": load, "achieved_mpackets_s": total / makespan_s / 1e6,
                "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                "submit_lag_p99_us": float(np.percentile(lag, 99)),
                "host_ns_per_request": (st1["submit_ns"] - st0["submit_ns"]) / n_req,
                "launches": st1["launches"] - st0["launches"],
                "ok": bool(rc == fw.FW_OK and np.all(status == 0) and st1["device_status"] == 0),
                "same_as_scan": bool(torch.equal(out_i, ref_i) and torch.equal(out_a, ref_a))}
    dq.destroy()
    ceiling = total / (1e-3 * t_plan) / 1e6
    rec["loads"] = loads
    rec["mpackets_s"] = max(v["achieved_mpackets_s"] for v in loads.values())
    rec["saturation_frac_of_ceiling"] = rec["mpackets_s"] / ceiling
    rec["device_queue"] = {"loads": dq_loads, "clocks": clk.summary(),
                           "mpackets_s": max(v["achieved_mpackets_s"] for v in dq_loads.values()),
                           "config": {"ring": 4096, "chunk_packets": 256, "blocks_per_sm": 2, "idle_us": 1000}}
    rec["device_queue"]["saturation_frac_of_ceiling"] = rec["device_queue"]["mpackets_s"] / ceiling
    rec["one_plan_ceiling"] = {"ms": t_plan, "mpackets_s": ceiling, "same_as_scan": plan_same,
                               "what": "the same requests, all present at once, as one graph-replayed batched plan"}
    rec["note"] = ("offered 128 G/s is past saturation: its achieved rate is the saturation throughput; "
                   "`loads`: host scheduler (fw_server, a launch per group); `device_queue`: fw_dqueue (one "
                   "persistent kernel takes the requests from a host ring); `sustained`: the same at 128 G/s "
                   "offered over 16,000 requests, whose rate is less a matter of the burst's start and end")
    rec["sustained"] = serving_sustained(ctx, sets, dpools, pool_n)
    if ctx["cpu"]:
        import oracle
        cores = os.cpu_count() or 1
        ok, pk, t_all = True, 0, 0.0
        ref_i_h, ref_a_h = ref_i.cpu().numpy(), ref_a.cpu().numpy()
        for k in range(64):  # the first 64 requests in full
            s, o, m, off = int(req_set[k]), int(req_off[k]), int(req_n[k]), int(offs[k])
            smp = {f: host_pools[s][f][o:o + m] for f in W.HEADER_FIELDS}
            t0 = time.perf_counter()
            o_idx, o_act, _ = oracle.classify(rules[s], smp, threads=cores)
            t_all += time.perf_counter() - t0
            pk += m
            ok &= bool(np.array_equal(ref_i_h[off:off + m], o_idx) and np.array_equal(ref_a_h[off:off + m], o_act))
        rec["cpu_baseline"] = {"value": pk / t_all / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": "the first 64 requests in full", "packets": pk, "parity_on_sample": ok}
    for r in sets:
        r.destroy()
    return rec


SIDE = {"plain_1k_x_100k": side_plain, "rule_split_10k_x_16m": side_rule_split,
        "variants_10k_x_16m": side_variants, "batched_256_sets": side_batched,
        "lindex_100k_x_64m": side_lindex, "serving_4_sets": side_serving}


def main():
    args = parse()
    ws, rank, local = replica.world()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import torch.distributed as dist

    from paper_1312_4188_gb300 import build, fw

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    w = W.WORKLOADS[args.workload]
    rules = W.gen_rules(w["n_rules"], w["rules_seed"])
    n = w["n_packets"]
    # weak scaling: every rank classifies its own batch of the same size
    hdr = W.gen_packets(rules, n, replica.packets_seed(w["packets_seed"], rank), zipf_s=w["zipf_s"],
                        workers=GEN_WORKERS)
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    pk, peak_src = peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    stream = torch.cuda.Stream()

    t0 = time.perf_counter()
    rs = fw.fw_ruleset_create(rules)
    create_ms = 1e3 * (time.perf_counter() - t0)
    dh = fw.headers_to_device(hdr)
    out_idx = torch.empty(n, dtype=torch.int32, device="cuda")
    out_act = torch.empty(n, dtype=torch.uint8, device="cuda")
    cfg = fw.make_config(args.mode)
    launches_per_step = 3 if args.mode == "rule_split_grid" else 1
    if args.mode.startswith("rule_split"):
        kernel = "k_rule_split"
    elif rs.filter()["words"] > 0:
        kernel = "k_packet_split_filter"
    else:
        kernel = "k_packet_split_compact_x2" if n >= COMPACT_MID_PACKETS else "k_packet_split"
    # inputs that fit in L2 are flushed out of it before every timed launch (a zeroed buffer of
    # twice its size, outside the launch's events); the rate then comes from the launch times
    l2_bytes = int(getattr(props, "L2_cache_size", 0) or (128 << 20))
    scrub = torch.empty(2 * l2_bytes // 4, dtype=torch.int32, device="cuda")
    flush = BYTES_PER_PACKET * n < 2 * l2_bytes

    # the INT32 roofline denominator, measured on this GPU before the timed region
    ip = measure_int32_peak(stream, sms, gpu_id)
    int_peak = max(ip["alu_lop3"], ip["fma_imad"], ip["mixed"])
    alu_peak = ip["alu_lop3"]

    def step(c=cfg):
        fw.fw_classify(rs, dh, n, out_idx, out_act, stream=stream, config=c)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    # The timed region: K steps back to back between two events (inputs larger than L2), or, for
    # inputs that fit in L2, each step between its own events after an L2 flush outside them.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(gpu_id) as clk:
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            g0.record(stream)
            for i in range(args.steps):
                if flush:
                    scrub.zero_()
                    ev[i][0].record(stream)
                step()
                if flush:
                    ev[i][1].record(stream)
            g1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in ev) if flush else g0.elapsed_time(g1)
    total_ms = replica.max_over_ranks(total_ms, device="cuda")
    # per-launch latency (the roofline's launch duration): each launch between its own events,
    # after the timed region
    per = sorted(events_ms(step, stream, max(args.steps, 20), 0, flush=(lambda: scrub.zero_()) if flush else None)) \
        if not flush else sorted(a.elapsed_time(b) for a, b in ev)
    mean_launch_ms = sum(per) / len(per)
    assert rs.check() == fw.FW_OK, "a bounded device wait timed out"

    # workload facts from this step's verdicts (post-processing, not timed)
    N = int(w["n_rules"])
    depth_sum = depth_sum_of(out_idx, N)
    unmatched = float((out_idx < 0).float().mean().item())
    value = replica.job_rate(n, args.steps, ws, total_ms)
    # the default packet split scans the sub-list of the packet's partition class: the checks it
    # executes are the rules of that sub-list up to the match
    partitioned = args.mode in ("auto", "packet_split")
    part = rs.partition()
    scan_sum = (partition_depth(rules, out_idx.cpu().numpy(), hdr, part["key_field"], part["key_bits"])
                if partitioned else depth_sum)
    fr = fractions(n, depth_sum, scan_sum, mean_launch_ms, int_peak, alu_peak, pk["hbm_gbs"])
    traffic, traffic_note = recorded_traffic(kernel, args.workload, args.mode)
    peak_note = (f"measured in this run: fw_int32_peak_launch, best of lop3-only {ip['alu_lop3'] / 1e12:.2f}, "
                 f"imad-only {ip['fma_imad'] / 1e12:.2f} and 1:1 mixed {ip['mixed'] / 1e12:.2f} T instr/s "
                 f"({ip['launch']}; SM clock median {ip['clocks'].get('sm_mhz')} MHz)")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": workload_config(args.workload),
        "run": {"mode": args.mode, "kernel": kernel,
                "l2": (f"L2 flushed before every timed launch ({2 * l2_bytes >> 20} MiB zeroed outside the "
                       f"launch events; {BYTES_PER_PACKET * n / 1e6:.1f} MB of headers+verdicts per step); "
                       "value and ms_per_step from the launch events" if flush else
                       f"inputs larger than L2 ({BYTES_PER_PACKET * n / 1e6:.0f} MB of headers+verdicts per step)"),
                "parallelism": f"replicas x{ws} (packet split across GPUs, no collective)"},
        "roofline": roofline_object(kernel, fr, int_peak, pk["hbm_gbs"], peak_src, peak_note, traffic, traffic_note),
        "roofline_fractions": {
            **fr, "alu_pipe_peak_tops": alu_peak / 1e12, "int32_peak_tops": int_peak / 1e12,
            "hbm_peak_gbs": pk["hbm_gbs"], "hbm_peak_source": f"{peak_src} (MEASURED_PEAKS.json copy bandwidth)",
            "ops_per_check": OPS_PER_CHECK, "bytes_per_packet": BYTES_PER_PACKET,
            "int32_executed_note": ("checks of the packet's class sub-list up to the match (what the partitioned scan "
                                    "kernels execute; the filter kernel tests only its bucket candidates)")},
        "int32_peak_measured": {k: (v / 1e12 if isinstance(v, float) else v) for k, v in ip.items()},
        "rule_checks_per_s": depth_sum / (mean_launch_ms * 1e-3),
        "executed_checks_per_s": scan_sum / (mean_launch_ms * 1e-3),
        "latency_ms": {"launch_p50": pct(per, 0.5), "launch_p99": pct(per, 0.99),
                       "launch_mean": mean_launch_ms, "packets_per_launch": n,
                       "how": ("each launch between its own CUDA events, after the timed region" if not flush else
                               "the timed launches, each between its own CUDA events")},
        "workload_stats": {"first_catch_all": rs.first_catch_all, "mean_depth": depth_sum / n,
                           "mean_scan_depth": scan_sum / n, "unmatched_frac": unmatched,
                           "partition": part},
        "create_ms": create_ms,
        "clocks": clk.summary(),
        "gpu_launches": launches_per_step * args.steps,
    }

    if rank == 0 and args.modes:
        modes = {}
        variants = {"packet_split_filter_512t_3bps": ("packet_split", {"filter": 1, "block_threads": 512,
                                                                       "blocks_per_sm": 3}),
                    "packet_split_filter_384t_4bps": ("packet_split", {"filter": 1, "block_threads": 384,
                                                                       "blocks_per_sm": 4}),
                    "packet_split_filter_pairs": ("packet_split", {"filter": 1, "lane_packets": 2}),
                    "packet_split_filter_pairs_256t_8bps": ("packet_split", {"filter": 1, "lane_packets": 2,
                                                                             "block_threads": 256, "blocks_per_sm": 7}),
                    "packet_split_scan_x2": ("packet_split", {"filter": 2}),
                    "packet_split_one_lane": ("packet_split", {"lane_packets": 1}),
                    "packet_split_dense": ("packet_split", {"block_threads": 768, "blocks_per_sm": 2, "smem_rules": 1024}),
                    "packet_split_whole_list": ("packet_split", {"partition": 2}),
                    "packet_split_lockstep": ("packet_split", {"compact": 2}),
                    "packet_split_lockstep_whole_list": ("packet_split", {"compact": 2, "partition": 2}),
                    "packet_split_lockstep_clamp": ("packet_split", {"compact": 2, "predicate": fw.FW_PRED_CLAMP}),
                    "rule_split_warp_seg2": ("rule_split_warp", {"segment_rules": 2}),
                    "rule_split_warp_seg8": ("rule_split_warp", {"segment_rules": 8}),
                    "rule_split_warp_seg16": ("rule_split_warp", {"segment_rules": 16}),
                    "rule_split_warp_whole_list": ("rule_split_warp", {"partition": 2}),
                    "rule_split_block_whole_list": ("rule_split_block", {"partition": 2}),
                    "rule_split_grid_whole_list": ("rule_split_grid", {"partition": 2})}
        tmp_i, tmp_a = torch.empty_like(out_idx), torch.empty_like(out_act)
        for name, (mname, kw) in variants.items():
            c = fw.make_config(mname, **kw)
            ts = events_ms(lambda: fw.fw_classify(rs, dh, n, tmp_i, tmp_a, stream=stream, config=c), stream, 10, 3)
            modes[name] = {"mpackets_s": n / (statistics.median(ts) * 1e-3) / 1e6,
                           "same": bool(torch.equal(tmp_i, out_idx) and torch.equal(tmp_a, out_act))}
        line["modes_mpackets_s"] = modes

    # end to end through the public API with host buffers (copies inside the timed region), every rank
    if args.e2e_steps > 0:
        line["e2e"] = measure_e2e(args, fw, rs, hdr, n, cfg, out_idx, out_act, ws)

    # CPU baseline leg: the oracle on a bounded sample, and the sample's bit-exact check
    oracle_sample = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        m = min(n, 1 << 20)
        pos = W.sample_positions(n, m, seed=99)
        sample = W.take(hdr, pos)
        pt = torch.from_numpy(pos).cuda()
        g_idx = out_idx[pt].cpu().numpy()
        g_act = out_act[pt].cpu().numpy()
        cb = oracle_leg(rules, sample, g_idx, g_act, threads=cores)
        m1 = min(m, 1 << 17)
        s1 = {f: sample[f][:m1] for f in W.HEADER_FIELDS}
        t0 = time.perf_counter()
        o1 = oracle.classify(rules, s1, threads=1)
        t_one = time.perf_counter() - t0
        cb.update({"sample": f"{m} packets at fixed seeded positions of the {n}-packet batch "
                             f"(mean depth {cb['mean_depth']:.1f})", "single_thread_value": m1 / t_one / 1e6})
        line["cpu_baseline"] = cb
        o_idx, o_act, _ = oracle.classify(rules, sample, threads=cores)
        oracle_sample = (pt, o_idx, o_act)
        del o1

    if ws == 1 and not args.no_side:
        ctx = {"stream": stream, "gpu_id": gpu_id, "int_peak": int_peak, "alu_peak": alu_peak,
               "hbm_gbs": pk["hbm_gbs"], "cpu": not args.no_cpu_baseline, "flush": lambda: scrub.zero_(),
               "main": {"rs": rs, "dh": dh, "n": n, "out_idx": out_idx, "out_act": out_act, "depth_sum": depth_sum,
                        "workload": args.workload, "value_1gpu": value, "oracle_sample": oracle_sample}}
        only = [s for s in args.only_side.split(",") if s]
        configs = {}
        for name, fn in SIDE.items():
            if only and name not in only:
                continue
            t0 = time.perf_counter()
            try:
                configs[name] = fn(ctx)
            except Exception as e:  # a failed record is reported, never silently dropped
                configs[name] = {"error": f"{type(e).__name__}: {e}"}
            configs[name]["wall_s"] = time.perf_counter() - t0
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        line["configs"] = configs

    if rank == 0:
        print(json.dumps(line), flush=True)
    rs.destroy()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
