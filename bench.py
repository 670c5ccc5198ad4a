"""Benchmark of first-match packet classification on GB300.

One step = one fw_classify call over one batch of synthetic packet headers
already resident in device memory (the scan at scale: 10,000 rules x
16,777,216 packets, Zipf(1.1) rule choice for in-rule traffic). Prints one
JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1312_4188_gb300 import workload as W  # noqa: E402
from paper_1312_4188_gb300.metrics import partition_depth  # noqa: E402,F401

METRIC = "Mpackets/s first-match at 10K rules; rule-checks/s vs INT32 peak; p99 latency"
UNIT = "Mpackets/s"
# Algorithmic work per rule check: 3 masked-equality tests (src, dst, proto:
# one 3-input logic op each), 2 subtractions and 2 unsigned compares for the
# port ranges, 1 combine = 8 INT32 operations.
OPS_PER_CHECK = 8
# Algorithmic bytes per packet: 13 B of header in + 4 B index + 1 B action out.
BYTES_PER_PACKET = 18
INT32_LANES_PER_SM_CLK = 128  # 4 schedulers x 32 lanes, one warp instruction per clock each
FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "sms": 152}
KERNEL_SOURCES = ["paper_1312_4188_gb300/csrc/fw_scan.cu", "paper_1312_4188_gb300/csrc/fw_scan.cuh",
                  "paper_1312_4188_gb300/csrc/fw_internal.cuh"]
# the kernel the default (auto) configuration launches for this workload: the compacting scan of
# the partitioned lists (protocol class and address key) with two packets per lane
KERNEL_NAME = "k_packet_split_compact_x2"
TRAFFIC_RECORD = "profiles/k_packet_split_compact_x2_scan_10k_x_16m.md"
TRAFFIC_WORKLOAD = "scan_10k_x_16m_zipf"  # the workload and mode (auto) the record was captured on
COMPACT_MID_PACKETS = 98_304  # smallest batch the auto mode classifies with the compacting kernel


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="scan_10k_x_16m_zipf", choices=sorted(W.WORKLOADS))
    ap.add_argument("--mode", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--modes", action="store_true", help="also time every decomposition / record form (side lines)")
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


def sources_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes from the committed ncu summary, if it is for the current kernel source."""
    path = os.path.join(ROOT, TRAFFIC_RECORD)
    if not os.path.exists(path):
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_sha:\s*([0-9a-f]+)", open(path).read())
    if not m or m.group(2) != sources_sha():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

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


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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
    full = W.gen_packets(rules, w["n_packets"], w["packets_seed"], zipf_s=w["zipf_s"])
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
        "config": {"workload": args.workload, "rules": w["n_rules"], "packets": w["n_packets"],
                   "zipf_s": w["zipf_s"], "rules_seed": w["rules_seed"], "packets_seed": w["packets_seed"],
                   "parallelism": f"CPU oracle on {cores} host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{m} packets at fixed seeded positions of the {w['n_packets']}-packet batch per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import torch.distributed as dist

    from paper_1312_4188_gb300 import build, fw

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    pk, peak_src = peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    alu_peak = sms * INT32_LANES_PER_SM_CLK * pk["sm_max_mhz"] * 1e6  # int ops / s

    w = W.WORKLOADS[args.workload]
    rules = W.gen_rules(w["n_rules"], w["rules_seed"])
    n = w["n_packets"]
    # weak scaling: every rank classifies its own batch of the same size
    hdr = W.gen_packets(rules, n, w["packets_seed"] + 1000 * rank, zipf_s=w["zipf_s"])
    t0 = time.perf_counter()
    rs = fw.fw_ruleset_create(rules)
    create_ms = 1e3 * (time.perf_counter() - t0)
    dh = fw.headers_to_device(hdr)
    out_idx = torch.empty(n, dtype=torch.int32, device="cuda")
    out_act = torch.empty(n, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    cfg = fw.make_config(args.mode)
    launches_per_step = 3 if args.mode == "rule_split_grid" else 1
    if args.mode.startswith("rule_split"):
        kernel = "k_rule_split"
    else:
        kernel = KERNEL_NAME if n >= COMPACT_MID_PACKETS else "k_packet_split"
    # inputs that fit in L2 are flushed out of it before every timed launch (a zeroed buffer of
    # twice its size, outside the launch's events); the rate then comes from the launch times
    l2_bytes = int(getattr(props, "L2_cache_size", 0) or (128 << 20))
    flush = BYTES_PER_PACKET * n < 2 * l2_bytes
    scrub = torch.empty(2 * l2_bytes // 4, dtype=torch.int32, device="cuda") if flush else None

    def step(c=cfg):
        fw.fw_classify(rs, dh, n, out_idx, out_act, stream=stream, config=c)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
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
                ev[i][1].record(stream)
            g1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in ev) if flush else g0.elapsed_time(g1)
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    per = sorted(a.elapsed_time(b) for a, b in ev)
    mean_launch_ms = sum(per) / len(per)
    assert rs.check() == fw.FW_OK, "a bounded device wait timed out"

    # workload facts from this step's verdicts (post-processing, not timed)
    N = int(w["n_rules"])
    depth = torch.where(out_idx >= 0, out_idx.to(torch.int64) + 1, torch.full_like(out_idx, N, dtype=torch.int64))
    depth_sum = int(depth.sum().item())
    unmatched = float((out_idx < 0).float().mean().item())

    value = ws * n * args.steps / (total_ms * 1e-3) / 1e6
    checks_per_s = depth_sum / (mean_launch_ms * 1e-3)
    # the default packet split scans the sub-list of the packet's partition class: its algorithmic
    # work is the rules of that sub-list up to the match, which is what the roofline counts
    partitioned = args.mode in ("auto", "packet_split")
    part = rs.partition()
    scan_sum = (partition_depth(rules, out_idx.cpu().numpy(), hdr, part["key_field"], part["key_bits"])
                if partitioned else depth_sum)
    scan_checks_per_s = scan_sum / (mean_launch_ms * 1e-3)
    ops_per_s = scan_checks_per_s * OPS_PER_CHECK
    hbm_gbs = BYTES_PER_PACKET * n / (mean_launch_ms * 1e-3) / 1e9
    traffic = recorded_traffic() if (args.workload, args.mode) == (TRAFFIC_WORKLOAD, "auto") else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "rules": N, "packets": n, "mode": args.mode,
                   "zipf_s": w["zipf_s"], "rules_seed": w["rules_seed"], "packets_seed": w["packets_seed"],
                   "l2": (f"L2 flushed before every timed launch ({2 * l2_bytes >> 20} MiB zeroed outside the "
                          f"launch events; {BYTES_PER_PACKET * n / 1e6:.1f} MB of headers+verdicts per step); "
                          "value and ms_per_step from the launch events" if flush else
                          f"inputs larger than L2 ({BYTES_PER_PACKET * n / 1e6:.0f} MB of headers+verdicts per step)"),
                   "parallelism": f"replicas x{ws} (packet split across GPUs, no collective)"},
        "roofline": {"bound": "alu", "achieved": ops_per_s / 1e12, "peak": alu_peak / 1e12, "unit": "Tops/s",
                     "frac": ops_per_s / alu_peak, "traffic": traffic,
                     "peak_source": f"derived: {sms} SMs x {INT32_LANES_PER_SM_CLK} INT32 lanes/clk x "
                                    f"{pk['sm_max_mhz']:.0f} MHz ({peak_src} max clock)",
                     "ops_per_check": OPS_PER_CHECK, "kernel": kernel},
        "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": pk["hbm_gbs"], "frac": hbm_gbs / pk["hbm_gbs"],
                "peak_source": peak_src, "bytes_per_packet": BYTES_PER_PACKET},
        "rule_checks_per_s": checks_per_s,
        "scan_checks_per_s": scan_checks_per_s,
        "rule_checks_note": ("rule_checks_per_s counts first-match index + 1 (N if unmatched) per packet over "
                             "the whole list; scan_checks_per_s counts the rules of the sub-list of the packet's "
                             "partition class that the partitioned scan examines (the roofline numerator)"),
        "latency_ms": {"launch_p50": per[len(per) // 2], "launch_p99": per[min(len(per) - 1, int(0.99 * len(per)))],
                       "launch_mean": mean_launch_ms, "packets_per_launch": n},
        "workload_stats": {"first_catch_all": rs.first_catch_all, "mean_depth": depth_sum / n,
                           "mean_scan_depth": scan_sum / n, "unmatched_frac": unmatched},
        "create_ms": create_ms,
        "clocks": clk.summary(),
        "gpu_launches": launches_per_step * args.steps,
    }

    if rank == 0 and args.modes:
        modes = {}
        variants = {"packet_split": ("packet_split", {}),
                    "packet_split_one_lane": ("packet_split", {"lane_packets": 1}),
                    "packet_split_dense": ("packet_split", {"block_threads": 768, "blocks_per_sm": 2, "smem_rules": 1024}),
                    "packet_split_whole_list": ("packet_split", {"partition": 2}),
                    "packet_split_lockstep": ("packet_split", {"compact": 2}),
                    "packet_split_lockstep_whole_list": ("packet_split", {"compact": 2, "partition": 2}),
                    "packet_split_lockstep_clamp": ("packet_split", {"compact": 2, "predicate": fw.FW_PRED_CLAMP}),
                    "rule_split_warp": ("rule_split_warp", {}),
                    "rule_split_block": ("rule_split_block", {}),
                    "rule_split_grid": ("rule_split_grid", {})}
        for name, (mname, kw) in variants.items():
            c = fw.make_config(mname, **kw)
            with torch.cuda.stream(stream):
                for _ in range(3):
                    step(c)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 20
            a.record(stream)
            for _ in range(reps):
                step(c)
            b.record(stream)
            torch.cuda.synchronize()
            modes[name] = n * reps / (a.elapsed_time(b) * 1e-3) / 1e6
        line["modes_mpackets_s"] = modes
        step()  # leave the default mode's verdicts in out_idx/out_act
        torch.cuda.synchronize()

    # end to end through the public API with host buffers (copies inside the timed region)
    if rank == 0 or ws > 1:
        pin = {f: torch.from_numpy(np.ascontiguousarray(hdr[f]).view(
            {"src": np.int32, "dst": np.int32, "sport": np.int16, "dport": np.int16, "proto": np.uint8}[f])
        ).pin_memory() for f in W.HEADER_FIELDS}
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
            e2e[sname] = {"mpackets_s": n / statistics.median(ts) / 1e6, "same_as_device_path": ok}
        pl.destroy()
        best = max(e2e, key=lambda k: e2e[k]["mpackets_s"])
        line["e2e"] = {"value": ws * e2e[best]["mpackets_s"], "unit": UNIT, "h2d_bytes_per_step": 13 * n,
                       "d2h_bytes_per_step": 5 * n, "strategy": best, "strategies": e2e,
                       "api": "fw_classify_host (pinned host SoA headers in, host verdicts out)"}

    # CPU baseline leg: the oracle on a bounded sample, and the sample's bit-exact check
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        m = min(n, 1 << 20)
        pos = W.sample_positions(n, m, seed=99)
        sample = W.take(hdr, pos)
        t0 = time.perf_counter()
        o_idx, o_act, o_depth = oracle.classify(rules, sample, threads=cores)
        t_all = time.perf_counter() - t0
        m1 = min(m, 1 << 17)
        s1 = {f: sample[f][:m1] for f in W.HEADER_FIELDS}
        t0 = time.perf_counter()
        oracle.classify(rules, s1, threads=1)
        t_one = time.perf_counter() - t0
        pt = torch.from_numpy(pos).cuda()
        g_idx = out_idx[pt].cpu().numpy()
        g_act = out_act[pt].cpu().numpy()
        line["cpu_baseline"] = {
            "value": m / t_all / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} packets at fixed seeded positions of the {n}-packet batch (mean depth {o_depth / m:.1f})",
            "single_thread_value": m1 / t_one / 1e6,
            "parity_on_sample": bool(np.array_equal(g_idx, o_idx) and np.array_equal(g_act, o_act)),
        }

    if rank == 0:
        print(json.dumps(line), flush=True)
    rs.destroy()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
