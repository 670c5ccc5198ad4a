"""bench.py on a GPU: the JSON line keeps its contract and every parity flag it carries is true.

A short run (two timed steps, one record) so that the check stays cheap; the round-end bench runs
the full default.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_contract_and_parity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
                        "--e2e-steps", "2", "--only-side", "plain_1k_x_100k"],
                       capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    rf = d["roofline"]
    assert rf["bound"] in ("hbm", "alu") and rf["peak"] > 0 and rf["achieved"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["parity_on_sample"] is True
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == 13 * d["config"]["packets"]
    assert all(v["same_as_device_path"] for v in e["strategies"].values())
    peaks = d["int32_peak_measured"]
    assert peaks["mixed"] >= max(peaks["alu_lop3"], peaks["fma_imad"]) * 0.95
    rec = d["configs"]["plain_1k_x_100k"]
    assert "error" not in rec, rec.get("error")
    assert rec["cpu_baseline"]["parity_on_sample"] is True
    assert all(f.get("same_as_auto", True) for f in rec["forms"].values())
