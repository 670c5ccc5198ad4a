"""The C-ABI library loads, exports what include/*.h declares, and rejects bad arguments on the host.

No call here launches GPU work; these run without a GPU.
"""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1312_4188_gb300 import build as B
from paper_1312_4188_gb300 import fw, workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return fw.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(fw_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ("fw_ruleset_create", "fw_ruleset_create_ex", "fw_classify", "fw_classify_ex", "fw_ruleset_destroy",
              "fw_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        getattr(L, n)


def test_library_is_built_for_sm_103a():
    # the object files carry the target named on the command line
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)


def test_rule_layout(L):
    assert L.fw_rule_size() == 24 == W.RULE_DTYPE.itemsize
    assert L.fw_abi_version() >= 1


def test_status_strings(L):
    for s in (0, -1, -2, -3, -4, -5, -6, -7, -99):
        assert isinstance(L.fw_status_string(s), bytes)


def _create(L, rules):
    out = ctypes.c_void_p()
    r = np.ascontiguousarray(rules.astype(W.RULE_DTYPE))
    return L.fw_ruleset_create_ex(r.ctypes.data_as(ctypes.c_void_p), len(r), ctypes.byref(out)), out


@pytest.mark.parametrize("field,value", [
    ("src_prefix", 33), ("dst_prefix", 40), ("action", 2), ("action", 255),
])
def test_create_rejects_bad_rules(L, field, value):
    rules = W.gen_rules(10, 1)
    rules[field][5] = value
    s, out = _create(L, rules)
    assert s == fw.FW_EINVAL and not out.value


def test_create_rejects_inverted_ranges(L):
    rules = W.gen_rules(10, 1)
    rules["sport_lo"][3], rules["sport_hi"][3] = 10, 9
    assert _create(L, rules)[0] == fw.FW_EINVAL
    rules = W.gen_rules(10, 1)
    rules["dport_lo"][0], rules["dport_hi"][0] = 65535, 0
    assert _create(L, rules)[0] == fw.FW_EINVAL


def test_create_rejects_reserved_bytes(L):
    raw = np.zeros(3, dtype=W.RULE_DTYPE)
    raw["sport_hi"] = raw["dport_hi"] = 65535
    b = raw.view(np.uint8).reshape(3, 24).copy()
    b[1, 22] = 7
    out = ctypes.c_void_p()
    s = L.fw_ruleset_create_ex(b.ctypes.data_as(ctypes.c_void_p), 3, ctypes.byref(out))
    assert s == fw.FW_EINVAL


def test_create_rejects_null_and_negative(L):
    out = ctypes.c_void_p()
    assert L.fw_ruleset_create_ex(None, 5, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_ruleset_create_ex(None, -1, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_ruleset_create_ex(None, 0, None) == fw.FW_EINVAL
    assert L.fw_ruleset_create(None, -3) is None
    assert L.fw_last_status() == fw.FW_EINVAL


def test_classify_rejects_bad_arguments(L):
    h = fw.fw_headers()
    assert L.fw_classify(None, ctypes.byref(h), 10, None, None, None) == fw.FW_EINVAL
    fake = ctypes.c_void_p(1)  # never dereferenced: argument checks come first
    assert L.fw_classify(fake, ctypes.byref(h), -1, None, None, None) == fw.FW_EINVAL
    assert L.fw_classify(fake, ctypes.byref(h), 10, None, None, None) == fw.FW_EINVAL
    assert L.fw_classify(fake, None, 10, None, None, None) == fw.FW_EINVAL
    assert L.fw_classify(fake, ctypes.byref(h), 0, None, None, None) == fw.FW_OK  # empty batch: no-op
    hp = fw.fw_headers(*([ctypes.c_void_p(16)] * 5))  # never dereferenced
    cfg = fw.make_config(fw.FW_MODE_PACKET_SPLIT)
    cfg.reserved[0] = 1
    assert L.fw_classify_ex(fake, ctypes.byref(hp), 8, fake, fake, None, ctypes.byref(cfg)) == fw.FW_EINVAL
    cfg = fw.make_config(99)
    assert L.fw_classify_ex(fake, ctypes.byref(hp), 8, fake, fake, None, ctypes.byref(cfg)) == fw.FW_EINVAL


def test_ruleset_filter_rejects_null(L):
    w, b = ctypes.c_int32(), ctypes.c_int64()
    assert L.fw_ruleset_filter(None, ctypes.byref(w), ctypes.byref(b)) == fw.FW_EINVAL
    fake = ctypes.c_void_p(64)  # never dereferenced: argument checks come first
    assert L.fw_ruleset_filter(fake, None, ctypes.byref(b)) == fw.FW_EINVAL
    assert L.fw_ruleset_filter(fake, ctypes.byref(w), None) == fw.FW_EINVAL


def test_filter_field_out_of_range_is_rejected(L):
    fake = ctypes.c_void_p(1)  # never dereferenced: argument checks come first
    hp = fw.fw_headers(*([ctypes.c_void_p(16)] * 5))
    for v in (-1, 3):
        cfg = fw.make_config(fw.FW_MODE_PACKET_SPLIT, filter=v)
        assert L.fw_classify_ex(fake, ctypes.byref(hp), 8, fake, fake, None, ctypes.byref(cfg)) == fw.FW_EINVAL


def test_int32_peak_rejects_bad_arguments(L):
    ops = ctypes.c_int64()
    fake = ctypes.c_void_p(256)  # never dereferenced: argument checks come first
    for kind, iters, blocks, threads, sink, out in ((3, 1, 1, 32, fake, ops), (-1, 1, 1, 32, fake, ops),
                                                    (0, 0, 1, 32, fake, ops), (0, 1 << 25, 1, 32, fake, ops),
                                                    (0, 1, 0, 32, fake, ops), (0, 1, 1, 48, fake, ops),
                                                    (0, 1, 1, 1024, fake, ops), (0, 1, 1, 32, None, ops)):
        assert L.fw_int32_peak_launch(kind, iters, blocks, threads, sink, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_int32_peak_launch(0, 1, 1, 32, fake, None, None) == fw.FW_EINVAL


STRUCTS = ("fw_headers", "fw_config", "fw_lindex_config", "fw_lindex_stats", "fw_job", "fw_plan_config",
           "fw_server_config", "fw_server_stats", "fw_request", "fw_dqueue_config", "fw_dqueue_stats")


def test_binding_structs_match_header(tmp_path):
    """Every ctypes struct of the binding has the header's size and field offsets (gcc's view)."""
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fw.h"', "int main(void) {"]
    want = []
    for name in STRUCTS:
        cls = getattr(fw, name)
        lines.append(f'printf("%zu\\n", sizeof({name}));')
        want.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({name}, {field}));')
            want.append(getattr(cls, field).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want


def _cfg(cls, **kw):
    c = cls()
    for k, v in kw.items():
        if isinstance(v, tuple):
            getattr(c, k)[0] = v[0]
        else:
            setattr(c, k, v)
    return c


def test_plan_rejects_bad_arguments(L):
    out = ctypes.c_void_p()
    assert L.fw_plan_create(None, 0, None, None) == fw.FW_EINVAL
    assert L.fw_plan_create(None, -1, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_plan_create(None, 2, None, ctypes.byref(out)) == fw.FW_EINVAL
    # shared memory: 32 warps x 4,096 queue entries x 16 B is past the 227 KB a block may hold
    for kw in ({"n_classes": 5}, {"packets_per_item": (100,)}, {"packets_per_item": (8192,)},
               {"segment_rules": (6,)}, {"block_threads": 48}, {"block_threads": 2048},
               {"block_threads": 1024, "packets_per_item": (4096,)}):
        cfg = _cfg(fw.fw_plan_config, **kw)
        assert L.fw_plan_create(None, 0, ctypes.byref(cfg), ctypes.byref(out)) == fw.FW_EINVAL, kw
        assert out.value is None
    jobs = (fw.fw_job * 1)()
    jobs[0].n = 10  # no rule set
    assert L.fw_plan_create(jobs, 1, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_plan_launch(None, None) == fw.FW_EINVAL
    assert L.fw_plan_launch_graph(None, None) == fw.FW_EINVAL
    assert L.fw_plan_items(None) == -1
    L.fw_plan_destroy(None)


def test_lindex_rejects_bad_arguments(L):
    out = ctypes.c_void_p()
    r = np.ascontiguousarray(W.gen_rules(10, 1))
    ptr = r.ctypes.data_as(ctypes.c_void_p)
    assert L.fw_lindex_create(ptr, 10, None, None) == fw.FW_EINVAL
    assert L.fw_lindex_create(None, 5, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_lindex_create(ptr, -1, None, ctypes.byref(out)) == fw.FW_EINVAL
    for kw in ({"segments": 3}, {"segments": 1 << 17}, {"truncate": 3}, {"truncate": -1}):
        cfg = _cfg(fw.fw_lindex_config, **kw)
        assert L.fw_lindex_create(ptr, 10, ctypes.byref(cfg), ctypes.byref(out)) == fw.FW_EINVAL, kw
    bad = r.copy()
    bad["sport_lo"][2], bad["sport_hi"][2] = 9, 3
    assert L.fw_lindex_create(bad.ctypes.data_as(ctypes.c_void_p), 10, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert out.value is None
    fake = ctypes.c_void_p(1)  # never dereferenced: argument checks come first
    h = fw.fw_headers()
    assert L.fw_lindex_classify(None, ctypes.byref(h), 10, None, None, None) == fw.FW_EINVAL
    assert L.fw_lindex_classify(fake, ctypes.byref(h), -1, None, None, None) == fw.FW_EINVAL
    assert L.fw_lindex_classify(fake, ctypes.byref(h), 0, None, None, None) == fw.FW_OK
    assert L.fw_lindex_classify(fake, ctypes.byref(h), 10, None, None, None) == fw.FW_EINVAL
    assert L.fw_lindex_get_stats(None, None) == fw.FW_EINVAL
    L.fw_lindex_destroy(None)


def test_server_rejects_bad_arguments(L):
    out = ctypes.c_void_p()
    sets = (ctypes.c_void_p * 2)(1, 1)  # never dereferenced: configuration checks come first
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert L.fw_server_create(sets, 2, None, None) == fw.FW_EINVAL
    assert L.fw_server_create(sets, 0, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_server_create(None, 2, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_server_create(nulls, 2, None, ctypes.byref(out)) == fw.FW_EINVAL
    for kw in ({"mode": 3}, {"slots": 17}, {"slots": -1}, {"max_group_requests": -1}, {"max_pending": -1},
               {"max_group_packets": -1}, {"arena_bytes": 1000}, {"packets_per_item": 100},
               {"packets_per_item": 8192}, {"segment_rules": 6}, {"block_threads": 33}, {"block_threads": 2048},
               {"block_threads": 1024, "packets_per_item": 4096}, {"items_per_warp": -1}, {"busy_groups": -1}):
        cfg = _cfg(fw.fw_server_config, **kw)
        assert L.fw_server_create(sets, 2, ctypes.byref(cfg), ctypes.byref(out)) == fw.FW_EINVAL, kw
        assert out.value is None
    cfg = fw.fw_server_config()
    cfg.reserved[1] = 1  # reserved fields must be zero
    assert L.fw_server_create(sets, 2, ctypes.byref(cfg), ctypes.byref(out)) == fw.FW_EINVAL
    ticket = ctypes.c_uint64()
    h = fw.fw_headers()
    assert L.fw_server_submit(None, 0, ctypes.byref(h), 10, None, None, ctypes.byref(ticket)) == fw.FW_EINVAL
    assert L.fw_server_wait(None, 1, 0, None) == fw.FW_EINVAL
    assert L.fw_server_drain(None, 0) == fw.FW_EINVAL
    assert L.fw_server_get_stats(None, None) == fw.FW_EINVAL
    assert L.fw_server_register_buffer(None, None, 0) == fw.FW_EINVAL
    assert L.fw_server_unregister_buffer(None, None) == fw.FW_EINVAL
    assert L.fw_server_replay(None, None, 0, 0) == fw.FW_EINVAL
    L.fw_server_destroy(None)


def test_dqueue_rejects_bad_arguments(L):
    out = ctypes.c_void_p()
    sets = (ctypes.c_void_p * 2)(1, 1)  # never dereferenced: configuration checks come first
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert L.fw_dqueue_create(sets, 2, None, None) == fw.FW_EINVAL
    assert L.fw_dqueue_create(sets, 0, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_dqueue_create(None, 2, None, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_dqueue_create(nulls, 2, None, ctypes.byref(out)) == fw.FW_EINVAL
    for kw in ({"ring": 63}, {"ring": 100}, {"ring": 1 << 17}, {"ring": -64}, {"chunk_packets": 32},
               {"chunk_packets": 100}, {"chunk_packets": -64}, {"blocks_per_sm": 3}, {"blocks_per_sm": -1},
               {"idle_us": -1}, {"life_ms": -1}, {"poll_ns": -1}, {"max_request_packets": -1},
               {"max_request_packets": 1 << 31}):
        cfg = _cfg(fw.fw_dqueue_config, **kw)
        assert L.fw_dqueue_create(sets, 2, ctypes.byref(cfg), ctypes.byref(out)) == fw.FW_EINVAL, kw
        assert out.value is None
    cfg = fw.fw_dqueue_config()
    cfg.reserved[2] = 1  # reserved fields must be zero
    assert L.fw_dqueue_create(sets, 2, ctypes.byref(cfg), ctypes.byref(out)) == fw.FW_EINVAL
    ticket = ctypes.c_uint64()
    h = fw.fw_headers()
    assert L.fw_dqueue_submit(None, 0, ctypes.byref(h), 10, None, None, ctypes.byref(ticket)) == fw.FW_EINVAL
    assert L.fw_dqueue_wait(None, 1, 0, None) == fw.FW_EINVAL
    assert L.fw_dqueue_get_stats(None, None) == fw.FW_EINVAL
    assert L.fw_dqueue_register_buffer(None, None, 0) == fw.FW_EINVAL
    assert L.fw_dqueue_replay(None, None, 0, 0) == fw.FW_EINVAL
    L.fw_dqueue_destroy(None)


def test_host_pipeline_rejects_bad_arguments(L):
    out = ctypes.c_void_p()
    assert L.fw_host_pipeline_create(0, 0, None) == fw.FW_EINVAL
    assert L.fw_host_pipeline_create(-1, 0, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_host_pipeline_create(0, 9, ctypes.byref(out)) == fw.FW_EINVAL
    assert L.fw_host_pipeline_create(0, -1, ctypes.byref(out)) == fw.FW_EINVAL
    fake = ctypes.c_void_p(1)  # never dereferenced: argument checks come first
    h = fw.fw_headers()
    copy = fw.FW_HOST_COPY
    assert L.fw_classify_host(None, fake, ctypes.byref(h), 10, None, None, copy, None) == fw.FW_EINVAL
    assert L.fw_classify_host(fake, None, ctypes.byref(h), 10, None, None, copy, None) == fw.FW_EINVAL
    assert L.fw_classify_host(fake, fake, ctypes.byref(h), -1, None, None, copy, None) == fw.FW_EINVAL
    assert L.fw_classify_host(fake, fake, ctypes.byref(h), 0, None, None, copy, None) == fw.FW_OK
    assert L.fw_classify_host(fake, fake, ctypes.byref(h), 10, None, None, copy, None) == fw.FW_EINVAL
    L.fw_host_pipeline_destroy(None)


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_compiles_alone_without_warnings(tmp_path, lang):
    """include/fw.h is self-contained and warning-free as strict C11 and C++17."""
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "fw.h"\nint main(void) { return (int)sizeof(fw_rule) - 24; }\n')
    cc, std = ("gcc", "-std=c11") if lang == "c" else ("g++", "-std=c++17")
    subprocess.run([cc, std, "-Wall", "-Wextra", "-Wpedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(tmp_path / "h")], check=True)
    assert subprocess.run([str(tmp_path / "h")]).returncode == 0
