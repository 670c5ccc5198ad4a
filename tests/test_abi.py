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


STRUCTS = ("fw_headers", "fw_config", "fw_lindex_config", "fw_lindex_stats", "fw_job", "fw_plan_config",
           "fw_server_config", "fw_server_stats", "fw_request")


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
