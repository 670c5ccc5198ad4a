"""CPU oracle for first-match, default-deny classification.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg may import this package; the product path
(``paper_1312_4188_gb300``) never does. The oracle is a plain sequential C
loop (``fw_oracle.c``) over the rules in list order, following the first-match
and default-deny policy of Sec. I and the wildcard-field rule model of Sec. IV.
It is compiled here with gcc and loaded through ctypes; it shares no code with
the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from paper_1312_4188_gb300.workload import RULE_DTYPE

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(src: str = _SRC, out: str = _LIB_PATH, force: bool = False) -> str:
    """Compile ``src`` into a shared library at ``out`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` loads another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _bind(lib):
    P = ctypes.c_void_p
    lib.oracle_classify.restype = ctypes.c_int64
    lib.oracle_classify.argtypes = [P, ctypes.c_int64, P, P, P, P, P, ctypes.c_int64, P, P, ctypes.c_int]
    lib.oracle_rule_size.restype = ctypes.c_int
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def classify(rules: np.ndarray, headers: dict, threads: int = 1, lib=None):
    """Return ``(idx int32[n], action uint8[n], depth_sum)`` for SoA ``headers``.

    ``rules`` is a structured array with the 24-byte rule layout
    (``paper_1312_4188_gb300.workload.RULE_DTYPE``).
    """
    lib = lib or load()
    if rules.dtype != RULE_DTYPE:  # e.g. numpy's packed result of concatenate
        rules = rules.astype(RULE_DTYPE)
    assert rules.dtype.itemsize == lib.oracle_rule_size() == 24
    rules = np.ascontiguousarray(rules)
    h = {
        "src": np.ascontiguousarray(headers["src"], dtype=np.uint32),
        "dst": np.ascontiguousarray(headers["dst"], dtype=np.uint32),
        "sport": np.ascontiguousarray(headers["sport"], dtype=np.uint16),
        "dport": np.ascontiguousarray(headers["dport"], dtype=np.uint16),
        "proto": np.ascontiguousarray(headers["proto"], dtype=np.uint8),
    }
    n = int(h["src"].shape[0])
    for f in h.values():
        assert f.shape[0] == n
    idx = np.empty(n, dtype=np.int32)
    act = np.empty(n, dtype=np.uint8)
    depth = lib.oracle_classify(_ptr(rules), int(rules.shape[0]), _ptr(h["src"]), _ptr(h["dst"]),
                                _ptr(h["sport"]), _ptr(h["dport"]), _ptr(h["proto"]), n,
                                _ptr(idx), _ptr(act), int(threads))
    return idx, act, int(depth)
