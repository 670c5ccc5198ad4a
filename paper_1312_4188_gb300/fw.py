"""Thin Python binding of the C ABI in ``include/fw.h`` (ctypes).

Argument marshalling only: every step of classification runs in the CUDA
library ``libfw.so``. PyTorch supplies device memory and streams. If the
library is missing the calls raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .workload import HEADER_FIELDS, RULE_DTYPE

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfw.so")

FW_OK = 0
FW_EINVAL = -1
FW_ENOMEM = -2
FW_ECUDA = -3
FW_EALIGN = -4
FW_ETIMEOUT = -5
FW_EBUSY = -6
FW_ERANGE = -7
FW_NOALLOC_MAX_PACKETS = 1 << 20

FW_DROP = 0
FW_ACCEPT = 1

FW_MODE_AUTO = 0
FW_MODE_PACKET_SPLIT = 1
FW_MODE_RULE_SPLIT_WARP = 2
FW_MODE_RULE_SPLIT_BLOCK = 3
FW_MODE_RULE_SPLIT_GRID = 4
MODES = {
    "auto": FW_MODE_AUTO,
    "packet_split": FW_MODE_PACKET_SPLIT,
    "rule_split_warp": FW_MODE_RULE_SPLIT_WARP,
    "rule_split_block": FW_MODE_RULE_SPLIT_BLOCK,
    "rule_split_grid": FW_MODE_RULE_SPLIT_GRID,
}
FW_PRED_CLAMP = 1
FW_PRED_CMP = 2
FW_PRED_ARITH = 3
FW_PRED_RANGE = 4
FW_HOST_COPY = 1
FW_HOST_ZEROCOPY = 2


class FwError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})" if what else status_string(status))


class fw_headers(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("sport", ctypes.c_void_p),
                ("dport", ctypes.c_void_p), ("proto", ctypes.c_void_p)]


class fw_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("smem_rules", ctypes.c_int32), ("packets_per_group", ctypes.c_int32),
                ("rule_slices", ctypes.c_int32), ("compact", ctypes.c_int32), ("predicate", ctypes.c_int32),
                ("segment_rules", ctypes.c_int32), ("partition", ctypes.c_int32), ("lane_packets", ctypes.c_int32),
                ("filter", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


def make_config(mode=FW_MODE_AUTO, **kw) -> fw_config:
    if isinstance(mode, str):
        mode = MODES[mode]
    c = fw_config()
    c.mode = mode
    for k, v in kw.items():
        setattr(c, k, int(v))
    return c


class fw_lindex_config(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int32), ("truncate", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class fw_lindex_stats(ctypes.Structure):
    _fields_ = [("rules", ctypes.c_int64), ("rules_indexed", ctypes.c_int64), ("words_per_row", ctypes.c_int64),
                ("segments", ctypes.c_int64), ("intervals", ctypes.c_int64 * 5), ("max_error", ctypes.c_int32 * 5),
                ("bitmap_bytes", ctypes.c_int64), ("fallbacks", ctypes.c_int64), ("classes", ctypes.c_int64),
                ("key_field", ctypes.c_int32), ("key_bits", ctypes.c_int32)]


class fw_job(ctypes.Structure):
    _fields_ = [("rs", ctypes.c_void_p), ("hdrs", fw_headers), ("n", ctypes.c_int64),
                ("out_rule_idx", ctypes.c_void_p), ("out_action", ctypes.c_void_p)]


class fw_plan_config(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("class_max_rules", ctypes.c_int32 * 4), ("packets_per_item", ctypes.c_int32 * 4),
                ("segment_rules", ctypes.c_int32 * 4), ("reserved", ctypes.c_int32 * 5)]


class fw_server_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("slots", ctypes.c_int32), ("max_group_requests", ctypes.c_int32),
                ("max_pending", ctypes.c_int32), ("max_group_packets", ctypes.c_int64),
                ("arena_bytes", ctypes.c_int64), ("packets_per_item", ctypes.c_int32),
                ("segment_rules", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("items_per_warp", ctypes.c_int32), ("busy_groups", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class fw_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "packets", "groups",
                                               "max_group_requests", "max_inflight_groups", "arena_high_water",
                                               "pending", "submit_ns", "launch_ns", "complete_ns")]


class fw_request(ctypes.Structure):
    _fields_ = [("set", ctypes.c_int32), ("status", ctypes.c_int32), ("hdrs", fw_headers), ("n", ctypes.c_int64),
                ("out_rule_idx", ctypes.c_void_p), ("out_action", ctypes.c_void_p), ("arrival_us", ctypes.c_double),
                ("latency_us", ctypes.c_double), ("submit_lag_us", ctypes.c_double)]


class fw_dqueue_config(ctypes.Structure):
    _fields_ = [("ring", ctypes.c_int32), ("chunk_packets", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("idle_us", ctypes.c_int32), ("max_request_packets", ctypes.c_int64), ("life_ms", ctypes.c_int32),
                ("poll_ns", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class fw_dqueue_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "packets", "launches", "idle_exits",
                                               "life_exits", "fed_requests", "fed_items", "device_status",
                                               "submit_ns", "feed_ns", "feeds", "feed_read_ns", "work_ns",
                                               "items_done")]


_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I64 = ctypes.c_int64

SIGNATURES = {
    "fw_ruleset_create_ex": (ctypes.c_int, [P, I64, ctypes.POINTER(P)]),
    "fw_ruleset_create": (P, [P, I64]),
    "fw_ruleset_destroy": (None, [P]),
    "fw_ruleset_size": (I64, [P]),
    "fw_ruleset_first_catch_all": (I64, [P]),
    "fw_ruleset_partition": (ctypes.c_int, [P, P, P, P]),
    "fw_partition_plan": (ctypes.c_int, [P, I64, ctypes.c_int32, P, P, P, P, P]),
    "fw_ruleset_check": (ctypes.c_int, [P]),
    "fw_ruleset_filter": (ctypes.c_int, [P, P, P]),
    "fw_filter_plan": (ctypes.c_int, [P, I64, P, I64, P, P, P, P]),
    "fw_classify": (ctypes.c_int, [P, ctypes.POINTER(fw_headers), I64, P, P, P]),
    "fw_classify_ex": (ctypes.c_int, [P, ctypes.POINTER(fw_headers), I64, P, P, P, ctypes.POINTER(fw_config)]),
    "fw_host_pipeline_create": (ctypes.c_int, [I64, ctypes.c_int, ctypes.POINTER(P)]),
    "fw_host_pipeline_destroy": (None, [P]),
    "fw_classify_host": (ctypes.c_int, [P, P, ctypes.POINTER(fw_headers), I64, P, P, ctypes.c_int,
                                        ctypes.POINTER(fw_config)]),
    "fw_selftest_wait_timeout": (ctypes.c_int, [P, I64, P]),
    "fw_selftest_fail_alloc": (ctypes.c_int, [I64]),
    "fw_classify_rule_split_noalloc": (ctypes.c_int, [P, ctypes.POINTER(fw_headers), I64, P, P, P,
                                                      ctypes.POINTER(fw_config)]),
    "fw_lindex_create": (ctypes.c_int, [P, I64, ctypes.POINTER(fw_lindex_config), ctypes.POINTER(P)]),
    "fw_lindex_destroy": (None, [P]),
    "fw_lindex_classify": (ctypes.c_int, [P, ctypes.POINTER(fw_headers), I64, P, P, P]),
    "fw_lindex_get_stats": (ctypes.c_int, [P, ctypes.POINTER(fw_lindex_stats)]),
    "fw_plan_create": (ctypes.c_int, [ctypes.POINTER(fw_job), I64, ctypes.POINTER(fw_plan_config),
                                      ctypes.POINTER(P)]),
    "fw_plan_launch": (ctypes.c_int, [P, P]),
    "fw_plan_launch_graph": (ctypes.c_int, [P, P]),
    "fw_plan_items": (I64, [P]),
    "fw_plan_kernel": (ctypes.c_int, [P]),
    "fw_plan_destroy": (None, [P]),
    "fw_server_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(fw_server_config),
                                        ctypes.POINTER(P)]),
    "fw_server_destroy": (None, [P]),
    "fw_server_submit": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(fw_headers), I64, P, P,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "fw_server_wait": (ctypes.c_int, [P, ctypes.c_uint64, I64, ctypes.POINTER(ctypes.c_double)]),
    "fw_server_drain": (ctypes.c_int, [P, I64]),
    "fw_server_register_buffer": (ctypes.c_int, [P, P, ctypes.c_size_t]),
    "fw_server_unregister_buffer": (ctypes.c_int, [P, P]),
    "fw_server_get_stats": (ctypes.c_int, [P, ctypes.POINTER(fw_server_stats)]),
    "fw_server_replay": (ctypes.c_int, [P, ctypes.POINTER(fw_request), I64, I64]),
    "fw_dqueue_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(fw_dqueue_config),
                                        ctypes.POINTER(P)]),
    "fw_dqueue_destroy": (None, [P]),
    "fw_dqueue_register_buffer": (ctypes.c_int, [P, P, ctypes.c_size_t]),
    "fw_dqueue_submit": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(fw_headers), I64, P, P,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "fw_dqueue_wait": (ctypes.c_int, [P, ctypes.c_uint64, I64, ctypes.POINTER(ctypes.c_double)]),
    "fw_dqueue_get_stats": (ctypes.c_int, [P, ctypes.POINTER(fw_dqueue_stats)]),
    "fw_dqueue_replay": (ctypes.c_int, [P, ctypes.POINTER(fw_request), I64, I64]),
    "fw_int32_peak_launch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P,
                                            ctypes.POINTER(I64)]),
    "fw_last_status": (ctypes.c_int, []),
    "fw_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fw_abi_version": (ctypes.c_int, []),
    "fw_rule_size": (ctypes.c_int, []),
}


def lib(path: str | None = None):
    """Load ``libfw.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} is missing (run paper_1312_4188_gb300.build.build())")
        L = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.fw_rule_size() != RULE_DTYPE.itemsize:
            raise RuntimeError("fw_rule layout mismatch between library and binding")
        if path is None:
            _lib = L
        return L


def status_string(s: int) -> str:
    try:
        return lib().fw_status_string(int(s)).decode()
    except RuntimeError:
        return f"status {s}"


def _check(s: int, what: str):
    if s != FW_OK:
        raise FwError(s, what)


def _as_rules(rules) -> np.ndarray:
    """Copy rules field by field into a zeroed 24-byte-record array.

    numpy leaves the padding bytes of structured copies (fancy indexing,
    concatenate) uninitialised; the library rejects non-zero reserved bytes.
    """
    rules = np.asarray(rules)
    out = np.zeros(rules.shape[0], dtype=RULE_DTYPE)
    for f in RULE_DTYPE.names:
        out[f] = rules[f]
    return out


class Ruleset:
    """Owning wrapper of an ``fw_ruleset*`` handle."""

    def __init__(self, handle: int, n: int):
        self.handle = ctypes.c_void_p(handle)
        self.n = n

    @property
    def first_catch_all(self) -> int:
        return int(lib().fw_ruleset_first_catch_all(self.handle))

    def partition(self) -> dict:
        """{"classes", "key_field" (0 none, 1 src, 2 dst), "key_bits"} of the partitioned scan."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().fw_ruleset_partition(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "fw_ruleset_partition")
        return {"classes": a.value, "key_field": b.value, "key_bits": c.value}

    def filter(self) -> dict:
        """{"words" (0 = no bucket filter), "bytes"} of the rule set's bucket filter."""
        w, b = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().fw_ruleset_filter(self.handle, ctypes.byref(w), ctypes.byref(b)), "fw_ruleset_filter")
        return {"words": w.value, "bytes": b.value}

    def size(self) -> int:
        return int(lib().fw_ruleset_size(self.handle))

    def check(self) -> int:
        return int(lib().fw_ruleset_check(self.handle))

    def destroy(self):
        if self.handle is not None and self.handle.value:
            lib().fw_ruleset_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fw_partition_plan(rules, granule: int = 1) -> dict:
    """The partition of ``rules`` as given (host only): {"classes", "key_field", "key_bits",
    "class_len" (per class), "proto_class" (256 protocol classes)}."""
    r = _as_rules(rules)
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    lens = np.zeros(8, dtype=np.int64)
    pc = np.zeros(256, dtype=np.uint8)
    s = lib().fw_partition_plan(r.ctypes.data_as(P) if r.size else None, int(r.shape[0]), int(granule),
                                ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), lens.ctypes.data_as(P),
                                pc.ctypes.data_as(P))
    _check(s, "fw_partition_plan")
    return {"classes": a.value, "key_field": b.value, "key_bits": c.value, "class_len": lens[:a.value].tolist(),
            "proto_class": pc}


def fw_filter_plan(rules) -> dict:
    """The bucket filter a rule set of ``rules`` would hold, built on the host: {"words", "block"
    (uint8 array, empty without a filter), "class_off", "class_len"}."""
    r = _as_rules(rules)
    nb, w = ctypes.c_int64(), ctypes.c_int32()
    off = np.zeros(8, dtype=np.int32)
    ln = np.zeros(8, dtype=np.int32)
    rp = r.ctypes.data_as(P) if r.size else None
    _check(lib().fw_filter_plan(rp, int(r.shape[0]), None, 0, ctypes.byref(nb), ctypes.byref(w), None, None),
           "fw_filter_plan")
    blk = np.zeros(max(nb.value, 0), dtype=np.uint8)
    _check(lib().fw_filter_plan(rp, int(r.shape[0]), blk.ctypes.data_as(P) if blk.size else None, int(blk.size),
                                ctypes.byref(nb), ctypes.byref(w), off.ctypes.data_as(P), ln.ctypes.data_as(P)),
           "fw_filter_plan")
    return {"words": w.value, "block": blk, "class_off": off, "class_len": ln}


def fw_ruleset_create(rules) -> Ruleset:
    r = _as_rules(rules)
    out = ctypes.c_void_p()
    s = lib().fw_ruleset_create_ex(r.ctypes.data_as(P) if r.size else None, int(r.shape[0]), ctypes.byref(out))
    _check(s, "fw_ruleset_create")
    return Ruleset(out.value, int(r.shape[0]))


def headers_struct(h: dict) -> fw_headers:
    """``fw_headers`` from a dict of tensors (or objects with data_ptr) keyed by field."""
    return fw_headers(*[ctypes.c_void_p(int(h[f].data_ptr())) for f in HEADER_FIELDS])


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def headers_to_device(h: dict, device="cuda") -> dict:
    """Copy numpy SoA headers to device tensors (same bytes, signed views for torch)."""
    import torch
    views = {"src": np.int32, "dst": np.int32, "sport": np.int16, "dport": np.int16, "proto": np.uint8}
    return {f: torch.from_numpy(np.ascontiguousarray(h[f]).view(views[f])).to(device) for f in HEADER_FIELDS}


def fw_classify(rs: Ruleset, hdrs: dict, n: int | None = None, out_idx=None, out_act=None, stream=None,
                config: fw_config | None = None):
    """Classify device headers; returns (out_idx int32 tensor, out_act uint8 tensor)."""
    import torch
    if n is None:
        n = int(hdrs["src"].shape[0])
    dev = hdrs["src"].device
    if out_idx is None:
        out_idx = torch.empty(n, dtype=torch.int32, device=dev)
    if out_act is None:
        out_act = torch.empty(n, dtype=torch.uint8, device=dev)
    hs = headers_struct(hdrs)
    st = _stream_handle(stream)
    if config is None:
        s = lib().fw_classify(rs.handle, ctypes.byref(hs), int(n), ctypes.c_void_p(out_idx.data_ptr()),
                              ctypes.c_void_p(out_act.data_ptr()), st)
    else:
        s = lib().fw_classify_ex(rs.handle, ctypes.byref(hs), int(n), ctypes.c_void_p(out_idx.data_ptr()),
                                 ctypes.c_void_p(out_act.data_ptr()), st, ctypes.byref(config))
    _check(s, "fw_classify")
    return out_idx, out_act


fw_classify_ex = fw_classify


class HostPipeline:
    """Owning wrapper of an ``fw_host_pipeline*``."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    def destroy(self):
        if self.handle is not None and self.handle.value:
            lib().fw_host_pipeline_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fw_host_pipeline_create(chunk_packets: int = 0, n_streams: int = 0) -> HostPipeline:
    out = ctypes.c_void_p()
    _check(lib().fw_host_pipeline_create(int(chunk_packets), int(n_streams), ctypes.byref(out)),
           "fw_host_pipeline_create")
    return HostPipeline(out.value)


def fw_classify_host(pl: HostPipeline, rs: Ruleset, host_hdrs: dict, out_idx, out_act, n: int | None = None,
                     strategy: int = FW_HOST_COPY, config: fw_config | None = None):
    """Classify headers held in host memory (tensors or numpy arrays); verdicts land in host ``out_*``."""
    def ptr(a):
        return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
    if n is None:
        n = int(host_hdrs["src"].shape[0])
    hs = fw_headers(*[ptr(host_hdrs[f]) for f in HEADER_FIELDS])
    s = lib().fw_classify_host(pl.handle, rs.handle, ctypes.byref(hs), int(n), ptr(out_idx), ptr(out_act),
                               int(strategy), ctypes.byref(config) if config is not None else None)
    _check(s, "fw_classify_host")


class LIndex:
    """Owning wrapper of an ``fw_lindex*`` (learned-index decomposition classifier)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    def stats(self) -> dict:
        st = fw_lindex_stats()
        _check(lib().fw_lindex_get_stats(self.handle, ctypes.byref(st)), "fw_lindex_get_stats")
        return {"rules": st.rules, "rules_indexed": st.rules_indexed, "words_per_row": st.words_per_row,
                "segments": st.segments, "intervals": list(st.intervals), "max_error": list(st.max_error),
                "bitmap_bytes": st.bitmap_bytes, "fallbacks": st.fallbacks, "classes": st.classes,
                "key_field": st.key_field, "key_bits": st.key_bits}

    def destroy(self):
        if self.handle is not None and self.handle.value:
            lib().fw_lindex_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fw_lindex_create(rules, segments: int = 0, truncate: int = 0) -> LIndex:
    r = _as_rules(rules)
    cfg = fw_lindex_config()
    cfg.segments, cfg.truncate = int(segments), int(truncate)
    out = ctypes.c_void_p()
    s = lib().fw_lindex_create(r.ctypes.data_as(P) if r.size else None, int(r.shape[0]), ctypes.byref(cfg),
                               ctypes.byref(out))
    _check(s, "fw_lindex_create")
    return LIndex(out.value)


def fw_lindex_classify(li: LIndex, hdrs: dict, n: int | None = None, out_idx=None, out_act=None, stream=None):
    import torch
    if n is None:
        n = int(hdrs["src"].shape[0])
    dev = hdrs["src"].device
    if out_idx is None:
        out_idx = torch.empty(n, dtype=torch.int32, device=dev)
    if out_act is None:
        out_act = torch.empty(n, dtype=torch.uint8, device=dev)
    hs = headers_struct(hdrs)
    s = lib().fw_lindex_classify(li.handle, ctypes.byref(hs), int(n), ctypes.c_void_p(out_idx.data_ptr()),
                                 ctypes.c_void_p(out_act.data_ptr()), _stream_handle(stream))
    _check(s, "fw_lindex_classify")
    return out_idx, out_act


def make_plan_config(classes=None, block_threads=0, blocks_per_sm=0) -> fw_plan_config:
    """``classes``: list of (max_rules, packets_per_item, segment_rules); the last max_rules is ignored."""
    c = fw_plan_config()
    c.block_threads, c.blocks_per_sm = int(block_threads), int(blocks_per_sm)
    classes = classes or []
    c.n_classes = len(classes)
    for i, (mx, ppi, seg) in enumerate(classes):
        c.class_max_rules[i], c.packets_per_item[i], c.segment_rules[i] = int(mx), int(ppi), int(seg)
    return c


class Plan:
    """Owning wrapper of an ``fw_plan*``; keeps the jobs' tensors alive."""

    def __init__(self, handle: int, keep):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep

    def items(self) -> int:
        return int(lib().fw_plan_items(self.handle))

    def kernel(self) -> int:
        """0: the general batched kernel; 2 or 3: the filter-only kernel (its resident blocks per SM)."""
        return int(lib().fw_plan_kernel(self.handle))

    def launch(self, stream=None, graph: bool = True):
        fn = lib().fw_plan_launch_graph if graph else lib().fw_plan_launch
        _check(fn(self.handle, _stream_handle(stream)), "fw_plan_launch")

    def destroy(self):
        if self.handle is not None and self.handle.value:
            lib().fw_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fw_plan_create(jobs, config: fw_plan_config | None = None) -> Plan:
    """``jobs``: list of (Ruleset, device header dict, out_idx tensor, out_act tensor)."""
    arr = (fw_job * max(1, len(jobs)))()
    for i, (rs, h, oi, oa) in enumerate(jobs):
        n = int(h["src"].shape[0])
        arr[i] = fw_job(rs.handle, headers_struct(h), n, ctypes.c_void_p(oi.data_ptr()), ctypes.c_void_p(oa.data_ptr()))
    out = ctypes.c_void_p()
    s = lib().fw_plan_create(arr, len(jobs), ctypes.byref(config) if config is not None else None, ctypes.byref(out))
    _check(s, "fw_plan_create")
    return Plan(out.value, list(jobs))


class Server:
    """Owning wrapper of an ``fw_server*`` (continuous-batching classification service)."""

    def __init__(self, rulesets, **cfg):
        self._sets = list(rulesets)
        arr = (ctypes.c_void_p * len(self._sets))(*[r.handle.value for r in self._sets])
        c = fw_server_config()
        for k, v in cfg.items():
            setattr(c, k, int(v))
        out = ctypes.c_void_p()
        _check(lib().fw_server_create(arr, len(self._sets), ctypes.byref(c), ctypes.byref(out)), "fw_server_create")
        self.handle = out

    def submit(self, set_index: int, hdrs: dict, out_idx, out_act, n: int | None = None) -> int:
        """Queue a request; returns its ticket. Raises FwError (e.g. FW_EBUSY when the queue is full)."""
        if n is None:
            n = int(hdrs["src"].shape[0])
        hs = headers_struct(hdrs)
        t = ctypes.c_uint64()
        s = lib().fw_server_submit(self.handle, int(set_index), ctypes.byref(hs), int(n),
                                   ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_act.data_ptr()),
                                   ctypes.byref(t))
        _check(s, "fw_server_submit")
        return int(t.value)

    def wait(self, ticket: int, timeout_us: int = -1):
        """(status, latency_us) of a request; releases the ticket."""
        lat = ctypes.c_double()
        s = lib().fw_server_wait(self.handle, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(lat))
        return int(s), float(lat.value)

    def register(self, tensor):
        """Zero-copy mode: register a tensor's storage as a request buffer (see fw_server_register_buffer)."""
        _check(lib().fw_server_register_buffer(self.handle, ctypes.c_void_p(tensor.data_ptr()),
                                               tensor.numel() * tensor.element_size()), "fw_server_register_buffer")

    def drain(self, timeout_us: int = -1) -> int:
        return int(lib().fw_server_drain(self.handle, int(timeout_us)))

    def stats(self) -> dict:
        st = fw_server_stats()
        _check(lib().fw_server_get_stats(self.handle, ctypes.byref(st)), "fw_server_get_stats")
        return {k: int(getattr(st, k)) for k, _ in fw_server_stats._fields_}

    def replay(self, specs, timeout_us: int = 60_000_000):
        """``specs``: list of (set, hdrs dict, out_idx, out_act, arrival_us). Returns (status array, latency array)."""
        arr = (fw_request * len(specs))()
        for i, (st, h, oi, oa, t) in enumerate(specs):
            arr[i] = fw_request(int(st), 0, headers_struct(h), int(h["src"].shape[0]), ctypes.c_void_p(oi.data_ptr()),
                                ctypes.c_void_p(oa.data_ptr()), float(t), 0.0)
        s = lib().fw_server_replay(self.handle, arr, len(specs), int(timeout_us))
        status = np.array([r.status for r in arr], dtype=np.int32)
        lat = np.array([r.latency_us for r in arr], dtype=np.float64)
        # time each request waited for the submitting thread (part of its latency)
        self.last_submit_lag_us = np.array([r.submit_lag_us for r in arr], dtype=np.float64)
        return int(s), status, lat

    def destroy(self):
        if self.handle is not None and self.handle.value:
            lib().fw_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class DeviceQueue:
    """Owning wrapper of an ``fw_dqueue*`` (continuous batching scheduled on the device by one
    persistent kernel). Request buffers must lie in registered tensors."""

    def __init__(self, rulesets, **cfg):
        self._sets = list(rulesets)
        arr = (ctypes.c_void_p * len(self._sets))(*[r.handle.value for r in self._sets])
        c = fw_dqueue_config()
        for k, v in cfg.items():
            setattr(c, k, int(v))
        out = ctypes.c_void_p()
        _check(lib().fw_dqueue_create(arr, len(self._sets), ctypes.byref(c), ctypes.byref(out)), "fw_dqueue_create")
        self.handle = out

    def register(self, tensor):
        """Declare a tensor's storage as holding request buffers (see fw_dqueue_register_buffer)."""
        _check(lib().fw_dqueue_register_buffer(self.handle, ctypes.c_void_p(tensor.data_ptr()),
                                               tensor.numel() * tensor.element_size()), "fw_dqueue_register_buffer")

    def submit(self, set_index: int, hdrs: dict, out_idx, out_act, n: int | None = None) -> int:
        """Queue a request; returns its ticket. Raises FwError (e.g. FW_EBUSY when its ring entry is held)."""
        if n is None:
            n = int(hdrs["src"].shape[0])
        hs = headers_struct(hdrs)
        t = ctypes.c_uint64()
        s = lib().fw_dqueue_submit(self.handle, int(set_index), ctypes.byref(hs), int(n),
                                   ctypes.c_void_p(out_idx.data_ptr()), ctypes.c_void_p(out_act.data_ptr()),
                                   ctypes.byref(t))
        _check(s, "fw_dqueue_submit")
        return int(t.value)

    def wait(self, ticket: int, timeout_us: int = -1):
        """(status, latency_us) of a request; FW_OK releases the ticket."""
        lat = ctypes.c_double()
        s = lib().fw_dqueue_wait(self.handle, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(lat))
        return int(s), float(lat.value)

    def stats(self) -> dict:
        st = fw_dqueue_stats()
        _check(lib().fw_dqueue_get_stats(self.handle, ctypes.byref(st)), "fw_dqueue_get_stats")
        return {k: int(getattr(st, k)) for k, _ in fw_dqueue_stats._fields_}

    def replay(self, specs, timeout_us: int = 60_000_000):
        """``specs``: list of (set, hdrs dict, out_idx, out_act, arrival_us). Returns (status, status array,
        latency array); ``last_submit_lag_us`` keeps each request's wait for the submitting thread."""
        arr = (fw_request * len(specs))()
        for i, (st, h, oi, oa, t) in enumerate(specs):
            arr[i] = fw_request(int(st), 0, headers_struct(h), int(h["src"].shape[0]), ctypes.c_void_p(oi.data_ptr()),
                                ctypes.c_void_p(oa.data_ptr()), float(t), 0.0)
        s = lib().fw_dqueue_replay(self.handle, arr, len(specs), int(timeout_us))
        status = np.array([r.status for r in arr], dtype=np.int32)
        lat = np.array([r.latency_us for r in arr], dtype=np.float64)
        self.last_submit_lag_us = np.array([r.submit_lag_us for r in arr], dtype=np.float64)
        return int(s), status, lat

    def destroy(self):
        if self.handle is not None and self.handle.value:
            lib().fw_dqueue_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def pinned_headers(h: dict) -> dict:
    """Pinned host tensors holding the bytes of numpy SoA headers."""
    import torch
    views = {"src": np.int32, "dst": np.int32, "sport": np.int16, "dport": np.int16, "proto": np.uint8}
    return {f: torch.from_numpy(np.ascontiguousarray(h[f]).view(views[f])).pin_memory() for f in HEADER_FIELDS}


INT32_PEAK_KINDS = {"alu_lop3": 0, "fma_imad": 1, "mixed": 2}


def fw_int32_peak_launch(kind: int, iters: int, blocks: int, threads: int, sink, stream=None) -> int:
    """Enqueue the integer-throughput microbenchmark (``sink``: device tensor of at least
    blocks*threads uint32); returns the instruction count of the launch (lanes x instructions)."""
    ops = ctypes.c_int64()
    s = lib().fw_int32_peak_launch(int(kind), int(iters), int(blocks), int(threads),
                                   ctypes.c_void_p(sink.data_ptr()), _stream_handle(stream), ctypes.byref(ops))
    _check(s, "fw_int32_peak_launch")
    return int(ops.value)
