"""ctypes wrapper around the CPU oracle (test infrastructure only).

Nothing here imports the GPU package; the oracle declares its own record
layouts for findings, site rows and the summary.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "odp_oracle.cpp")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# 48-byte finding record, as the oracle writes it.
FINDING_DTYPE = np.dtype(
    [
        ("kind", "u1"),
        ("pad0", "u1", (3,)),
        ("site", "<u4"),
        ("partner_site", "<u4"),
        ("pad1", "<u4"),
        ("event", "<u8"),
        ("partner", "<u8"),
        ("wasted_bytes", "<u8"),
        ("wasted_ns", "<u8"),
    ]
)
assert FINDING_DTYPE.itemsize == 48

SITE_DTYPE = np.dtype(
    [
        ("site", "<u4"),
        ("kind", "u1"),
        ("pad", "u1", (3,)),
        ("count", "<u8"),
        ("wasted_bytes", "<u8"),
        ("wasted_ns", "<u8"),
    ]
)
assert SITE_DTYPE.itemsize == 32

# The summary is a flat array of u64 in this order.
SUMMARY_FIELDS = (
    ["n_events", "n_transfers", "n_allocs", "n_deletes", "n_kernels", "n_pairs",
     "n_unpaired_allocs", "n_unmatched_deletes"]
    + [f"count{k}" for k in range(6)]
    + [f"wasted_bytes{k}" for k in range(6)]
    + [f"wasted_ns{k}" for k in range(6)]
    + ["trace_begin_ns", "trace_end_ns", "trace_span_ns", "saved_ns", "speedup_num",
       "speedup_den"]
)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, single-threaded code)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(
                ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC]
            )
            os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        so = ctypes.CDLL(_SO)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        so.orc_fp128.argtypes = [ctypes.c_void_p, ctypes.c_uint64, u64p]
        so.orc_fp128_many.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_uint64, ctypes.c_void_p]
        so.orc_constant.argtypes = [ctypes.c_int, u64p]
        so.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p]
        so.orc_chunk_leaf.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        so.orc_lane_state.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.c_void_p]
        so.orc_tree_node.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.c_void_p]
        so.orc_mix128.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        so.orc_chain_step.argtypes = [ctypes.c_int, ctypes.c_uint64, u64p]
        for name in ("orc_analyze",):
            getattr(so, name).argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_uint64, u64p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_uint64, u64p]
            getattr(so, name).restype = ctypes.c_int
        so.orc_analyze_bruteforce.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_uint64, u64p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                              u64p]
        so.orc_analyze_bruteforce.restype = ctypes.c_int
        _lib = so
    return _lib


def _as_u8(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    arr = np.ascontiguousarray(data)
    return arr.view(np.uint8).reshape(-1)


def fp128(data) -> tuple[int, int]:
    """FP128 v1 of a byte string / array; returns (lo, hi)."""
    buf = _as_u8(data)
    out = (ctypes.c_uint64 * 2)()
    ptr = buf.ctypes.data if buf.size else None
    lib().orc_fp128(ptr, buf.size, out)
    return int(out[0]), int(out[1])


def fp128_many(arena, offsets, sizes) -> np.ndarray:
    """FP128 of buffers inside one host arena; returns (n, 2) uint64."""
    buf = _as_u8(arena)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
    n = offsets.size
    out = np.zeros((n, 2), dtype=np.uint64)
    lib().orc_fp128_many(buf.ctypes.data, offsets.ctypes.data, sizes.ctypes.data, n,
                         out.ctypes.data)
    return out


@dataclass
class OracleResult:
    status: int
    count: int
    findings: np.ndarray
    summary: dict
    sites: np.ndarray
    n_sites: int


def _run(fn, events: np.ndarray, extra, capacity, site_capacity) -> OracleResult:
    ev = np.ascontiguousarray(events)
    assert ev.dtype.itemsize == 64
    n = ev.size
    if capacity is None:
        capacity = max(16, 6 * n)
    if site_capacity is None:
        site_capacity = 5 * 65536
    items = np.zeros(capacity, dtype=FINDING_DTYPE)
    sites = np.zeros(site_capacity, dtype=SITE_DTYPE)
    summary = np.zeros(len(SUMMARY_FIELDS), dtype=np.uint64)
    count = ctypes.c_uint64(0)
    n_sites = ctypes.c_uint64(0)
    args = [ev.ctypes.data if n else None, n]
    if extra is not None:
        args.append(extra)
    args += [items.ctypes.data, capacity, ctypes.byref(count), summary.ctypes.data,
             sites.ctypes.data, site_capacity, ctypes.byref(n_sites)]
    status = fn(*args)
    c = int(count.value)
    s = int(n_sites.value)
    return OracleResult(
        status=status,
        count=c,
        findings=items[: min(c, capacity)].copy(),
        summary={k: int(v) for k, v in zip(SUMMARY_FIELDS, summary)},
        sites=sites[: min(s, site_capacity)].copy(),
        n_sites=s,
    )


def analyze(events: np.ndarray, capacity=None, site_capacity=None) -> OracleResult:
    """Algorithms 1-5 over a 64-byte-record event log (numpy structured array)."""
    return _run(lib().orc_analyze, events, None, capacity, site_capacity)


def analyze_bruteforce(events: np.ndarray, payloads, capacity=None,
                       site_capacity=None) -> OracleResult:
    """Collision-check mode: content equality by comparing payload bytes.

    ``payloads[i]`` is the byte content of event i (ignored for non-transfers).
    """
    n = events.size
    keep = []
    ptrs = (ctypes.c_void_p * max(1, n))()
    for i in range(n):
        p = payloads[i]
        if p is None:
            ptrs[i] = None
            continue
        a = _as_u8(p)
        keep.append(a)
        ptrs[i] = a.ctypes.data if a.size else None
    return _run(lib().orc_analyze_bruteforce, events, ptrs, capacity, site_capacity)
