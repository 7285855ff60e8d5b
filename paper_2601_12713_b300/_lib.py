"""ctypes binding of libodp (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libodp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2601_12713_b300.build` "
        "(there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p

_lib.odp_status_string.argtypes = [ctypes.c_int]
_lib.odp_status_string.restype = ctypes.c_char_p
_lib.odp_fingerprint.argtypes = [_vp, _vp, ctypes.c_uint64, _vp, _vp]
_lib.odp_fingerprint.restype = ctypes.c_int
_lib.odp_fingerprint_one.argtypes = [_vp, ctypes.c_uint64, _vp, _vp]
_lib.odp_fingerprint_one.restype = ctypes.c_int
_lib.odp_fingerprint_noalloc.argtypes = [_vp, _vp, ctypes.c_uint64, _vp, _vp]
_lib.odp_fingerprint_noalloc.restype = ctypes.c_int
_lib.odp_fingerprint_log.argtypes = [_vp, _vp, ctypes.c_uint64, _vp]
_lib.odp_fingerprint_log.restype = ctypes.c_int
class FpSchedule(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tmin_scale", ctypes.c_int32), ("load_stages", ctypes.c_int32)]


_lib.odp_fingerprint_with.argtypes = [ctypes.POINTER(FpSchedule), _vp, _vp, ctypes.c_uint64, _vp,
                                      _vp]
_lib.odp_fingerprint_with.restype = ctypes.c_int
_lib.odp_autotune_fingerprint.argtypes = [_vp, _vp, ctypes.c_uint64, _vp, _vp, ctypes.c_int,
                                          ctypes.POINTER(FpSchedule),
                                          ctypes.POINTER(ctypes.c_float)]
_lib.odp_autotune_fingerprint.restype = ctypes.c_int
_lib.odp_autotune_clear.argtypes = []
_lib.odp_autotune_clear.restype = ctypes.c_int
_lib.odp_fingerprint_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
_lib.odp_fingerprint_status.restype = ctypes.c_int
_lib.odp_analyze.argtypes = [_vp, ctypes.c_uint64, _vp, _vp]
_lib.odp_analyze.restype = ctypes.c_int
_lib.odp_verify_fingerprints.argtypes = [_vp, _vp, ctypes.c_uint64, _vp, _vp, _vp]
_lib.odp_verify_fingerprints.restype = ctypes.c_int
_lib.odp_release_scratch.argtypes = []
_lib.odp_release_scratch.restype = ctypes.c_int

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_lib.odp_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, ctypes.c_void_p]
_lib.odp_set_allocator.restype = ctypes.c_int


def lib():
    return _lib


class OdpError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


def status_string(status: int) -> str:
    return _lib.odp_status_string(int(status)).decode()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _check(status: int, what: str) -> int:
    if status < 0:
        raise OdpError(status, what)
    return status


# ------------------------------------------------------------ fingerprint

def fingerprint(ptrs: torch.Tensor, sizes: torch.Tensor, out: torch.Tensor, stream=None) -> None:
    """FP128 of n buffers: ``ptrs``/``sizes`` int64 CUDA tensors of n entries,
    ``out`` an (n, 2) int64 CUDA tensor receiving (lo, hi)."""
    n = ptrs.numel()
    assert sizes.numel() == n and out.numel() == 2 * n
    for t in (ptrs, sizes, out):
        assert t.is_cuda and t.is_contiguous()
    _check(_lib.odp_fingerprint(ptrs.data_ptr() if n else None, sizes.data_ptr() if n else None,
                                n, out.data_ptr() if n else None, _stream(stream)),
           "odp_fingerprint")


def fingerprint_one(ptr: int, size: int, out: torch.Tensor, stream=None) -> None:
    """FP128 of one device buffer given by its address and size (host ints);
    ``out`` a CUDA tensor of at least 16 bytes receiving (lo, hi)."""
    assert out.is_cuda and out.is_contiguous() and out.numel() * out.element_size() >= 16
    _check(_lib.odp_fingerprint_one(ptr or None, size, out.data_ptr(), _stream(stream)),
           "odp_fingerprint_one")


def _fp_args(ptrs, sizes, out):
    n = ptrs.numel()
    assert sizes.numel() == n and out.numel() == 2 * n
    for t in (ptrs, sizes, out):
        assert t.is_cuda and t.is_contiguous()
    return (ptrs.data_ptr() if n else None, sizes.data_ptr() if n else None, n,
            out.data_ptr() if n else None)


def fingerprint_with(schedule, ptrs: torch.Tensor, sizes: torch.Tensor, out: torch.Tensor,
                     stream=None) -> None:
    """odp_fingerprint with an explicit (warps_per_cta, ctas_per_sm, tmin_scale[,
    load_stages])."""
    w, c, t = schedule[:3]
    st = schedule[3] if len(schedule) > 3 else 0
    sch = FpSchedule(w, c, t, st)
    _check(_lib.odp_fingerprint_with(ctypes.byref(sch), *_fp_args(ptrs, sizes, out),
                                     _stream(stream)), "odp_fingerprint_with")


def autotune_fingerprint(ptrs: torch.Tensor, sizes: torch.Tensor, out: torch.Tensor, reps=3,
                         stream=None):
    """Times every schedule on this batch, keeps the fastest for its size class;
    returns ((warps_per_cta, ctas_per_sm, tmin_scale, load_stages), ms per call)."""
    sch = FpSchedule()
    ms = ctypes.c_float(0)
    _check(_lib.odp_autotune_fingerprint(*_fp_args(ptrs, sizes, out), _stream(stream), reps,
                                         ctypes.byref(sch), ctypes.byref(ms)),
           "odp_autotune_fingerprint")
    return (sch.warps_per_cta, sch.ctas_per_sm, sch.tmin_scale, sch.load_stages), float(ms.value)


def autotune_clear() -> None:
    _check(_lib.odp_autotune_clear(), "odp_autotune_clear")


def fingerprint_noalloc(ptrs: torch.Tensor, sizes: torch.Tensor, out: torch.Tensor,
                        stream=None) -> None:
    """Like :func:`fingerprint` but through odp_fingerprint_noalloc, which uses
    a fixed device array instead of allocating scratch (at most 4096 buffers
    per call; calls must not overlap on the GPU)."""
    n = ptrs.numel()
    assert sizes.numel() == n and out.numel() == 2 * n
    for t in (ptrs, sizes, out):
        assert t.is_cuda and t.is_contiguous()
    _check(_lib.odp_fingerprint_noalloc(ptrs.data_ptr() if n else None,
                                        sizes.data_ptr() if n else None, n,
                                        out.data_ptr() if n else None, _stream(stream)),
           "odp_fingerprint_noalloc")


def fingerprint_tensors(tensors, stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """FP128 of the bytes of each CUDA tensor (any dtype, contiguous)."""
    dev = tensors[0].device if tensors else torch.device("cuda")
    n = len(tensors)
    ptr_h = torch.tensor([t.data_ptr() for t in tensors], dtype=torch.int64)
    size_h = torch.tensor([t.numel() * t.element_size() for t in tensors], dtype=torch.int64)
    ptrs = ptr_h.to(dev, non_blocking=False)
    sizes = size_h.to(dev, non_blocking=False)
    if out is None:
        out = torch.empty((n, 2), dtype=torch.int64, device=dev)
    fingerprint(ptrs, sizes, out, stream)
    return out


def fingerprint_status(stream=None) -> int:
    s = ctypes.c_int32(0)
    _check(_lib.odp_fingerprint_status(_stream(stream), ctypes.byref(s)), "odp_fingerprint_status")
    return int(s.value)


# ---------------------------------------------------------------- analysis

EVENT_DTYPE = np.dtype(
    [("t_start_ns", "<u8"), ("t_end_ns", "<u8"), ("host_addr", "<u8"), ("dev_addr", "<u8"),
     ("bytes", "<u8"), ("fp_lo", "<u8"), ("fp_hi", "<u8"), ("site_id", "<u4"), ("kind", "u1"),
     ("src_dev", "i1"), ("dst_dev", "i1"), ("flags", "u1")])
FINDING_DTYPE = np.dtype(
    [("kind", "u1"), ("pad0", "u1", (3,)), ("site", "<u4"), ("partner_site", "<u4"),
     ("pad1", "<u4"), ("event", "<u8"), ("partner", "<u8"), ("wasted_bytes", "<u8"),
     ("wasted_ns", "<u8")])
SITE_DTYPE = np.dtype(
    [("site", "<u4"), ("kind", "u1"), ("pad", "u1", (3,)), ("count", "<u8"),
     ("wasted_bytes", "<u8"), ("wasted_ns", "<u8")])
SUMMARY_FIELDS = (
    ["n_events", "n_transfers", "n_allocs", "n_deletes", "n_kernels", "n_pairs",
     "n_unpaired_allocs", "n_unmatched_deletes"]
    + [f"count{k}" for k in range(6)] + [f"wasted_bytes{k}" for k in range(6)]
    + [f"wasted_ns{k}" for k in range(6)]
    + ["trace_begin_ns", "trace_end_ns", "trace_span_ns", "saved_ns", "speedup_num",
       "speedup_den"])
assert EVENT_DTYPE.itemsize == 64 and FINDING_DTYPE.itemsize == 48 and SITE_DTYPE.itemsize == 32


class _OdpFindings(ctypes.Structure):
    _fields_ = [("items", _vp), ("capacity", ctypes.c_uint64), ("count", _vp), ("sites", _vp),
                ("sites_capacity", ctypes.c_uint64), ("sites_count", _vp), ("summary", _vp),
                ("status", _vp)]


class Findings:
    """Device-side output buffers of odp_analyze."""

    def __init__(self, capacity: int, sites_capacity: int = 5 * 65536, device="cuda"):
        self.capacity = int(capacity)
        self.sites_capacity = int(sites_capacity)
        self.items = torch.empty(max(1, self.capacity) * 48, dtype=torch.uint8, device=device)
        self.sites = torch.empty(max(1, self.sites_capacity) * 32, dtype=torch.uint8, device=device)
        # count, sites_count, status (+pad), summary
        self.small = torch.zeros(4 + len(SUMMARY_FIELDS), dtype=torch.int64, device=device)
        base = self.small.data_ptr()
        self.struct = _OdpFindings(self.items.data_ptr(), self.capacity, base,
                                   self.sites.data_ptr(), self.sites_capacity, base + 8,
                                   base + 32, base + 16)

    def to_host(self):
        small = self.small.cpu().numpy().view(np.uint64)
        count = int(small[0])
        n_sites = int(small[1])
        status = int(np.int32(np.uint32(small[2] & np.uint64(0xFFFFFFFF))))
        summary = {k: int(v) for k, v in zip(SUMMARY_FIELDS, small[4:])}
        k = min(count, self.capacity)
        items = self.items[: k * 48].cpu().numpy().view(FINDING_DTYPE).copy()
        s = min(n_sites, self.sites_capacity)
        sites = self.sites[: s * 32].cpu().numpy().view(SITE_DTYPE).copy()
        return {"status": status, "count": count, "findings": items, "summary": summary,
                "sites": sites, "n_sites": n_sites}


def analyze(events: torch.Tensor, n: int, out: Findings, stream=None) -> None:
    """Algorithms 1-5 over ``n`` 64-byte events held in a CUDA byte tensor."""
    assert events.is_cuda and events.numel() >= 64 * n
    _check(_lib.odp_analyze(events.data_ptr() if n else None, n, ctypes.byref(out.struct),
                            _stream(stream)), "odp_analyze")


def fingerprint_log(events: torch.Tensor, n: int, payload_ptrs: torch.Tensor,
                    stream=None) -> None:
    """Writes the fingerprint of every transfer's payload (``payload_ptrs``:
    int64 CUDA tensor of n device pointers) into its record of ``events``
    (a CUDA byte tensor of n 64-byte records)."""
    assert events.is_cuda and events.numel() >= 64 * n
    assert payload_ptrs.is_cuda and payload_ptrs.numel() >= n
    _check(_lib.odp_fingerprint_log(events.data_ptr() if n else None,
                                    payload_ptrs.data_ptr() if n else None, n, _stream(stream)),
           "odp_fingerprint_log")


def verify_fingerprints(events: torch.Tensor, n: int, payload_ptrs: torch.Tensor,
                        flags: torch.Tensor | None = None, stream=None) -> int:
    """Collision check: returns the number of transfers whose bytes differ
    from the first transfer with the same fingerprint (synchronises)."""
    count = torch.zeros(1, dtype=torch.int64, device=events.device)
    _check(_lib.odp_verify_fingerprints(events.data_ptr() if n else None,
                                        payload_ptrs.data_ptr() if n else None, n,
                                        count.data_ptr(),
                                        flags.data_ptr() if flags is not None else None,
                                        _stream(stream)), "odp_verify_fingerprints")
    return int(count.item())


# ---------------------------------------------------------------- serving

class ServerCfg(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("n_slots", ctypes.c_int32),
                ("device_budget_bytes", ctypes.c_uint64), ("max_events", ctypes.c_uint64),
                ("max_batch_events", ctypes.c_uint32), ("max_producers", ctypes.c_uint32),
                ("watermark_timeout_us", ctypes.c_uint32), ("batch_interval_us", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "events_submitted", "events_processed", "batches", "findings_streamed", "late_events",
        "latency_p50_ns", "latency_p99_ns", "latency_max_ns", "first_submit_ns", "last_done_ns",
        "rt_groups_at_flush", "stream_overflow", "queue_p50_ns", "queue_p99_ns",
        "device_bytes")]


_lib.odp_server_bytes.argtypes = [ctypes.POINTER(ServerCfg), ctypes.POINTER(ctypes.c_uint64)]
_lib.odp_server_bytes.restype = ctypes.c_int
_lib.odp_server_create.argtypes = [ctypes.POINTER(ServerCfg), ctypes.POINTER(_vp)]
_lib.odp_server_create.restype = ctypes.c_int
_lib.odp_server_submit.argtypes = [_vp, _vp, _vp, ctypes.c_uint64]
_lib.odp_server_submit.restype = ctypes.c_int
_lib.odp_server_attach.argtypes = [_vp, ctypes.c_uint64]
_lib.odp_server_attach.restype = ctypes.c_int
_lib.odp_server_begin.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64)]
_lib.odp_server_begin.restype = ctypes.c_int
_lib.odp_server_cancel.argtypes = [_vp, ctypes.c_uint64]
_lib.odp_server_cancel.restype = ctypes.c_int
_lib.odp_server_poll.argtypes = [_vp, _vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
_lib.odp_server_poll.restype = ctypes.c_int
_lib.odp_server_flush.argtypes = [_vp]
_lib.odp_server_flush.restype = ctypes.c_int
_lib.odp_server_log.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_uint64)]
_lib.odp_server_log.restype = ctypes.c_int
_lib.odp_server_origin.argtypes = [_vp, _vp, _vp, ctypes.c_uint64]
_lib.odp_server_origin.restype = ctypes.c_int
_lib.odp_server_stats_get.argtypes = [_vp, ctypes.POINTER(ServerStats)]
_lib.odp_server_stats_get.restype = ctypes.c_int
_lib.odp_server_destroy.argtypes = [_vp]
_lib.odp_server_destroy.restype = ctypes.c_int


def server_bytes(n_slots=4, max_events=1 << 23, max_batch_events=4096, max_producers=128) -> int:
    """Device bytes a Server of this shape reserves (odp_server_bytes)."""
    cfg = ServerCfg(0, n_slots, 0, max_events, max_batch_events, max_producers, 0, 0)
    b = ctypes.c_uint64(0)
    _check(_lib.odp_server_bytes(ctypes.byref(cfg), ctypes.byref(b)), "odp_server_bytes")
    return int(b.value)


class Server:
    """Continuous-batching serving loop (odp_server_*)."""

    def __init__(self, device=0, n_slots=4, device_budget_bytes=8 << 30, max_events=1 << 23,
                 max_batch_events=4096, max_producers=128, watermark_timeout_us=50_000,
                 batch_interval_us=50):
        cfg = ServerCfg(device, n_slots, device_budget_bytes, max_events, max_batch_events,
                        max_producers, watermark_timeout_us, batch_interval_us)
        self.h = None
        h = _vp()
        _check(_lib.odp_server_create(ctypes.byref(cfg), ctypes.byref(h)), "odp_server_create")
        self.h = h
        self.submit_fn = ctypes.cast(_lib.odp_server_submit, _vp).value
        self.attach_fn = ctypes.cast(_lib.odp_server_attach, _vp).value
        self.begin_fn = ctypes.cast(_lib.odp_server_begin, _vp).value

    def attach(self, start_t_ns: int = 0) -> None:
        _check(_lib.odp_server_attach(self.h, start_t_ns), "odp_server_attach")

    def begin(self) -> int:
        """Opens an event on the calling thread; returns its start time (ns)."""
        t = ctypes.c_uint64(0)
        _check(_lib.odp_server_begin(self.h, ctypes.byref(t)), "odp_server_begin")
        return int(t.value)

    def cancel(self, t_start_ns: int) -> None:
        """Closes an event opened by begin() without submitting it."""
        _check(_lib.odp_server_cancel(self.h, t_start_ns), "odp_server_cancel")

    def submit(self, events: np.ndarray, payload_ptrs) -> None:
        ev = np.ascontiguousarray(events)
        n = ev.size
        ptrs = np.ascontiguousarray(np.asarray(payload_ptrs, dtype=np.uint64))
        _check(_lib.odp_server_submit(self.h, ev.ctypes.data, ptrs.ctypes.data, n),
               "odp_server_submit")

    def poll(self, cap=1 << 20) -> np.ndarray:
        out = np.zeros(cap, dtype=FINDING_DTYPE)
        k = ctypes.c_uint64(0)
        _check(_lib.odp_server_poll(self.h, out.ctypes.data, cap, ctypes.byref(k)), "odp_server_poll")
        return out[: k.value].copy()

    def flush(self) -> None:
        _check(_lib.odp_server_flush(self.h), "odp_server_flush")

    def log(self):
        p = _vp()
        n = ctypes.c_uint64(0)
        _check(_lib.odp_server_log(self.h, ctypes.byref(p), ctypes.byref(n)), "odp_server_log")
        return int(p.value or 0), int(n.value)

    def origin(self, n):
        prod = np.zeros(n, dtype=np.uint32)
        seq = np.zeros(n, dtype=np.uint64)
        _check(_lib.odp_server_origin(self.h, prod.ctypes.data, seq.ctypes.data, n),
               "odp_server_origin")
        return prod, seq

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.odp_server_stats_get(self.h, ctypes.byref(st)), "odp_server_stats_get")
        return {k: int(getattr(st, k)) for k, _ in ServerStats._fields_}

    def close(self) -> None:
        if self.h:
            _lib.odp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def log_tensor(server: Server, n: int | None = None) -> torch.Tensor:
    """The server's resident log as a CUDA byte tensor view (no copy)."""
    ptr, m = server.log()
    n = m if n is None else n
    if n == 0:
        return torch.empty(64, dtype=torch.uint8, device="cuda")
    return _wrap_device(ptr, 64 * n)


def _wrap_device(ptr: int, nbytes: int) -> torch.Tensor:
    class _Holder:
        __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                    "version": 3, "strides": None}

    return torch.as_tensor(_Holder(), device="cuda")


# ---------------------------------------------------------------- memory

_keep = []


def _install(a, f) -> None:
    # odp_set_allocator frees the cached blocks through the previous
    # callbacks, so they must stay alive until it returns
    old = list(_keep)
    try:
        _check(_lib.odp_set_allocator(a if a is not None else _ALLOC_FN(),
                                      f if f is not None else _FREE_FN(), None),
               "odp_set_allocator")
        _keep[:] = [a, f] if a is not None else []
    finally:
        del old


def set_torch_allocator() -> None:
    """Route libodp scratch through torch's caching allocator."""

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _install(a, f)


def set_allocator(alloc, free) -> None:
    """Route libodp scratch through Python callables alloc(nbytes, stream) ->
    device pointer (0/None on failure) and free(ptr, stream); None, None
    restores cudaMallocAsync."""
    if alloc is None:
        _install(None, None)
        return
    a = _ALLOC_FN(lambda nbytes, stream, ctx: alloc(int(nbytes), stream))
    f = _FREE_FN(lambda ptr, stream, ctx: free(int(ptr or 0), stream))
    _install(a, f)


def release_scratch() -> None:
    _check(_lib.odp_release_scratch(), "odp_release_scratch")
