"""Python handle on the C++ load generator (``loadgen.cpp``): host threads
emitting mapping events with Poisson arrivals into an odp server."""

from __future__ import annotations

import ctypes
import os

_SO = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth_load.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise ImportError(f"{_SO} missing: run python -m paper_2601_12713_b300.build")
        so = ctypes.CDLL(_SO)
        so.synth_load_create.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_uint64]
        so.synth_load_create.restype = ctypes.c_void_p
        so.synth_load_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
        so.synth_load_run.restype = ctypes.c_int64
        so.synth_load_payload.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.c_uint64)]
        so.synth_load_payload.restype = ctypes.c_int
        so.synth_load_thread_of.argtypes = [ctypes.c_uint64]
        so.synth_load_thread_of.restype = ctypes.c_uint32
        so.synth_load_destroy.argtypes = [ctypes.c_void_p]
        _lib = so
    return _lib


class Load:
    """n_threads producers, aggregate Poisson rate events_per_s, for seconds;
    payloads are views of [min_payload, max_payload] bytes (log-uniform) into
    the device pool."""

    def __init__(self, n_threads, events_per_s, seconds, seed, pool_ptr, pool_bytes,
                 min_payload=256, max_payload=64 << 20):
        self.h = lib().synth_load_create(n_threads, events_per_s, seconds, seed, pool_ptr,
                                         pool_bytes, min_payload, max_payload)

    def run(self, server, announce: bool = True) -> int:
        """Runs the producers into ``server``.  With ``announce`` each event
        is opened with the server's begin call, which stamps its start time."""
        begin = server.begin_fn if announce else None
        return int(lib().synth_load_run(self.h, server.h, server.submit_fn, server.attach_fn,
                                        begin))

    def payload(self, thread, seq):
        off, size = ctypes.c_uint64(), ctypes.c_uint64()
        rc = lib().synth_load_payload(self.h, thread, seq, ctypes.byref(off), ctypes.byref(size))
        assert rc == 0
        return int(off.value), int(size.value)

    @staticmethod
    def thread_of(host_addr) -> int:
        return int(lib().synth_load_thread_of(int(host_addr)))

    def close(self):
        if self.h:
            lib().synth_load_destroy(self.h)
            self.h = None
