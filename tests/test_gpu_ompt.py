"""The OMPT front end (libodp_ompt.so) driven by a stand-in OpenMP runtime:
the test plays the runtime's part of the OMPT interface (ompt_start_tool,
the lookup of ompt_set_callback, the EMI target / data-op / submit
callbacks with begin and end endpoints) around real device buffers, and
checks the tool's log and findings against the oracle."""

import ctypes
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

HOST = 1  # the runtime's number for the host (one device: device 0)
BEGIN, END = 1, 2
ALLOC, TO_DEVICE, FROM_DEVICE, DELETE, ASSOCIATE = 1, 2, 3, 4, 5


class OmptData(ctypes.Union):
    _fields_ = [("value", ctypes.c_uint64), ("ptr", ctypes.c_void_p)]


class StartResult(ctypes.Structure):
    _fields_ = [("initialize", ctypes.c_void_p), ("finalize", ctypes.c_void_p),
                ("tool_data", OmptData)]


INIT = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(OmptData))
FINI = ctypes.CFUNCTYPE(None, ctypes.POINTER(OmptData))
LOOKUP = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_char_p)
SET_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_void_p)
TARGET_EMI = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(OmptData), ctypes.POINTER(OmptData),
                              ctypes.POINTER(OmptData), ctypes.c_void_p)
DATA_OP_EMI = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.POINTER(OmptData),
                               ctypes.POINTER(OmptData), ctypes.POINTER(ctypes.c_uint64),
                               ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p)
SUBMIT_EMI = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.POINTER(OmptData),
                              ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint)


class FakeRuntime:
    """Registers the tool's callbacks and issues them like an offload runtime."""

    def __init__(self, lib):
        self.cbs = {}

        @SET_CB
        def set_cb(event, fn):
            self.cbs[event] = fn
            return 5  # ompt_set_always

        @LOOKUP
        def lookup(name):
            return ctypes.cast(set_cb, ctypes.c_void_p).value if name == b"ompt_set_callback" else None

        self._keep = (set_cb, lookup)
        lib.ompt_start_tool.restype = ctypes.POINTER(StartResult)
        res = lib.ompt_start_tool(51, b"stand-in runtime")
        assert res
        self.res = res.contents
        self.tool_data = OmptData()
        ok = INIT(self.res.initialize)(ctypes.cast(lookup, ctypes.c_void_p).value, HOST,
                                       ctypes.byref(self.tool_data))
        assert ok == 1
        assert set(self.cbs) == {33, 34, 35}
        self.target = TARGET_EMI(self.cbs[33])
        self.data_op = DATA_OP_EMI(self.cbs[34])
        self.submit = SUBMIT_EMI(self.cbs[35])
        self.td = OmptData()

    def op(self, optype, src, src_dev, dst, dst_dev, nbytes, site, fill=None):
        hid = ctypes.c_uint64(0)
        self.data_op(BEGIN, None, ctypes.byref(self.td), ctypes.byref(hid), optype, src, src_dev,
                     dst, dst_dev, nbytes, site)
        if fill is not None:
            fill()
            torch.cuda.synchronize()
        self.data_op(END, None, ctypes.byref(self.td), ctypes.byref(hid), optype, src, src_dev,
                     dst, dst_dev, nbytes, site)

    def kernel(self, body=None):
        hid = ctypes.c_uint64(0)
        self.submit(BEGIN, ctypes.byref(self.td), ctypes.byref(hid), 1)
        if body is not None:
            body()
            torch.cuda.synchronize()
        self.submit(END, ctypes.byref(self.td), ctypes.byref(hid), 1)

    def region(self, begin):
        self.target(1, BEGIN if begin else END, 0, None, None, ctypes.byref(self.td), 0x400000)

    def finalize(self):
        FINI(self.res.finalize)(ctypes.byref(self.tool_data))


def test_ompt_tool_with_stand_in_runtime(cuda_ok, orc, tmp_path):
    import paper_2601_12713_b300 as odp

    lib = ctypes.CDLL(os.path.join(os.path.dirname(odp.__file__), "libodp_ompt.so"))
    lib.odp_ompt_server.restype = ctypes.c_void_p
    lib.odp_ompt_dropped.restype = ctypes.c_uint64
    rt = FakeRuntime(lib)
    nbytes = 1 << 16
    host = np.random.default_rng(7).integers(0, 256, nbytes, dtype=np.uint8)
    first_content = host.copy()
    host_t = torch.from_numpy(host)
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    hp, dp = host.ctypes.data, dev.data_ptr()

    def cycle(modify):
        rt.region(True)
        rt.op(ALLOC, hp, HOST, dp, 0, nbytes, 0x401000)
        rt.op(TO_DEVICE, hp, HOST, dp, 0, nbytes, 0x401010, fill=lambda: dev.copy_(host_t))
        rt.kernel((lambda: dev.add_(1)) if modify else None)
        rt.op(FROM_DEVICE, dp, 0, hp, HOST, nbytes, 0x401020,
              fill=lambda: host_t.copy_(dev.cpu()))
        rt.op(DELETE, dp, 0, hp, HOST, nbytes, 0x401030)
        rt.op(ASSOCIATE, hp, HOST, dp, 0, nbytes, 0x401040)   # no data moves: not logged
        rt.op(TO_DEVICE, hp, HOST, dp, 0, 0, 0x401050)        # empty: not logged
        rt.region(False)

    cycle(False)  # round trip: the content goes back unchanged
    cycle(False)  # the same content sent again (duplicate), the same range allocated again
    cycle(True)   # a kernel changes the data on the device
    cycle(False)
    prefix = str(tmp_path / "run")
    os.environ["ODP_OMPT_OUT"] = prefix
    try:
        rt.finalize()
    finally:
        del os.environ["ODP_OMPT_OUT"]
    assert lib.odp_ompt_dropped() == 0
    ev = np.fromfile(prefix + ".events", dtype=odp.EVENT_DTYPE)
    assert ev.size == 4 * 5
    assert list(ev["kind"][:5]) == [1, 2, 6, 3, 5]
    assert np.all(ev["dst_dev"][ev["kind"] == 2] == 0) and np.all(ev["src_dev"][ev["kind"] == 3] == 0)
    # the fingerprints are the oracle's of the bytes that were in device memory
    assert (int(ev["fp_lo"][1]), int(ev["fp_hi"][1])) == orc.fp128(first_content)
    assert (int(ev["fp_lo"][-2]), int(ev["fp_hi"][-2])) == orc.fp128(host)  # the last copy back
    sites = open(prefix + ".sites").read().split("\n")
    assert len([x for x in sites if x]) == 5  # four data-op code addresses + kernels
    o = orc.analyze(ev)
    counts = [o.summary[f"count{k}"] for k in range(1, 6)]
    assert counts[0] >= 1 and counts[1] >= 1 and counts[2] == 3  # DD, RT, RA
    # the findings streamed by the tool's server equal the oracle's
    srv = ctypes.c_void_p(lib.odp_ompt_server())
    out = np.zeros(256, dtype=odp.FINDING_DTYPE)
    k = ctypes.c_uint64(0)
    assert odp.lib().odp_server_poll(srv, out.ctypes.data, 256, ctypes.byref(k)) == 0
    st = out[: k.value]
    st = st[np.lexsort((st["partner"], st["event"], st["kind"]))]
    assert np.array_equal(st.view(np.uint8), o.findings.view(np.uint8))
    from paper_2601_12713_b300._lib import ServerStats

    stats = ServerStats()
    assert odp.lib().odp_server_stats_get(srv, ctypes.byref(stats)) == 0
    assert stats.late_events == 0 and stats.events_processed == ev.size
    lib.odp_ompt_shutdown()
