"""Host side of the OMPT front end, without a GPU: the tool's initializer, as
an OpenMP runtime calls it, declines with a message when its server cannot
be created, and ompt_start_tool honours ODP_OMPT_DISABLE."""

import ctypes
import os

import pytest


class OmptData(ctypes.Union):
    _fields_ = [("value", ctypes.c_uint64), ("ptr", ctypes.c_void_p)]


class StartResult(ctypes.Structure):
    _fields_ = [("initialize", ctypes.c_void_p), ("finalize", ctypes.c_void_p),
                ("tool_data", OmptData)]


INIT = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(OmptData))
LOOKUP = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_char_p)
SET_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_void_p)


@pytest.fixture(scope="module")
def tool():
    from paper_2601_12713_b300 import build

    build.build()
    lib = ctypes.CDLL(build.OMPT_LIB)
    lib.ompt_start_tool.argtypes = [ctypes.c_uint, ctypes.c_char_p]
    lib.ompt_start_tool.restype = ctypes.POINTER(StartResult)
    lib.odp_ompt_server.restype = ctypes.c_void_p
    return lib


def test_initializer_declines_an_unsupported_log_capacity(tool, capfd, monkeypatch):
    registered = []
    set_cb = SET_CB(lambda event, cb: registered.append(event) or 5)
    lookup = LOOKUP(lambda name: ctypes.cast(set_cb, ctypes.c_void_p).value
                    if name == b"ompt_set_callback" else None)
    monkeypatch.delenv("ODP_OMPT_DISABLE", raising=False)
    # above the server's 2^30 capacity limit: refused by host arithmetic alone
    monkeypatch.setenv("ODP_OMPT_MAX_EVENTS", str((1 << 30) + 1))
    res = tool.ompt_start_tool(51, b"stand-in runtime")
    assert res
    init = INIT(res.contents.initialize)
    data = OmptData()
    assert init(ctypes.cast(lookup, ctypes.c_void_p), 1, ctypes.byref(data)) == 0
    err = capfd.readouterr().err
    assert "tool inactive" in err and str((1 << 30) + 1) in err
    assert registered == []  # no callback was registered
    assert tool.odp_ompt_server() is None


def test_start_tool_honours_disable(tool, monkeypatch):
    monkeypatch.setenv("ODP_OMPT_DISABLE", "1")
    assert not tool.ompt_start_tool(51, b"x")
    monkeypatch.setenv("ODP_OMPT_DISABLE", "0")
    assert tool.ompt_start_tool(51, b"x")
