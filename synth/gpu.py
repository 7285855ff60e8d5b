"""Device-side materialisation of synthetic contents (CUDA fill kernels in
``gen.cu``); same bytes as :mod:`synth.content`."""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise ImportError(f"{_SO} missing: run python -m paper_2601_12713_b300.build")
        so = ctypes.CDLL(_SO)
        so.synth_fill.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                  ctypes.c_uint64, ctypes.c_void_p]
        so.synth_fill_many.argtypes = [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_void_p]
        _lib = so
    return _lib


def _stream():
    return torch.cuda.current_stream().cuda_stream


def fill(t: torch.Tensor, variant: int, seed: int, word_offset: int = 0, nbytes=None) -> None:
    """Fill the bytes of CUDA tensor ``t`` (or its first ``nbytes``)."""
    nb = t.numel() * t.element_size() if nbytes is None else nbytes
    rc = lib().synth_fill(t.data_ptr(), nb, variant, seed & 0xFFFFFFFFFFFFFFFF, word_offset,
                          _stream())
    assert rc == 0


def fill_at(ptr: int, nbytes: int, variant: int, seed: int, word_offset: int = 0) -> None:
    rc = lib().synth_fill(ptr, nbytes, variant, seed & 0xFFFFFFFFFFFFFFFF, word_offset, _stream())
    assert rc == 0


def fill_many(arena: torch.Tensor, offsets: np.ndarray, sizes: np.ndarray,
              seeds: np.ndarray) -> None:
    """Random-variant contents for many buffers packed in one arena."""
    dev = arena.device
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = np.asarray(sizes, dtype=np.int64)
    nwords = (sizes + 7) // 8
    npieces = (nwords + 8191) // 8192
    piece_buf = np.repeat(np.arange(sizes.size, dtype=np.int64), npieces)
    starts = np.zeros(sizes.size, dtype=np.int64)
    starts[1:] = np.cumsum(npieces)[:-1]
    piece_first = (np.arange(piece_buf.size, dtype=np.int64) - starts[piece_buf]) * 8192
    d_off = torch.from_numpy(offsets).to(dev)
    d_sz = torch.from_numpy(sizes).to(dev)
    d_seed = torch.from_numpy(np.asarray(seeds, dtype=np.uint64).view(np.int64)).to(dev)
    d_pb = torch.from_numpy(piece_buf).to(dev)
    d_pf = torch.from_numpy(piece_first).to(dev)
    rc = lib().synth_fill_many(arena.data_ptr(), d_off.data_ptr(), d_sz.data_ptr(),
                               d_seed.data_ptr(), d_pb.data_ptr(), d_pf.data_ptr(),
                               piece_buf.size, _stream())
    assert rc == 0
    torch.cuda.current_stream().synchronize()
