"""Buffer contents from counter-based SplitMix64 streams (host side).

A content descriptor is (variant, seed, word_offset):
  * ``random``: 8-byte little-endian word j is SplitMix64 output
    ``word_offset + j`` of the stream seeded with ``seed``;
  * ``zero``: all bytes zero;
  * ``page``: one random 4 KiB page (words 0..511 of the stream) tiled.
The CUDA fill kernel in ``gen.cu`` produces the same bytes on the device.
"""

from __future__ import annotations

import numpy as np

from . import prng

RANDOM, ZERO, PAGE = 0, 1, 2
VARIANTS = {"random": RANDOM, "zero": ZERO, "page": PAGE}


def words(variant: int, seed: int, word_offset: int, nwords: int) -> np.ndarray:
    if variant == ZERO:
        return np.zeros(nwords, dtype=np.uint64)
    if variant == PAGE:
        idx = (np.arange(word_offset, word_offset + nwords, dtype=np.uint64) % np.uint64(512))
        return prng.at(np.uint64(seed), idx)
    return prng.stream(seed, word_offset, nwords)


def bytes_of(variant: int, seed: int, nbytes: int, word_offset: int = 0) -> np.ndarray:
    """``nbytes`` bytes of the descriptor (uint8 array)."""
    nw = (nbytes + 7) // 8
    w = words(variant, seed, word_offset, nw).astype("<u8")
    return w.view(np.uint8)[:nbytes].copy()


def lognormal_sizes(seed: int, n: int, median: float, sigma: float, lo: int, hi: int,
                    total: int | None = None) -> np.ndarray:
    """Lognormal sizes clipped to [lo, hi], optionally rescaled to sum to ``total``."""
    r = prng.Rng(seed)
    z = r.normal(n)
    s = np.exp(np.log(median) + sigma * z)
    s = np.clip(s, lo, hi)
    if total is not None:
        for _ in range(8):
            s = np.clip(s * (total / s.sum()), lo, hi)
    out = np.maximum(np.floor(s).astype(np.int64), lo)
    if total is not None:
        # put the rounding remainder on the largest buffer below the cap
        diff = int(total - out.sum())
        order = np.argsort(out)[::-1]
        for j in order:
            room = hi - out[j] if diff > 0 else out[j] - lo
            step = min(abs(diff), int(room))
            out[j] += step if diff > 0 else -step
            diff -= step if diff > 0 else -step
            if diff == 0:
                break
    return out


def batched_ragged(seed: int, n: int = 1_000_000, total: int = 16 << 30,
                   median: int = 4096, dup_frac: float = 0.4, max_size: int = 256 << 20,
                   align: int = 16):
    """Ragged batch: lognormal sizes (median 4 KiB, sigma = sqrt(2 ln 4), so the
    mean is four times the median), clipped to [1 B, 256 MiB] and rescaled to
    ``total`` bytes; ``dup_frac`` of the buffers copy an earlier buffer's size
    and content exactly.

    Returns (sizes, offsets, seeds, dup_of) where offsets pack the buffers in one
    arena at ``align``-byte alignment and dup_of[i] is the earlier buffer copied
    (or -1).
    """
    sigma = float(np.sqrt(2.0 * np.log(4.0)))
    r = prng.Rng(prng.derive(seed, 3))
    sizes = lognormal_sizes(prng.derive(seed, 1), n, median, sigma, 1, max_size, total)
    is_dup = r.uniform(n) < dup_frac
    is_dup[0] = False
    src = (r.uniform(n) * np.arange(n)).astype(np.int64)  # uniform earlier index
    dup_of = np.where(is_dup, src, -1)
    # follow chains so that dup_of points at an original
    for _ in range(64):
        chained = dup_of >= 0
        chained &= dup_of[np.maximum(dup_of, 0)] >= 0
        if not chained.any():
            break
        dup_of = np.where(chained, dup_of[np.maximum(dup_of, 0)], dup_of)
    sizes = np.where(dup_of >= 0, sizes[np.maximum(dup_of, 0)], sizes)
    # put the remainder on the largest originals that nothing copies
    referenced = np.zeros(n, dtype=bool)
    referenced[dup_of[dup_of >= 0]] = True
    free = np.flatnonzero((dup_of < 0) & ~referenced)
    order = free[np.argsort(sizes[free])[::-1]]
    diff = int(total - sizes.sum())
    for j in order:
        if diff == 0:
            break
        room = max_size - sizes[j] if diff > 0 else sizes[j] - 1
        step = min(abs(diff), int(room))
        sizes[j] += step if diff > 0 else -step
        diff -= step if diff > 0 else -step
    base_seed = prng.derive(seed, 2)
    seeds = prng.at(np.uint64(base_seed), np.arange(n, dtype=np.uint64))
    seeds = np.where(dup_of >= 0, seeds[np.maximum(dup_of, 0)], seeds)
    padded = (sizes + align - 1) // align * align
    offsets = np.zeros(n, dtype=np.int64)
    offsets[1:] = np.cumsum(padded)[:-1]
    return sizes.astype(np.int64), offsets, seeds.astype(np.uint64), dup_of
