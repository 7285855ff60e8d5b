"""odp_fingerprint_noalloc against odp_fingerprint (GPU, through the C ABI).

The allocation-free entry point serves callers that cannot allocate device
memory when they need a fingerprint; it keeps its scratch in one fixed
device array shared by every call.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def batch(seed, n, max_size, big=None):
    """A ragged batch of views into one arena: any byte alignment, some empty
    buffers, optionally one large buffer appended."""
    from synth import content, gpu

    rng = np.random.default_rng(seed)
    sizes = rng.integers(0, max_size, n)
    sizes[rng.integers(0, n, max(1, n // 20))] = 0
    offs = np.zeros(n, dtype=np.int64)
    cur = 0
    for i in range(n):
        cur += int(rng.integers(0, 16))
        offs[i] = cur
        cur += int(sizes[i])
    total = cur + (big or 0) + 64
    arena = torch.empty(total, dtype=torch.uint8, device="cuda")
    gpu.fill(arena, content.RANDOM, seed)
    ptrs = list(arena.data_ptr() + offs)
    szs = list(sizes)
    if big:
        ptrs.append(arena.data_ptr() + cur + 16 - (cur % 16))
        szs.append(big - 16)
    d_ptrs = torch.tensor(ptrs, dtype=torch.int64, device="cuda")
    d_sizes = torch.tensor(szs, dtype=torch.int64, device="cuda")
    return arena, d_ptrs, d_sizes


def both(odp, d_ptrs, d_sizes):
    n = d_ptrs.numel()
    want = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    got = torch.full((n, 2), -1, dtype=torch.int64, device="cuda")
    odp.fingerprint(d_ptrs, d_sizes, want)
    odp.fingerprint_noalloc(d_ptrs, d_sizes, got)
    torch.cuda.synchronize()
    return got.cpu().numpy(), want.cpu().numpy()


def test_noalloc_matches_allocating_entry_point(cuda_ok):
    import paper_2601_12713_b300 as odp

    # two calls in a row with different batches: the shared array must not
    # carry anything from the first call into the second
    arena1, p1, s1 = batch(101, 1500, 90_000, big=96 << 20)
    got, want = both(odp, p1, s1)
    assert np.array_equal(got, want)
    arena2, p2, s2 = batch(202, 4096, 20_000)
    got, want = both(odp, p2, s2)
    assert np.array_equal(got, want)


def test_noalloc_rejects_too_many_buffers(cuda_ok):
    import paper_2601_12713_b300 as odp

    n = 4097
    p = torch.zeros(n, dtype=torch.int64, device="cuda")
    s = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(odp.OdpError) as e:
        odp.fingerprint_noalloc(p, s, out)
    assert e.value.status == -7


@pytest.mark.parametrize("big,n_small", [((3 << 30) + 12345, 300), ((6 << 30) + 777, 1)])
def test_noalloc_large_tiles_match(cuda_ok, big, n_small):
    """Batches large enough that the fixed array's tile capacity forces tiles
    of 64 or 128 chunks (the stack merge inside a tile and the climb over
    spans above 32 chunks), with chunk counts that are not powers of two.
    odp_fingerprint cuts the same buffers into tiles of at most 32 chunks, so
    equality checks the larger tiles' tree shape independently."""
    import paper_2601_12713_b300 as odp

    arena, p, s = batch(303 + n_small, n_small, 50_000, big=big + 16)
    assert int(s.sum()) > (5 << 29)
    got, want = both(odp, p, s)
    del arena
    torch.cuda.empty_cache()
    assert np.array_equal(got, want)


def test_noalloc_allocates_nothing(cuda_ok):
    """After one call on the device (which looks up the array's address),
    calls succeed with an allocator that refuses every request installed, and
    the device's free memory is the same before and after a call."""
    import paper_2601_12713_b300 as odp

    arena, p, s = batch(404, 2000, 40_000, big=8 << 20)
    n = p.numel()
    want = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    odp.fingerprint(p, s, want)
    got = torch.full((n, 2), -1, dtype=torch.int64, device="cuda")
    odp.fingerprint_noalloc(p, s, got)  # warm-up: address lookup, modules loaded
    torch.cuda.synchronize()
    calls = []
    try:
        odp.set_allocator(lambda nbytes, stream: calls.append(nbytes) or 0, lambda q, st: None)
        got.fill_(-1)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        odp.fingerprint_noalloc(p, s, got)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
    finally:
        odp.set_allocator(None, None)
    assert calls == []
    assert free0 == free1
    assert torch.equal(got, want)
