"""Every launch schedule (and the autotuner's choice) gives the oracle's
fingerprints bit for bit (GPU, through the C ABI)."""

import itertools

import numpy as np
import pytest
import torch

from synth import content

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def odp():
    import paper_2601_12713_b300 as odp

    return odp


@pytest.fixture(scope="module")
def batch(orc):
    from synth import gpu

    rng = np.random.default_rng(31)
    n = 2500
    sizes = np.concatenate([rng.integers(0, 5000, n - 6),
                            [0, 1, 4097, 32 * 4096 + 1, 40 << 20, (24 << 20) + 7]])
    offs = np.zeros(n, dtype=np.int64)
    cur = 0
    for i in range(n):
        cur += int(rng.integers(0, 16))
        offs[i] = cur
        cur += int(sizes[i])
    arena = torch.empty(cur + 64, dtype=torch.uint8, device="cuda")
    gpu.fill(arena, content.RANDOM, 77)
    want = orc.fp128_many(arena.cpu().numpy(), offs, sizes)
    ptrs = torch.tensor(arena.data_ptr() + offs, dtype=torch.int64, device="cuda")
    sz = torch.tensor(sizes, dtype=torch.int64, device="cuda")
    return arena, ptrs, sz, want


SCHEDULES = [s for s in itertools.product((4, 8, 16), (0, 1, 3), (1, 2, 4, 16), (0, 2, 4))
             if not (s[0] == 16 and s[3] == 4)]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_schedule_invariance_batch(cuda_ok, odp, batch, sched):
    arena, ptrs, sizes, want = batch
    out = torch.empty((ptrs.numel(), 2), dtype=torch.int64, device="cuda")
    odp.fingerprint_with(sched, ptrs, sizes, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)


@pytest.mark.parametrize("sched", [(4, 0, 1), (8, 1, 2), (16, 0, 64), (8, 0, 1 << 20),
                                   (4, 0, 1, 4), (8, 0, 2, 2), (16, 0, 8, 2), (8, 0, 1 << 20, 4)])
def test_schedule_invariance_single_buffer(cuda_ok, orc, odp, sched):
    from synth import gpu

    size = (96 << 20) + 12345
    t = torch.empty(size, dtype=torch.uint8, device="cuda")
    gpu.fill(t, content.RANDOM, 5)
    ptrs = torch.tensor([t.data_ptr()], dtype=torch.int64, device="cuda")
    sz = torch.tensor([size], dtype=torch.int64, device="cuda")
    out = torch.empty((1, 2), dtype=torch.int64, device="cuda")
    odp.fingerprint_with(sched, ptrs, sz, out)
    assert tuple(out.cpu().numpy().view(np.uint64)[0]) == orc.fp128(t.cpu().numpy())


def test_autotune_keeps_results(cuda_ok, odp, batch):
    arena, ptrs, sizes, want = batch
    out = torch.empty((ptrs.numel(), 2), dtype=torch.int64, device="cuda")
    sched, ms = odp.autotune_fingerprint(ptrs, sizes, out, reps=2)
    assert sched[0] in (4, 8, 16) and ms > 0
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    out.zero_()
    odp.fingerprint(ptrs, sizes, out)  # now uses the tuned schedule
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    odp.autotune_clear()


def test_invalid_schedule_rejected(cuda_ok, odp, batch):
    arena, ptrs, sizes, want = batch
    out = torch.empty((ptrs.numel(), 2), dtype=torch.int64, device="cuda")
    with pytest.raises(odp.OdpError):
        odp.fingerprint_with((5, 0, 1), ptrs, sizes, out)
    with pytest.raises(odp.OdpError):
        odp.fingerprint_with((8, 0, 0), ptrs, sizes, out)
    with pytest.raises(odp.OdpError):
        odp.fingerprint_with((8, 0, 1, 3), ptrs, sizes, out)
    with pytest.raises(odp.OdpError):
        odp.fingerprint_with((16, 0, 1, 4), ptrs, sizes, out)


def test_repeated_calls_reset_counters(cuda_ok, orc, odp):
    """Tree counters reset themselves: many calls of changing shapes on one
    stream keep giving the oracle's values."""
    from synth import gpu

    arena = torch.empty(200 << 20, dtype=torch.uint8, device="cuda")
    gpu.fill(arena, content.RANDOM, 9)
    host = arena.cpu().numpy()
    rng = np.random.default_rng(4)
    for it in range(12):
        n = int(rng.integers(1, 40))
        sizes = rng.integers(0, 6 << 20, n)
        offs = rng.integers(0, (200 << 20) - (6 << 20), n)
        ptrs = torch.tensor(arena.data_ptr() + offs, dtype=torch.int64, device="cuda")
        sz = torch.tensor(sizes, dtype=torch.int64, device="cuda")
        out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
        odp.fingerprint(ptrs, sz, out)
        assert np.array_equal(out.cpu().numpy().view(np.uint64),
                              orc.fp128_many(host, offs, sizes)), it


def test_batch_size_changes_on_one_stream(cuda_ok, orc, odp):
    """A large batch (long tile list) followed by single-buffer and small-batch
    calls on the same stream: the tree counters of every call start at zero."""
    from synth import gpu

    arena = torch.empty(96 << 20, dtype=torch.uint8, device="cuda")
    gpu.fill(arena, content.RANDOM, 21)
    host = arena.cpu().numpy()
    n = 300_000
    offs = np.arange(n, dtype=np.int64) * 112
    sizes = np.full(n, 100, dtype=np.int64)
    ptrs = torch.tensor(arena.data_ptr() + offs, dtype=torch.int64, device="cuda")
    sz = torch.tensor(sizes, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    odp.fingerprint(ptrs, sz, out)
    sample = np.arange(0, n, 997)
    assert np.array_equal(out.cpu().numpy().view(np.uint64)[sample],
                          orc.fp128_many(host, offs[sample], sizes[sample]))
    for size in (4097, 33 * 4096, 200 * 4096 + 5, 5 << 20, 40 << 20):
        views = [arena[1024:1024 + size]]
        got = odp.fingerprint_tensors(views).cpu().numpy().view(np.uint64)[0]
        assert tuple(got) == orc.fp128(host[1024:1024 + size]), size
    offs2 = np.arange(50, dtype=np.int64) * (1 << 20)
    sizes2 = np.full(50, 700_001, dtype=np.int64)
    ptrs2 = torch.tensor(arena.data_ptr() + offs2, dtype=torch.int64, device="cuda")
    sz2 = torch.tensor(sizes2, dtype=torch.int64, device="cuda")
    out2 = torch.empty((50, 2), dtype=torch.int64, device="cuda")
    odp.fingerprint(ptrs2, sz2, out2)
    assert np.array_equal(out2.cpu().numpy().view(np.uint64), orc.fp128_many(host, offs2, sizes2))
