"""GPU parity of odp_fingerprint against the oracle's FP128 (bit-exact).

Calls go through the C ABI (ctypes binding); inputs are seeded synthetic
contents materialised on the device by the fill kernels and, for the oracle,
copied back or regenerated on the host.
"""

import numpy as np
import pytest
import torch

from synth import content

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def odp():
    import paper_2601_12713_b300 as odp

    return odp


def dev_buffer(nbytes, variant=content.RANDOM, seed=1, pad=64):
    from synth import gpu

    t = torch.zeros(nbytes + pad, dtype=torch.uint8, device="cuda")
    if nbytes:
        gpu.fill(t, variant, seed, nbytes=nbytes)
    return t


def gpu_fp(odp, views):
    out = odp.fingerprint_tensors(views)
    torch.cuda.synchronize()
    return [tuple(int(v) & ((1 << 64) - 1) for v in row) for row in out.cpu().tolist()]


SIZES = [1, 2, 15, 16, 17, 31, 100, 511, 512, 4095, 4096, 4097, 8191, 8192, 12293,
         32 * 4096 - 1, 32 * 4096, 32 * 4096 + 1, 33 * 4096 + 17, (1 << 20) + 3, 5 << 20]


@pytest.mark.parametrize("size", SIZES)
@pytest.mark.parametrize("variant", [content.RANDOM, content.ZERO, content.PAGE])
def test_single_buffer_matches_oracle(cuda_ok, orc, odp, size, variant):
    t = dev_buffer(size, variant, seed=size)
    host = t[:size].cpu().numpy()
    assert np.array_equal(host, content.bytes_of(variant, size, size))
    assert gpu_fp(odp, [t[:size]]) == [orc.fp128(host)]


@pytest.mark.parametrize("off", list(range(1, 16)))
def test_misaligned_views(cuda_ok, orc, odp, off):
    size = 3 * 4096 + 77
    t = dev_buffer(size + 32, seed=99 + off)
    v = t[off:off + size]
    assert gpu_fp(odp, [v]) == [orc.fp128(v.cpu().numpy())]


def test_empty_and_zero_sized(cuda_ok, orc, odp):
    t = dev_buffer(100)
    assert gpu_fp(odp, [t[:0]]) == [orc.fp128(b"")]
    # n == 0 is a no-op
    z = torch.empty(0, dtype=torch.int64, device="cuda")
    odp.fingerprint(z, z, torch.empty((0, 2), dtype=torch.int64, device="cuda"))


def test_ragged_batch_mixed_alignment(cuda_ok, orc, odp):
    rng = np.random.default_rng(5)
    n = 3000
    sizes = np.concatenate([rng.integers(0, 300, n // 3), rng.integers(1, 70_000, n // 3),
                            rng.integers(4000, 4200, n - 2 * (n // 3))])
    rng.shuffle(sizes)
    offs = np.zeros(n, dtype=np.int64)
    cur = 0
    for i in range(n):
        cur += int(rng.integers(0, 16))       # arbitrary byte alignment
        offs[i] = cur
        cur += int(sizes[i])
    arena = dev_buffer(cur + 64, seed=7)
    host = arena.cpu().numpy()
    views = [arena[o:o + s] for o, s in zip(offs, sizes)]
    got = gpu_fp(odp, views)
    want = orc.fp128_many(host, offs, sizes)
    assert got == [(int(a), int(b)) for a, b in want]


def test_duplicates_and_aliases(cuda_ok, orc, odp):
    t = dev_buffer(200_000, seed=3)
    views = [t[:100_000], t[:100_000], t[5:100_005], t[:0], t[:100_000]]
    got = gpu_fp(odp, views)
    assert got[0] == got[1] == got[4]
    assert got[2] != got[0]
    assert got == [orc.fp128(v.cpu().numpy()) for v in views]


def test_large_batch_multiblock_plan(cuda_ok, orc, odp):
    # more buffers than the single-block plan handles
    rng = np.random.default_rng(8)
    n = 20_000
    sizes = rng.integers(0, 9000, n)
    offs = np.concatenate([[0], np.cumsum((sizes + 15) // 16 * 16)[:-1]])
    arena = dev_buffer(int(offs[-1] + sizes[-1]) + 64, seed=11)
    host = arena.cpu().numpy()
    ptrs = torch.tensor(arena.data_ptr() + offs, dtype=torch.int64, device="cuda")
    sz = torch.tensor(sizes, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    odp.fingerprint(ptrs, sz, out)
    got = out.cpu().numpy().view(np.uint64)
    want = orc.fp128_many(host, offs, sizes)
    assert np.array_equal(got, want)


def test_null_pointer_reports_status(cuda_ok, odp):
    ptrs = torch.zeros(2, dtype=torch.int64, device="cuda")
    sizes = torch.tensor([0, 10], dtype=torch.int64, device="cuda")
    out = torch.full((2, 2), 7, dtype=torch.int64, device="cuda")
    odp.fingerprint(ptrs, sizes, out)
    assert odp.fingerprint_status() == -1
    assert out[1].tolist() == [0, 0]
    assert odp.fingerprint_status() == 0


@pytest.mark.parametrize("variant", [content.ZERO, content.PAGE, content.RANDOM])
def test_sweep_sizes_16mib_and_up(cuda_ok, orc, odp, variant):
    """The bandwidth sweep's sizes from 16 MiB up, one buffer per call as
    benchmarked: zero and page contents at every size to 4 GiB, random bytes
    to 1 GiB (4 GiB of random bytes has a test of its own)."""
    import concurrent.futures

    top = 4 << 30 if variant != content.RANDOM else 1 << 30
    size = 16 << 20
    cases = []
    while size <= top:
        t = dev_buffer(size, variant, seed=0x0DB2 + size.bit_length(), pad=0)
        got = gpu_fp(odp, [t])[0]
        host = t.cpu().numpy()
        del t
        torch.cuda.empty_cache()
        cases.append((size, got, host))
        size *= 4
    with concurrent.futures.ThreadPoolExecutor(len(cases)) as ex:
        wants = list(ex.map(lambda c: orc.fp128(c[2]), cases))
    for (size, got, _), want in zip(cases, wants):
        assert got == want, size


def test_full_size_4gib_buffer(cuda_ok, orc, odp):
    """The bandwidth sweep's largest buffer (4 GiB, random bytes) in the launch
    configuration the benchmark times, checked against the oracle."""
    size = 4 << 30
    t = dev_buffer(size, seed=0x0DB2, pad=0)
    got = gpu_fp(odp, [t])
    host = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    assert got == [orc.fp128(host)]


def oracle_all_cores(orc, host, offs, sizes):
    """The oracle's FP128 of every buffer, split over the host's cores (the
    oracle call releases the interpreter lock)."""
    import concurrent.futures
    import os

    n = sizes.size
    parts = np.array_split(np.arange(n), max(1, 4 * (os.cpu_count() or 1)))
    want = np.zeros((n, 2), dtype=np.uint64)

    def run(idx):
        if idx.size:
            want[idx] = orc.fp128_many(host, offs[idx], sizes[idx])

    with concurrent.futures.ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        list(ex.map(run, parts))
    return want


def test_full_scale_batched_ragged(cuda_ok, orc, odp):
    """The 10^6-buffer, 16 GiB ragged batch in one call (as benchmarked):
    every buffer equals the oracle (the arena's bytes copied to the host and
    hashed on all host cores), duplicates share fingerprints, and distinct
    contents get distinct fingerprints."""
    from synth import gpu

    sizes, offs, seeds, dup_of = content.batched_ragged(seed=0x0DB3)
    n = sizes.size
    arena = torch.empty(int(offs[-1] + sizes[-1]) + 64, dtype=torch.uint8, device="cuda")
    gpu.fill_many(arena, offs, sizes, seeds)
    ptrs = torch.from_numpy(arena.data_ptr() + offs).cuda()
    sz = torch.from_numpy(sizes).cuda()
    out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    odp.fingerprint(ptrs, sz, out)
    fps = out.cpu().numpy().view(np.uint64)
    host = arena.cpu().numpy()
    del arena
    torch.cuda.empty_cache()
    rng = np.random.default_rng(99)
    for i in np.concatenate([rng.choice(n, 50, replace=False), np.argsort(sizes)[-2:]]):
        data = content.bytes_of(content.RANDOM, int(seeds[i]), int(sizes[i]))
        assert np.array_equal(host[offs[i]:offs[i] + sizes[i]], data), i
    want = oracle_all_cores(orc, host, offs, sizes)
    del host
    bad = np.flatnonzero((fps != want).any(axis=1))
    assert bad.size == 0, f"{bad.size} buffers differ, first {bad[:5]}"
    d = np.flatnonzero(dup_of >= 0)
    assert np.array_equal(fps[d], fps[dup_of[d]])
    orig = fps[dup_of < 0]
    assert np.unique(orig, axis=0).shape[0] == orig.shape[0]


def test_fingerprint_one_equals_batched_call(cuda_ok, orc, odp):
    """odp_fingerprint_one (host-side pointer and size, launch sized to the
    buffer) gives the same fingerprints as odp_fingerprint, for sizes from 0
    to 256 MiB and start offsets that break 16-byte alignment."""
    big = dev_buffer((256 << 20) + 64, seed=0x0DB7, pad=0)
    out1 = torch.empty(2, dtype=torch.int64, device="cuda")
    for size in (0, 1, 15, 16, 17, 4095, 4096, 4097, 65536, (1 << 20) + 7, (64 << 20) + 13,
                 256 << 20):
        for off in (0, 1, 16, 4099):
            if off + size > big.numel():
                continue
            ptr = big.data_ptr() + off
            odp.fingerprint_one(ptr, size, out1)
            ptrs = torch.tensor([ptr], dtype=torch.int64, device="cuda")
            sizes = torch.tensor([size], dtype=torch.int64, device="cuda")
            out = torch.empty((1, 2), dtype=torch.int64, device="cuda")
            odp.fingerprint(ptrs, sizes, out)
            assert out1.tolist() == out[0].tolist(), (size, off)
            if size <= (1 << 20) + 7 and off in (0, 1):
                host = big[off:off + size].cpu().numpy()
                got = tuple(int(x) for x in out1.cpu().numpy().view(np.uint64))
                assert got == orc.fp128(host), (size, off)
    assert odp.fingerprint_status() == 0
    odp.fingerprint_one(0, 10, out1)  # null pointer with bytes: zero and a status
    assert odp.fingerprint_status() == -1
    assert out1.tolist() == [0, 0]


def test_reference_vectors(cuda_ok, odp):
    """The GPU reproduces the reference vectors of tests/golden (written by the
    oracle), each buffer alone and all of them in one batched call."""
    import sys

    sys.path.insert(0, __import__("os").path.dirname(__file__))
    from test_oracle_fp128 import load_vectors

    vecs = load_vectors()
    bufs = []
    for _, data, _ in vecs:
        t = torch.zeros(len(data) + 64, dtype=torch.uint8, device="cuda")
        if data:
            t[: len(data)] = torch.frombuffer(bytearray(data), dtype=torch.uint8).cuda()
        bufs.append(t[: len(data)])
    want = [w for _, _, w in vecs]
    assert gpu_fp(odp, bufs) == want
    for b, w in zip(bufs, want):
        assert gpu_fp(odp, [b]) == [w]


def test_worked_examples(cuda_ok, odp):
    """The GPU reproduces the FP128 v1 worked examples of tests/golden (each
    step of which the CPU tests check against the definition by inversion),
    alone, in one batch, and at an odd start address."""
    import sys

    sys.path.insert(0, __import__("os").path.dirname(__file__))
    from test_oracle_fp128_lanes import WORKED_NAMES, load_worked, worked_input

    _, ex = load_worked()
    t = torch.zeros(3 * 8192, dtype=torch.uint8, device="cuda")
    views, want = [], []
    for k, name in enumerate(WORKED_NAMES):
        data = worked_input(name)
        for off in (8192 * (k % 3), 8192 * (k % 3) + 4097):
            if off + len(data) > t.numel():
                continue
            if data:
                t[off:off + len(data)] = torch.frombuffer(bytearray(data), dtype=torch.uint8).cuda()
            v = t[off:off + len(data)]
            assert gpu_fp(odp, [v]) == [ex[name]["out"]], (name, off)
            views.append(v.clone())
            want.append(ex[name]["out"])
    assert gpu_fp(odp, views) == want


def test_fingerprint_log_fills_transfer_records(cuda_ok, orc, odp):
    """odp_fingerprint_log over the plain-small trace: every transfer record
    gets the oracle's fingerprint of its payload (payloads packed at mixed
    alignments), every other record is left byte for byte unchanged, and a
    second call over the filled log changes nothing."""
    from synth import gpu, traces

    b = traces.plain_small()
    ev = b.events.copy()
    ev["fp_lo"] = 0x1111
    ev["fp_hi"] = 0x2222
    n = ev.size
    xfer = np.flatnonzero(np.isin(ev["kind"], [2, 3, 4]))
    sizes = ev["bytes"][xfer].astype(np.int64)
    rng = np.random.default_rng(3)
    offs = np.zeros(xfer.size, dtype=np.int64)
    cur = 0
    for k in range(xfer.size):
        cur += int(rng.integers(0, 16)) * 16 + (k % 3)  # some starts off 16-byte boundaries
        offs[k] = cur
        cur += int(sizes[k])
    arena = torch.empty(cur + 64, dtype=torch.uint8, device="cuda")
    gpu.fill_many(arena, offs, sizes, b.payload_seed[xfer].astype(np.uint64))
    ptrs = np.zeros(n, dtype=np.int64)
    ptrs[xfer] = arena.data_ptr() + offs
    d_ptrs = torch.from_numpy(ptrs).cuda()
    d_ev = torch.from_numpy(ev.view(np.uint8).reshape(-1).copy()).cuda()
    odp.fingerprint_log(d_ev, n, d_ptrs)
    got = d_ev.cpu().numpy().view(traces.EVENT_DTYPE)
    assert odp.fingerprint_status() == 0
    host = arena.cpu().numpy()
    want = orc.fp128_many(host, offs, sizes)
    assert np.array_equal(got["fp_lo"][xfer], want[:, 0])
    assert np.array_equal(got["fp_hi"][xfer], want[:, 1])
    other = np.setdiff1d(np.arange(n), xfer)
    assert np.array_equal(got[other].view(np.uint8), ev[other].view(np.uint8))
    keep = ev.copy()
    keep["fp_lo"][xfer], keep["fp_hi"][xfer] = want[:, 0], want[:, 1]
    assert np.array_equal(got.view(np.uint8), keep.view(np.uint8))
    odp.fingerprint_log(d_ev, n, d_ptrs)
    assert np.array_equal(d_ev.cpu().numpy(), keep.view(np.uint8).reshape(-1))
    with pytest.raises(odp.OdpError):
        odp.fingerprint_log(d_ev[4:], n - 1, d_ptrs)  # records not 8-byte aligned


def test_batch_with_large_buffers_in_multiblock_plan(cuda_ok, orc, odp):
    """More than 8,192 buffers (the multi-block plan), some of them large
    enough for many tiles each: their tile lists are written by the plan's
    per-buffer pass and its warp-per-buffer pass; every fingerprint equals the
    oracle's."""
    rng = np.random.default_rng(21)
    n = 12_000
    sizes = rng.integers(0, 20_000, n)
    big = rng.choice(n, 40, replace=False)
    sizes[big] = rng.integers(1 << 20, 24 << 20, big.size)  # 256..6,144 chunks
    offs = np.concatenate([[0], np.cumsum((sizes + 15) // 16 * 16)[:-1]])
    arena = dev_buffer(int(offs[-1] + sizes[-1]) + 64, seed=23)
    host = arena.cpu().numpy()
    ptrs = torch.tensor(arena.data_ptr() + offs, dtype=torch.int64, device="cuda")
    sz = torch.tensor(sizes, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    for schedule in [(8, 0, 1, 0), (8, 0, 16, 2), (4, 0, 2, 0)]:
        out.fill_(-1)
        odp.fingerprint_with(schedule, ptrs, sz, out)
        got = out.cpu().numpy().view(np.uint64)
        want = orc.fp128_many(host, offs, sizes)
        assert np.array_equal(got, want), schedule


def test_fingerprint_log_null_payload(cuda_ok, odp):
    """A transfer record whose payload pointer is null gets {0, 0} and
    ODP_ERR_INVALID_ARG in the status word; the other transfers are hashed."""
    from synth import traces

    b = traces.listing2(3)
    ev = b.events.copy()
    n = ev.size
    xfer = np.flatnonzero(np.isin(ev["kind"], [2, 3, 4]))
    t = dev_buffer(8192, seed=5)
    ptrs = np.zeros(n, dtype=np.int64)
    ptrs[xfer] = t.data_ptr()
    ptrs[xfer[1]] = 0
    d_ev = torch.from_numpy(ev.view(np.uint8).reshape(-1).copy()).cuda()
    odp.fingerprint_log(d_ev, n, torch.from_numpy(ptrs).cuda())
    got = d_ev.cpu().numpy().view(traces.EVENT_DTYPE)
    assert odp.fingerprint_status() == -1
    assert got["fp_lo"][xfer[1]] == 0 and got["fp_hi"][xfer[1]] == 0
    same = gpu_fp(odp, [t[:int(ev["bytes"][xfer[0]])]])[0]
    assert (int(got["fp_lo"][xfer[0]]), int(got["fp_hi"][xfer[0]])) == same
