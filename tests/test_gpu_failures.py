"""Failure paths without faulting the GPU: an allocator that fails, the torch
caching allocator as scratch source, and a producer that stalls in serving."""

import threading
import time

import numpy as np
import pytest
import torch

from synth import content

pytestmark = pytest.mark.gpu


def test_failing_allocator_reports_oom(cuda_ok):
    import paper_2601_12713_b300 as odp

    t = torch.ones(1 << 20, dtype=torch.uint8, device="cuda")
    calls = []
    try:
        odp.set_allocator(lambda nbytes, stream: calls.append(nbytes) or 0, lambda p, s: None)
        with pytest.raises(odp.OdpError) as e:
            odp.fingerprint_tensors([t[:1000], t[:5000]])
        assert e.value.status == -3 and calls
    finally:
        odp.set_allocator(None, None)
    out = odp.fingerprint_tensors([t[:1000], t[:5000]])  # default allocator works again
    assert out.shape == (2, 2)


def test_torch_allocator_gives_same_results(cuda_ok, orc):
    import paper_2601_12713_b300 as odp
    from synth import gpu, traces

    t = torch.empty(3 << 20, dtype=torch.uint8, device="cuda")
    gpu.fill(t, content.RANDOM, 4)
    views = [t[:100], t[7:1 << 20], t[:3 << 20]]
    ref = odp.fingerprint_tensors(views).cpu()
    b = traces.listing2(5)
    traces.fill_fp_from_content(b)
    ev = torch.from_numpy(b.events.view(np.uint8).reshape(-1).copy()).cuda()
    try:
        odp.set_torch_allocator()
        assert torch.equal(odp.fingerprint_tensors(views).cpu(), ref)
        out = odp.Findings(64)
        odp.analyze(ev, b.events.size, out)
        r = out.to_host()
        assert r["count"] == orc.analyze(b.events).count
    finally:
        odp.set_allocator(None, None)


def test_stalled_producer_does_not_block_serving(cuda_ok):
    """A thread that attaches and never submits holds the merge only for the
    watermark timeout; the other producers' events are processed without a
    flush."""
    import paper_2601_12713_b300 as odp
    from synth import gpu, load

    pool = torch.empty(16 << 20, dtype=torch.uint8, device="cuda")
    gpu.fill(pool, content.RANDOM, 8)
    torch.cuda.synchronize()
    srv = odp.Server(n_slots=2, max_events=1 << 18, max_batch_events=1024,
                     device_budget_bytes=2 << 30, watermark_timeout_us=100_000)
    stop = threading.Event()

    def stalled():
        srv.attach(0)
        stop.wait(30)

    th = threading.Thread(target=stalled)
    th.start()
    lg = load.Load(4, 8000, 1.0, 3, pool.data_ptr(), 16 << 20, 256, 1 << 16)
    try:
        time.sleep(0.05)
        n = lg.run(srv)
        deadline = time.time() + 10
        while time.time() < deadline and srv.stats()["events_processed"] < n:
            time.sleep(0.02)
        s = srv.stats()
        assert s["events_processed"] == n, s
        srv.flush()
    finally:
        stop.set()
        th.join()
        srv.close()
        lg.close()


def test_scan_lookback_wait_is_bounded(cuda_ok, tmp_path):
    """The scan's look-back waits on status words of earlier tiles with a
    bounded poll count.  A hook (tests/hooks/scan_timeout.cu) starts the tile
    counter past tile 0, so the wait can only run out: the kernel ends, the
    fault word is set (odp_analyze reports it as ODP_ERR_TIMEOUT), and a
    normal scan right after is correct."""
    import ctypes
    import os
    import shutil
    import subprocess

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = str(tmp_path / "libscan_timeout.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                    "-Xcompiler", "-fPIC", "-I", os.path.join(root, "include"),
                    "-I", os.path.join(root, "paper_2601_12713_b300", "csrc"),
                    os.path.join(root, "tests", "hooks", "scan_timeout.cu"), "-o", so],
                   check=True)
    lib = ctypes.CDLL(so)
    fault, correct = ctypes.c_uint32(0), ctypes.c_uint32(0)
    assert lib.scan_timeout_case(ctypes.byref(fault), ctypes.byref(correct)) == 0
    assert fault.value == 1
    assert correct.value == 1


def test_bulk_copy_wait_is_bounded(cuda_ok, tmp_path):
    """The fingerprint kernel's waits for its bulk chunk copies are bounded in
    time.  The test builds the library's fingerprint sources with each ring
    slot's mbarrier expecting 8,192 bytes per 4,096-byte chunk copy, so no
    phase can complete and every wait runs out with nothing left in flight.
    The calls (batched and single-buffer) must end within seconds and report
    ODP_ERR_TIMEOUT; the same library's register-load path must then give
    correct fingerprints with a clean status, so no tree or tile counter was
    left set by the abandoned tiles."""
    import ctypes
    import os
    import shutil
    import subprocess
    import time

    import paper_2601_12713_b300 as odp
    from paper_2601_12713_b300._lib import FpSchedule
    from synth import gpu

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_2601_12713_b300", "csrc")
    so = str(tmp_path / "libodp_ring_hook.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-shared", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                    "-Xlinker", "-Bsymbolic", "-DODP_RING_TX_BYTES=8192u",
                    "-I", os.path.join(root, "include"), "-I", csrc,
                    *(os.path.join(csrc, f) for f in ("fingerprint.cu", "runtime.cu",
                                                      "autotune.cu")),
                    "-o", so], check=True)
    hook = ctypes.CDLL(so)
    vp = ctypes.c_void_p
    hook.odp_fingerprint_with.argtypes = [ctypes.POINTER(FpSchedule), vp, vp, ctypes.c_uint64,
                                          vp, vp]
    hook.odp_fingerprint_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]

    t = torch.empty((3 << 20) + 8192, dtype=torch.uint8, device="cuda")
    gpu.fill(t, content.RANDOM, 21)
    stream = torch.cuda.current_stream().cuda_stream

    def case(views):
        ptrs = torch.tensor([v.data_ptr() for v in views], dtype=torch.int64, device="cuda")
        sizes = torch.tensor([v.numel() for v in views], dtype=torch.int64, device="cuda")
        want = torch.empty((len(views), 2), dtype=torch.int64, device="cuda")
        odp.fingerprint(ptrs, sizes, want)
        return ptrs, sizes, want

    def run(schedule, ptrs, sizes):
        out = torch.full((ptrs.numel(), 2), -1, dtype=torch.int64, device="cuda")
        rc = hook.odp_fingerprint_with(ctypes.byref(schedule), ptrs.data_ptr(), sizes.data_ptr(),
                                       ptrs.numel(), out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        st = ctypes.c_int32(0)
        assert hook.odp_fingerprint_status(stream, ctypes.byref(st)) == 0
        return out, st.value

    ring, regs = FpSchedule(8, 0, 2, 2), FpSchedule(8, 0, 2, 0)
    for views in ([t[:2 << 20], t[4096:4096 + (1 << 20) + 100]], [t[8192:8192 + (3 << 20)]]):
        ptrs, sizes, want = case(views)
        t0 = time.monotonic()
        _, status = run(ring, ptrs, sizes)
        assert time.monotonic() - t0 < 20
        assert status == -4  # ODP_ERR_TIMEOUT
        for _ in range(2):
            out, status = run(regs, ptrs, sizes)
            assert status == 0
            assert torch.equal(out, want)
