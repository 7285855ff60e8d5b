"""Serving loop (GPU, through the C ABI): producers on host threads, the
merged log, streamed findings against the offline analysis of the same log,
and every request's fingerprints alone versus in the mix."""

import numpy as np
import pytest
import torch

from synth import content

pytestmark = pytest.mark.gpu


def run_server(odp, n_threads, rate, seconds, n_slots, max_batch, seed, max_payload=1 << 20,
               announce=True):
    from synth import gpu, load

    pool_bytes = 64 << 20
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    gpu.fill(pool, content.RANDOM, seed)
    torch.cuda.synchronize()
    srv = odp.Server(n_slots=n_slots, max_events=1 << 20, max_batch_events=max_batch,
                     device_budget_bytes=4 << 30, watermark_timeout_us=200_000)
    lg = load.Load(n_threads, rate, seconds, seed, pool.data_ptr(), pool_bytes, 256, max_payload)
    n = lg.run(srv, announce=announce)
    assert n > 0
    srv.flush()
    return srv, lg, pool, n


def payload_views(srv, lg, ev):
    n = ev.size
    prod, seq = srv.origin(n)
    views = np.zeros((n, 2), dtype=np.int64)
    is_x = np.isin(ev["kind"], [2, 3, 4])
    for i in np.flatnonzero(is_x):
        k = lg.thread_of(ev["host_addr"][i])
        views[i] = lg.payload(k, int(seq[i]))
    return views, is_x


def sorted_findings(st):
    return st[np.lexsort((st["partner"], st["event"], st["kind"]))]


@pytest.mark.parametrize("n_slots,max_batch,announce", [(1, 512, False), (4, 2048, True),
                                                         (2, 256, True)])
def test_streamed_findings_equal_offline(cuda_ok, orc, n_slots, max_batch, announce):
    """Producers that stamp events themselves (the merge waits for each
    one's next event) or open them with begin (it waits only for open ones)."""
    import paper_2601_12713_b300 as odp

    srv, lg, pool, n = run_server(odp, 8, 20_000, 1.5, n_slots, max_batch, 5 + n_slots,
                                  announce=announce)
    try:
        ptr, m = srv.log()
        assert m == n
        log = odp.log_tensor(srv, n)
        ev = log.cpu().numpy().view(odp.EVENT_DTYPE).copy()
        assert np.all(np.diff(ev["t_start_ns"].astype(np.int64)) >= 0)
        # the full analysis of the merged log on the GPU equals the oracle
        out = odp.Findings(6 * n)
        odp.analyze(log, n, out)
        g = out.to_host()
        o = orc.analyze(ev)
        assert g["status"] == o.status == 0 and g["count"] == o.count
        assert np.array_equal(g["findings"].view(np.uint8), o.findings.view(np.uint8))
        # the streamed findings (all five kinds) are exactly the offline ones
        st = sorted_findings(srv.poll())
        off = g["findings"]
        assert st.size == off.size and st.size > 0
        assert np.array_equal(st.view(np.uint8), off.view(np.uint8))
        assert (st["kind"] == 3).sum() > 0
        # every transfer's fingerprint, alone, equals the one computed in the mix
        views, is_x = payload_views(srv, lg, ev)
        idx = np.flatnonzero(is_x)
        ptrs = torch.tensor(pool.data_ptr() + views[idx, 0], dtype=torch.int64, device="cuda")
        sizes = torch.tensor(views[idx, 1], dtype=torch.int64, device="cuda")
        alone = torch.empty((idx.size, 2), dtype=torch.int64, device="cuda")
        odp.fingerprint(ptrs, sizes, alone)
        mixed = np.stack([ev["fp_lo"][idx], ev["fp_hi"][idx]], axis=1)
        assert np.array_equal(alone.cpu().numpy().view(np.uint64), mixed)
        host_pool = pool.cpu().numpy()
        for j in idx[:: max(1, idx.size // 40)]:
            o_ = int(views[j, 0])
            assert orc.fp128(host_pool[o_:o_ + int(views[j, 1])]) == (int(ev["fp_lo"][j]),
                                                                       int(ev["fp_hi"][j]))
        s = srv.stats()
        assert s["events_processed"] == n and s["late_events"] == 0
        assert s["latency_p50_ns"] > 0 and s["latency_p99_ns"] >= s["latency_p50_ns"]
        assert s["rt_groups_at_flush"] == 0
    finally:
        srv.close()
        lg.close()


def kernel_event(odp, t):
    e = np.zeros(1, dtype=odp.EVENT_DTYPE)
    e["t_start_ns"], e["t_end_ns"], e["kind"], e["src_dev"], e["dst_dev"] = t, t + 10, 6, -1, 0
    return e


def test_begin_holds_the_merge_only_while_open(cuda_ok):
    """An open event holds back every later event of other threads until
    it is submitted; a thread with nothing open does not hold the merge; an
    event closed by cancel stops holding it; a thread that stamps its own
    events holds the merge at its last one."""
    import threading
    import time

    import paper_2601_12713_b300 as odp

    srv = odp.Server(n_slots=1, max_events=1 << 10, max_batch_events=64,
                     device_budget_bytes=1 << 30, watermark_timeout_us=30_000_000)
    none = np.zeros(1, dtype=np.uint64)

    def processed():
        return srv.stats()["events_processed"]

    def wait_processed(k, secs=10.0):
        t_end = time.time() + secs
        while processed() < k and time.time() < t_end:
            time.sleep(0.01)
        return processed()

    opened, go, done_a = threading.Event(), threading.Event(), threading.Event()
    t_a = {}

    def thread_a():
        t_a["t"] = srv.begin()
        opened.set()
        go.wait(30)
        srv.submit(kernel_event(odp, t_a["t"]), none)
        done_a.set()

    def thread_b(k):
        for _ in range(k):
            srv.submit(kernel_event(odp, srv.begin()), none)

    try:
        a = threading.Thread(target=thread_a)
        a.start()
        assert opened.wait(30)
        b = threading.Thread(target=thread_b, args=(8,))
        b.start()
        b.join()
        time.sleep(0.3)
        assert processed() == 0          # all of B's events start after A's open one
        go.set()
        a.join()
        assert wait_processed(9) == 9    # no flush: nothing is open any more
        # a cancelled event stops holding the merge
        c_open, c_go = threading.Event(), threading.Event()

        def thread_c():
            t = srv.begin()
            c_open.set()
            c_go.wait(30)
            srv.cancel(t)
            with pytest.raises(odp.OdpError):
                srv.cancel(t)            # no longer open

        c = threading.Thread(target=thread_c)
        c.start()
        assert c_open.wait(30)
        thread_b(4)
        time.sleep(0.3)
        assert processed() == 9
        c_go.set()
        c.join()
        assert wait_processed(13) == 13
        # a self-stamping thread holds the merge at its last start time (the
        # server's clock is the monotonic clock)
        t_d = time.monotonic_ns()
        d = threading.Thread(target=lambda: srv.submit(kernel_event(odp, t_d), none))
        d.start()
        d.join()
        assert wait_processed(14) == 14
        b2 = threading.Thread(target=thread_b, args=(3,))
        b2.start()
        b2.join()
        time.sleep(0.3)
        assert processed() == 14         # held at D's last start time
        srv.flush()
        assert processed() == 17
        st = srv.stats()
        assert st["late_events"] == 0
        log = odp.log_tensor(srv, 17).cpu().numpy().view(odp.EVENT_DTYPE)
        assert np.all(np.diff(log["t_start_ns"].astype(np.int64)) >= 0)
        assert int(log["t_start_ns"][0]) == t_a["t"]
    finally:
        srv.close()


def xfer_events(odp, n, t0, host0, host_step, nbytes=256):
    e = np.zeros(n, dtype=odp.EVENT_DTYPE)
    e["t_start_ns"] = t0 + 10 * np.arange(n)
    e["t_end_ns"] = e["t_start_ns"] + 5
    e["host_addr"] = host0 + host_step * np.arange(n)
    e["dev_addr"] = 0xA00
    e["bytes"] = nbytes
    e["kind"], e["src_dev"], e["dst_dev"] = 2, -1, 0
    return e


def test_batch_with_many_findings_and_overflow_report(cuda_ok, orc):
    """A one-event batch (a kernel) that decides 599 waiting unused
    transfers: its findings exceed the copy made with the batch and are
    fetched in full.  A server whose waiting lists are too small reports the
    decisions it could not keep."""
    import time

    import paper_2601_12713_b300 as odp

    pool = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    srv = odp.Server(n_slots=1, max_events=4096, max_batch_events=4096,
                     device_budget_bytes=2 << 30)
    try:
        srv.attach(0)
        x = xfer_events(odp, 600, 1000, 0xA000, 0)      # one host range, overwritten 599 times
        srv.submit(x, np.full(600, pool.data_ptr(), dtype=np.uint64))
        t_end = time.time() + 30
        while srv.stats()["events_processed"] < 600 and time.time() < t_end:
            time.sleep(0.01)
        assert srv.stats()["events_processed"] == 600
        srv.submit(kernel_event(odp, 1000 + 10 * 600 + 100), np.zeros(1, dtype=np.uint64))
        srv.flush()
        st = srv.stats()
        assert st["events_processed"] == 601 and st["batches"] >= 2
        assert st["stream_overflow"] == 0
        log = odp.log_tensor(srv, 601).cpu().numpy().view(odp.EVENT_DTYPE).copy()
        o = orc.analyze(log)
        assert (o.findings["kind"] == 5).sum() == 599
        got = sorted_findings(srv.poll())
        assert np.array_equal(got.view(np.uint8), o.findings.view(np.uint8))
    finally:
        srv.close()
    # 40 transfers to distinct ranges wait for a kernel; one-event batches
    # keep 16 waiting at most
    srv = odp.Server(n_slots=1, max_events=256, max_batch_events=1, device_budget_bytes=1 << 30)
    try:
        srv.attach(0)
        x = xfer_events(odp, 40, 1000, 0xB000, 0x1000)
        srv.submit(x, np.full(40, pool.data_ptr(), dtype=np.uint64))
        srv.flush()
        st = srv.stats()
        assert st["events_processed"] == 40
        assert st["stream_overflow"] == 40 - 16
    finally:
        srv.close()


def test_submit_argument_errors(cuda_ok):
    import paper_2601_12713_b300 as odp

    srv = odp.Server(n_slots=1, max_events=16, max_batch_events=8, device_budget_bytes=1 << 30)
    try:
        ev = np.zeros(20, dtype=odp.EVENT_DTYPE)
        with pytest.raises(odp.OdpError):
            srv.submit(ev, np.zeros(20, dtype=np.uint64))   # beyond the log capacity
        srv.flush()
        assert srv.log()[1] == 0
    finally:
        srv.close()


def pairs_trace():
    """One producer's events with explicit times (ns): allocations used by a
    kernel in the same or a later batch, unused ones (no kernel, or a kernel
    on another device), a repeated allocation, a kernel that starts while a
    delete runs, allocations never deleted (one covered by a later kernel),
    an unmatched delete, and to-device transfers between, during and after
    kernels on two devices."""
    from synth import traces

    T, rows = traces, []

    def ev(t0, t1, kind, dev=0, host=0, daddr=0, nbytes=0, site=0):
        src, dst = (-1, dev) if kind != T.FROM_DEV else (dev, -1)
        rows.append((t0, t1, host, daddr, nbytes, 0, 0, site, kind, src, dst, 0))

    t = 1000
    for i in range(6):                       # used: ALLOC, TO_DEV, KERNEL, FROM_DEV, DELETE
        ev(t, t + 5, T.ALLOC, 0, 0x1000, 0x100, 4096, 1)
        ev(t + 10, t + 20, T.TO_DEV, 0, 0x1000, 0x100, 4096, 2)
        ev(t + 30, t + 80, T.KERNEL, 0, site=3)
        ev(t + 90, t + 99, T.FROM_DEV, 0, 0x1000, 0x100, 4096, 4)
        ev(t + 100, t + 105, T.DELETE, 0, 0x1000, 0x100, 4096, 5)
        t += 200
    for i in range(4):                       # unused, repeated <host, dev, bytes>
        ev(t, t + 5, T.ALLOC, 0, 0x2000, 0x200, 8192, 6)
        ev(t + 10, t + 15, T.DELETE, 0, 0x2000, 0x200, 8192, 7)
        t += 50
    ev(t, t + 5, T.ALLOC, 1, 0x3000, 0x300, 64, 8)   # a kernel on device 0 only: unused
    ev(t + 10, t + 40, T.KERNEL, 0, site=9)
    ev(t + 50, t + 55, T.DELETE, 1, 0x3000, 0x300, 64, 10)
    t += 100
    ev(t, t + 5, T.ALLOC, 0, 0x4000, 0x400, 64, 11)   # a kernel starts while the delete runs
    ev(t + 10, t + 500, T.DELETE, 0, 0x4000, 0x400, 64, 12)
    ev(t + 20, t + 30, T.KERNEL, 0, site=13)
    t += 600
    ev(t, t + 5, T.DELETE, 0, 0x9000, 0x900, 64, 14)  # unmatched
    ev(t + 10, t + 15, T.ALLOC, 0, 0x5000, 0x500, 64, 15)  # never deleted, later kernel
    ev(t + 20, t + 25, T.ALLOC, 1, 0x6000, 0x600, 64, 16)  # never deleted, no kernel on 1
    ev(t + 30, t + 90, T.KERNEL, 0, site=17)
    t += 100
    for i in range(5):                       # more unused allocations, same key
        ev(t, t + 5, T.ALLOC, 1, 0x7000, 0x700, 128, 18)
        ev(t + 10, t + 15, T.DELETE, 1, 0x7000, 0x700, 128, 19)
        t += 30
    # unused transfers: overwritten before the next kernel, a transfer during
    # a kernel (barrier), one that starts with the next kernel (barrier), and
    # transfers after the last kernel of their device
    for i in range(3):
        ev(t, t + 50, T.KERNEL, 0, site=20)
        ev(t + 60, t + 65, T.TO_DEV, 0, 0xA000, 0xA00, 256, 21)
        ev(t + 70, t + 75, T.TO_DEV, 0, 0xA000, 0xA00, 256, 22)
        ev(t + 80, t + 85, T.TO_DEV, 0, 0xB000, 0xB00, 256, 23)
        ev(t + 90, t + 95, T.TO_DEV, 1, 0xA000, 0xA00, 256, 24)
        ev(t + 100, t + 150, T.KERNEL, 0, site=25)
        ev(t + 120, t + 125, T.TO_DEV, 0, 0xA000, 0xA00, 256, 26)
        ev(t + 200, t + 205, T.TO_DEV, 0, 0xA000, 0xA00, 256, 27)
        ev(t + 300, t + 305, T.TO_DEV, 0, 0xA000, 0xA00, 256, 28)
        ev(t + 300, t + 350, T.KERNEL, 0, site=29)
        t += 400
    for i in range(3):
        ev(t, t + 5, T.TO_DEV, 0, 0xC000, 0xC00, 512, 30)
        ev(t + 10, t + 15, T.TO_DEV, 1, 0xC000, 0xC00, 512, 31)
        t += 20
    return np.array(rows, dtype=T.EVENT_DTYPE)


def kernel_heavy_trace(seed, n_cycles=800):
    """Allocation cycles on three devices (ALLOC, one or two TO_DEV of the
    same host range, DELETE) among kernels of random length on random
    devices, many of them overlapping several cycles; contents repeat, so
    duplicates and overwritten transfers occur.  Cycles of one <host, device,
    bytes> key never overlap, and content goes only from the host to one
    device."""
    from synth import traces as T

    rng = np.random.default_rng(seed)
    rows, t = [], 1000
    for c in range(n_cycles):
        dev, key = int(rng.integers(0, 3)), c % 40
        host, daddr, nbytes = 0x10000 + key * 0x1000, 0x100 * (key + 1), 256 * (1 + key % 3)
        site = int(rng.integers(0, 32))
        d_end = t + int(rng.integers(60, 400))
        rows.append((t, t + 5, host, daddr, nbytes, 0, 0, site, T.ALLOC, -1, dev, 0))
        for j in range(int(rng.integers(1, 3))):
            t1 = t + 10 + 20 * j
            content = int(rng.integers(0, 6)) * 16 + dev
            rows.append((t1, t1 + 5, host, daddr, nbytes, content + 1, 0, site, T.TO_DEV, -1, dev, 0))
        if rng.random() < 0.6:
            k0 = t + int(rng.integers(0, 300))
            kd = int(rng.integers(0, 3))
            rows.append((k0, k0 + int(rng.integers(1, 3000)), 0, 0, 0, 0, 0, site, T.KERNEL, -1, kd, 0))
        rows.append((d_end, d_end + 5, host, daddr, nbytes, 0, 0, site, T.DELETE, -1, dev, 0))
        t += int(rng.integers(20, 200))
    ev = np.array(rows, dtype=T.EVENT_DTYPE)
    ev = ev[np.argsort(ev["t_start_ns"], kind="stable")]
    ev["flags"] = np.where(np.isin(ev["kind"], [2, 3, 4]), 1, 0)  # fingerprints given
    return ev


@pytest.mark.parametrize("max_batch", [64, 4096, 16384])
def test_streamed_kernel_heavy_batches_equal_offline(cuda_ok, orc, max_batch):
    """Batches holding hundreds of kernels on three devices (the per-device
    kernel index of a batch) stream the same findings as the offline
    analysis."""
    import paper_2601_12713_b300 as odp

    # 16384-event batches sort with the multi-pass radix sort inside the graph
    ev = kernel_heavy_trace(11, n_cycles=800 if max_batch < 16384 else 3600)
    srv = odp.Server(n_slots=2, max_events=1 << 15, max_batch_events=max_batch,
                     device_budget_bytes=2 << 30)
    try:
        srv.attach(0)
        srv.submit(ev, np.zeros(ev.size, dtype=np.uint64))
        srv.flush()
        st = srv.stats()
        assert st["events_processed"] == ev.size
        assert st["stream_overflow"] == 0 and st["rt_groups_at_flush"] == 0
        log = odp.log_tensor(srv, ev.size).cpu().numpy().view(odp.EVENT_DTYPE).copy()
        o = orc.analyze(log)
        counts = [int((o.findings["kind"] == k).sum()) for k in range(1, 6)]
        assert counts[0] > 50 and counts[2] > 50 and counts[3] > 10 and counts[4] > 10
        got = sorted_findings(srv.poll())
        assert np.array_equal(got.view(np.uint8), o.findings.view(np.uint8))
    finally:
        srv.close()


@pytest.mark.parametrize("max_batch", [1, 3, 8, 4096])
def test_streamed_pairs_equal_offline(cuda_ok, orc, max_batch):
    """Streamed repeated allocations, unused allocations and unused transfers
    on a hand-made trace, in batches of 1 to 4096 events (decided in their
    own batch, waiting across batches, and at the flush), equal the oracle's
    over the log."""
    import paper_2601_12713_b300 as odp

    ev = pairs_trace()
    pool = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    is_x = np.isin(ev["kind"], [2, 3, 4])
    ptrs = np.where(is_x, pool.data_ptr(), 0).astype(np.uint64)
    srv = odp.Server(n_slots=2, max_events=1 << 12, max_batch_events=max_batch,
                     device_budget_bytes=2 << 30)
    try:
        srv.attach(0)
        srv.submit(ev, ptrs)
        srv.flush()
        log = odp.log_tensor(srv, ev.size)
        merged = log.cpu().numpy().view(odp.EVENT_DTYPE).copy()
        o = orc.analyze(merged)
        off = o.findings[np.isin(o.findings["kind"], [3, 4, 5])]
        st = sorted_findings(srv.poll())
        st = st[np.isin(st["kind"], [3, 4, 5])]
        assert (off["kind"] == 3).sum() >= 6 and (off["kind"] == 4).sum() >= 8
        assert (off["kind"] == 5).sum() >= 9
        assert np.array_equal(st.view(np.uint8), off.view(np.uint8))
    finally:
        srv.close()


@pytest.mark.parametrize("n_slots, max_events, max_batch", [(1, 1 << 12, 1), (2, 1 << 16, 2048),
                                                            (4, 1 << 20, 4096)])
def test_allocation_within_the_reservation(cuda_ok, n_slots, max_events, max_batch):
    import paper_2601_12713_b300 as odp

    shape = dict(n_slots=n_slots, max_events=max_events, max_batch_events=max_batch,
                 max_producers=16)
    need = odp.server_bytes(**shape)
    srv = odp.Server(device_budget_bytes=need, watermark_timeout_us=1000, **shape)
    try:
        got = srv.stats()["device_bytes"]
        # every allocated block is counted; the rest is per slot the fingerprint
        # plan's scratch (about 58 MB for a batch of at most 4,096) and 20 MB
        assert need - n_slots * (100 << 20) <= got <= need
    finally:
        srv.close()


def multi_endpoint_events(seed, n_transfers, n_devices, stretch=1):
    """Transfers among the host and n_devices devices (device-to-device
    included) whose content groups gain a third endpoint along the trace,
    fingerprints given; times stretched by `stretch`."""
    from synth import traces as T

    b = T.multi_endpoint(seed, n_transfers=n_transfers, n_contents=40, n_devices=n_devices)
    T.fill_fp_from_content(b)
    ev = b.events.copy()
    ev["t_start_ns"] *= stretch
    ev["t_end_ns"] = ev["t_start_ns"] + 10
    ev["flags"] = 1
    return ev


@pytest.mark.parametrize("seed,n_devices,max_batch", [(1, 2, 128), (2, 2, 256), (3, 3, 512),
                                                      (4, 7, 4096), (5, 127, 16384)])
def test_streamed_round_trips_with_three_or_more_endpoints(cuda_ok, orc, seed, n_devices,
                                                           max_batch):
    """Content groups that reach a third endpoint (devices 2 to 127, device-to-
    device transfers): their round trips after that are reported at the
    flush by replaying Alg. 2's queues (in rounds when they outnumber the
    findings buffer), so after the flush the streamed duplicate transfers,
    round trips and unused transfers equal the oracle's over the log, in
    batches of 128 to 16384 events (every to-device transfer waits for a
    kernel that never comes, so the waiting list, 16 batches long, must hold
    them)."""
    import paper_2601_12713_b300 as odp

    ev = multi_endpoint_events(seed, 4000 if max_batch < 16384 else 40_000, n_devices)
    srv = odp.Server(n_slots=2, max_events=1 << 16, max_batch_events=max_batch,
                     device_budget_bytes=4 << 30)
    try:
        srv.attach(0)
        srv.submit(ev, np.zeros(ev.size, dtype=np.uint64))
        srv.flush()
        st = srv.stats()
        assert st["events_processed"] == ev.size and st["stream_overflow"] == 0
        assert st["rt_groups_at_flush"] > 0
        log = odp.log_tensor(srv, ev.size).cpu().numpy().view(odp.EVENT_DTYPE).copy()
        o = orc.analyze(log)
        assert int((o.findings["kind"] == 2).sum()) > 100
        got = sorted_findings(srv.poll(1 << 20))
        assert np.array_equal(got.view(np.uint8), o.findings.view(np.uint8))
    finally:
        srv.close()


def test_streamed_mixed_trace_with_multi_endpoint_groups(cuda_ok, orc):
    """The kernel-heavy allocation cycles on three devices interleaved with
    multi-endpoint transfers: all five kinds streamed, the multi-endpoint
    round trips completed at the flush, equal to the oracle's over the log."""
    import paper_2601_12713_b300 as odp

    a = kernel_heavy_trace(12, n_cycles=800)
    b = multi_endpoint_events(6, 3000, 3, stretch=25)
    ev = np.concatenate([a, b])
    ev = ev[np.argsort(ev["t_start_ns"], kind="stable")]
    srv = odp.Server(n_slots=2, max_events=1 << 15, max_batch_events=256,
                     device_budget_bytes=2 << 30)
    try:
        srv.attach(0)
        srv.submit(ev, np.zeros(ev.size, dtype=np.uint64))
        srv.flush()
        st = srv.stats()
        assert st["stream_overflow"] == 0 and st["rt_groups_at_flush"] > 0
        log = odp.log_tensor(srv, ev.size).cpu().numpy().view(odp.EVENT_DTYPE).copy()
        o = orc.analyze(log)
        counts = [int((o.findings["kind"] == k).sum()) for k in range(1, 6)]
        assert all(c > 0 for c in counts)
        got = sorted_findings(srv.poll(1 << 20))
        assert np.array_equal(got.view(np.uint8), o.findings.view(np.uint8))
    finally:
        srv.close()


def nested_completions(ev):
    """Pairs (the nearest open ALLOC of the same device and device address,
    closed by a DELETE) that complete while an earlier allocation of their
    <host address, device, bytes> key is still open."""
    from synth import traces as T

    stacks, open_by_key, nested = {}, {}, 0
    for i, e in enumerate(ev):
        pk = (int(e["dst_dev"]), int(e["dev_addr"]))
        if e["kind"] == T.ALLOC:
            stacks.setdefault(pk, []).append(i)
            k = (int(e["host_addr"]), int(e["dst_dev"]), int(e["bytes"]))
            open_by_key.setdefault(k, set()).add(i)
        elif e["kind"] == T.DELETE and stacks.get(pk):
            a = stacks[pk].pop()
            k = (int(ev[a]["host_addr"]), int(ev[a]["dst_dev"]), int(ev[a]["bytes"]))
            open_by_key[k].discard(a)
            nested += any(x < a for x in open_by_key[k])
    return nested


@pytest.mark.parametrize("seed,max_batch", [(1, 64), (2, 256), (3, 1024), (4, 4096)])
def test_streamed_random_traces_with_nested_allocations(cuda_ok, orc, seed, max_batch):
    """Random traces over three devices with device-to-device transfers,
    overlapping allocations and deletes that close any open allocation: pairs
    of one <host address, device, bytes> key complete out of allocation order
    (a pair waits while an earlier allocation of its key is open), and content
    groups reach three endpoints.  After the flush the streamed findings of all
    five kinds equal the oracle's over the log."""
    import paper_2601_12713_b300 as odp
    from synth import traces as T

    b = T.random_small(seed, n_ops=4000, n_contents=8, n_hosts=3, n_devices=3, d2d=True)
    T.fill_fp_from_content(b)
    ev = b.events.copy()
    ev["flags"] = np.where(np.isin(ev["kind"], [2, 3, 4]), 1, 0)
    assert nested_completions(ev) > 20
    srv = odp.Server(n_slots=2, max_events=1 << 14, max_batch_events=max_batch,
                     device_budget_bytes=2 << 30)
    try:
        srv.attach(0)
        srv.submit(ev, np.zeros(ev.size, dtype=np.uint64))
        srv.flush()
        st = srv.stats()
        assert st["events_processed"] == ev.size and st["stream_overflow"] == 0
        log = odp.log_tensor(srv, ev.size).cpu().numpy().view(odp.EVENT_DTYPE).copy()
        o = orc.analyze(log)
        counts = [int((o.findings["kind"] == k).sum()) for k in range(1, 6)]
        assert counts[2] > 50, counts
        got = sorted_findings(srv.poll(1 << 20))
        assert np.array_equal(got.view(np.uint8), o.findings.view(np.uint8))
    finally:
        srv.close()


def test_flush_round_trips_in_rounds(cuda_ok, orc):
    """More round trips are left to the flush (content groups with three
    endpoints) than one batch's findings buffer holds (3 * 128 + 2,048 + 64):
    the flush replays the groups in rounds until none is dropped.  Kernels on
    both devices every 40 events keep the unused-transfer lists short."""
    import paper_2601_12713_b300 as odp
    from synth import traces as T

    x = multi_endpoint_events(7, 24_000, 2, stretch=10)
    kern = np.zeros(x.size // 40, dtype=x.dtype)
    kern["kind"] = T.KERNEL
    kern["src_dev"] = -1
    kern["dst_dev"] = np.arange(kern.size) % 2
    kern["t_start_ns"] = x["t_start_ns"][::40][: kern.size] + 3
    kern["t_end_ns"] = kern["t_start_ns"] + 4
    ev = np.concatenate([x, kern])
    ev = ev[np.argsort(ev["t_start_ns"], kind="stable")]
    srv = odp.Server(n_slots=2, max_events=1 << 16, max_batch_events=128,
                     device_budget_bytes=2 << 30)
    try:
        srv.attach(0)
        srv.submit(ev, np.zeros(ev.size, dtype=np.uint64))
        srv.flush()
        st = srv.stats()
        assert st["stream_overflow"] == 0 and st["rt_groups_at_flush"] > 0
        log = odp.log_tensor(srv, ev.size).cpu().numpy().view(odp.EVENT_DTYPE).copy()
        o = orc.analyze(log)
        rt = o.findings[o.findings["kind"] == 2]
        assert rt.size > 3 * (3 * 128 + 2048 + 64)
        got = sorted_findings(srv.poll(1 << 20))
        assert np.array_equal(got.view(np.uint8), o.findings.view(np.uint8))
    finally:
        srv.close()
