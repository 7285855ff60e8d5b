"""Serving loop (GPU, through the C ABI): producers on host threads, the
merged log, streamed findings against the offline analysis of the same log,
and every request's fingerprints alone versus in the mix."""

import numpy as np
import pytest
import torch

from synth import content

pytestmark = pytest.mark.gpu


def run_server(odp, n_threads, rate, seconds, n_slots, max_batch, seed, max_payload=1 << 20):
    from synth import gpu, load

    pool_bytes = 64 << 20
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
    gpu.fill(pool, content.RANDOM, seed)
    torch.cuda.synchronize()
    srv = odp.Server(n_slots=n_slots, max_events=1 << 20, max_batch_events=max_batch,
                     device_budget_bytes=4 << 30, watermark_timeout_us=200_000)
    lg = load.Load(n_threads, rate, seconds, seed, pool.data_ptr(), pool_bytes, 256, max_payload)
    n = lg.run(srv)
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


@pytest.mark.parametrize("n_slots,max_batch", [(1, 512), (4, 2048)])
def test_streamed_findings_equal_offline(cuda_ok, orc, n_slots, max_batch):
    import paper_2601_12713_b300 as odp

    srv, lg, pool, n = run_server(odp, 8, 20_000, 1.5, n_slots, max_batch, 5 + n_slots)
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
        # streamed DD and RT findings are exactly the offline ones
        st = srv.poll()
        key = np.lexsort((st["partner"], st["event"], st["kind"]))
        st = st[key]
        off = g["findings"][np.isin(g["findings"]["kind"], [1, 2])]
        assert st.size == off.size and st.size > 0
        assert np.array_equal(st.view(np.uint8), off.view(np.uint8))
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
        assert s["rt_groups_unstreamed"] == 0
    finally:
        srv.close()
        lg.close()


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
