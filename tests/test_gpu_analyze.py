"""GPU parity of odp_analyze against the oracle (bit-exact findings, site
rows, summary and status), through the C ABI."""

import itertools

import numpy as np
import pytest
import torch

from synth import content, traces

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def odp():
    import paper_2601_12713_b300 as odp

    return odp


def gpu_analyze(odp, events, capacity=None, site_capacity=5 * 65536):
    n = events.size
    if capacity is None:
        capacity = max(16, 6 * n)
    ev = torch.from_numpy(events.view(np.uint8).reshape(-1).copy()).cuda() if n else \
        torch.empty(64, dtype=torch.uint8, device="cuda")
    out = odp.Findings(capacity, site_capacity)
    odp.analyze(ev, n, out)
    torch.cuda.synchronize()
    return out.to_host()


def assert_same(g, o):
    assert g["status"] == o.status
    assert g["count"] == o.count
    assert g["summary"] == o.summary
    assert g["n_sites"] == o.n_sites
    assert np.array_equal(g["findings"].view(np.uint8), o.findings.view(np.uint8)), \
        first_diff(g["findings"], o.findings)
    assert np.array_equal(g["sites"].view(np.uint8), o.sites.view(np.uint8))


def first_diff(a, b):
    for i in range(min(a.size, b.size)):
        if a[i].tobytes() != b[i].tobytes():
            return f"first difference at {i}: gpu {a[i]} oracle {b[i]}"
    return f"sizes {a.size} vs {b.size}"


def check(odp, orc, events, **kw):
    g = gpu_analyze(odp, events, **kw)
    o = orc.analyze(events, **{k: v for k, v in kw.items()})
    assert_same(g, o)
    return g


def with_fp(bundle):
    traces.fill_fp_from_content(bundle)
    return bundle.events


def test_listings(cuda_ok, orc, odp):
    check(odp, orc, with_fp(traces.listing1()))
    for n in (1, 2, 8, 50):
        check(odp, orc, with_fp(traces.listing2(n)))
    check(odp, orc, with_fp(traces.repeated_runs(500, 4096)))


def test_empty_trace(cuda_ok, orc, odp):
    ev = np.zeros(0, dtype=traces.EVENT_DTYPE)
    g = gpu_analyze(odp, ev)
    assert g["status"] == 0 and g["count"] == 0 and g["n_sites"] == 0
    assert all(v == 0 for v in g["summary"].values())


@pytest.mark.parametrize("seed", range(60))
def test_random_small_traces(cuda_ok, orc, odp, seed):
    n_dev = 1 + seed % 3
    b = traces.random_small(seed, n_ops=10 + (seed * 7) % 60, n_devices=n_dev, d2d=seed % 2 == 0)
    check(odp, orc, with_fp(b))


def test_random_medium_traces(cuda_ok, orc, odp):
    for seed in range(8):
        b = traces.random_small(1000 + seed, n_ops=20_000, n_contents=50, n_hosts=40,
                                n_devices=1 + seed % 4, d2d=True)
        check(odp, orc, with_fp(b))


@pytest.mark.parametrize("where", ["near_2_64", "span_over_2_63"])
def test_extreme_time_ranges(cuda_ok, orc, odp, where):
    """Times near 2^64 ns and kernel spans over 2^63 ns (the widest buckets
    of the per-device kernel index, whose bucket starts saturate): Alg. 4
    and 5 still agree with the oracle."""
    b = traces.random_small(77, n_ops=5000, n_contents=30, n_hosts=20, n_devices=3, d2d=True)
    ev = with_fp(b).copy()
    t0 = ev["t_start_ns"].astype(object)
    t1 = ev["t_end_ns"].astype(object)
    lo, hi = min(t0), max(t1)
    if where == "near_2_64":
        base, scale = (1 << 64) - 1 - (hi - lo) * 4, 4
    else:
        base, scale = 0, ((1 << 63) + (1 << 62)) // (hi - lo)
    ev["t_start_ns"] = np.array([base + (t - lo) * scale for t in t0], dtype=np.uint64)
    ev["t_end_ns"] = np.array([base + (t - lo) * scale for t in t1], dtype=np.uint64)
    assert int(ev["t_end_ns"].max()) < (1 << 64)
    g = check(odp, orc, ev)
    assert g["summary"]["count4"] + g["summary"]["count5"] > 0


def test_exhaustive_two_endpoint_rt(cuda_ok, orc, odp):
    # every direction pattern of length 6 over 2 contents, concatenated with
    # distinct content ids per pattern so the groups stay independent
    import itertools

    dirs_all, cont_all = [], []
    for k, dirs in enumerate(itertools.product((0, 1), repeat=6)):
        for cs in itertools.product((0, 1), repeat=6):
            dirs_all += list(dirs)
            cont_all += [2 * (k * 64 + int("".join(map(str, cs)), 2)) + c for c in cs]
    b = traces.two_endpoint_sequence(dirs_all, cont_all)
    check(odp, orc, with_fp(b))


def _all_sequences(endpoints, max_len):
    pairs = [(a, b) for a in endpoints for b in endpoints if a != b]
    seqs, conts = [], []
    k = 0
    for length in range(1, max_len + 1):
        for seq in itertools.product(pairs, repeat=length):
            seqs += list(seq)
            conts += [k] * length
            k += 1
    return seqs, conts


def test_exhaustive_three_endpoint_rt(cuda_ok, orc, odp):
    # every transfer sequence of length <= 6 among the host and devices 0, 1,
    # and of length <= 5 among devices 1, 2 and 127 (endpoint codes across
    # 32-bit words of the per-segment source sets); one content per sequence
    for endpoints, max_len in (((-1, 0, 1), 6), ((1, 2, 127), 5)):
        seqs, conts = _all_sequences(endpoints, max_len)
        check(odp, orc, with_fp(traces.endpoint_sequence(seqs, conts)))


@pytest.mark.parametrize("n_devices", [2, 3, 4, 8, 128])
def test_multi_endpoint_random(cuda_ok, orc, odp, n_devices):
    for seed in range(3):
        b = traces.multi_endpoint(7000 + seed, 40_000 + 30_000 * seed, n_contents=200 * (seed + 1),
                                  n_devices=n_devices)
        check(odp, orc, with_fp(b))


def test_multi_endpoint_one_long_group(cuda_ok, orc, odp):
    # one content moved 300,000 times among the host and 128 devices (129
    # endpoints, the most the record allows), with and without chains
    for follow in (0.9, 0.0):
        b = traces.multi_endpoint(7100, 300_000, n_contents=1, n_devices=128, hot=1.0,
                                  follow=follow)
        check(odp, orc, with_fp(b))


def test_graph_capture_and_concurrent_streams(cuda_ok, orc, odp):
    """odp_analyze captured in a CUDA graph and replayed, and two calls in
    flight on two streams at once, give the oracle's results."""
    b1 = traces.random_small(4242, n_ops=20_000, n_contents=50, n_hosts=40, n_devices=3, d2d=True)
    b2 = traces.multi_endpoint(4243, 30_000, n_contents=300, n_devices=4)
    e1, e2 = with_fp(b1), with_fp(b2)
    o1, o2 = orc.analyze(e1), orc.analyze(e2)

    def dev(e):
        return torch.from_numpy(e.view(np.uint8).reshape(-1).copy()).cuda()

    d1, d2 = dev(e1), dev(e2)
    s = torch.cuda.Stream()
    out = odp.Findings(6 * e1.size)
    with torch.cuda.stream(s):
        odp.analyze(d1, e1.size, out, s)  # first call on the stream allocates its scratch
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        odp.analyze(d1, e1.size, out, s)
    out.items.zero_()
    out.small.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert_same(out.to_host(), o1)

    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    oa, ob = odp.Findings(6 * e1.size), odp.Findings(6 * e2.size)
    for _ in range(3):
        odp.analyze(d1, e1.size, oa, sa)
        odp.analyze(d2, e2.size, ob, sb)
    torch.cuda.synchronize()
    assert_same(oa.to_host(), o1)
    assert_same(ob.to_host(), o2)


def test_plain_small_with_payload_fingerprints(cuda_ok, orc, odp):
    """Plain small workload: every transfer fingerprinted on the GPU, one
    buffer per launch, then the whole log analysed; every fingerprint and the
    findings checked against the oracle, and the text report rendered from
    the GPU result equals the one rendered from the oracle's."""
    from paper_2601_12713_b300 import report
    from synth import gpu

    b = traces.plain_small()
    ev = b.events
    idx = np.flatnonzero(b.content >= 0)
    fps_gpu = np.zeros((ev.size, 2), dtype=np.uint64)
    for i in idx:
        nbytes = int(ev["bytes"][i])
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        gpu.fill(t, content.RANDOM, int(b.payload_seed[i]))
        out = odp.fingerprint_tensors([t])
        fps_gpu[i] = out.cpu().numpy().view(np.uint64)[0]
    for i in idx:
        data = content.bytes_of(content.RANDOM, int(b.payload_seed[i]), int(ev["bytes"][i]))
        assert tuple(int(x) for x in fps_gpu[i]) == orc.fp128(data), i
    ev_g = ev.copy()
    ev_g["fp_lo"][idx] = fps_gpu[idx, 0]
    ev_g["fp_hi"][idx] = fps_gpu[idx, 1]
    g = check(odp, orc, ev_g)
    assert g["summary"]["count1"] > 0 and g["summary"]["count3"] > 0
    o = orc.analyze(ev_g)
    names = {k: f"plain_small.c:{100 + k}" for k in range(32)}
    text = report.render(g, site_names=names)
    assert text == report.render({"summary": o.summary, "sites": o.sites, "status": o.status},
                                 site_names=names)
    for kind in range(1, 6):
        assert f"findings: {g['summary'][f'count{kind}']}," in text
    assert "predicted speedup" in text


@pytest.mark.parametrize("n_iter,n_arrays,per_iter,p_skip",
                         [(20, 400, 100, 0.0), (60, 2000, 500, 0.0), (60, 2000, 500, 0.1),
                          (200, 5000, 2500, 0.05)])
def test_iterative_solver_reduced(cuda_ok, orc, odp, n_iter, n_arrays, per_iter, p_skip):
    """Reduced iterative-solver traces; the last one (10^6 transfers) makes a
    content table of 2^21 slots, which is inserted into partition by
    partition."""
    b = traces.iterative_solver(n_iter=n_iter, n_arrays=n_arrays, per_iter=per_iter, n_sites=50,
                                p_skip_kernel=p_skip)
    g = check(odp, orc, with_fp(b))
    if p_skip:
        assert g["summary"]["count4"] > 0 and g["summary"]["count5"] > 0


def test_validation_errors(cuda_ok, orc, odp):
    b = traces.listing2(4)
    base = with_fp(b)
    cases = []
    e = base.copy(); e["kind"][3] = 9; cases.append(e)
    e = base.copy(); e["t_start_ns"][7] = e["t_start_ns"][6] - 1; cases.append(e)
    e = base.copy(); e["t_end_ns"][2] = e["t_start_ns"][2] - 1; cases.append(e)
    e = base.copy(); e["bytes"][1] = 0; cases.append(e)
    e = base.copy(); e["site_id"][5] = 70000; cases.append(e)
    e = base.copy(); e["src_dev"][1] = 0; cases.append(e)          # to-device from a device
    e = base.copy(); e["t_start_ns"][3] = 0; e["kind"][8] = 0; cases.append(e)
    for e in cases:
        g = gpu_analyze(odp, e)
        o = orc.analyze(e)
        assert g["status"] == o.status < 0
        assert g["count"] == 0 and g["n_sites"] == 0
        assert all(v == 0 for v in g["summary"].values())


def test_truncation(cuda_ok, orc, odp):
    ev = with_fp(traces.repeated_runs(50, 64))
    check(odp, orc, ev, capacity=10, site_capacity=1)


def test_unmatched_and_nested_pairs(cuda_ok, orc, odp):
    bld = traces._Builder()
    D = traces.DELETE
    A = traces.ALLOC
    # nested allocations of one device address, an unmatched delete, a
    # never-deleted allocation, and a kernel that overlaps only some lifetimes
    bld.add(D, 10, dst=0, host_addr=0x10, dev_addr=0x100, nbytes=8)
    bld.add(A, 10, dst=0, host_addr=0x10, dev_addr=0x100, nbytes=8)
    bld.add(A, 10, dst=0, host_addr=0x10, dev_addr=0x100, nbytes=8)
    bld.add(traces.KERNEL, 50, dst=0)
    bld.add(D, 10, dst=0, host_addr=0x10, dev_addr=0x100, nbytes=8)
    bld.add(D, 10, dst=0, host_addr=0x10, dev_addr=0x100, nbytes=8)
    bld.add(A, 10, dst=0, host_addr=0x10, dev_addr=0x100, nbytes=8)
    bld.add(A, 10, dst=1, host_addr=0x20, dev_addr=0x100, nbytes=8)
    bld.add(D, 10, dst=0, host_addr=0x10, dev_addr=0x100, nbytes=8)
    bld.add(A, 10, dst=0, host_addr=0x30, dev_addr=0x200, nbytes=8)
    g = check(odp, orc, with_fp(bld.done()))
    assert g["summary"]["n_unmatched_deletes"] == 1


def test_misaligned_events_rejected(cuda_ok, odp):
    ev = with_fp(traces.listing2(3))
    raw = torch.zeros(ev.size * 64 + 16, dtype=torch.uint8, device="cuda")
    raw[8:8 + ev.size * 64] = torch.from_numpy(ev.view(np.uint8).reshape(-1).copy()).cuda()
    out = odp.Findings(64)
    with pytest.raises(odp.OdpError) as e:
        odp.analyze(raw[8:], ev.size, out)
    assert e.value.status == -1


@pytest.mark.parametrize("p_skip", [0.0, 0.03])
def test_full_scale_iterative_solver(cuda_ok, orc, odp, p_skip):
    """The 5·10^7-event trace at full size, as the benchmark times it: the GPU
    output equals the oracle's bit for bit (the oracle takes minutes).  The
    second case moves 3 % of the iterations' kernels to another device, so
    unused allocations and unused transfers are found at full size too."""
    b = traces.iterative_solver(p_skip_kernel=p_skip)
    traces.fill_fp_from_content(b)
    n = b.events.size
    assert n == 50_002_000
    ev = torch.from_numpy(b.events.view(np.uint8).reshape(-1)).cuda()
    out = odp.Findings(n)
    odp.analyze(ev, n, out)
    torch.cuda.synchronize()
    del ev
    g = out.to_host()
    del out
    torch.cuda.empty_cache()
    o = orc.analyze(b.events, capacity=n)
    assert g["status"] == o.status == 0
    assert g["count"] == o.count and g["summary"] == o.summary and g["n_sites"] == o.n_sites
    assert np.array_equal(g["sites"].view(np.uint8), o.sites.view(np.uint8))
    assert np.array_equal(g["findings"].view(np.uint8), o.findings.view(np.uint8))
    if p_skip:
        assert g["summary"]["count4"] > 100_000 and g["summary"]["count5"] > 10_000


@pytest.mark.parametrize("seed", range(4))
def test_all_ones_and_zero_fingerprints(cuda_ok, orc, odp, seed):
    """Contents whose fingerprint is all ones (the hash table's empty key,
    kept in a slot of its own) or all zeros group like any other content."""
    b = traces.random_small(2000 + seed, n_ops=3000 + 2000 * seed, n_contents=12, n_hosts=9,
                            n_devices=1 + seed % 3, d2d=seed % 2 == 0)
    ev = with_fp(b)
    xfer = np.isin(ev["kind"], [traces.TO_DEV, traces.FROM_DEV, traces.DEV_TO_DEV])
    cont = b.content
    ones = xfer & (cont == cont[xfer].min())
    zeros = xfer & (cont == cont[xfer].max())
    assert ones.any() and zeros.any()
    ev["fp_lo"][ones] = ev["fp_hi"][ones] = np.uint64(0xFFFFFFFFFFFFFFFF)
    ev["fp_lo"][zeros] = ev["fp_hi"][zeros] = 0
    g = check(odp, orc, ev)
    assert g["count"] > 0


def many_keys_trace(seed, n_arrays, n_rounds, n_devices):
    """n_arrays arrays (one host address, device address and device each),
    each mapped n_rounds times at random times (ALLOC, TO_DEV, FROM_DEV,
    DELETE), with kernels at random times on random devices; content versions
    change at random.  More than 2^16 distinct (device, device address) keys
    and candidate host addresses."""
    rng = np.random.default_rng(seed)
    m = n_arrays * n_rounds
    arr = np.repeat(np.arange(n_arrays), n_rounds)
    start = 1000 + 4 * rng.integers(0, 40 * m, m)
    dev = arr % n_devices
    ver = rng.integers(0, 3, (m, 2))
    n_k = m // 50
    ev = np.zeros(4 * m + n_k, dtype=traces.EVENT_DTYPE)
    content = np.full(ev.size, -1, dtype=np.int64)
    parts = [(0, traces.ALLOC), (1, traces.TO_DEV), (20, traces.FROM_DEV), (21, traces.DELETE)]
    for j, (off, kind) in enumerate(parts):
        sl = slice(j * m, (j + 1) * m)
        ev["t_start_ns"][sl] = start + off
        ev["kind"][sl] = kind
        ev["host_addr"][sl] = 0x1000 * (1 + arr)
        ev["dev_addr"][sl] = 0x100 * (1 + arr)
        ev["bytes"][sl] = 64 * (1 + arr % 3)
        ev["site_id"][sl] = arr % 500
        ev["src_dev"][sl] = dev if kind == traces.FROM_DEV else traces.HOST
        ev["dst_dev"][sl] = traces.HOST if kind == traces.FROM_DEV else dev
        if kind == traces.TO_DEV:
            content[sl] = 10 * arr + ver[:, 0]
        elif kind == traces.FROM_DEV:
            content[sl] = 10 * arr + ver[:, 1]
    sl = slice(4 * m, None)
    ev["t_start_ns"][sl] = 1000 + rng.integers(0, 160 * m, n_k)
    ev["kind"][sl] = traces.KERNEL
    ev["src_dev"][sl] = traces.HOST
    ev["dst_dev"][sl] = rng.integers(0, n_devices, n_k)
    ev["t_end_ns"] = ev["t_start_ns"] + 2
    ev["t_end_ns"][sl] = ev["t_start_ns"][sl] + 5
    order = np.argsort(ev["t_start_ns"], kind="stable")
    b = traces.TraceBundle(events=ev[order], content=content[order])
    return with_fp(b)


@pytest.mark.parametrize("n_devices", [1, 3])
def test_grouping_sorts_past_16_bits(cuda_ok, orc, odp, n_devices):
    """More than 2^16 distinct allocation keys and candidate host addresses:
    the grouping sorts on dense ids need more than two passes."""
    ev = many_keys_trace(17 + n_devices, 100_000, 2, n_devices)
    al = ev[ev["kind"] == traces.ALLOC]
    assert np.unique(al["dev_addr"]).size > 1 << 16
    g = check(odp, orc, ev)
    assert g["count"] > 0


def test_many_contents(cuda_ok, orc, odp):
    """600,000 transfers of 361,000 distinct contents on two devices (a
    content table of 2^20 slots, three in five of its inserts new)."""
    ev = many_keys_trace(31, 150_000, 2, 2)
    xfer = ev[np.isin(ev["kind"], [traces.TO_DEV, traces.FROM_DEV])]
    assert 1.25 * xfer.size > (1 << 19)
    fps = np.unique(np.stack([xfer["fp_lo"], xfer["fp_hi"]], axis=1), axis=0)
    assert fps.shape[0] > (1 << 18)
    g = check(odp, orc, ev)
    assert g["count"] > 0
