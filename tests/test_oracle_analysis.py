"""Pins for the oracle's Algorithms 1-5 (CPU only).

Expectations come from the paper's worked examples (Listings 1 and 2, Sec. 4),
the count semantics of Table 2, hand-derived traces, exhaustive enumeration
of small two-endpoint transfer sequences against a closed form, and
brute-force restatements of Definitions 1, 3 and 4 and of the unused-transfer
rule on random small traces.
"""

import itertools

import numpy as np
import pytest

from synth import traces, content as synth_content

NONE = (1 << 64) - 1
DD, RT, RA, UA, UT = 1, 2, 3, 4, 5


def run(orc, bundle, **kw):
    traces.fill_fp_from_content(bundle)
    r = orc.analyze(bundle.events, **kw)
    assert r.status in (0, 1), r.status
    return r


def by_kind(r, kind):
    f = r.findings[r.findings["kind"] == kind]
    return [(int(e), int(p)) for e, p in zip(f["event"], f["partner"])]


def counts(r):
    return [r.summary[f"count{k}"] for k in range(1, 6)]


def golden_counts(name, n=None):
    """Expected per-kind counts from tests/golden (values the paper prints or
    states for its examples); `N-1` is evaluated with the given n."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    vals = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, v = line.split()
        vals[kind] = n - 1 if v == "N-1" else int(v)
    return [vals[k] for k in ("DD", "RT", "RA", "UA", "UT")]


def test_listing1(orc):
    b = traces.listing1()
    r = run(orc, b)
    assert counts(r) == golden_counts("listing1_counts.txt")
    ev = b.events
    to = np.flatnonzero((ev["kind"] == traces.TO_DEV) & (ev["host_addr"] == 0x10000))
    assert by_kind(r, DD) == [(int(to[1]), int(to[0]))]
    al = np.flatnonzero((ev["kind"] == traces.ALLOC) & (ev["host_addr"] == 0x10000))
    assert by_kind(r, RA) == [(int(al[1]), int(al[0]))]


@pytest.mark.parametrize("n_iter", [1, 2, 3, 8, 50])
def test_listing2(orc, n_iter):
    b = traces.listing2(n_iter)
    r = run(orc, b)
    assert counts(r) == golden_counts("listing2_counts.txt", n_iter)
    ev = b.events
    frm = np.flatnonzero(ev["kind"] == traces.FROM_DEV)
    to = np.flatnonzero(ev["kind"] == traces.TO_DEV)
    # the round trip is device -> host -> device: (D2H_i, H2D_{i+1})
    assert by_kind(r, RT) == [(int(frm[i]), int(to[i + 1])) for i in range(n_iter - 1)]
    # wasted union: the return trips plus the re-allocations and deletes
    d = (ev["t_end_ns"] - ev["t_start_ns"]).astype(np.int64)
    al = np.flatnonzero(ev["kind"] == traces.ALLOC)
    de = np.flatnonzero(ev["kind"] == traces.DELETE)
    saved = d[to[1:]].sum() + d[al[1:]].sum() + d[de[1:]].sum()
    assert r.summary["saved_ns"] == saved
    span = int(ev["t_end_ns"].max() - ev["t_start_ns"].min())
    assert r.summary["trace_span_ns"] == span
    assert (r.summary["speedup_num"], r.summary["speedup_den"]) == (span, span - saved)


def test_repeated_runs_table2_count_semantics(orc):
    # 500 runs: each group of n equal events yields n - 1 findings (Table 2
    # reports DD = RA = 499 for babelstream's 500 repetitions).
    r = run(orc, traces.repeated_runs(500, 4096))
    assert counts(r) == golden_counts("table2_babelstream_counts.txt")


def test_three_endpoint_literal_quirk(orc):
    """Alg. 2 literally: H->D0, D0->D1, D1->H of one content.  The first
    transfer pairs with the later D1->H; the D1->H transfer peeks the D0->D1
    reception at D1 even though it precedes it."""
    b = traces._Builder()
    b.add(traces.TO_DEV, 10, src=-1, dst=0, nbytes=8, content=1)
    b.add(traces.DEV_TO_DEV, 10, src=0, dst=1, nbytes=8, content=1)
    b.add(traces.FROM_DEV, 10, src=1, dst=-1, nbytes=8, content=1)
    r = run(orc, b.done())
    assert by_kind(r, RT) == [(0, 2), (2, 1)]
    assert by_kind(r, DD) == []


def test_peek_does_not_dequeue(orc):
    # two sends of the same content then one return: both sends pair with it
    r = run(orc, traces.two_endpoint_sequence([0, 0, 1], [7, 7, 7]))
    assert by_kind(r, RT) == [(0, 2), (1, 2)]
    assert by_kind(r, DD) == [(1, 0)]


def closed_form_rt(dirs, cont):
    """Two endpoints: tx e from A pairs with the first later reception at A of
    the same content (Sec. 5.2 queues reduce to this when only two endpoints
    exist)."""
    out = []
    for e, (d, c) in enumerate(zip(dirs, cont)):
        # reception at A = transfer whose destination is A
        for j in range(e + 1, len(dirs)):
            dest_of_j_is_host = dirs[j] == 1
            src_of_e_is_host = d == 0
            if cont[j] == c and dest_of_j_is_host == src_of_e_is_host:
                out.append((e, j))
                break
    return out


def brute_dd(dirs, cont):
    out = []
    first = {}
    for e, (d, c) in enumerate(zip(dirs, cont)):
        key = (c, d)
        if key in first:
            out.append((e, first[key]))
        else:
            first[key] = e
    return out


def restricted_growth(length, k):
    def rec(prefix, m):
        if len(prefix) == length:
            yield list(prefix)
            return
        for v in range(min(m + 1, k)):
            yield from rec(prefix + [v], max(m, v + 1))
    yield from rec([], 0)


def test_round_trips_exhaustive_two_endpoints(orc):
    n_checked = 0
    for length in range(1, 8):
        for cont in restricted_growth(length, 3):
            for dirs in itertools.product((0, 1), repeat=length):
                b = traces.two_endpoint_sequence(dirs, cont)
                r = run(orc, b)
                assert sorted(by_kind(r, RT)) == closed_form_rt(dirs, cont), (dirs, cont)
                assert sorted(by_kind(r, DD)) == brute_dd(dirs, cont)
                n_checked += 1
    assert n_checked > 50_000


def test_round_trips_random_length8(orc):
    rng = np.random.default_rng(21)
    for _ in range(1500):
        dirs = [int(x) for x in rng.integers(0, 2, 8)]
        cont = [int(x) for x in rng.integers(0, 3, 8)]
        r = run(orc, traces.two_endpoint_sequence(dirs, cont))
        assert sorted(by_kind(r, RT)) == closed_form_rt(dirs, cont)


# --- brute-force definitions on random small traces -------------------------

def bf_dd(ev, cont):
    """Def. 1: a device (or host) receives data that it had received before."""
    out = []
    for i in range(ev.size):
        if ev["kind"][i] not in traces.TRANSFER_KINDS:
            continue
        for j in range(i):
            if (ev["kind"][j] in traces.TRANSFER_KINDS and cont[j] == cont[i]
                    and ev["dst_dev"][j] == ev["dst_dev"][i]):
                out.append((i, j))
                break
    return out


def bf_pairs(ev):
    """A delete closes the nearest earlier open alloc of the same (dev, addr)."""
    n = ev.size
    used = [False] * n
    pairs = []
    for j in range(n):
        if ev["kind"][j] != traces.DELETE:
            continue
        for i in range(j - 1, -1, -1):
            if (ev["kind"][i] == traces.ALLOC and not used[i]
                    and ev["dst_dev"][i] == ev["dst_dev"][j] and ev["dev_addr"][i] == ev["dev_addr"][j]):
                used[i] = True
                pairs.append((i, j))
                break
    return sorted(pairs), [i for i in range(n) if ev["kind"][i] == traces.ALLOC and not used[i]]


def bf_ra(ev):
    """Def. 3: the same (host address, device, bytes) allocated and deleted
    more than once; each pair after the first is a finding."""
    pairs, _ = bf_pairs(ev)
    out = []
    for k, (a, _d) in enumerate(pairs):
        key = (ev["host_addr"][a], ev["dst_dev"][a], ev["bytes"][a])
        earlier = [p for p, _ in pairs[:k]
                   if (ev["host_addr"][p], ev["dst_dev"][p], ev["bytes"][p]) == key]
        if earlier:
            out.append((a, earlier[0]))
    return out


def bf_ua(ev):
    """Def. 4 for allocations: no kernel on the device overlaps the closed
    lifetime [alloc start, delete end] (open allocations end at trace end)."""
    pairs, unpaired = bf_pairs(ev)
    end = int(ev["t_end_ns"].max()) if ev.size else 0
    lives = [(a, d, int(ev["t_end_ns"][d])) for a, d in pairs] + [(a, NONE, end) for a in unpaired]
    out = []
    for a, d, dend in lives:
        dev = ev["dst_dev"][a]
        used = False
        for k in range(ev.size):
            if ev["kind"][k] == traces.KERNEL and ev["dst_dev"][k] == dev:
                if ev["t_start_ns"][k] <= dend and ev["t_end_ns"][k] >= ev["t_start_ns"][a]:
                    used = True
        if not used:
            out.append((a, d))
    return sorted(out)


def bf_ut(ev):
    """Unused transfers, restated without the pointer walk: for a to-device
    transfer, p = the first kernel of its device (start order) whose end is
    not before the transfer's start.  No such kernel: unused (after the last
    kernel).  A transfer is overwritten when a later to-device transfer of the
    same device and host address has the same p, both start before kernel p
    starts, and no transfer of that device overlapping kernel p lies between."""
    n = ev.size
    out = []
    info = {}
    for i in range(n):
        if ev["kind"][i] != traces.TO_DEV:
            continue
        dev = ev["dst_dev"][i]
        ks = [k for k in range(n) if ev["kind"][k] == traces.KERNEL and ev["dst_dev"][k] == dev]
        p = next((q for q, k in enumerate(ks) if ev["t_end_ns"][k] >= ev["t_start_ns"][i]), None)
        if p is None:
            info[i] = ("after", None)
        elif ev["t_start_ns"][ks[p]] > ev["t_start_ns"][i]:
            info[i] = ("cand", p)
        else:
            info[i] = ("barrier", p)
    for i, (cls, p) in info.items():
        if cls == "after":
            out.append((i, NONE))
            continue
        if cls != "cand":
            continue
        for j in range(i + 1, n):
            if j not in info or ev["dst_dev"][j] != ev["dst_dev"][i]:
                continue
            cj, pj = info[j]
            if pj != p or cj == "after":
                break
            if cj == "barrier":
                break
            if ev["host_addr"][j] == ev["host_addr"][i]:
                out.append((i, j))
                break
    return sorted(out)


@pytest.mark.parametrize("seed", range(120))
def test_random_small_against_definitions(orc, seed):
    n_dev = 1 + seed % 3
    b = traces.random_small(seed, n_ops=18 + seed % 17, n_devices=n_dev)
    r = run(orc, b)
    ev = b.events
    assert sorted(by_kind(r, DD)) == bf_dd(ev, b.content)
    assert sorted(by_kind(r, RA)) == bf_ra(ev)
    assert sorted(by_kind(r, UA)) == bf_ua(ev)
    assert sorted(by_kind(r, UT)) == bf_ut(ev)
    if n_dev == 1:
        # host + one device: the round-trip closed form applies
        dirs = []
        idx = []
        for i in range(ev.size):
            if ev["kind"][i] in (traces.TO_DEV, traces.FROM_DEV):
                idx.append(i)
                dirs.append(0 if ev["kind"][i] == traces.TO_DEV else 1)
        cont = [int(b.content[i]) for i in idx]
        want = [(idx[e], idx[j]) for e, j in closed_form_rt(dirs, cont)]
        assert sorted(by_kind(r, RT)) == want


def test_bruteforce_mode_matches_hash_mode(orc):
    for seed in range(6):
        b = traces.random_small(seed, n_ops=40, n_devices=2, d2d=True)
        payloads = []
        for i in range(b.events.size):
            c = int(b.content[i])
            if c < 0:
                payloads.append(None)
                continue
            data = synth_content.bytes_of(0, 1000 + c, int(b.events["bytes"][i]))
            payloads.append(data)
            lo, hi = orc.fp128(data)
            b.events["fp_lo"][i] = lo
            b.events["fp_hi"][i] = hi
        r_hash = orc.analyze(b.events)
        r_bf = orc.analyze_bruteforce(b.events, payloads)
        assert r_hash.status == r_bf.status == 0
        assert np.array_equal(r_hash.findings, r_bf.findings)


def test_plain_small_ground_truth(orc):
    b = traces.plain_small(n_cycles=300)
    r = run(orc, b)
    ev = b.events
    dd = dict(by_kind(r, DD))
    for e in b.labels["dd"]:
        assert e in dd
    for e, p in dd.items():
        assert b.content[e] == b.content[p] and ev["dst_dev"][e] == ev["dst_dev"][p]
    rt_rx = {p for _, p in by_kind(r, RT)}
    rt_tx = {e for e, _ in by_kind(r, RT)}
    for e in b.labels["rt"]:
        assert e in rt_rx or e in rt_tx
    ra = dict(by_kind(r, RA))
    for e in b.labels["ra"]:
        assert e in ra
    ua = dict(by_kind(r, UA))
    for e in b.labels["ua"]:
        assert e in ua
    ut = dict(by_kind(r, UT))
    for e in b.labels["ut"]:
        assert e in ut
    assert r.summary["n_events"] == ev.size
    n_data_ops = int(np.isin(ev["kind"], [1, 2, 3, 4, 5]).sum())
    assert n_data_ops == 4 * 300


def test_validation_status(orc):
    b = traces.listing2(3)
    traces.fill_fp_from_content(b)
    ev = b.events.copy()
    ev["kind"][4] = 9
    assert orc.analyze(ev).status == -5
    ev = b.events.copy()
    ev["t_start_ns"][6] = ev["t_start_ns"][5] - 1
    assert orc.analyze(ev).status == -6
    ev = b.events.copy()
    ev["t_end_ns"][2] = ev["t_start_ns"][2] - 1
    assert orc.analyze(ev).status == -5
    ev = b.events.copy()
    ev["bytes"][1] = 0      # a transfer of zero bytes
    assert orc.analyze(ev).status == -5
    ev = b.events.copy()   # malformed later than an unsorted index: unsorted wins
    ev["t_start_ns"][3] = 0
    ev["kind"][8] = 0
    assert orc.analyze(ev).status == -6
    assert orc.analyze(b.events[:0]).status == 0


def test_truncation(orc):
    b = traces.repeated_runs(50, 64)
    traces.fill_fp_from_content(b)
    full = orc.analyze(b.events)
    part = orc.analyze(b.events, capacity=10)
    assert part.status == 1 and part.count == full.count == 98
    assert np.array_equal(part.findings, full.findings[:10])
    assert part.summary == full.summary


def test_site_rows(orc):
    b = traces.plain_small(n_cycles=200)
    r = run(orc, b)
    f = r.findings
    rows = {}
    for x in f:
        k = (int(x["kind"]), int(x["site"]))
        c, by, ns = rows.get(k, (0, 0, 0))
        rows[k] = (c + 1, by + int(x["wasted_bytes"]), ns + int(x["wasted_ns"]))
    got = {(int(s["kind"]), int(s["site"])): (int(s["count"]), int(s["wasted_bytes"]),
                                               int(s["wasted_ns"])) for s in r.sites}
    assert got == rows
    keys = [(int(s["kind"]), int(s["site"])) for s in r.sites]
    assert keys == sorted(keys)


# --- more than two endpoints ------------------------------------------------

def closed_form_rt_general(events):
    """Alg. 2 restated without queues, for any number of endpoints, on one
    content group given as (src, dst) pairs in order.  With n_A receptions at
    A and last_A the index of the last one:
      * a transfer from A at t succeeds iff t < last_A or some reception at A
        failed (if all A-receptions lie before t, the queue of A is non-empty
        exactly when not every one of them was popped);
      * a reception r from X fails iff r > last_X and every reception at X
        succeeded (allOK_X) -- so allOK is settled endpoint by endpoint in
        increasing order of last;
      * the partner is the k-th reception at A, k = receptions at A before t
        that succeeded."""
    rec = {}
    for t, (s, d) in enumerate(events):
        rec.setdefault(d, []).append(t)
    last = {d: v[-1] for d, v in rec.items()}
    all_ok = {}
    failed = [False] * len(events)
    for d in sorted(rec, key=lambda x: last[x]):
        ok = True
        for r in rec[d]:
            x = events[r][0]
            f = x in last and r > last[x] and all_ok[x]
            if x not in last:
                f = True  # the source never receives: its queue is empty
            failed[r] = f
            ok &= not f
        all_ok[d] = ok
    out = []
    for t, (a, _d) in enumerate(events):
        if a not in rec:
            continue
        if not (t < last[a] or not all_ok[a]):
            continue
        k = sum(1 for r in rec[a] if r < t and not failed[r])
        out.append((t, rec[a][k]))
    return out


def literal_rt(events):
    """Alg. 2 on one content group with the queues, for comparison."""
    from collections import deque
    q = {}
    for t, (s, d) in enumerate(events):
        q.setdefault(d, deque()).append(t)
    out = []
    for t, (a, b) in enumerate(events):
        if a not in q or not q[a]:
            continue
        out.append((t, q[a][0]))
        q[b].popleft()
    return out


def test_general_closed_form_three_endpoints(orc):
    """Every sequence of up to 6 transfers among three endpoints: the queue
    walk, the oracle and the closed form agree."""
    eps = (-1, 0, 1)
    pairs = [(a, b) for a in eps for b in eps if a != b]
    n = 0
    for length in range(1, 7):
        for seq in itertools.product(pairs, repeat=length):
            want = literal_rt(seq)
            assert closed_form_rt_general(seq) == want, seq
            n += 1
            if length <= 4:
                b = traces._Builder(gap_ns=1)
                for s, d in seq:
                    kind = traces.TO_DEV if s == -1 else traces.FROM_DEV if d == -1 else traces.DEV_TO_DEV
                    b.add(kind, 5, src=s, dst=d, nbytes=8, content=0)
                r = run(orc, b.done())
                assert by_kind(r, RT) == want, seq
    assert n > 50_000


def test_oracle_rt_many_endpoints(orc):
    """The oracle's Alg. 2 on traces over the host and 128 devices (129
    endpoints) against the queue-free closed form, group by group."""
    for seed, follow in ((1, 0.7), (2, 0.0)):
        b = traces.multi_endpoint(seed, 3000, n_contents=5, n_devices=128, follow=follow)
        r = run(orc, b)
        got = by_kind(r, RT)
        want = []
        for c in np.unique(b.content):
            idx = np.nonzero(b.content == c)[0]
            seq = [(int(b.events["src_dev"][i]), int(b.events["dst_dev"][i])) for i in idx]
            want += [(int(idx[t]), int(idx[p])) for t, p in closed_form_rt_general(seq)]
        assert sorted(got) == sorted(want)
        assert len(want) > 100
