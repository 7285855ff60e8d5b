"""Seeded synthetic mapping-event logs shaped like the paper's workloads.

Events use the 64-byte little-endian record (``EVENT_DTYPE``): t_start_ns,
t_end_ns, host_addr, dev_addr, bytes, fp_lo, fp_hi (u64 each), site_id (u32),
kind (u8), src_dev (i8), dst_dev (i8), flags (u8).  The host is device -1.

Transfers carry a *content id* on the side (``TraceBundle.content``): equal ids
mean byte-identical payloads.  It is the generator's own ground truth and is
independent of any fingerprint.  For traces with real payload bytes the
content id is also a :mod:`synth.content` descriptor (``payload_seed``) that
the host and the device can materialise.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import prng

EVENT_DTYPE = np.dtype(
    [
        ("t_start_ns", "<u8"),
        ("t_end_ns", "<u8"),
        ("host_addr", "<u8"),
        ("dev_addr", "<u8"),
        ("bytes", "<u8"),
        ("fp_lo", "<u8"),
        ("fp_hi", "<u8"),
        ("site_id", "<u4"),
        ("kind", "u1"),
        ("src_dev", "i1"),
        ("dst_dev", "i1"),
        ("flags", "u1"),
    ]
)
assert EVENT_DTYPE.itemsize == 64

ALLOC, TO_DEV, FROM_DEV, DEV_TO_DEV, DELETE, KERNEL = 1, 2, 3, 4, 5, 6
HOST = -1
TRANSFER_KINDS = (TO_DEV, FROM_DEV, DEV_TO_DEV)


@dataclass
class TraceBundle:
    events: np.ndarray                 # EVENT_DTYPE
    content: np.ndarray                # int64 content id per event (-1: none)
    payload_seed: np.ndarray = None    # uint64 payload seed per event (transfers)
    labels: dict = field(default_factory=dict)


def _empty(n: int) -> np.ndarray:
    return np.zeros(n, dtype=EVENT_DTYPE)


class _Builder:
    """Appends events on a sequential timeline (one event after another)."""

    def __init__(self, gap_ns: int = 100):
        self.rows = []
        self.content = []
        self.t = 1_000
        self.gap = gap_ns

    def add(self, kind, dur_ns, src=HOST, dst=0, host_addr=0, dev_addr=0, nbytes=0,
            site=0, content=-1):
        t0 = self.t
        t1 = t0 + int(dur_ns)
        self.rows.append((t0, t1, host_addr, dev_addr, nbytes, 0, 0, site, kind, src, dst, 0))
        self.content.append(content)
        self.t = t1 + self.gap
        return len(self.rows) - 1

    def done(self) -> TraceBundle:
        ev = np.array(self.rows, dtype=EVENT_DTYPE) if self.rows else _empty(0)
        return TraceBundle(events=ev, content=np.array(self.content, dtype=np.int64))


def fill_fp_from_content(bundle: TraceBundle, seed: int = 0x0DB0) -> np.ndarray:
    """Synthetic 128-bit fingerprints: a PRNG of the content id (no payload bytes).

    Used where the payload volume would be impractical; equal content ids give
    equal fingerprints and distinct ids distinct ones (checked by the caller).
    """
    ev = bundle.events
    c = bundle.content
    m = c >= 0
    cu = c[m].astype(np.uint64)
    ev["fp_lo"][m] = prng.at(np.uint64(prng.derive(seed, 1)), cu)
    ev["fp_hi"][m] = prng.at(np.uint64(prng.derive(seed, 2)), cu)
    return ev


def transfer_duration(nbytes):
    """Timing model: 2 us + bytes / 25 GB/s."""
    return 2_000 + np.asarray(nbytes, dtype=np.int64) * 1_000 // 25_000


# ---------------------------------------------------------------------------
# The paper's worked examples (Sec. 4, Listings 1 and 2)
# ---------------------------------------------------------------------------

def listing1(n_bytes: int = 4096) -> TraceBundle:
    """Listing 1: `a` is mapped `to` in two target regions with unchanged
    content; `sum` and `prod` are `tofrom` with distinct contents.  Each region
    allocates and deletes its mappings."""
    b = _Builder()
    A, SUM, PROD = 0x10000, 0x20000, 0x30000
    # region 1: map(to:a) map(tofrom:sum)
    b.add(ALLOC, 1000, dst=0, host_addr=A, dev_addr=0xA000, nbytes=n_bytes, site=1)
    b.add(TO_DEV, transfer_duration(n_bytes), src=HOST, dst=0, host_addr=A, dev_addr=0xA000,
          nbytes=n_bytes, site=1, content=1)
    b.add(ALLOC, 1000, dst=0, host_addr=SUM, dev_addr=0xB000, nbytes=4, site=1)
    b.add(TO_DEV, transfer_duration(4), src=HOST, dst=0, host_addr=SUM, dev_addr=0xB000,
          nbytes=4, site=1, content=2)          # sum = 0
    b.add(KERNEL, 50_000, dst=0, site=1)
    b.add(FROM_DEV, transfer_duration(4), src=0, dst=HOST, host_addr=SUM, dev_addr=0xB000,
          nbytes=4, site=1, content=3)          # sum of a
    b.add(DELETE, 1000, dst=0, host_addr=SUM, dev_addr=0xB000, nbytes=4, site=1)
    b.add(DELETE, 1000, dst=0, host_addr=A, dev_addr=0xA000, nbytes=n_bytes, site=1)
    # region 2: map(to:a) map(tofrom:prod)
    b.add(ALLOC, 1000, dst=0, host_addr=A, dev_addr=0xA000, nbytes=n_bytes, site=2)
    b.add(TO_DEV, transfer_duration(n_bytes), src=HOST, dst=0, host_addr=A, dev_addr=0xA000,
          nbytes=n_bytes, site=2, content=1)    # same a: duplicate
    b.add(ALLOC, 1000, dst=0, host_addr=PROD, dev_addr=0xC000, nbytes=4, site=2)
    b.add(TO_DEV, transfer_duration(4), src=HOST, dst=0, host_addr=PROD, dev_addr=0xC000,
          nbytes=4, site=2, content=4)          # prod = 1
    b.add(KERNEL, 50_000, dst=0, site=2)
    b.add(FROM_DEV, transfer_duration(4), src=0, dst=HOST, host_addr=PROD, dev_addr=0xC000,
          nbytes=4, site=2, content=5)
    b.add(DELETE, 1000, dst=0, host_addr=PROD, dev_addr=0xC000, nbytes=4, site=2)
    b.add(DELETE, 1000, dst=0, host_addr=A, dev_addr=0xA000, nbytes=n_bytes, site=2)
    return b.done()


def listing2(n_iter: int = 8, n_bytes: int = 4096) -> TraceBundle:
    """Listing 2: a target region inside a loop with implicit tofrom mapping of
    `a`; iteration i allocates, sends v_i, runs the kernel, returns v_{i+1} and
    deletes.  The host does not modify `a` between iterations."""
    b = _Builder()
    A = 0x10000
    for i in range(n_iter):
        b.add(ALLOC, 1000, dst=0, host_addr=A, dev_addr=0xA000, nbytes=n_bytes, site=7)
        b.add(TO_DEV, transfer_duration(n_bytes), src=HOST, dst=0, host_addr=A,
              dev_addr=0xA000, nbytes=n_bytes, site=7, content=i)
        b.add(KERNEL, 40_000, dst=0, site=7)
        b.add(FROM_DEV, transfer_duration(n_bytes), src=0, dst=HOST, host_addr=A,
              dev_addr=0xA000, nbytes=n_bytes, site=7, content=i + 1)
        b.add(DELETE, 1000, dst=0, host_addr=A, dev_addr=0xA000, nbytes=n_bytes, site=7)
    return b.done()


def repeated_runs(n_runs: int = 500, n_bytes: int = 1 << 20) -> TraceBundle:
    """Shaped after the babelstream description (Sec. 7.5): the same array is
    re-allocated and re-sent with unchanged content for every repeated run,
    with the result read back changed each run."""
    b = _Builder()
    A = 0x4000_0000
    for i in range(n_runs):
        b.add(ALLOC, 1000, dst=0, host_addr=A, dev_addr=0x9000_0000, nbytes=n_bytes, site=3)
        b.add(TO_DEV, transfer_duration(n_bytes), src=HOST, dst=0, host_addr=A,
              dev_addr=0x9000_0000, nbytes=n_bytes, site=3, content=0)
        b.add(KERNEL, 30_000, dst=0, site=4)
        b.add(FROM_DEV, transfer_duration(8), src=0, dst=HOST, host_addr=A + n_bytes,
              dev_addr=0x9100_0000, nbytes=8, site=5, content=1 + i)
        b.add(DELETE, 1000, dst=0, host_addr=A, dev_addr=0x9000_0000, nbytes=n_bytes, site=3)
    return b.done()


# ---------------------------------------------------------------------------
# Random small traces (exhaustive / brute-force tests)
# ---------------------------------------------------------------------------

def random_small(seed: int, n_ops: int = 24, n_contents: int = 3, n_hosts: int = 3,
                 n_devices: int = 1, kernel_p: float = 0.15, d2d: bool = False) -> TraceBundle:
    """A random, well-formed mix of allocs, transfers, kernels and deletes over
    a few host addresses, devices and contents; some allocations stay open and
    some intervals overlap."""
    r = prng.Rng(prng.derive(seed, 77))
    b = _Builder(gap_ns=0)
    open_allocs = []  # (dev, dev_addr, host, nbytes)
    t = 1000
    rows = []
    content = []
    for _ in range(n_ops):
        u = float(r.uniform(1)[0])
        dev = int(r.integers(0, n_devices, 1)[0])
        host = 0x1000 * (1 + int(r.integers(0, n_hosts, 1)[0]))
        nbytes = 64 * (1 + int(r.integers(0, 2, 1)[0]))
        dur = int(r.integers(1, 40, 1)[0])
        t += int(r.integers(0, 20, 1)[0])  # starts nondecreasing, may overlap
        c = int(r.integers(0, n_contents, 1)[0])
        if u < kernel_p:
            rows.append((t, t + 3 * dur, 0, 0, 0, 0, 0, 1, KERNEL, HOST, dev, 0)); content.append(-1)
        elif u < 0.30:
            dev_addr = 0x100 * (1 + int(r.integers(0, n_hosts, 1)[0]))
            rows.append((t, t + dur, host, dev_addr, nbytes, 0, 0, 2, ALLOC, HOST, dev, 0)); content.append(-1)
            open_allocs.append((dev, dev_addr))
        elif u < 0.42 and open_allocs:
            k = int(r.integers(0, len(open_allocs), 1)[0])
            dv, da = open_allocs.pop(k)
            rows.append((t, t + dur, host, da, nbytes, 0, 0, 3, DELETE, HOST, dv, 0)); content.append(-1)
        else:
            w = float(r.uniform(1)[0])
            if d2d and n_devices > 1 and w < 0.2:
                src = dev
                dst = (dev + 1 + int(r.integers(0, n_devices - 1, 1)[0])) % n_devices
                kind = DEV_TO_DEV
            elif w < 0.6:
                kind, src, dst = TO_DEV, HOST, dev
            else:
                kind, src, dst = FROM_DEV, dev, HOST
            rows.append((t, t + dur, host, 0x100, nbytes, 0, 0, 4 + (kind - 2), kind, src, dst, 0))
            content.append(c)
    ev = np.array(rows, dtype=EVENT_DTYPE) if rows else _empty(0)
    return TraceBundle(events=ev, content=np.array(content, dtype=np.int64))


def two_endpoint_sequence(dirs, contents, host_addr=0x1000) -> TraceBundle:
    """Transfers only, between the host and device 0: dirs[i] is 0 for
    host->device and 1 for device->host; contents[i] the content id."""
    b = _Builder(gap_ns=1)
    for d, c in zip(dirs, contents):
        if d == 0:
            b.add(TO_DEV, 10, src=HOST, dst=0, host_addr=host_addr, nbytes=64, site=1, content=c)
        else:
            b.add(FROM_DEV, 10, src=0, dst=HOST, host_addr=host_addr, nbytes=64, site=2, content=c)
    return b.done()


def endpoint_sequence(pairs, contents, host_addr=0x1000) -> TraceBundle:
    """Transfers only: pairs[i] = (src, dst) with the host as -1 (host->device,
    device->host or device->device by the endpoints); contents[i] the content
    id."""
    b = _Builder(gap_ns=1)
    for (src, dst), c in zip(pairs, contents):
        kind = TO_DEV if src == HOST else FROM_DEV if dst == HOST else DEV_TO_DEV
        b.add(kind, 10, src=src, dst=dst, host_addr=host_addr, nbytes=64, site=kind, content=c)
    return b.done()


def multi_endpoint(seed: int, n_transfers: int, n_contents: int, n_devices: int,
                   hot: float = 0.3, follow: float = 0.7) -> TraceBundle:
    """Transfers among the host and ``n_devices`` devices.  A fraction ``hot``
    of the transfers moves content 0 (one long content group), the rest pick
    one of ``n_contents`` contents uniformly; with probability ``follow`` a
    transfer starts where the content last arrived (data moving along a chain
    of devices), else at a random endpoint."""
    r = prng.Rng(prng.derive(seed, 91))
    u = r.uniform(2 * n_transfers).reshape(2, -1)
    pick = r.integers(1, max(2, n_contents), n_transfers)
    e_src = r.integers(0, n_devices + 1, n_transfers) - 1
    e_off = r.integers(1, n_devices + 1, n_transfers)
    last = {}
    pairs, contents = [], []
    for i in range(n_transfers):
        c = 0 if u[0, i] < hot else int(pick[i])
        src = last[c] if (c in last and u[1, i] < follow) else int(e_src[i])
        # a destination other than src among the n_devices + 1 endpoints
        dst = ((src + 1) + int(e_off[i])) % (n_devices + 1) - 1
        pairs.append((src, dst))
        contents.append(c)
        last[c] = dst
    return endpoint_sequence(pairs, contents)


# ---------------------------------------------------------------------------
# Plain small workload: 128 host buffers, 1,000 map cycles, 4,000 data ops
# ---------------------------------------------------------------------------

def plain_small(seed: int = 0x0DB1, n_buffers: int = 128, n_cycles: int = 1000,
                p_dd: float = 0.30, p_rt: float = 0.10, p_ra: float = 0.05,
                p_unused_alloc: float = 0.02, p_double_send: float = 0.02,
                n_sites: int = 32) -> TraceBundle:
    """Map cycles of ALLOC, TO_DEV, KERNEL, FROM_DEV, DELETE on random
    page-aligned sub-ranges of 128 host buffers (log-uniform 4 KiB .. 1 MiB).

    * p_dd of the to-device transfers resend an earlier transfer's content;
    * p_rt of the cycles return the content unmodified;
    * p_ra of the allocations reuse an exactly freed <host_addr, bytes>;
    * p_unused_alloc of the cycles run no kernel (unused allocation);
    * p_double_send of the cycles send twice before the kernel and skip the
      read-back (the first send is overwritten unused).
    Every cycle has exactly four data-op events.  Payloads are random bytes
    from ``payload_seed`` (see :mod:`synth.content`).
    """
    r = prng.Rng(prng.derive(seed, 11))
    sizes = np.exp(np.log(4096) + r.uniform(n_buffers) * (np.log(1 << 20) - np.log(4096)))
    sizes = (np.floor(sizes / 4096).astype(np.int64) * 4096).clip(4096, 1 << 20)
    bases = 0x7F00_0000_0000 + np.concatenate([[0], np.cumsum(sizes + 65536)[:-1]])
    enter_site = r.integers(0, n_sites, n_buffers)
    exit_site = r.integers(0, n_sites, n_buffers)
    b = _Builder(gap_ns=500)
    next_content = [0]
    sent = []           # (content, nbytes) of earlier to-device transfers
    freed = []          # (buf, host_addr, nbytes) freed regions
    dev_free = {}       # nbytes -> [dev_addr]  (exact-size reuse)
    dev_top = [0x1_0000_0000]
    labels = {"dd": [], "rt": [], "ra": [], "ua": [], "ut": []}

    def new_content():
        next_content[0] += 1
        return next_content[0] - 1

    def dev_alloc(nbytes):
        lst = dev_free.get(nbytes)
        if lst:
            return lst.pop()
        a = dev_top[0]
        dev_top[0] += (nbytes + 4095) // 4096 * 4096
        return a

    for _ in range(n_cycles):
        u = r.uniform(4)
        buf = int(r.integers(0, n_buffers, 1)[0])
        dd = u[0] < p_dd and len(sent) > 0
        if u[1] < p_ra and freed:
            k = int(r.integers(0, len(freed), 1)[0])
            buf, host_addr, nbytes = freed[k]
            is_ra = True
        else:
            is_ra = False
            if dd:
                c_prev, nbytes = sent[int(r.integers(0, len(sent), 1)[0])]
                cand = np.flatnonzero(sizes >= nbytes)
                buf = int(cand[int(r.integers(0, cand.size, 1)[0])])
            else:
                nbytes = int(4096 + r.integers(0, int(sizes[buf]) - 4096 + 1, 1)[0])
            span = int(sizes[buf]) - nbytes
            off = int(r.integers(0, span // 4096 + 1, 1)[0]) * 4096
            host_addr = int(bases[buf]) + off
        if dd and is_ra:
            # resend content of the same size
            same = [c for c, nb in sent if nb == nbytes]
            if same:
                c_prev = same[int(r.integers(0, len(same), 1)[0])]
            else:
                dd = False
        c_in = c_prev if dd else new_content()
        dev_addr = dev_alloc(nbytes)
        es, xs = int(enter_site[buf]), int(exit_site[buf])
        ia = b.add(ALLOC, 1000, dst=0, host_addr=host_addr, dev_addr=dev_addr, nbytes=nbytes,
                   site=es)
        if is_ra:
            labels["ra"].append(ia)
        t1 = b.add(TO_DEV, transfer_duration(nbytes), src=HOST, dst=0, host_addr=host_addr,
                   dev_addr=dev_addr, nbytes=nbytes, site=es, content=c_in)
        if dd:
            labels["dd"].append(t1)
        sent.append((c_in, nbytes))
        if u[2] < p_double_send:
            c2 = new_content()
            t2 = b.add(TO_DEV, transfer_duration(nbytes), src=HOST, dst=0, host_addr=host_addr,
                       dev_addr=dev_addr, nbytes=nbytes, site=es, content=c2)
            sent.append((c2, nbytes))
            labels["ut"].append(t1)
            b.add(KERNEL, int(50_000 * np.exp(r.uniform(1)[0] * np.log(100))), dst=0, site=es)
        else:
            if u[3] < p_unused_alloc:
                labels["ua"].append(ia)
            else:
                b.add(KERNEL, int(50_000 * np.exp(r.uniform(1)[0] * np.log(100))), dst=0,
                      site=es)
            rt = float(r.uniform(1)[0]) < p_rt
            c_out = c_in if rt else new_content()
            ro = b.add(FROM_DEV, transfer_duration(nbytes), src=0, dst=HOST, host_addr=host_addr,
                       dev_addr=dev_addr, nbytes=nbytes, site=xs, content=c_out)
            if rt:
                labels["rt"].append(ro)
        b.add(DELETE, 1000, dst=0, host_addr=host_addr, dev_addr=dev_addr, nbytes=nbytes,
              site=xs)
        dev_free.setdefault(nbytes, []).append(dev_addr)
        freed.append((buf, host_addr, nbytes))
    out = b.done()
    out.labels = labels
    # payload seeds: one random stream per content id
    base = prng.derive(seed, 12)
    ps = np.zeros(out.events.size, dtype=np.uint64)
    m = out.content >= 0
    ps[m] = prng.at(np.uint64(base), out.content[m].astype(np.uint64))
    out.payload_seed = ps
    return out


# ---------------------------------------------------------------------------
# Trace at scale: an iterative offload solver
# ---------------------------------------------------------------------------

def skip_kernels(events: np.ndarray, fraction: float, seed: int, device: int = 0) -> np.ndarray:
    """Moves a seeded ``fraction`` of the KERNEL events of ``device`` to device
    ``device + 1`` (in place) and returns their indices.  In the iterative
    solver trace such an iteration launches nothing on the device its arrays
    are mapped to: its allocations are unused (Alg. 4), and its to-device
    transfers wait for the next iteration's kernel, where a resend of the same
    array overwrites them unused (Alg. 5)."""
    k = np.flatnonzero((events["kind"] == KERNEL) & (events["dst_dev"] == device))
    r = prng.Rng(prng.derive(seed, 23))
    moved = k[r.uniform(k.size) < fraction]
    events["dst_dev"][moved] = device + 1
    return moved


def iterative_solver(seed: int = 0x0DB4, n_iter: int = 2000, n_arrays: int = 25_000,
                     per_iter: int = 6_250, p_change: float = 0.2, n_sites: int = 500,
                     device: int = 0, p_skip_kernel: float = 0.0) -> TraceBundle:
    """Each iteration maps a seeded sample of ``per_iter`` float64 arrays
    (sizes log-uniform 1 KiB .. 64 MiB): ALLOC and TO_DEV at region entry, one
    KERNEL, FROM_DEV and DELETE at exit -- 4 * per_iter data-op events plus one
    kernel per iteration.  Before every transfer the array's content version
    changes with probability ``p_change``.  Content ids are (array, version);
    fingerprints are filled with :func:`fill_fp_from_content`.  With
    ``p_skip_kernel`` > 0 that fraction of the iterations runs its kernel on
    another device (:func:`skip_kernels`), which gives unused allocations
    and unused transfers.
    """
    r = prng.Rng(prng.derive(seed, 21))
    lo, hi = np.log(1024.0), np.log(64.0 * (1 << 20))
    sizes = (np.exp(lo + r.uniform(n_arrays) * (hi - lo)) // 8 * 8).astype(np.int64)
    sizes = np.maximum(sizes, 1024)
    host_base = 0x7F00_0000_0000 + np.concatenate([[0], np.cumsum(sizes + 4096)[:-1]])
    dev_base = 0x2_0000_0000 + np.concatenate([[0], np.cumsum((sizes + 4095) // 4096 * 4096)[:-1]])
    enter_site = r.integers(0, n_sites, n_arrays)
    exit_site = r.integers(0, n_sites, n_arrays)

    # arrays mapped per iteration: first per_iter of a seeded permutation
    mapped = np.empty((n_iter, per_iter), dtype=np.int64)
    for it in range(n_iter):
        keys = r.u64(n_arrays)
        mapped[it] = np.argpartition(keys, per_iter - 1)[:per_iter]
        mapped[it].sort()

    # content versions: two transfers per (iteration, array), in time order
    flat_arr = mapped.reshape(-1)
    n_maps = flat_arr.size
    change = (r.uniform(2 * n_maps) < p_change).reshape(n_maps, 2)
    order = np.lexsort((np.repeat(np.arange(n_iter), per_iter), flat_arr))  # by array, iter
    ch_sorted = change[order].reshape(-1)
    arr_sorted = np.repeat(flat_arr[order], 2)
    cs = np.cumsum(ch_sorted)
    # restart the count at each array
    starts = np.flatnonzero(np.r_[True, arr_sorted[1:] != arr_sorted[:-1]])
    base_cs = np.zeros_like(cs)
    seg_id = np.cumsum(np.r_[True, arr_sorted[1:] != arr_sorted[:-1]]) - 1
    prev = np.r_[0, cs[starts[1:] - 1]] if starts.size > 1 else np.array([0])
    base_cs = prev[seg_id]
    ver_sorted = (cs - base_cs).reshape(n_maps, 2)
    version = np.empty_like(ver_sorted)
    version[order] = ver_sorted
    content_to = flat_arr * 100_000 + version[:, 0]
    content_from = flat_arr * 100_000 + version[:, 1]

    # event layout per iteration: (ALLOC, TO_DEV) * per_iter, KERNEL,
    # (FROM_DEV, DELETE) * per_iter
    per = 4 * per_iter + 1
    n = n_iter * per
    ev = np.zeros(n, dtype=EVENT_DTYPE)
    content = np.full(n, -1, dtype=np.int64)
    it_idx = np.repeat(np.arange(n_iter), per_iter)
    j = np.tile(np.arange(per_iter), n_iter)
    base = it_idx * per
    i_alloc = base + 2 * j
    i_to = i_alloc + 1
    i_kernel = np.arange(n_iter) * per + 2 * per_iter
    i_from = base + 2 * per_iter + 1 + 2 * j
    i_del = i_from + 1
    a = flat_arr
    sz = sizes[a]
    for idx, kind in ((i_alloc, ALLOC), (i_to, TO_DEV), (i_from, FROM_DEV), (i_del, DELETE)):
        ev["kind"][idx] = kind
        ev["host_addr"][idx] = host_base[a]
        ev["dev_addr"][idx] = dev_base[a]
        ev["bytes"][idx] = sz
        ev["dst_dev"][idx] = device
        ev["src_dev"][idx] = HOST
    ev["src_dev"][i_from] = device
    ev["dst_dev"][i_from] = HOST
    ev["site_id"][i_alloc] = enter_site[a]
    ev["site_id"][i_to] = enter_site[a]
    ev["site_id"][i_from] = exit_site[a]
    ev["site_id"][i_del] = exit_site[a]
    content[i_to] = content_to
    content[i_from] = content_from
    ev["kind"][i_kernel] = KERNEL
    ev["dst_dev"][i_kernel] = device
    ev["src_dev"][i_kernel] = HOST
    ev["site_id"][i_kernel] = r.integers(0, n_sites, n_iter)

    dur = np.zeros(n, dtype=np.int64)
    dur[i_alloc] = 1_000
    dur[i_del] = 1_000
    dur[i_to] = transfer_duration(sz)
    dur[i_from] = transfer_duration(sz)
    dur[i_kernel] = (50_000 * np.exp(r.uniform(n_iter) * np.log(100.0))).astype(np.int64)
    gap = 200
    start = 1_000 + np.concatenate([[0], np.cumsum(dur + gap)[:-1]])
    ev["t_start_ns"] = start
    ev["t_end_ns"] = start + dur
    if p_skip_kernel > 0:
        skip_kernels(ev, p_skip_kernel, seed, device)
    return TraceBundle(events=ev, content=content)
