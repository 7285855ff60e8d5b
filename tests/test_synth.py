"""CPU checks of the seeded input generators (shapes, determinism, the
properties the workloads are defined by)."""

import numpy as np

from synth import content, prng, traces


def test_content_words_are_splitmix_outputs():
    w = content.words(content.RANDOM, 0, 0, 3)
    assert [int(x) for x in w] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    page = content.words(content.PAGE, 5, 0, 1024)
    assert np.array_equal(page[:512], page[512:])
    assert not content.bytes_of(content.ZERO, 1, 100).any()
    b = content.bytes_of(content.RANDOM, 7, 13, word_offset=2)
    assert np.array_equal(b, content.words(content.RANDOM, 7, 2, 2).view(np.uint8)[:13])


def test_batched_ragged_shape():
    sizes, offs, seeds, dup_of = content.batched_ragged(seed=1, n=20_000, total=320 << 20,
                                                        max_size=32 << 20)
    assert sizes.sum() == 320 << 20
    assert sizes.min() >= 1 and sizes.max() <= 32 << 20
    assert np.all(offs % 16 == 0) and np.all(np.diff(offs) >= sizes[:-1])
    d = np.flatnonzero(dup_of >= 0)
    assert 0.37 < d.size / sizes.size < 0.43
    assert np.all(dup_of[d] < d) and np.all(dup_of[dup_of[d]] < 0)
    assert np.array_equal(sizes[d], sizes[dup_of[d]]) and np.array_equal(seeds[d], seeds[dup_of[d]])
    med = np.median(sizes)
    assert 3000 < med < 5500
    again = content.batched_ragged(seed=1, n=20_000, total=320 << 20, max_size=32 << 20)
    assert all(np.array_equal(x, y) for x, y in zip((sizes, offs, seeds, dup_of), again))


def test_plain_small_shape():
    b = traces.plain_small()
    ev = b.events
    ops = np.isin(ev["kind"], [1, 2, 3, 4, 5])
    assert ops.sum() == 4000
    assert np.all(np.diff(ev["t_start_ns"].astype(np.int64)) >= 0)
    assert np.all(ev["t_end_ns"] >= ev["t_start_ns"])
    sent = ev["kind"] == traces.TO_DEV
    assert sent.sum() >= 1000
    assert len(b.labels["dd"]) > 200 and len(b.labels["rt"]) > 50


def test_iterative_solver_shape():
    b = traces.iterative_solver(n_iter=10, n_arrays=1000, per_iter=250, n_sites=50)
    ev = b.events
    assert ev.size == 10 * (4 * 250 + 1)
    assert (ev["kind"] == traces.KERNEL).sum() == 10
    assert np.all(np.diff(ev["t_start_ns"].astype(np.int64)) >= 0)
    per = 4 * 250 + 1
    first = ev[:per]
    assert list(first["kind"][:4]) == [traces.ALLOC, traces.TO_DEV, traces.ALLOC, traces.TO_DEV]
    assert first["kind"][500] == traces.KERNEL
    # each array mapped at most once per iteration
    to = ev["kind"] == traces.TO_DEV
    it = np.arange(ev.size) // per
    pairs = set(zip(it[to].tolist(), ev["host_addr"][to].tolist()))
    assert len(pairs) == to.sum()


def test_synthetic_fingerprints_follow_content_ids():
    b = traces.iterative_solver(n_iter=6, n_arrays=300, per_iter=100, n_sites=10)
    traces.fill_fp_from_content(b)
    ev = b.events
    m = b.content >= 0
    fp = ev["fp_lo"][m].astype(object) * (1 << 64) + ev["fp_hi"][m].astype(object)
    c = b.content[m]
    by_c = {}
    for ci, f in zip(c.tolist(), fp.tolist()):
        assert by_c.setdefault(ci, f) == f
    assert len(set(by_c.values())) == len(by_c)


def test_rng_draws():
    r = prng.Rng(3)
    x = r.integers(5, 9, 10_000)
    assert x.min() == 5 and x.max() == 8
    u = prng.Rng(4).uniform(10_000)
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.02
