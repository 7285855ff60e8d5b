"""Collision check (App. B) on the GPU: forged fingerprint collisions are
found exactly, genuine duplicates verify clean (through the C ABI)."""

import numpy as np
import pytest
import torch

from synth import content, traces

pytestmark = pytest.mark.gpu


def setup_trace(odp, orc, forge, misalign):
    from synth import gpu

    b = traces.plain_small(n_cycles=300)
    ev = b.events.copy()
    idx = np.flatnonzero(b.content >= 0)
    sizes = ev["bytes"][idx].astype(np.int64)
    offs = np.zeros(idx.size, dtype=np.int64)
    cur = 0
    rng = np.random.default_rng(3)
    for j in range(idx.size):
        cur += int(rng.integers(0, 16)) if misalign else (-cur) % 16
        offs[j] = cur
        cur += int(sizes[j])
    arena = torch.empty(cur + 64, dtype=torch.uint8, device="cuda")
    for j, i in enumerate(idx):
        gpu.fill_at(arena.data_ptr() + int(offs[j]), int(sizes[j]), content.RANDOM,
                    int(b.payload_seed[i]))
    views = [arena[o:o + s] for o, s in zip(offs, sizes)]
    fps = odp.fingerprint_tensors(views).cpu().numpy().view(np.uint64)
    ev["fp_lo"][idx] = fps[:, 0]
    ev["fp_hi"][idx] = fps[:, 1]
    # forge collisions: give some transfers the fingerprint of another
    # transfer with different bytes of the same length
    forged = []
    if forge:
        by_len = {}
        for j, i in enumerate(idx):
            by_len.setdefault(int(sizes[j]), []).append(j)
        for j, i in enumerate(idx):
            if len(forged) >= 12:
                break
            for k in by_len[int(sizes[j])]:
                if k < j and b.content[idx[k]] != b.content[i]:
                    ev["fp_lo"][i] = ev["fp_lo"][idx[k]]
                    ev["fp_hi"][i] = ev["fp_hi"][idx[k]]
                    forged.append(i)
                    break
        # and one with a different length
        ev["fp_lo"][idx[-1]], ev["fp_hi"][idx[-1]] = ev["fp_lo"][idx[0]], ev["fp_hi"][idx[0]]
    ptrs = np.zeros(ev.size, dtype=np.int64)
    ptrs[idx] = arena.data_ptr() + offs
    host = arena.cpu().numpy()
    payload = {int(i): host[offs[j]:offs[j] + sizes[j]] for j, i in enumerate(idx)}
    return ev, ptrs, payload, arena


def brute_collisions(ev, payload):
    first = {}
    out = []
    for i in sorted(payload):
        key = (int(ev["fp_lo"][i]), int(ev["fp_hi"][i]))
        if key not in first:
            first[key] = i
            continue
        r = first[key]
        if payload[i].size != payload[r].size or not np.array_equal(payload[i], payload[r]):
            out.append(i)
    return out


@pytest.mark.parametrize("forge,misalign", [(False, False), (True, False), (True, True)])
def test_collision_check(cuda_ok, orc, forge, misalign):
    import paper_2601_12713_b300 as odp

    ev, ptrs, payload, arena = setup_trace(odp, orc, forge, misalign)
    want = brute_collisions(ev, payload)
    assert (len(want) > 0) == forge
    d_ev = torch.from_numpy(ev.view(np.uint8).reshape(-1).copy()).cuda()
    d_ptrs = torch.from_numpy(ptrs).cuda()
    flags = torch.full((ev.size,), 7, dtype=torch.uint8, device="cuda")
    n = odp.verify_fingerprints(d_ev, ev.size, d_ptrs, flags)
    f = flags.cpu().numpy()
    assert n == len(want)
    assert sorted(np.flatnonzero(f == 1).tolist()) == want
    xfer = np.isin(ev["kind"], [2, 3, 4])
    assert np.all(np.isin(f[xfer], [0, 1])) and np.all(f[~xfer] == 7)
    # the oracle's brute-force mode and hash mode differ exactly where
    # collisions were forged
    payloads = [payload.get(i) for i in range(ev.size)]
    r_hash = orc.analyze(ev)
    r_bf = orc.analyze_bruteforce(ev, payloads)
    same = np.array_equal(r_hash.findings, r_bf.findings)
    assert same == (not forge)
