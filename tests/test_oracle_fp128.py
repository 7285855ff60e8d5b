"""Pins for the oracle's FP128 v1 (CPU only).

FP128 is project-defined, so nothing outside the project prints its values.
These tests pin the oracle against what the definition and mathematics fix:
published SplitMix64 vectors for the constants, explicit inverses of every
mixer (bijectivity, and that the stated operations run in the stated order),
lane linearity of the chunk combine (which word feeds which lane), the
left-balanced tree shape via a second tree algorithm, injectivity of every
single bit and 16-byte word, padding/length separation and collision checks.
"""

import ctypes
import itertools

import numpy as np
import pytest

from synth import content, prng

M64 = (1 << 64) - 1


def sm64(seed, i):
    """SplitMix64 output i from its published definition (Steele et al. 2014)."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def inv_odd(k):
    """Inverse of an odd k modulo 2**64 (Newton iteration)."""
    x = k
    for _ in range(6):
        x = (x * (2 - k * x)) & M64
    assert (x * k) & M64 == 1
    return x


def const(orc, i):
    o = ctypes.c_uint64()
    orc.lib().orc_constant(i, ctypes.byref(o))
    return o.value


FP_SEED = int.from_bytes(b"FP128_v1", "big")


def test_splitmix64_published_vectors(orc):
    # Published outputs for seeds 0 and 1234567.
    want0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    want1 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
             4593380528125082431, 16408922859458223821]
    o = ctypes.c_uint64()
    for i, w in enumerate(want0):
        orc.lib().orc_splitmix64(0, i, ctypes.byref(o))
        assert o.value == w
        assert int(prng.stream(0, i, 1)[0]) == w
    for i, w in enumerate(want1):
        orc.lib().orc_splitmix64(1234567, i, ctypes.byref(o))
        assert o.value == w
        assert int(prng.stream(1234567, i, 1)[0]) == w


def test_constants_are_splitmix_outputs(orc):
    assert FP_SEED == 0x46503132385F7631
    for i in range(96):
        assert const(orc, i) == sm64(FP_SEED, i)


def test_chain_step_inverse(orc):
    ks = [const(orc, i) | 1 for i in range(4)]
    rng = np.random.default_rng(1)
    o = ctypes.c_uint64()
    for which, (k1, k2) in ((0, (ks[0], ks[1])), (1, (ks[2], ks[3]))):
        for v in [0, 1, M64, 1 << 63] + [int(x) for x in rng.integers(0, 2**63, 200)]:
            orc.lib().orc_chain_step(which, v, ctypes.byref(o))
            t = (o.value * inv_odd(k2)) & M64
            t ^= t >> 32
            t = (t * inv_odd(k1)) & M64
            assert t == v


def inv_mix128(x, y, k):
    k0, k1, k2, k3 = (inv_odd(c) for c in k)
    x ^= y >> 29
    y = (y * k3) & M64
    y ^= x >> 32
    x = (x * k2) & M64
    x ^= y >> 32
    y = (y * k1) & M64
    y ^= x >> 29
    x = (x * k0) & M64
    return x, y


@pytest.mark.parametrize("which,base", [(0, 6), (1, 10), (2, 14)])
def test_mix128_inverse(orc, which, base):
    k = [const(orc, base + i) | 1 for i in range(4)]
    rng = np.random.default_rng(2 + which)
    inp = (ctypes.c_uint64 * 2)()
    out = (ctypes.c_uint64 * 2)()
    vals = [(0, 0), (1, 0), (0, 1), (M64, M64)] + [
        (int(a), int(b)) for a, b in rng.integers(0, 2**63, (200, 2))]
    for x, y in vals:
        inp[0], inp[1] = x, y
        orc.lib().orc_mix128(which, inp, out)
        assert inv_mix128(out[0], out[1], k) == (x, y)


def leaf(orc, data: bytes, r=None):
    buf = np.frombuffer(data, dtype=np.uint8).copy()
    out = (ctypes.c_uint64 * 2)()
    orc.lib().orc_chunk_leaf(buf.ctypes.data, len(data) if r is None else r, out)
    return out[0], out[1]


def leaf_root(orc, data: bytes):
    """Undo the leaf finalisation with the test's own inverse of Q."""
    kq = [const(orc, 6 + i) | 1 for i in range(4)]
    lx, ly = leaf(orc, data)
    x, y = inv_mix128(lx, ly, kq)
    return x ^ len(data) ^ const(orc, 18), y ^ const(orc, 19)


def test_lane_combine_is_linear_across_lanes(orc):
    """Words w1, w2 in different lanes (w mod 32 differs) enter independent
    chains combined by xor-linear maps, so the four chunk roots of
    {a,a'} x {b,b'} xor to zero; for two words of the same lane they do not."""
    rng = np.random.default_rng(5)
    base = bytearray(rng.integers(0, 256, 4096, dtype=np.uint8).tobytes())

    def with_words(w1, v1, w2, v2):
        d = bytearray(base)
        d[16 * w1:16 * w1 + 16] = v1
        d[16 * w2:16 * w2 + 16] = v2
        return bytes(d)

    def xor4(w1, w2):
        a, a2, b, b2 = (rng.integers(0, 256, 16, dtype=np.uint8).tobytes() for _ in range(4))
        roots = [leaf_root(orc, with_words(w1, p, w2, q)) for p in (a, a2) for q in (b, b2)]
        x = y = 0
        for rx, ry in roots:
            x ^= rx
            y ^= ry
        return x, y

    for w1, w2 in [(0, 1), (3, 200), (31, 32), (17, 255), (0, 64 + 1)]:
        assert w1 % 32 != w2 % 32
        assert xor4(w1, w2) == (0, 0)
    for w1, w2 in [(0, 32), (5, 229), (31, 255), (64, 96)]:
        assert w1 % 32 == w2 % 32
        assert xor4(w1, w2) != (0, 0)


def fp(orc, data):
    return orc.fp128(data)


def test_final_and_empty_formula(orc):
    kz = [const(orc, 14 + i) | 1 for i in range(4)]
    # empty input: Z(K_empty ^ (0, 0 ^ D_final))
    h = fp(orc, b"")
    x, y = inv_mix128(h[0], h[1], kz)
    assert (x, y) == (const(orc, 22), const(orc, 23) ^ const(orc, 21))
    # one chunk: root = leaf
    rng = np.random.default_rng(9)
    for n in (1, 15, 16, 17, 4095, 4096):
        d = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        h = fp(orc, d)
        x, y = inv_mix128(h[0], h[1], kz)
        lx, ly = leaf(orc, d)
        assert (x ^ n, y ^ 1 ^ const(orc, 21)) == (lx, ly)


def test_tree_shape_bottom_up_equivalence(orc):
    """The left-balanced tree equals bottom-up pairing where an unpaired last
    node is promoted unchanged (the RFC 6962 equivalence); node tweak = leaf
    count of the subtree."""
    kz = [const(orc, 14 + i) | 1 for i in range(4)]
    rng = np.random.default_rng(11)
    out = (ctypes.c_uint64 * 2)()
    for n_chunks in list(range(1, 40)) + [63, 64, 65, 100]:
        size = 4096 * (n_chunks - 1) + int(rng.integers(1, 4097))
        d = rng.integers(0, 256, size, dtype=np.uint8).tobytes()
        nodes = []
        for c in range(n_chunks):
            part = d[4096 * c:4096 * (c + 1)]
            nodes.append((leaf(orc, part), 1))
        while len(nodes) > 1:
            nxt = []
            for i in range(0, len(nodes), 2):
                if i + 1 == len(nodes):
                    nxt.append(nodes[i])
                    continue
                (l, cl), (r, cr) = nodes[i], nodes[i + 1]
                lt = (ctypes.c_uint64 * 2)(*l)
                rt = (ctypes.c_uint64 * 2)(*r)
                orc.lib().orc_tree_node(lt, rt, cl + cr, out)
                nxt.append(((out[0], out[1]), cl + cr))
            nodes = nxt
        root = nodes[0][0]
        h = fp(orc, d)
        x, y = inv_mix128(h[0], h[1], kz)
        assert (x ^ size, y ^ n_chunks ^ const(orc, 21)) == root


def test_tree_node_operand_order(orc):
    """node(L, R) must distinguish the left operand from the right."""
    kp = [const(orc, 10 + i) | 1 for i in range(4)]
    out = (ctypes.c_uint64 * 2)()
    L, R = (11, 22), (33, 44)
    orc.lib().orc_tree_node((ctypes.c_uint64 * 2)(*L), (ctypes.c_uint64 * 2)(*R), 2, out)
    x, y = inv_mix128(out[0], out[1], kp)
    # left enters as-is, right through G(x, y) = (y, x ^ y), count into x
    assert x == L[0] ^ R[1] ^ 2
    assert y == L[1] ^ R[0] ^ R[1] ^ const(orc, 20)


@pytest.mark.parametrize("size", [1, 15, 16, 17, 100, 4095, 4096, 4097, 12293, 16384])
def test_every_single_bit_flip_changes_hash(orc, size):
    rng = np.random.default_rng(size)
    buf = rng.integers(0, 256, size, dtype=np.uint8)
    h0 = fp(orc, buf)
    seen = {h0}
    for byte in range(size):
        orig = buf[byte]
        for bit in range(8):
            buf[byte] = orig ^ (1 << bit)
            h = fp(orc, buf)
            assert h not in seen
            seen.add(h)
        buf[byte] = orig


def test_single_word_changes_change_hash(orc):
    rng = np.random.default_rng(3)
    buf = rng.integers(0, 256, 3 * 4096 + 5, dtype=np.uint8)
    h0 = fp(orc, buf)
    for _ in range(400):
        w = int(rng.integers(0, buf.size // 16))
        save = buf[16 * w:16 * w + 16].copy()
        buf[16 * w:16 * w + 16] = rng.integers(0, 256, 16, dtype=np.uint8)
        if not np.array_equal(save, buf[16 * w:16 * w + 16]):
            assert fp(orc, buf) != h0
        buf[16 * w:16 * w + 16] = save


def test_length_and_padding_are_separated(orc):
    seen = {}
    for n in list(range(0, 300)) + [4095, 4096, 4097, 8191, 8192, 8193]:
        h = fp(orc, bytes(n))
        assert h not in seen, (n, seen.get(h))
        seen[h] = n
    rng = np.random.default_rng(4)
    for n in (1, 15, 16, 4095, 4096):
        x = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert fp(orc, x) != fp(orc, x + b"\0")


def test_position_sensitivity(orc):
    rng = np.random.default_rng(6)
    a = rng.integers(0, 256, 4096, dtype=np.uint8).tobytes()
    b = rng.integers(0, 256, 4096, dtype=np.uint8).tobytes()
    assert fp(orc, a + b) != fp(orc, b + a)
    assert fp(orc, a + a + b) != fp(orc, a + b + a)
    w = bytearray(a)
    w[0:16], w[16:32] = a[16:32], a[0:16]
    assert fp(orc, bytes(w)) != fp(orc, a)
    w = bytearray(a)
    w[0:16], w[512:528] = a[512:528], a[0:16]   # same lane, consecutive steps
    assert fp(orc, bytes(w)) != fp(orc, a)


def test_equal_content_any_alignment(orc):
    rng = np.random.default_rng(8)
    data = rng.integers(0, 256, 10_000, dtype=np.uint8)
    h = fp(orc, data)
    for off in range(1, 17):
        big = np.zeros(data.size + 32, dtype=np.uint8)
        big[off:off + data.size] = data
        assert fp(orc, big[off:off + data.size]) == h


def test_no_collisions_over_many_buffers(orc):
    seen = {}
    for variant in (content.RANDOM, content.ZERO, content.PAGE):
        for seed in range(40):
            for n in (1, 63, 4096, 4097, 20000):
                d = content.bytes_of(variant, seed, n)
                key = d.tobytes()
                h = fp(orc, d)
                if h in seen:
                    assert seen[h] == key
                seen[h] = key


def test_avalanche(orc):
    rng = np.random.default_rng(12)
    flips = []
    for _ in range(300):
        n = int(rng.integers(1, 9000))
        buf = rng.integers(0, 256, n, dtype=np.uint8)
        h0 = fp(orc, buf)
        i = int(rng.integers(0, n))
        buf[i] ^= 1 << int(rng.integers(0, 8))
        h1 = fp(orc, buf)
        flips.append(bin(h0[0] ^ h1[0]).count("1") + bin(h0[1] ^ h1[1]).count("1"))
    assert abs(np.mean(flips) - 64.0) < 2.0


def load_vectors():
    """(name, data, (lo, hi)) from tests/golden/fp128_vectors.txt with the
    inputs of the script that wrote it."""
    import importlib.util
    import os

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_fp128_vectors",
                                                  os.path.join(here, "make_fp128_vectors.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    data = dict(mod.inputs())
    out = []
    for line in open(os.path.join(here, "fp128_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, length, lo, hi = line.split()
        assert len(data[name]) == int(length)
        out.append((name, data[name], (int(lo, 16), int(hi, 16))))
    return out


def test_reference_vectors_reproduce():
    import oracle

    vecs = load_vectors()
    assert len(vecs) == 8
    for name, data, want in vecs:
        assert oracle.fp128(data) == want, name
