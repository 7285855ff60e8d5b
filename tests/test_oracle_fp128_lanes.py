"""Pins for the chunk-leaf lane stage of the oracle's FP128 v1 (CPU only).

The lane stage of a chunk is: two 64-bit chains per lane started from
C[32+2l] and C[33+2l], one chain step per word of the lane, a two-round
Feistel finish (a ^= b*Kodd4, then b ^= a*Kodd5), a 32-lane tree with
node = L ^ G(R), and the leaf = Q(root ^ (r ^ C[18], C[19])) (the FP128 v1
definition beside odp_fingerprint in include/odp.h; the paper, Sec. 5.1,
asks only for a collision-free hash of each transfer's bytes).

Nothing here recomputes the forward definition.  Each test runs a step
backwards with the test's own inverses, or checks a closed form the tree
implies, so a swapped start constant, a Feistel finish in the other order,
G on the left operand or a wrong leaf constant each fail:

  * inverting the Feistel finish and the eight chain steps of every lane,
    with the chunk's own words, must land on SplitMix64 outputs 32+2l and
    33+2l of the FP128 seed;
  * in the 32-lane tree the right operand goes through G at each level
    where the lane is a right child, so lane l reaches the root through
    G^(popcount(l) mod 3) (G has order 3); a change confined to lane l must
    move the pre-Q root by exactly that image of the lane's change;
  * inverting Q of a leaf and removing the closed-form root must leave
    (r ^ C[18], C[19]) for every valid length r;
  * the worked examples in tests/golden/fp128_worked.txt pass all of the
    above step by step, and the oracle reproduces every stored value.
"""

import ctypes
import os

import numpy as np
import pytest

M64 = (1 << 64) - 1
FP_SEED = int.from_bytes(b"FP128_v1", "big")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fp128_worked.txt")


def sm64(seed, i):
    """SplitMix64 output i from its published definition (Steele et al. 2014)."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def C(i):
    return sm64(FP_SEED, i)


def Kodd(i):
    return C(i) | 1


def inv_odd(k):
    x = k
    for _ in range(6):
        x = (x * (2 - k * x)) & M64
    assert (x * k) & M64 == 1
    return x


def inv_chain(t, k1, k2):
    """Inverse of S(v) = ((v*k1) ^ (v*k1) >> 32) * k2."""
    t = (t * inv_odd(k2)) & M64
    t ^= t >> 32  # the fold keeps the top half, so it is its own inverse
    return (t * inv_odd(k1)) & M64


def inv_feistel(a, b):
    """Inverse of a ^= b*Kodd(4); b ^= a*Kodd(5) (undo the second round first)."""
    b ^= (a * Kodd(5)) & M64
    a ^= (b * Kodd(4)) & M64
    return a, b


def inv_mix(x, y, base):
    k0, k1, k2, k3 = (inv_odd(Kodd(base + i)) for i in range(4))
    x ^= y >> 29
    y = (y * k3) & M64
    y ^= x >> 32
    x = (x * k2) & M64
    x ^= y >> 32
    y = (y * k1) & M64
    y ^= x >> 29
    x = (x * k0) & M64
    return x, y


def G(x, y):
    return y, x ^ y


def G_pow(v, k):
    for _ in range(k % 3):
        v = G(*v)
    return v


def words_of(chunk: bytes):
    """The chunk zero-padded to 4096 bytes as 256 little-endian (lo, hi) words."""
    p = chunk + bytes(4096 - len(chunk))
    return [(int.from_bytes(p[16 * i:16 * i + 8], "little"),
             int.from_bytes(p[16 * i + 8:16 * i + 16], "little")) for i in range(256)]


def lane_state(orc, chunk: bytes, lane: int):
    buf = np.frombuffer(chunk, dtype=np.uint8).copy()
    out = (ctypes.c_uint64 * 2)()
    orc.lib().orc_lane_state(buf.ctypes.data, len(chunk), lane, out)
    return out[0], out[1]


def leaf(orc, chunk: bytes):
    buf = np.frombuffer(chunk, dtype=np.uint8).copy()
    out = (ctypes.c_uint64 * 2)()
    orc.lib().orc_chunk_leaf(buf.ctypes.data, len(chunk), out)
    return out[0], out[1]


def unwind_lane(a, b, words, lane):
    """Run lane `lane` backwards from its finished state to its start state."""
    a, b = inv_feistel(a, b)
    for j in reversed(range(8)):
        lo, hi = words[lane + 32 * j]
        a = inv_chain(a, Kodd(0), Kodd(1)) ^ lo
        b = inv_chain(b, Kodd(2), Kodd(3)) ^ hi
    return a, b


def closed_form_root(lanes):
    x = y = 0
    for lane, s in enumerate(lanes):
        gx, gy = G_pow(s, bin(lane).count("1"))
        x ^= gx
        y ^= gy
    return x, y


def chunks():
    rng = np.random.default_rng(2024)
    out = [bytes(4096), b"\0", b"\x61"]
    for r in (1, 15, 16, 17, 512, 2000, 4095, 4096):
        out.append(rng.integers(0, 256, r, dtype=np.uint8).tobytes())
    return out


@pytest.mark.parametrize("idx", range(11))
def test_lanes_unwind_to_their_start_constants(orc, idx):
    chunk = chunks()[idx]
    words = words_of(chunk)
    for lane in range(32):
        a, b = lane_state(orc, chunk, lane)
        assert unwind_lane(a, b, words, lane) == (C(32 + 2 * lane), C(33 + 2 * lane)), lane


def test_unwinding_discriminates_the_lane_variants(orc):
    """The unwinding above fails for the plausible mistakes it is meant to
    catch: Feistel rounds undone in the other order, a lane read as
    consecutive words, or the start constants of the two chains swapped."""
    rng = np.random.default_rng(7)
    chunk = rng.integers(0, 256, 4096, dtype=np.uint8).tobytes()
    words = words_of(chunk)
    starts = [(C(32 + 2 * l), C(33 + 2 * l)) for l in range(32)]
    for lane in (0, 5, 31):
        a, b = lane_state(orc, chunk, lane)
        # other Feistel order
        a2 = a ^ ((b * Kodd(4)) & M64)
        b2 = b ^ ((a2 * Kodd(5)) & M64)
        for j in reversed(range(8)):
            lo, hi = words[lane + 32 * j]
            a2 = inv_chain(a2, Kodd(0), Kodd(1)) ^ lo
            b2 = inv_chain(b2, Kodd(2), Kodd(3)) ^ hi
        assert (a2, b2) != starts[lane]
        # words 8*lane .. 8*lane+7 instead of lane, lane+32, ...
        a3, b3 = inv_feistel(a, b)
        for j in reversed(range(8)):
            lo, hi = words[8 * lane + j]
            a3 = inv_chain(a3, Kodd(0), Kodd(1)) ^ lo
            b3 = inv_chain(b3, Kodd(2), Kodd(3)) ^ hi
        assert (a3, b3) != starts[lane]
        assert unwind_lane(a, b, words, lane) != starts[lane][::-1]


def test_lane_tree_applies_G_to_right_operands(orc):
    """A change confined to lane l moves the pre-Q root by G^popcount(l) of the
    lane's change, for every lane; with G on the left operand the exponent
    would be (5 - popcount(l)), which differs for every lane whose popcount is
    not 1 mod 3 away -- checked to fail below."""
    rng = np.random.default_rng(11)
    base = rng.integers(0, 256, 4096, dtype=np.uint8).tobytes()
    base_lanes = [lane_state(orc, base, l) for l in range(32)]
    bq = inv_mix(*leaf(orc, base), 6)
    left_variant_fails = 0
    for lane in range(32):
        j = int(rng.integers(0, 8))
        w = lane + 32 * j
        mod = bytearray(base)
        mod[16 * w:16 * w + 16] = rng.integers(0, 256, 16, dtype=np.uint8).tobytes()
        mod = bytes(mod)
        for other in range(32):
            if other != lane:
                assert lane_state(orc, mod, other) == base_lanes[other]
        ml = lane_state(orc, mod, lane)
        d_lane = (ml[0] ^ base_lanes[lane][0], ml[1] ^ base_lanes[lane][1])
        assert d_lane != (0, 0)
        mq = inv_mix(*leaf(orc, mod), 6)
        d_root = (mq[0] ^ bq[0], mq[1] ^ bq[1])
        pc = bin(lane).count("1")
        assert d_root == G_pow(d_lane, pc), lane
        if d_root != G_pow(d_lane, 5 - pc):
            left_variant_fails += 1
    assert left_variant_fails >= 20


@pytest.mark.parametrize("idx", range(11))
def test_leaf_constants(orc, idx):
    """Q^-1(leaf) = closed-form root ^ (r ^ C[18], C[19])."""
    chunk = chunks()[idx]
    root = closed_form_root([lane_state(orc, chunk, l) for l in range(32)])
    x, y = inv_mix(*leaf(orc, chunk), 6)
    assert x ^ root[0] == len(chunk) ^ C(18)
    assert y ^ root[1] == C(19)


def load_worked():
    consts, ex = {}, {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "const":
            consts[int(f[1])] = int(f[2], 16)
            continue
        name, step = f[0], f[1]
        d = ex.setdefault(name, {})
        if len(f) == 5:
            d.setdefault(step, {})[int(f[2])] = (int(f[3], 16), int(f[4], 16))
        else:
            d[step] = (int(f[2], 16), int(f[3], 16))
    return consts, ex


def worked_input(name):
    if name == "empty":
        return b""
    if name == "byte61":
        return b"\x61"
    if name == "word37":
        d = bytearray(4096)
        d[16 * 37:16 * 37 + 8] = (0x0123456789ABCDEF).to_bytes(8, "little")
        d[16 * 37 + 8:16 * 37 + 16] = (0xFEDCBA9876543210).to_bytes(8, "little")
        return bytes(d)
    if name == "zero4096_01":
        return bytes(4096) + b"\x01"
    raise KeyError(name)


WORKED_NAMES = ["empty", "byte61", "word37", "zero4096_01"]


def test_worked_examples_are_consistent_with_the_definition():
    """Every stored step of the worked examples is checked by inversion or by
    the closed-form lane tree, against constants the test derives itself."""
    consts, ex = load_worked()
    assert sorted(ex) == sorted(WORKED_NAMES)
    for i, v in consts.items():
        assert v == C(i)
    for name in ("byte61", "word37"):
        data = worked_input(name)
        e = ex[name]
        words = words_of(data)
        lanes = [e["lane"][l] for l in range(32)]
        for l, (a, b) in enumerate(lanes):
            assert unwind_lane(a, b, words, l) == (C(32 + 2 * l), C(33 + 2 * l))
        (step_name,) = [k for k in e if k.endswith("_step")]
        lane = int(step_name[4:-5])
        steps = e[step_name]
        a, b = C(32 + 2 * lane), C(33 + 2 * lane)
        for j in range(8):
            lo, hi = words[lane + 32 * j]
            sa, sb = steps[j]
            assert inv_chain(sa, Kodd(0), Kodd(1)) ^ lo == a
            assert inv_chain(sb, Kodd(2), Kodd(3)) ^ hi == b
            a, b = sa, sb
        assert inv_feistel(*lanes[lane]) == (a, b)
        assert e["lane_root"] == closed_form_root(lanes)
        r = len(data)
        assert e["leaf_in"] == (e["lane_root"][0] ^ r ^ C(18), e["lane_root"][1] ^ C(19))
        assert inv_mix(*e["leaf"], 6) == e["leaf_in"]
        assert e["final_in"] == (e["leaf"][0] ^ r, e["leaf"][1] ^ 1 ^ C(21))
        assert inv_mix(*e["out"], 14) == e["final_in"]
    e = ex["zero4096_01"]
    for k in ("leaf0", "leaf1"):
        rx, ry = e[k + "_root"]
        r = 4096 if k == "leaf0" else 1
        assert inv_mix(*e[k], 6) == (rx ^ r ^ C(18), ry ^ C(19))
    gx, gy = G(*e["leaf1"])
    assert e["node_in"] == (e["leaf0"][0] ^ gx ^ 2, e["leaf0"][1] ^ gy ^ C(20))
    assert inv_mix(*e["node"], 10) == e["node_in"]
    assert e["final_in"] == (e["node"][0] ^ 4097, e["node"][1] ^ 2 ^ C(21))
    assert inv_mix(*e["out"], 14) == e["final_in"]
    e = ex["empty"]
    assert e["final_in"] == (C(22), C(23) ^ C(21))
    assert inv_mix(*e["out"], 14) == e["final_in"]


def test_oracle_reproduces_worked_examples(orc):
    _, ex = load_worked()
    for name in WORKED_NAMES:
        data = worked_input(name)
        e = ex[name]
        assert orc.fp128(data) == e["out"], name
        if "lane" in e:
            for l in range(32):
                assert lane_state(orc, data, l) == e["lane"][l], (name, l)
            assert leaf(orc, data) == e["leaf"]
    e = ex["zero4096_01"]
    data = worked_input("zero4096_01")
    assert leaf(orc, data[:4096]) == e["leaf0"]
    assert leaf(orc, data[4096:]) == e["leaf1"]
    assert closed_form_root([lane_state(orc, data[:4096], l) for l in range(32)]) == e["leaf0_root"]
    assert closed_form_root([lane_state(orc, data[4096:], l) for l in range(32)]) == e["leaf1_root"]
