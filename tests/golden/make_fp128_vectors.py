"""Writes fp128_vectors.txt: FP128 v1 of a few fixed inputs, computed by the
oracle alone (reference values for anyone implementing the hash; the tests
check that both the oracle and the GPU reproduce them).

    python tests/golden/make_fp128_vectors.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def inputs():
    """(name, bytes) pairs: empty, short, chunk-boundary and pattern inputs."""
    yield "empty", b""
    yield "one_zero_byte", b"\x00"
    yield "abc", b"abc"
    yield "zeros_4096", bytes(4096)
    yield "zeros_4097", bytes(4097)
    yield "ramp_8192", bytes(i & 0xFF for i in range(8192))
    yield "ramp_100000", bytes((i * 7 + 3) & 0xFF for i in range(100000))
    yield "ones_65536", b"\xff" * 65536


def main():
    path = os.path.join(HERE, "fp128_vectors.txt")
    with open(path, "w") as f:
        f.write("# FP128 v1 reference vectors, written by make_fp128_vectors.py from the\n")
        f.write("# oracle: name, byte length, fp_lo, fp_hi (hex).  Inputs: see inputs().\n")
        for name, data in inputs():
            lo, hi = oracle.fp128(data)
            f.write(f"{name} {len(data)} {lo:016x} {hi:016x}\n")


if __name__ == "__main__":
    main()
