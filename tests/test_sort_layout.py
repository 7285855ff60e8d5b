"""The radix sort's digit layout (host logic, no GPU): for every key width
the passes are even in number, each takes 1 to 8 bits, and together they
cover the key's bits exactly once from bit 0 up.  The same function gives
the layout on the device, where a bound on the keys known only there lowers
the width and leaves the later launched passes inactive."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("sort_layout") / "sort_layout")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2601_12713_b300", "csrc"),
                    os.path.join(ROOT, "tests", "hooks", "sort_layout.cu"), "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = {}
    for line in out.splitlines():
        f = line.split()
        kb, np_ = int(f[0]), int(f[1])
        rows[kb] = (np_, f[2:])
    return rows


def test_every_width_is_covered(layout):
    assert sorted(layout) == list(range(33))
    for kb, (npass, cells) in layout.items():
        assert npass % 2 == 0, kb
        assert npass == 0 if kb == 0 else npass >= 2
        active = [c for c in cells if c != "-"]
        assert len(active) == npass, kb
        assert all(c == "-" for c in cells[npass:]), kb  # passes past the count do nothing
        shift = 0
        for c in active:
            s, b = (int(x) for x in c.split(":"))
            assert s == shift and 1 <= b <= 8, (kb, c)
            shift += b
        # the bits are covered; a pass past them (an even count for an odd
        # number of digits) takes one bit above the keys: a stable copy
        assert shift >= kb and shift - kb <= npass, (kb, active)


def test_pass_counts(layout):
    # fewest even number of passes of at most 8 bits
    assert [layout[kb][0] for kb in (1, 8, 9, 15, 16, 17, 24, 26, 27, 32)] == \
        [2, 2, 2, 2, 2, 4, 4, 4, 4, 4]
    # 15 bits (25,000 distinct grouping keys) in two passes of 8 and 7
    assert layout[15][1][:2] == ["0:8", "8:7"]
