"""The plane slot swizzle of the compile-time cube kernels (internal.h
plane_swizzle), compiled for the host: a permutation of each row that is its
own inverse and keeps 16-element blocks in place, and, at 96^3 with the tile
passes' thread mapping (384 threads, radix 12 then 8 along x), every
half-warp's 16 accesses of both x stages and of the y stages fall on 16
distinct 8-byte bank pairs -- the property the row rotation of the swizzle
word was chosen for."""
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2110_07670_gb300", "csrc")
DRIVER = r"""
#include <cstdio>
#include "internal.h"
int main() {
    const int ns[4] = {32, 80, 96, 160};
    for (int n : ns)
        for (int y = 0; y < n; ++y)
            for (int p = 0; p < n; ++p) std::printf("%d\n", ace::plane_swizzle(p, y, n));
}
"""


@pytest.fixture(scope="module")
def slots(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if gxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("swz")
    (d / "swz.cpp").write_text(DRIVER)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", cuda_inc, str(d / "swz.cpp"), "-o", str(d / "swz")],
                   check=True)
    vals = np.array(subprocess.run([str(d / "swz")], capture_output=True, text=True, check=True).stdout.split(),
                    dtype=np.int64)
    out, pos = {}, 0
    for n in (32, 80, 96, 160):
        out[n] = vals[pos:pos + n * n].reshape(n, n)  # [y][p]
        pos += n * n
    return out


@pytest.mark.parametrize("n", [32, 80, 96, 160])
def test_swizzle_is_a_block_preserving_involution(slots, n):
    s = slots[n]
    p = np.arange(n)
    for y in range(n):
        assert sorted(s[y]) == list(range(n))  # a permutation of the row
        assert (s[y][s[y]] == p).all()  # its own inverse
        assert (s[y] >> 4 == p >> 4).all()  # 16-element blocks stay in place


def _distinct_bank_pairs(addrs):
    """8-byte accesses of one half-warp, in elements: all on distinct 8-byte bank pairs (16 per 128 bytes)."""
    return len({a % 16 for a in addrs}) == len(addrs)


def test_tile_pass_stages_conflict_free_at_96(slots):
    n, s = 96, slots[96]  # butterfly b = thread + k 384: a half-warp's 16 lanes take 16 consecutive b
    for radix, lb in ((12, 96), (8, 8)):  # x stages: strided (radix 12), then adjacent (radix 8)
        m, nb = lb // radix, n // radix
        for base in range(0, nb * n, 16):  # half-warps: 16 consecutive butterflies
            lanes = range(base, min(base + 16, nb * n))
            for q in range(radix):
                rows = []
                for b in lanes:
                    line, i = b // nb, b % nb
                    beta, j = i // m, i % m
                    rows.append(line * n + s[line][beta * lb + j + q * m])
                assert _distinct_bank_pairs(rows), (radix, base, q)
        for base in range(0, nb * n, 16):  # y stages: lanes along x, one row per access
            lanes = range(base, min(base + 16, nb * n))
            for q in range(radix):
                cols = []
                for b in lanes:
                    i, x = b // n, b % n
                    beta, j = i // m, i % m
                    y = beta * lb + j + q * m
                    cols.append(y * n + s[y][x])
                assert _distinct_bank_pairs(cols), (radix, base, q)
