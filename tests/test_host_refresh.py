"""Host-side check of the refresh word ranges the CUDA library derives for
each slice (the words holding the ACT blocks that Algorithm 2 checks when a
slice opens), for the staggered blocks of Sec. 3 and for the aligned variant
(one block), against a brute force over every AT: the ranges must cover
every word holding an AT whose new ACT is 0 or k, stay inside the ATV, and
start and end on such words; with the paired block order of timestamp pools
(blocks b and b + k side by side) they must form one range.  Built with the
host compiler, no GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "refresh_ranges.cpp")
BUILD = os.path.join(ROOT, "tests", "host", "_build")


@pytest.fixture(scope="module")
def ranges_tool():
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "refresh_ranges")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1807_01527_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, SRC, "-o", exe], check=True)
    return exe


def _cases():
    out = []
    for k in (1, 2, 3, 4, 5, 9, 10, 30, 60, 127):
        for g in sorted({2 * k, 2 * k + 1, 3 * k + 2, 128, 130, 512, 1024, 4096}):
            if g < 2 * k:
                continue
            for w in (ww for ww in range(1, 9) if (1 << ww) > 2 * k):
                F = 32 // w
                for aligned, paired in ((False, False), (False, True), (True, False)):
                    blk = g if aligned else g // (2 * k)
                    for t in range(1, 2 * k + 2):
                        out.append((k, g, blk, F, t, int(paired), aligned))
                break  # the AT width of this k
    return out


def test_refresh_ranges_cover_exactly_the_checked_blocks(ranges_tool):
    cases = _cases()
    inp = "".join("%d %d %d %d %d %d\n" % c[:6] for c in cases)
    res = subprocess.run([ranges_tool], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    assert len([r for r in res if r]) == len(cases)
    for (k, g, blk, F, t, paired, aligned), line in zip(cases, res):
        c0n, n, lo0, hi0, lo1, hi1 = map(int, line.split())
        k2 = 2 * k
        assert c0n == t % k2
        nblk = 1 if aligned else k2
        need = set()
        for h in range(g):
            b = min(h // blk, nblk - 1)
            # storage position of AT h: paired slots 0, k, 1, k+1, ... (all of blk ATs but the last block)
            pos = h - b * blk + (2 * b if b < k else 2 * (b - k) + 1) * blk if paired else h
            if (c0n + b) % k2 in (0, k):
                need.add(pos // F)
        ranges = [(lo0, hi0), (lo1, hi1)][:n]
        covered = set()
        for lo, hi in ranges:
            assert lo <= hi and hi < -(-g // F), (k, g, aligned, t, ranges)
            assert lo in need and hi in need, (k, g, aligned, t, ranges)
            covered |= set(range(lo, hi + 1))
        assert need <= covered, (k, g, aligned, t, sorted(need - covered))
        assert (n == 0) == (not need)
        if paired:
            assert n == 1, (k, g, t, ranges)
        if aligned:
            # one block: the whole ATV every k slices, nothing in between
            assert (n == 1) == (t % k == 0)
