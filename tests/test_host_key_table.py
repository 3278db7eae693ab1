"""Host-side checks of the ingest's key table helpers: the 48-bit key mix is
a bijection (so a table entry's slot and tag identify its (aip, BH(bip)) key
exactly and a claim can never be mistaken for another key's), checked by
inverting every step; and the table size policy.  Built with the host
compiler, no GPU needed."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "key_table.cpp")
BUILD = os.path.join(ROOT, "tests", "host", "_build")
M48 = (1 << 48) - 1
C1, C2 = 0x9E3779B97F4B, 0xC2B2AE3D27D5


@pytest.fixture(scope="module")
def tool():
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "key_table")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1807_01527_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, SRC, "-o", exe], check=True)

    def run(lines):
        out = subprocess.run([exe], input="".join(l + "\n" for l in lines), capture_output=True, text=True,
                             check=True).stdout.split()
        assert len(out) == len(lines)
        return [int(v) for v in out]
    return run


def _unxorshift(y, s):
    x = y
    for _ in range(48 // s + 1):
        x = y ^ (x >> s)
    return x


def _unmix(m):
    """The inverse of every step of the mix, applied in reverse order."""
    x = _unxorshift(m, 21)
    x = (x * pow(C2, -1, 1 << 48)) & M48
    x = _unxorshift(x, 23)
    return (x * pow(C1, -1, 1 << 48)) & M48


def test_key_mix_is_a_bijection(tool):
    rng = random.Random(7)
    keys = [(0, 0), (0, 4095), (0xFFFFFFFF, 0), (0xFFFFFFFF, 4095), (1, 1), (0x80000000, 2048)]
    keys += [(rng.getrandbits(32), rng.randrange(4096)) for _ in range(20000)]
    # neighbouring keys (same host, adjacent h; adjacent hosts, same h)
    keys += [(12345, h) for h in range(4096)] + [(a, 77) for a in range(4096)]
    mixed = tool(["M %d %d" % k for k in keys])
    for (aip, h), m in zip(keys, mixed):
        assert 0 <= m <= M48
        assert _unmix(m) == (aip << 16) | h, (aip, h)
    assert len(set(mixed)) == len(set(keys))


@pytest.mark.parametrize("n_atv,pool_bytes,l2,mode,want", [
    (262144, 92 << 20, 126 << 20, 0, 0),        # link pool fits L2: no table by default
    (262144, 92 << 20, 126 << 20, 1, 20),       # forced on: 4 entries per ATV
    (262144, 92 << 20, 126 << 20, 2, 0),        # forced off
    (1 << 20, 1 << 30, 126 << 20, 0, 22),       # long pool: table, 4 M entries
    (1 << 24, 1 << 34, 126 << 20, 0, 22),       # capped at 2^22
    (4096, 1 << 20, 1 << 19, 0, 17),            # at least 2^17 (tags below 2^31)
    (4096, 1 << 20, 1 << 19, 1, 17),
    ((1 << 18) + 1, 1 << 30, 1, 0, 21),         # rounded up to a power of two
])
def test_key_table_size_policy(tool, n_atv, pool_bytes, l2, mode, want):
    assert tool(["S %d %d %d %d" % (n_atv, pool_bytes, l2, mode)]) == [want]
