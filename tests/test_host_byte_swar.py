"""Host-side check of the word-level tests on byte-wide counter fields
(seven-bit counters in eight bits, four to a word), which the scan uses to
count active ATs (Algorithm 1), clear them (Algorithm 2) and age the aging
counters: exhaustive over every value and range of a byte, in every byte
position, against the per-byte definitions.  Built with the host compiler,
no GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "byte_swar.cpp")
BUILD = os.path.join(ROOT, "tests", "host", "_build")


def test_byte_swar_exhaustive():
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "vector_types.h")):
        pytest.skip("needs g++ and the CUDA headers")
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "byte_swar")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1807_01527_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, SRC, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.split()[-1] == "ok", out.stdout
