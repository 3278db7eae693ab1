"""Host-side logic of bench.py, no GPU: the two arms of one command line
print the same config; the counter kind follows the pool's size against the
L2 cache; the scan's algorithmic bytes follow their definition (the pool read
once plus the words the refresh rewrites)."""
import argparse

import pytest

import bench
import synth


def _args(**kw):
    a = dict(counter="auto", key_table="auto", cluster=0)
    a.update(kw)
    return argparse.Namespace(**a)


@pytest.mark.parametrize("name", ["tiny_b", "link", "long"])
def test_both_arms_share_the_config(name, monkeypatch):
    w = synth.workload(name, seed=1)
    monkeypatch.setenv("WORLD_SIZE", "1")
    a = bench.line_config(w, _args(), 1)
    assert a == bench.line_config(w, _args(), 1)
    assert a["parallelism"] == "single" and bench.line_config(w, _args(), 2)["parallelism"] == "replicas"
    assert a["k"] == w.k and a["g"] == w.g and a["pairs_per_slice"] == w.n_per_slice
    assert a["counter"] == bench.counter_for(_args(), w).upper()


def test_counter_choice_follows_pool_size_against_l2():
    # link: 4 x 65,536 ATVs x 88 words x 4 B = 92 MB, inside the 129 MB L2
    assert bench.auto_counter(10, 512, 4, 16) == "at"
    # long: 4 x 262,144 x 256 words x 4 B = 1.07 GB
    assert bench.auto_counter(60, 1024, 4, 18) == "hist"
    # an explicit choice wins
    assert bench.counter_for(_args(counter="ace"), synth.workload("long", seed=1)) == "ace"


def test_scan_bytes_are_the_pool_plus_the_refreshed_words():
    w = synth.workload("long", seed=1)
    words = 4 * (1 << 18) * 256
    info = {"pool_words": words, "words": 256, "w": 8, "fields": 4, "E": 1 << 18}
    got = bench.scan_alg_bytes(w, info, "at")
    want = 4.0 * words * (1 + 2.0 / (2 * w.k))      # two of the 2k ACT blocks rewritten
    assert got == pytest.approx(want, rel=1e-9)
