"""Parity at the full size of the long-window workload (k=60, 32 Mi pairs
per slice, 4 x 262,144 ATVs of g=1024 ATs: a 1 GB AT pool, 0.87 GB with
aging counters), for the first two slices, with each counter kind: the
state after ingest and after the refresh, counts, loads, candidates and
report against the oracle (timestamps, aging counters, and timestamps with
slice counts)."""
import numpy as np
import pytest

import synth
from gpu_util import assert_state_equal, check_close, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1807_01527_gb300 import asse, build
    build.build()
    oracle.build()
    return asse, oracle, torch


@pytest.fixture(scope="module")
def long_slices():
    w = synth.workload("long")
    return w, [w.pairs(t) for t in range(2)]


@pytest.mark.parametrize("counter", ["at", "ace", "hist"])
def test_long_full_size_two_slices(mods, long_slices, counter):
    asse, oracle, torch = mods
    w, slices = long_slices
    pool = asse.Pool(w.params, counter=counter)
    orc = oracle.Oracle.from_params(w.params, mode=1 if counter == "ace" else 0)
    for t, pairs in enumerate(slices):
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        assert_state_equal(pool, orc, "after ingest t=%d" % t)
        check_close(pool, orc, w.k)
        orc.advance()
        assert_state_equal(pool, orc, "after refresh t=%d" % t)
    pool.close()
