"""The bounded device-side waits: a wait on an mbarrier that nothing
completes gives up after its bound and reports ASSE_ETIMEOUT, the kernel
returns, and the CUDA context stays usable (a pool closes a slice exactly as
the oracle does right after it).  The failure is made by a barrier that
nothing arrives at, with a bound of about a millisecond: no fault, no trap,
no hang."""
import numpy as np
import pytest

import synth
from gpu_util import check_close, state, to_device

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


def test_wait_that_completes_returns_ok(mods):
    asse, _oracle, _torch = mods
    rc, waited = asse.probe_bounded_wait(1 << 30, complete=True)
    assert rc == asse.OK
    assert waited < 1 << 30


@pytest.mark.parametrize("limit", [1 << 12, 2_000_000])
def test_wait_that_never_completes_times_out(mods, limit):
    asse, oracle, torch = mods
    rc, waited = asse.probe_bounded_wait(limit, complete=False)
    assert rc == asse.ETIMEOUT
    assert limit < waited < limit + (1 << 24)      # gave up just after its bound
    assert asse.lib().asse_strerror(rc) == b"ASSE_ETIMEOUT"
    # the context is still usable: a small pool's close equals the oracle's
    w = synth.workload("tiny_b")
    pool = asse.Pool(w.params)
    orc = oracle.Oracle.from_params(w.params)
    pairs = w.pairs(0)
    pool.ingest(to_device(pairs))
    orc.ingest(pairs)
    check_close(pool, orc, w.k)
    orc.advance()
    np.testing.assert_array_equal(state(pool), orc.at())
    torch.cuda.synchronize()
    pool.close()
