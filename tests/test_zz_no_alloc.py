"""asse_restore_static, the restore for callers that cannot allocate device
memory while they close slices (their cudaMalloc/cudaFree could stall a
latency-bound pipeline, or their host forbids allocation after start-up),
must give exactly what asse_restore gives: the same candidates and the same
report, with identical NAT and estimates, on two calls in a row (the second
call reuses the fixed scratch the first one left behind).

This file is collected last on purpose; it also passes alone in a fresh
process, where its first call sets the scratch address up."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu


def _rows(arr):
    return sorted((int(r["aip"]), int(r["nat"]), float(r["est"]), int(r["flags"])) for r in arr)


def _same(got, want):
    g, w = _rows(got), _rows(want)
    assert [x[0] for x in g] == [x[0] for x in w]
    for a, b in zip(g, w):
        assert a[1] == b[1] and a[3] == b[3], (a, b)
        assert a[2] == b[2] or (np.isinf(a[2]) and np.isinf(b[2])), (a, b)   # the same restore kernel: bit-equal


def test_static_restore_matches_pool_restore_twice_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_01527_gb300 import asse, build
    build.build()
    L = asse.lib()
    w = synth.workload("tiny_b")
    pool = asse.Pool(w.params)
    cap = 4096
    cand = torch.zeros(cap * 4, dtype=torch.int32, device="cuda")      # cap 16-byte records
    rep = torch.zeros(cap * 4, dtype=torch.int32, device="cuda")
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    vp = ctypes.c_void_p
    checked = 0
    for t in range(4):
        pool.ingest(to_device(w.pairs(t)))
        pool.scan(w.k)
        pool.restore()
        want_c, want_r = pool.candidates(), pool.report()
        for _call in range(2):
            rc = L.asse_restore_static(pool._h, cap, vp(cand.data_ptr()), vp(rep.data_ptr()), cap,
                                       vp(counters.data_ptr()))
            assert rc == asse.OK, L.asse_last_error(pool._h)
            torch.cuda.synchronize()
            n = counters.cpu().numpy().view(np.uint64)
            assert n[3] == 0 and n[0] == want_c.size and n[1] == want_r.size
            _same(cand.cpu().numpy().view(asse.SP_DTYPE)[: int(n[0])], want_c)
            _same(rep.cpu().numpy().view(asse.SP_DTYPE)[: int(n[1])], want_r)
            checked += int(n[0])
        pool.advance()
    assert checked > 0
    # after a close of two windows, the call restores the selected window
    pool.ingest(to_device(w.pairs(4)))
    pool.close_slice_multi([w.k, 2])
    for m in (1, 0):
        pool.select_window(m)
        want_c = pool.candidates()
        rc = L.asse_restore_static(pool._h, cap, vp(cand.data_ptr()), vp(rep.data_ptr()), cap,
                                   vp(counters.data_ptr()))
        assert rc == asse.OK, L.asse_last_error(pool._h)
        torch.cuda.synchronize()
        n = counters.cpu().numpy().view(np.uint64)
        assert n[3] == 0 and n[0] == want_c.size
        _same(cand.cpu().numpy().view(asse.SP_DTYPE)[: int(n[0])], want_c)
    # sizes beyond the fixed scratch are refused with a clear error
    too_many = asse.lib().asse_restore_static(pool._h, 65537, vp(cand.data_ptr()), vp(rep.data_ptr()), cap,
                                              vp(counters.data_ptr()))
    assert too_many == asse.EINVAL
    assert b"exceeds the static restore scratch" in L.asse_last_error(pool._h)
    pool.close()
