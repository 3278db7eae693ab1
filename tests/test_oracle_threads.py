"""The oracle's multi-threaded calls (the timed CPU baseline runs them on
every host core) give exactly what the single-thread calls give: the same
AT state after ingest and refresh, the same counts, the same candidates in
the same order, the same NAT and Eq. 4 values."""
import numpy as np
import pytest

import synth


def _mixed(seed, t, n):
    idx = np.arange(n, dtype=np.uint64)
    h = synth.rand_u64(synth.key(seed, 1, t), idx) % np.uint64(300)
    heavy = h < np.uint64(4)
    d = np.where(heavy, np.uint64(400), np.uint64(6))
    j = synth.rand_u64(synth.key(seed, 2, t), idx) % d
    aip = synth.mix32(h.astype(np.uint32) + np.uint32(seed))
    with np.errstate(over="ignore"):
        bip = synth.mix32((synth.mix32(aip).astype(np.uint64) + j).astype(np.uint32))
    return np.stack([aip, bip], axis=1).astype(np.uint32)


@pytest.mark.parametrize("k,g,r,c,u,s,mode,threads", [
    (4, 128, 4, 10, 0, 8, 0, 3), (6, 150, 4, 9, 2, 7, 0, 4), (5, 77, 5, 7, 1, 6, 1, 5),
    (10, 128, 4, 8, 4, 7, 2, 8), (3, 61, 3, 11, 1, 10, 0, 2)])
def test_threads_equal_single(oracle_mod, k, g, r, c, u, s, mode, threads):
    p = dict(k=k, theta=max(8, g // 3), g=g, r=r, c=c, u=u, s=s, **synth.method_keys(k + g))
    one = oracle_mod.Oracle.from_params(p, mode=mode)
    many = oracle_mod.Oracle.from_params(p, mode=mode)
    for t in range(2 * k + 2):
        pairs = _mixed(k + g, t, 5000 + 37 * t)
        one.ingest(pairs)
        many.ingest(pairs, threads=threads)
        np.testing.assert_array_equal(many.at(), one.at(), err_msg="ingest t=%d" % t)
        kp = k if t % 3 else 1 + t % k
        np.testing.assert_array_equal(many.counts(kp, threads=threads), one.counts(kp))
        a = one.close_report(kp)
        b = many.close_report(kp, threads=threads)
        assert a["n_candidates"] == b["n_candidates"]
        assert [x[0] for x in a["candidates"]] == [x[0] for x in b["candidates"]]
        for x, y in zip(a["candidates"], b["candidates"]):
            assert x[2] == y[2] and (x[1] == y[1] or (np.isinf(x[1]) and np.isinf(y[1])))
        cnt = one.counts(kp)
        n1, c1 = one.restore(cnt, 1 << 16)
        n2, c2 = many.restore_mt(cnt, 1 << 16, 1 << 16, threads)
        assert n1 == n2 and list(c1) == list(c2)      # frame order kept
        one.advance()
        many.advance(threads=threads)
        np.testing.assert_array_equal(many.at(), one.at(), err_msg="refresh t=%d" % t)
