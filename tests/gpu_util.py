"""Helpers of the GPU parity tests: drive a library pool and the oracle on
the same seeded inputs and compare everything the close produces."""
import numpy as np

import synth

# Eq. 4: the oracle evaluates it in FP64; the library's restore evaluates it
# in FP32 where the result is provably within 8e-6 relative of the FP64 value
# (else in FP64) and stores FP32.  The 1e-5 relative bound covers both; the
# absolute floor only matters for estimates near 0, and the report decision
# (estimate >= theta) is always taken from an FP64 value near theta.
EST_RTOL = 1e-5
EST_ATOL = 1e-6


def to_device(pairs):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.uint32).view(np.int32)).cuda()


def mixed_pairs(seed: int, t: int, n: int, sizes, n_background: int = 200, bg_set: int = 6):
    """n pairs of slice t: heavy hosts with bip sets of the given sizes (each
    slice draws members at random), plus background hosts with small sets."""
    sizes = np.asarray(sizes, dtype=np.int64)
    hosts = np.concatenate([sizes, np.full(n_background, bg_set, dtype=np.int64)])
    weights = hosts.astype(np.float64) / hosts.sum()
    cdf = np.cumsum(weights)
    idx = np.arange(n, dtype=np.uint64)
    u = synth.rand_unit(synth.key(seed, 0xE0, t), idx)
    h = np.minimum(np.searchsorted(cdf, u, side="right"), len(hosts) - 1)
    j = (synth.rand_u64(synth.key(seed, 0xE1, t), idx) % hosts[h].astype(np.uint64)).astype(np.uint64)
    aip = synth.mix32(h.astype(np.uint32) + np.uint32(seed * 7919))
    with np.errstate(over="ignore"):
        bip = synth.mix32((synth.mix32(aip).astype(np.uint64) + j).astype(np.uint32))
    out = np.empty((n, 2), dtype=np.uint32)
    out[:, 0] = aip
    out[:, 1] = bip
    return out


def sp_rows(arr):
    return sorted((int(r["aip"]), float(r["est"]), int(r["nat"]), int(r["flags"])) for r in arr)


def compare_lists(gpu, oracle_rows, theta, what):
    """gpu: structured array; oracle_rows: (aip, est, nat) sorted by aip."""
    g = sp_rows(gpu)
    assert [x[0] for x in g] == [x[0] for x in oracle_rows], what
    for (aip, est, nat, flags), (aip2, est2, nat2) in zip(g, oracle_rows):
        assert nat == nat2, (what, aip, nat, nat2)
        if np.isinf(est2):
            assert np.isinf(est) and flags & 1, (what, aip)
        else:
            assert abs(est - est2) <= EST_RTOL * abs(est2) + EST_ATOL, (what, aip, est, est2)
        assert bool(flags & 2) == (est2 >= theta), (what, aip)


def check_close(pool, orc, kp, *, cap_ok=True):
    """Close the open slice on both sides and compare counts, loads,
    candidates (CSIP) and the report; returns the oracle result."""
    from paper_1807_01527_gb300 import asse
    res = orc.close_report(kp, cap=pool.out_cap, limit_extra=0)
    pool.close_slice(kp)
    np.testing.assert_array_equal(pool.counts(), res["counts"])
    np.testing.assert_array_equal(pool.loads(), res["aat"])
    if res["n_candidates"] <= pool.cap:
        compare_lists(pool.candidates(), res["candidates"], orc.theta, "csip")
        report_rows = [row for row in res["candidates"] if row[1] >= orc.theta]
        compare_lists(pool.report(), report_rows, orc.theta, "report")
    else:
        try:
            pool.candidates()
        except asse.AsseError as e:
            assert e.status == asse.ECAPACITY
        else:
            # the per-frame join can stay under the cap while the total is above it
            assert res["n_candidates"] <= pool.out_cap
    return res


def assert_state_equal(pool, orc, what="", chunk=16384):
    """The pool's counters equal the oracle's, decoded a block of ATVs at a
    time (a full-size pool holds up to a billion counters)."""
    from paper_1807_01527_gb300 import asse
    words = pool.read_pool()
    at = orc.at()
    info = dict(pool._info)
    E = words.shape[1]
    for e in range(0, E, chunk):
        part = np.ascontiguousarray(words[:, e:e + chunk])
        info["E"] = part.shape[1]
        np.testing.assert_array_equal(asse.unpack_pool(part, info, pool.g), at[:, e:e + chunk],
                                      err_msg="%s (ATVs %d..)" % (what, e))
