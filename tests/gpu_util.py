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


def mixed_pairs(seed: int, t: int, n: int, sizes, n_background: int = 200, bg_set: int = 6, live=None):
    """n pairs of slice t: heavy hosts with bip sets of the given sizes (each
    slice draws members at random), plus background hosts with small sets.
    live (one bool per heavy host) leaves the hosts that are not live out of
    this slice."""
    sizes = np.asarray(sizes, dtype=np.int64)
    hosts = np.concatenate([sizes, np.full(n_background, bg_set, dtype=np.int64)])
    weights = hosts.astype(np.float64)
    if live is not None:
        weights[: len(sizes)] *= np.asarray(live, dtype=np.float64)
    weights /= weights.sum()
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


def interval_pairs(seed: int, t: int, k: int, sizes, starts, lens, n_background: int = 3000):
    """Slice t of a stream whose heavy hosts enter and leave the window: host
    i is live in slices [starts[i], starts[i] + lens[i]) and then emits
    ceil(4 sizes[i] / k) members of its bip set per slice, cycling through
    the set, so its cardinality in a k-slice window grows over the first k/4
    live slices and falls back to zero k slices after its last one.  Plus
    n_background pairs of small background hosts.  Shuffled."""
    parts = []
    for i, (m, s0, ln) in enumerate(zip(sizes, starts, lens)):
        if not (s0 <= t < s0 + ln):
            continue
        per = -(-4 * int(m) // k)
        j = (np.arange(per, dtype=np.uint64) + np.uint64(t * per)) % np.uint64(m)
        aip = synth.mix32(np.full(per, 0x7F000000 + i + seed * 7919, dtype=np.uint32))
        with np.errstate(over="ignore"):
            bip = synth.mix32((synth.mix32(aip).astype(np.uint64) + j).astype(np.uint32))
        parts.append(np.stack([aip, bip], axis=1))
    parts.append(mixed_pairs(seed, t, n_background, [], n_background=400, bg_set=5))
    out = np.concatenate(parts).astype(np.uint32)
    order = np.argsort(synth.rand_u64(synth.key(seed, 0xE2, t), np.arange(out.shape[0], dtype=np.uint64)),
                       kind="stable")
    return np.ascontiguousarray(out[order])


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


def at_positions(info: dict, g: int) -> np.ndarray:
    """Storage position of every AT h of an ATV, as asse_info describes it:
    h itself, or with paired blocks (the 2k ACT blocks stored in the order 0,
    k, 1, k+1, ...) h - b*block + s*block for h in block b, s its slot."""
    h = np.arange(g)
    if not info["paired"]:
        return h
    k, blk = info["k"], info["block"]
    b = np.minimum(h // blk, 2 * k - 1)
    s = np.where(b < k, 2 * b, 2 * (b - k) + 1)
    return h - b * blk + s * blk


def unpack_pool(words: np.ndarray, info: dict, g: int) -> np.ndarray:
    """Packed pool words [r][E][words] -> counter values [r][E][g] (uint8):
    the counter at position p is field p % fields, bits [j*w, j*w+w), of word
    p // fields, and AT h sits at position at_positions(h) (w, fields and the
    block order as asse_info reports them)."""
    w, F = info["w"], info["fields"]
    words = words.reshape(-1, info["E"], info["words"])
    pos = at_positions(info, g)
    sel = words[:, :, pos // F]
    return ((sel >> ((pos % F) * w).astype(np.uint32)) & ((1 << w) - 1)).astype(np.uint8)


def state(pool) -> np.ndarray:
    """Counter values [r][E][g] of a library pool, decoded from its packed words."""
    return unpack_pool(pool.read_pool(), pool._info, pool.g)


def assert_state_equal(pool, orc, what="", chunk=16384):
    """The pool's counters equal the oracle's, decoded a block of ATVs at a
    time (a full-size pool holds up to a billion counters)."""
    words = pool.read_pool()
    at = orc.at()
    info = dict(pool._info)
    E = words.shape[1]
    for e in range(0, E, chunk):
        part = np.ascontiguousarray(words[:, e:e + chunk])
        info["E"] = part.shape[1]
        np.testing.assert_array_equal(unpack_pool(part, info, pool.g), at[:, e:e + chunk],
                                      err_msg="%s (ATVs %d..)" % (what, e))
