"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same
seeded inputs: the AT pool state bit-exact after every ingest and every
refresh, per-ATV counts and row-frame loads exact, candidate and report sets
exact, NAT exact, Eq. 4 estimates within 1e-5 relative."""
import numpy as np
import pytest

import synth
from gpu_util import check_close, compare_lists, interval_pairs, mixed_pairs, state, to_device

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


def _params(k, g, r, c, u, s, theta, seed=1):
    return dict(k=k, theta=theta, g=g, r=r, c=c, u=u, s=s, **synth.method_keys(seed))


def test_tiny_b_every_slice(mods):
    """Tiny workload with per-host bip sets (k=4, 16 slices of 65,536 pairs)."""
    asse, oracle, torch = mods
    w = synth.workload("tiny_b")
    pool = asse.Pool(w.params)
    orc = oracle.Oracle.from_params(w.params)
    for t in range(w.slices):
        pairs = w.pairs(t)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after ingest t={t}")
        res = check_close(pool, orc, w.k)
        assert set(w.planted_aip.tolist()) <= {a for a, e, _n in res["report"]}
        orc.advance()
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after refresh t={t}")
    pool.close()


def test_tiny_saturated_state_and_capacity(mods):
    """Tiny workload as specified (bips uniform over 2^24): the pool
    saturates, every ATV is super, and the restore must report that it needs
    more than restore_cap tuples instead of returning a partial list."""
    asse, oracle, torch = mods
    w = synth.workload("tiny")
    pool = asse.Pool(w.params)
    orc = oracle.Oracle.from_params(w.params)
    for t in range(6):
        pairs = w.pairs(t)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at())
        cnt = orc.counts(w.k)
        pool.close_slice(w.k)
        np.testing.assert_array_equal(pool.counts(), cnt)
        np.testing.assert_array_equal(pool.loads(), orc.aat(cnt))
        n_orc, _ = orc.restore(cnt, pool.cap, limit_extra=0)
        if n_orc > pool.cap:
            with pytest.raises(asse.AsseError) as ei:
                pool.report()
            assert ei.value.status == asse.ECAPACITY and ei.value.n_needed > pool.cap
        orc.advance()
        np.testing.assert_array_equal(state(pool), orc.at())


# (k, g, r, c, u, s, counter): every counter width 1..8, r from 2 to 8,
# frames 1..16, g not a multiple of the fields per word; ATVs of 8 to 88
# words, so both scan tile layouts (padded lane segments, and whole tiles
# when a segment is an odd number of 16-byte units) are covered.  Every case
# runs 2k+3 slices, past the point where C0 = t mod 2k wraps.
CASES = [
    (1, 37, 4, 8, 0, 8, "at"), (2, 29, 4, 8, 0, 8, "at"), (3, 61, 3, 11, 1, 10, "at"),
    (5, 130, 5, 7, 1, 6, "at"), (10, 211, 4, 9, 2, 7, "at"), (20, 97, 8, 6, 2, 4, "at"),
    (40, 257, 4, 8, 0, 8, "at"), (100, 333, 3, 11, 1, 10, "at"), (6, 37, 2, 16, 0, 16, "at"),
    (1, 64, 4, 8, 0, 8, "ace"), (3, 50, 4, 9, 2, 7, "ace"), (5, 77, 5, 7, 1, 6, "ace"),
    (10, 128, 4, 8, 0, 8, "ace"), (20, 101, 3, 11, 1, 10, "ace"), (40, 300, 4, 8, 0, 8, "ace"),
    (100, 250, 4, 8, 0, 8, "ace"), (10, 570, 4, 8, 0, 8, "ace"),
    # one ACT for the whole ATV: the refresh reaches every word every k slices
    (1, 37, 4, 8, 0, 8, "aligned"), (4, 130, 4, 9, 2, 7, "aligned"), (10, 512, 4, 8, 0, 8, "aligned"),
    (12, 1024, 4, 8, 0, 8, "aligned"),
    # timestamps with slice counts: the close counts from the counts kept by the ingest
    (1, 37, 4, 8, 0, 8, "hist"), (3, 61, 3, 11, 1, 10, "hist"), (5, 130, 5, 7, 1, 6, "hist"),
    (10, 211, 4, 9, 2, 7, "hist"), (40, 257, 4, 8, 0, 8, "hist"),
]

MODE = {"at": 0, "ace": 1, "aligned": 2, "hist": 0}

@pytest.mark.parametrize("k,g,r,c,u,s,counter", CASES)
def test_random_configs_every_slice(mods, k, g, r, c, u, s, counter):
    asse, oracle, torch = mods
    theta = max(4, g // 3)
    p = _params(k, g, r, c, u, s, theta, seed=k + g)
    mode = MODE[counter]
    # half of the cases with the ingest's key table (small pools have none by default)
    pool = asse.Pool(p, counter=counter, restore_cap=1 << 14, key_table="on" if (k + g) % 2 else "auto")
    orc = oracle.Oracle.from_params(p, mode=mode)
    heavy = [theta // 2, theta, 2 * theta, 3 * theta]
    n_slices = 2 * k + 3
    rng = np.random.default_rng(k * 31 + g)
    for t in range(n_slices):
        n = int(rng.integers(0, 3000)) | 1 if t % 5 else int(rng.integers(0, 3))
        pairs = mixed_pairs(k + g, t, n, heavy)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after ingest t={t}")
        kp = k if t % 3 else 1 + (t % k)
        check_close(pool, orc, kp)
        orc.advance()
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after refresh t={t}")
    pool.close()


# The long workload's counters at small E: k = 60 (timestamps of 7 bits held
# in byte-wide fields, four to a word, or 6-bit aging counters) with g = 1024
# (an ATV of 256 words, scanned by eight lanes), and k = 30 (6-bit / 5-bit).
EDGE_CASES = [(60, 1024, 4, 8, 1, 8, "at"), (60, 1024, 4, 8, 1, 8, "ace"), (60, 1024, 4, 8, 1, 8, "aligned"),
              (60, 1024, 4, 8, 1, 8, "hist"), (30, 512, 4, 9, 2, 7, "at"), (30, 512, 4, 9, 2, 7, "ace")]


@pytest.mark.parametrize("k,g,r,c,u,s,counter", EDGE_CASES)
def test_window_edges_full_cycle(mods, k, g, r, c, u, s, counter):
    """2k+3 slices (a full cycle of C0 and the wrap) of a stream whose heavy
    hosts enter and leave the window at random slices: they become super
    points, stay while the window holds enough of their bips, and vanish k
    slices after their last packet (Sec. 3, Algorithms 1-2).  State after
    every ingest and refresh, counts, loads, candidates and report against
    the oracle, for k' = k and for shorter windows."""
    asse, oracle, torch = mods
    theta = g // 3
    p = _params(k, g, r, c, u, s, theta, seed=k + 3 * g)
    mode = MODE[counter]
    pool = asse.Pool(p, counter=counter, restore_cap=1 << 12)
    orc = oracle.Oracle.from_params(p, mode=mode)
    rng = np.random.default_rng(k * 7 + g)
    n_heavy = 10
    sizes = (theta * rng.uniform(0.5, 4.0, n_heavy)).astype(np.int64)
    starts = rng.integers(0, k + 3, n_heavy)
    lens = rng.integers(k // 4, k + 1, n_heavy)
    reported, vanished = set(), set()
    for t in range(2 * k + 3):
        pairs = interval_pairs(k + g, t, k, sizes, starts, lens)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after ingest t={t}")
        kp = k if t % 4 else max(1, k // (1 + t % 3))
        res = check_close(pool, orc, kp)
        now = {a for a, _e, _n in res["report"]}
        if kp == k:
            vanished |= reported - now
        reported |= now
        orc.advance()
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after refresh t={t}")
    assert len(reported) >= 3 and len(vanished) >= 3, (reported, vanished)   # hosts entered and left
    pool.close()


def test_aligned_stepwise_and_staggered_equivalence(mods):
    """The aligned pool through the stepwise calls (scan, restore, the
    separate refresh kernel of asse_advance) equals the oracle's aligned mode,
    and its per-ATV counts equal the staggered pool's on the same input: both
    count exactly the ATs set in the latest k' slices."""
    asse, oracle, torch = mods
    p = _params(5, 200, 4, 9, 2, 7, 60, seed=8)
    al = asse.Pool(p, counter="aligned")
    st = asse.Pool(p)
    orc = oracle.Oracle.from_params(p, mode=2)
    assert al.info()["block"] == 200
    for t in range(24):
        pairs = mixed_pairs(8, t, 3001, [40, 90, 300])
        for pl in (al, st):
            pl.ingest(to_device(pairs))
        orc.ingest(pairs)
        kp = 1 + t % 5
        al.scan(kp)
        st.close_slice(kp)
        cnt = orc.counts(kp)
        np.testing.assert_array_equal(al.counts(), cnt)
        np.testing.assert_array_equal(st.counts(), cnt, err_msg=f"staggered t={t}")
        al.restore()
        compare_lists(al.candidates(), orc.close_report(kp)["candidates"], p["theta"], "csip")
        al.advance()
        orc.advance()
        np.testing.assert_array_equal(state(al), orc.at(), err_msg=f"after refresh t={t}")
    for pl in (al, st):
        pl.close()


def test_stepwise_equals_fused_and_estimate(mods):
    """scan -> restore -> estimate -> advance gives the fused close's results,
    and the estimate of any host equals the oracle's Algorithm 5 + Eq. 4."""
    asse, oracle, torch = mods
    p = _params(6, 150, 4, 9, 2, 7, 60, seed=5)
    fused = asse.Pool(p)
    step = asse.Pool(p)
    orc = oracle.Oracle.from_params(p)
    for t in range(16):
        pairs = mixed_pairs(5, t, 4001, [30, 60, 120, 400])
        for pl in (fused, step):
            pl.ingest(to_device(pairs))
        orc.ingest(pairs)
        kp = 1 + t % 6
        step.scan(kp)
        step.restore()
        cnt = orc.counts(kp)
        aat = orc.aat(cnt)
        hosts = np.unique(pairs[:, 0])[:50]
        est = step.estimate(hosts)
        for row in est:
            e2, n2 = orc.estimate(aat, int(row["aip"]), kp)
            assert row["nat"] == n2
            assert abs(row["est"] - e2) <= 1e-5 * abs(e2) + 1e-6 or (np.isinf(e2) and np.isinf(row["est"]))
        res = orc.close_report(kp)
        step.advance()
        fused.close_slice(kp)
        for pl in (fused, step):
            np.testing.assert_array_equal(pl.counts(), res["counts"])
            compare_lists(pl.candidates(), res["candidates"], p["theta"], "csip")
        orc.advance()
        np.testing.assert_array_equal(fused.read_pool(), step.read_pool())
        np.testing.assert_array_equal(state(fused), orc.at())


def test_host_ingest_chunks_and_snapshot(mods):
    """Host input staged by the copy engines (pageable memory in ten
    double-buffered chunks, and pinned memory) gives the oracle's state and
    report, as device input does; a snapshot restored into a fresh pool
    continues identically, also against the oracle."""
    asse, oracle, torch = mods
    p = _params(4, 128, 4, 10, 0, 8, 64, seed=3)
    a = asse.Pool(p, max_batch=1001)
    b = asse.Pool(p)
    c_pin = asse.Pool(p)
    orc = oracle.Oracle.from_params(p)
    for t in range(5):
        pairs = mixed_pairs(3, t, 9999, [100, 200])
        a.ingest(pairs)                  # numpy: pageable host memory, staged in 10 chunks
        b.ingest(to_device(pairs))
        c_pin.ingest(torch.from_numpy(pairs.view(np.int32)).pin_memory())   # pinned: staged in one chunk
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(a), orc.at(), err_msg=f"staged ingest t={t}")
        np.testing.assert_array_equal(state(c_pin), orc.at(), err_msg=f"pinned ingest t={t}")
        np.testing.assert_array_equal(b.read_pool(), a.read_pool())
        res = check_close(a, orc, 4)
        for pl in (b, c_pin):
            pl.close_slice()
            compare_lists(pl.report(), res["report"], orc.theta, "report t=%d" % t)
        orc.advance()
        np.testing.assert_array_equal(state(a), orc.at(), err_msg=f"after refresh t={t}")
    img = a.snapshot()
    c = asse.Pool(p)
    c.load(img)
    assert c.info()["slice"] == a.info()["slice"] == 5
    for t in range(5, 9):
        pairs = mixed_pairs(3, t, 5000, [100, 200])
        for pl in (a, c):
            pl.ingest(pairs)
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(c), orc.at(), err_msg=f"loaded pool t={t}")
        res = check_close(c, orc, 4)
        a.close_slice()
        compare_lists(a.report(), res["report"], orc.theta, "report t=%d" % t)
        orc.advance()
        np.testing.assert_array_equal(a.read_pool(), c.read_pool())
    bad = asse.Pool(_params(5, 128, 4, 10, 0, 8, 64, seed=3))
    with pytest.raises(asse.AsseError) as ei:
        bad.load(img)
    assert ei.value.status == asse.EINVAL


def test_slice_counts_stepwise_and_snapshot(mods):
    """A pool with slice counts: the stepwise calls (scan, restore, estimate,
    advance) give the oracle's counts, candidates and estimates, and a
    snapshot loaded into a fresh pool (whose counts are rebuilt from the
    words) continues with the same counts and reports as the original."""
    asse, oracle, torch = mods
    p = _params(6, 150, 4, 9, 2, 7, 60, seed=15)
    a = asse.Pool(p, counter="hist")
    orc = oracle.Oracle.from_params(p)
    for t in range(15):
        pairs = mixed_pairs(15, t, 4001, [30, 60, 120, 400])
        a.ingest(to_device(pairs))
        orc.ingest(pairs)
        kp = 1 + t % 6
        a.scan(kp)
        np.testing.assert_array_equal(a.counts(), orc.counts(kp), err_msg=f"t={t}")
        a.restore()
        res = orc.close_report(kp)
        compare_lists(a.candidates(), res["candidates"], p["theta"], "csip t=%d" % t)
        a.advance()
        orc.advance()
        np.testing.assert_array_equal(state(a), orc.at(), err_msg=f"after refresh t={t}")
    b = asse.Pool(p, counter="hist")
    b.load(a.snapshot())
    for t in range(15, 30):
        pairs = mixed_pairs(15, t, 4001, [30, 60, 120, 400])
        for pl in (a, b):
            pl.ingest(to_device(pairs))
        orc.ingest(pairs)
        res = check_close(b, orc, 6)
        a.close_slice(6)
        np.testing.assert_array_equal(a.counts(), b.counts())
        compare_lists(a.report(), res["report"], p["theta"], "report t=%d" % t)
        orc.advance()
    for pl in (a, b):
        pl.close()


def test_key_table_repeats_and_slice_wrap(mods):
    """The ingest skips a (aip, BH(bip)) key already set in the open slice,
    remembered in a key table shared by all blocks and tagged with the low 32
    bits of the slice.  Batches that repeat and overlap within a slice, with a
    stepwise scan in between, give the oracle's state; a pool loaded at slice
    2^32 - 1 (the same ACT phase, k = 4) passes the tag wrap, where the table
    is emptied, and stays equal to the pool it was copied from."""
    import ctypes
    asse, oracle, torch = mods
    p = _params(4, 128, 4, 10, 0, 8, 64, seed=5)
    a = asse.Pool(p, key_table="on")
    orc = oracle.Oracle.from_params(p)
    s0 = ((1 << 32) - 1) % 8          # slices 2^32 - 1 and s0 share C0 = t mod 2k
    for t in range(s0):
        x = mixed_pairs(5, t, 6001, [150, 300])
        y = np.concatenate([x[::3], mixed_pairs(5, 100 + t, 2001, [150])])
        for batch in (x, x, y):
            a.ingest(to_device(batch))
            orc.ingest(batch)
        np.testing.assert_array_equal(state(a), orc.at(), err_msg=f"after repeated batches t={t}")
        a.scan(4)
        a.ingest(to_device(x[::2]))
        np.testing.assert_array_equal(state(a), orc.at(), err_msg=f"after a batch past a scan t={t}")
        check_close(a, orc, 4)
        orc.advance()
        np.testing.assert_array_equal(state(a), orc.at(), err_msg=f"after refresh t={t}")
    img = bytearray(a.snapshot())
    off = 16 + ctypes.sizeof(asse.Config)
    assert int.from_bytes(img[off:off + 8], "little") == s0
    img[off:off + 8] = ((1 << 32) - 1).to_bytes(8, "little")
    b = asse.Pool(p, key_table="on")
    b.load(bytes(img))
    assert b.info()["slice"] == (1 << 32) - 1
    for t in range(s0, s0 + 4):
        x = mixed_pairs(5, t, 7001, [200, 300])
        for pl in (a, b):
            pl.ingest(to_device(x))
            pl.ingest(to_device(x[::2]))
        orc.ingest(x)
        np.testing.assert_array_equal(b.read_pool(), a.read_pool(), err_msg=f"slice {t}")
        np.testing.assert_array_equal(state(a), orc.at())
        check_close(a, orc, 4)
        b.close_slice(4)
        orc.advance()
        np.testing.assert_array_equal(b.read_pool(), a.read_pool(), err_msg=f"after close {t}")
        assert sorted(b.report()["aip"].tolist()) == sorted(a.report()["aip"].tolist())
    assert b.info()["slice"] == (1 << 32) + 3
    for pl in (a, b):
        pl.close()


@pytest.mark.parametrize("cluster", [2, 4, 8])
def test_cluster_shared_seen_table(mods, cluster):
    """The ingest whose table of seen keys is shared by the CTAs of a
    thread-block cluster (each CTA holds the keys that hash to it, the others
    reach it through distributed shared memory) gives the oracle's state,
    counts and reports: tiny_b for 8 slices, a pool with slice counts and the
    key table, and the link workload at full size for one slice."""
    asse, oracle, torch = mods
    w = synth.workload("tiny_b")
    pool = asse.Pool(w.params, cluster=cluster)
    orc = oracle.Oracle.from_params(w.params)
    for t in range(8):
        pairs = w.pairs(t)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"tiny_b t={t}")
        check_close(pool, orc, w.k)
        orc.advance()
    pool.close()
    p = _params(10, 211, 4, 9, 2, 7, 70, seed=cluster)
    pool = asse.Pool(p, counter="hist", key_table="on", cluster=cluster)
    orc = oracle.Oracle.from_params(p)
    for t in range(23):
        pairs = mixed_pairs(cluster, t, 20001, [35, 70, 140, 280])
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"hist t={t}")
        check_close(pool, orc, 10 if t % 3 else 4)
        orc.advance()
    pool.close()
    if cluster == 4:
        wl = synth.workload("link")
        pool = asse.Pool(wl.params, cluster=cluster)
        orc = oracle.Oracle.from_params(wl.params)
        pairs = wl.pairs(0)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg="link slice 0")
        check_close(pool, orc, wl.k)
        pool.close()


def test_random_read_probe_leaves_pool_unchanged(mods):
    """The random-read probe (the ingest's random-access roofline) issues at
    least the reads asked for, on the pool's stream, and changes nothing."""
    asse, oracle, torch = mods
    w = synth.workload("tiny_b")
    pool = asse.Pool(w.params)
    pool.ingest(to_device(w.pairs(0)))
    before = pool.read_pool()
    assert pool.probe_random_reads(0) == 0
    n = pool.probe_random_reads(1 << 20)
    assert n >= 1 << 20
    np.testing.assert_array_equal(pool.read_pool(), before)
    with pytest.raises(asse.AsseError) as ei:
        pool.probe_random_reads((1 << 34) + 1)
    assert ei.value.status == asse.EINVAL
    pool.close()


def test_edge_cases(mods):
    asse, oracle, torch = mods
    p = _params(3, 40, 4, 8, 0, 8, 10, seed=9)
    pool = asse.Pool(p, restore_cap=8)
    orc = oracle.Oracle.from_params(p)
    pool.close_slice()                          # empty slice
    assert pool.report().size == 0 and pool.candidates().size == 0
    orc.advance()
    one = mixed_pairs(9, 0, 1, [5])
    pool.ingest(to_device(one))                 # a single pair (tail path only)
    orc.ingest(one)
    np.testing.assert_array_equal(state(pool), orc.at())
    pool.ingest(one[:0])                        # empty batch
    with pytest.raises(asse.AsseError) as ei:
        pool.close_slice(4)                     # k' > k
    assert ei.value.status == asse.EINVAL
    with pytest.raises(asse.AsseError) as ei:
        pool.estimate(np.array([1], dtype=np.uint32))   # no scan of this slice
    assert ei.value.status == asse.ESTATE
    with pytest.raises(asse.AsseError):
        pool.ingest(to_device(mixed_pairs(9, 1, 9, [5]))[1:])  # misaligned device pointer
    # overflow of a tiny restore capacity is reported with the needed size
    heavy = mixed_pairs(9, 2, 20000, [60] * 40, n_background=0)
    pool.ingest(to_device(heavy))
    pool.close_slice()
    with pytest.raises(asse.AsseError) as ei:
        pool.report()
    assert ei.value.status == asse.ECAPACITY and ei.value.n_needed > 8


def test_link_full_size_three_slices(mods):
    """Link-scale workload at full size (k=10, 8 Mi pairs per slice, 4 x
    65,536 x 512 ATs): state after ingest and after refresh, counts, loads,
    candidates and report, for the first three slices."""
    asse, oracle, torch = mods
    w = synth.workload("link")
    pool = asse.Pool(w.params)
    orc = oracle.Oracle.from_params(w.params)
    for t in range(3):
        pairs = w.pairs(t)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after ingest t={t}")
        check_close(pool, orc, w.k)
        orc.advance()
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after refresh t={t}")


@pytest.mark.parametrize("k,g,r,c,u,s,counter,n_win", [
    (6, 150, 4, 9, 2, 7, "at", 3), (10, 211, 4, 9, 2, 7, "at", 4), (5, 77, 5, 7, 1, 6, "ace", 4),
    (1, 64, 4, 8, 0, 8, "ace", 2), (20, 97, 8, 6, 2, 4, "at", 2), (40, 257, 4, 8, 0, 8, "at", 4),
    (10, 570, 4, 8, 0, 8, "ace", 3), (60, 1024, 4, 8, 1, 8, "at", 3), (10, 211, 4, 9, 2, 7, "hist", 4)])
def test_multi_window_close(mods, k, g, r, c, u, s, counter, n_win):
    """One pass over the pool for several windows k' <= k: every window's
    counts, loads, candidates and report equal the oracle's close for that
    window on the same state, and the refreshed state equals the oracle's."""
    asse, oracle, torch = mods
    theta = max(4, g // 3)
    p = _params(k, g, r, c, u, s, theta, seed=3 * k + g)
    pool = asse.Pool(p, counter=counter, restore_cap=1 << 14)
    orc = oracle.Oracle.from_params(p, mode=MODE[counter])
    heavy = [theta // 2, theta, 2 * theta, 3 * theta]
    rng = np.random.default_rng(k + 7 * g)
    for t in range(2 * k + 3):
        n = int(rng.integers(1, 4000)) | 1
        pairs = mixed_pairs(k + g + 1, t, n, heavy)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        kps = [k, max(1, k - 2), 1, (k + 1) // 2][:n_win]
        if t % 4 == 3:
            kps = kps[::-1]
        pool.close_slice_multi(kps)
        for m, kp in enumerate(kps):
            pool.select_window(m)
            res = orc.close_report(kp, cap=pool.out_cap, limit_extra=0)
            np.testing.assert_array_equal(pool.counts(), res["counts"], err_msg=f"t={t} window {m} k'={kp}")
            np.testing.assert_array_equal(pool.loads(), res["aat"])
            assert res["n_candidates"] <= pool.cap
            compare_lists(pool.candidates(), res["candidates"], orc.theta, "csip")
            compare_lists(pool.report(), [row for row in res["candidates"] if row[1] >= orc.theta], orc.theta,
                          "report")
        with pytest.raises(asse.AsseError):
            pool.select_window(len(kps))
        orc.advance()
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after refresh t={t}")
    pool.close()


def test_long_report_beyond_the_early_copy(mods):
    """asse_close_slice copies the status and the first 4,096 report entries
    to pinned host memory so that a short report takes one wait; a report
    longer than that is read from device memory.  Both against the oracle."""
    asse, oracle, torch = mods
    p = _params(2, 64, 4, 10, 8, 5, 6, seed=17)
    pool = asse.Pool(p, restore_cap=1 << 12)
    orc = oracle.Oracle.from_params(p)
    sizes = [40] * 4500
    for t in range(2):
        pairs = mixed_pairs(23, t, 300_000, sizes, n_background=0)
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        res = check_close(pool, orc, 2)
        if t == 1:
            assert len(res["report"]) > 4096, len(res["report"])
        orc.advance()


@pytest.mark.parametrize("counter,key_table", [("at", "off"), ("at", "on"), ("hist", "on"), ("ace", "off")])
def test_replayed_permuted_and_truncated_batches(mods, counter, key_table):
    """SetAT is idempotent within a slice (Sec. 4.4): a batch cut short
    leaves the pool as the oracle fed the same prefix, and that prefix
    ingested again, then again in another order, changes nothing: the state,
    the counts (for slice-count pools, the counts the ingest keeps) and the
    report stay the oracle's, slice after slice over a full 2k cycle."""
    asse, oracle, torch = mods
    k, g, r, c, u, s, theta = 6, 150, 4, 9, 2, 7, 50
    p = _params(k, g, r, c, u, s, theta, seed=11)
    pool = asse.Pool(p, counter=counter, key_table=key_table)
    orc = oracle.Oracle.from_params(p, mode=1 if counter == "ace" else 0)
    rng = np.random.default_rng(4)
    for t in range(2 * k + 3):
        pairs = mixed_pairs(21, t, 20001, [theta // 2, theta, 3 * theta])
        cut = int(rng.integers(1, pairs.shape[0]))
        pool.ingest(to_device(pairs[:cut]))
        orc.ingest(pairs[:cut])
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"truncated batch, t={t}")
        pool.ingest(to_device(pairs[:cut]))
        pool.ingest(to_device(np.ascontiguousarray(pairs[:cut][rng.permutation(cut)])))
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"replayed batch, t={t}")
        check_close(pool, orc, k)
        orc.advance()
        np.testing.assert_array_equal(state(pool), orc.at(), err_msg=f"after refresh t={t}")
    pool.close()
