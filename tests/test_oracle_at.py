"""Pins of the oracle's counter arithmetic (Sec. 3 and the ACE counter of
Sec. 2.3) against facts the paper and plain mathematics fix:

* the k = 9 worked example of preserveAT (golden fixture);
* a naive absolute-timestamp model: an AT is active for the latest k' slices
  iff it was last set at most k'-1 slices ago (the meaning Sec. 3 gives to
  "active"), checked by brute force over random set patterns, every block
  offset, every k' <= k, for many k;
* the same model for the aging-counter variant;
* the refresh touches only ATs whose ACT is 0 or k, i.e. two of the 2k blocks
  per slice, once every k slices per block;
* k = 1 is the discrete window: the pool holds the current slice only;
* the aligned variant (one ACT for the whole ATV) meets the same naive model
  and checks every AT at once, every k slices.
"""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_preserve_k9_example(oracle_mod):
    ex = json.load(open(os.path.join(GOLDEN, "preserve_k9.json")))
    k, inactive = ex["k"], ex["inactive"]
    assert inactive == 2 * k
    for act in range(2 * k):
        cleared = set(ex["cleared_at_act"].get(str(act), []))
        for v in range(2 * k + 1):
            out = oracle_mod.preserve_at(v, act, k)
            if v in cleared:
                assert out == inactive, (act, v)
            else:
                assert out == v, (act, v)
    # only two of the 2k ACT values trigger a check
    touching = [a for a in range(2 * k) if any(oracle_mod.preserve_at(v, a, k) != v for v in range(2 * k))]
    assert len(touching) == ex["checks_per_2k_slices"]


def _naive_single_at(oracle_mod, k, offset, pattern):
    """Drive one AT whose block has ACT (t + offset) mod 2k through the set
    pattern; compare checkAT with t - last_set <= k'-1 at every slice."""
    value = 2 * k
    last = None
    for t, hit in enumerate(pattern):
        act = (t + offset) % (2 * k)
        value = oracle_mod.preserve_at(value, act, k)       # beginning of slice t
        if hit:
            value = act                                     # SetAT
            last = t
        for kp in range(1, k + 1):
            want = last is not None and t - last <= kp - 1
            got = oracle_mod.check_at(value, act, k, kp)
            assert got == want, (k, offset, t, kp, value, act, last)
        assert 0 <= value <= 2 * k


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 9, 10, 16, 30])
def test_check_and_preserve_match_naive_timestamps(oracle_mod, k):
    rng = np.random.default_rng(k)
    T = 6 * k + 7
    for offset in range(2 * k):
        for density in (0.05, 0.3, 0.9):
            _naive_single_at(oracle_mod, k, offset, rng.random(T) < density)
        # sets exactly k-1, k, k+1, 2k-1, 2k, 2k+1 slices apart (window edges, ACT wrap)
        for gap in (k - 1, k, k + 1, 2 * k - 1, 2 * k, 2 * k + 1):
            if gap < 1:
                continue
            pat = np.zeros(T, dtype=bool)
            pat[::gap] = True
            _naive_single_at(oracle_mod, k, offset, pat)


def test_check_and_preserve_k60_edges(oracle_mod):
    k = 60
    for offset in (0, 1, 59, 60, 61, 119):
        for gap in (59, 60, 61, 119, 120, 121):
            pat = np.zeros(4 * k + 3, dtype=bool)
            pat[3::gap] = True
            _naive_single_at(oracle_mod, k, offset, pat)


def _small_params(k, g, seed=3, u=0):
    c, s = (8, 8) if u == 0 else (7, 7)
    # r=4 windows of c bits cover LBS(f, 32-u): c + 3s >= 32 - u
    p = dict(k=k, theta=8, g=g, r=4, c=c, u=u, s=s, **synth.method_keys(seed))
    return p


@pytest.mark.parametrize("k,g,mode", [(3, 16, 0), (4, 24, 0), (5, 10, 0), (2, 9, 0), (4, 16, 1), (1, 8, 0),
                                      (3, 16, 2), (4, 24, 2), (1, 8, 2)])
def test_whole_pool_matches_naive_timestamps(oracle_mod, k, g, mode):
    """Every AT of a small pool, every slice, every k': the oracle's activity
    equals the naive 'last set at most k'-1 slices ago' model.  The naive
    model takes the AT positions from RRH/BH (pinned separately)."""
    p = _small_params(k, g)
    o = oracle_mod.Oracle.from_params(p, mode=mode)
    last = np.full((o.r, o.E, o.g), -(10 ** 9), dtype=np.int64)
    hosts = synth.random_pairs(5, 0, 40, n_hosts=40)[:, 0]
    for t in range(5 * k + 4):
        n = int(np.random.default_rng(t).integers(0, 120))
        pairs = synth.random_pairs(11, t, n, n_hosts=40, n_bips=64)
        pairs[:, 0] = hosts[pairs[:, 0] % 40]
        o.ingest(pairs)
        for aip, bip in pairs.tolist():
            x, z = o.rrh(aip)
            h = o.bh(bip)
            for i in range(o.r):
                last[i, (z << o.c) | x[i], h] = t
        for kp in range(1, k + 1):
            want = ((t - last) <= kp - 1).sum(axis=2)
            np.testing.assert_array_equal(o.counts(kp), want, err_msg=f"t={t} kp={kp}")
        o.advance()


def test_refresh_touches_two_blocks_per_slice(oracle_mod):
    """Sec. 3: with the 2k blocks' ACTs all different, only two blocks are
    checked per slice, and each block once every k slices."""
    k, g = 5, 23  # a = 2, last block holds 23 - 2*9 = 5 ATs
    p = _small_params(k, g)
    o = oracle_mod.Oracle.from_params(p)
    blocks = [o.block(h) for h in range(g)]
    a = g // (2 * k)
    assert blocks == [min(h // a, 2 * k - 1) for h in range(g)]
    assert blocks.count(2 * k - 1) == g - a * (2 * k - 1)
    seen = {b: [] for b in range(2 * k)}
    for t in range(4 * k):
        acts = {}
        for h in range(g):
            acts.setdefault(blocks[h], set()).add(o.act(h))
        assert all(len(v) == 1 for v in acts.values())            # one ACT per block
        act_of = {b: v.pop() for b, v in acts.items()}
        assert sorted(act_of.values()) == list(range(2 * k))        # all different
        refreshed = [b for b, a_ in act_of.items() if a_ % k == 0]
        assert len(refreshed) == 2
        for b in refreshed:
            seen[b].append(t)
        o.advance()
    for b, ts in seen.items():
        assert np.all(np.diff(ts) == k), (b, ts)


def test_aligned_refresh_checks_whole_pool_every_k_slices(oracle_mod):
    """Aligned variant: every AT shares the ACT C0 = t mod 2k, so preserveAT
    acts on the whole pool at the slices where C0 is 0 or k and on nothing in
    between; an AT set at slice t is cleared by the first such check at least
    k slices later, exactly when the naive model stops counting it."""
    k, g = 4, 24
    p = _small_params(k, g)
    o = oracle_mod.Oracle.from_params(p, mode=2)
    assert [o.block(h) for h in range(g)] == [0] * g
    pairs = synth.random_pairs(6, 0, 300, n_hosts=30, n_bips=200)
    changed_at = []
    for t in range(5 * k):
        assert all(o.act(h) == t % (2 * k) for h in range(g))
        if t % 3 == 0:
            o.ingest(pairs[(t // 3) * 40:(t // 3) * 40 + 40])
        before = o.at().copy()
        o.advance()
        after = o.at()
        if not np.array_equal(before, after):
            changed_at.append(t + 1)
        assert np.all((after == before) | (after == 2 * k))    # a check only clears
    assert changed_at and all(t1 % k == 0 for t1 in changed_at), changed_at


def test_k1_is_discrete_window(oracle_mod):
    """Sec. 2.3: k = 1 is the discrete window; the pool then acts as the
    one-bit linear estimator of the current slice."""
    p = _small_params(1, 8)
    o = oracle_mod.Oracle.from_params(p)
    for t in range(6):
        pairs = synth.random_pairs(2, t, 200, n_hosts=30, n_bips=50)
        o.ingest(pairs)
        touched = set()
        for aip, bip in pairs.tolist():
            x, z = o.rrh(aip)
            for i in range(o.r):
                touched.add((i, (z << o.c) | x[i], o.bh(bip)))
        cnt = o.counts(1)
        want = np.zeros_like(cnt)
        for i, e, _h in touched:
            want[i, e] += 1
        np.testing.assert_array_equal(cnt, want)
        o.advance()


def test_ingest_idempotent_and_order_free(oracle_mod):
    p = _small_params(4, 32)
    pairs = synth.random_pairs(9, 1, 500, n_hosts=50, n_bips=300)
    a = oracle_mod.Oracle.from_params(p)
    b = oracle_mod.Oracle.from_params(p)
    a.ingest(pairs)
    b.ingest(pairs[::-1])
    b.ingest(pairs[np.random.default_rng(1).permutation(len(pairs))])
    np.testing.assert_array_equal(a.at(), b.at())
