"""Pins of the feature definition of the learned estimators (oracle/features.py)
against an independent model: every AT's last set slice kept by hand.  An AT
set d slices ago, d < k', is active and falls in age bin d (Sec. 3's meaning
of "active in the latest k' slices"); bins add up to the active count; the
load features are the row-frame loads of Sec. 4.3 and their product and mean."""
import numpy as np
import pytest

import synth
from oracle import features as ofeat
from oracle import mlp as omlp


def _params(k, g, seed=3):
    # r=4 windows of c=7 bits over LBS(f, 31): c + 3s >= 31, two frames
    return dict(k=k, theta=8, g=g, r=4, c=7, u=1, s=8, **synth.method_keys(seed))


@pytest.mark.parametrize("k,g,mode", [(3, 16, 0), (5, 40, 0), (4, 24, 1), (6, 50, 2), (10, 64, 0)])
def test_age_bins_match_last_set_slice(oracle_mod, k, g, mode):
    o = oracle_mod.Oracle.from_params(_params(k, g), mode=mode)
    last = np.full((o.r, o.E, o.g), -(10 ** 9), dtype=np.int64)
    hosts = synth.random_pairs(5, 0, 30, n_hosts=30)[:, 0]
    for t in range(3 * k + 2):
        n = int(np.random.default_rng(t).integers(0, 150))
        pairs = synth.random_pairs(17, t, n, n_hosts=30, n_bips=90)
        pairs[:, 0] = hosts[pairs[:, 0] % 30]
        o.ingest(pairs)
        for aip, bip in pairs.tolist():
            x, z = o.rrh(aip)
            h = o.bh(bip)
            for i in range(o.r):
                last[i, (z << o.c) | x[i], h] = t
        for kp in sorted({1, max(1, k // 2), k}):
            rows = ofeat.pool_rows(o, kp).reshape(o.r, o.E, ofeat.FEAT)
            d = t - last
            want_cnt = ((d >= 0) & (d < kp)).sum(axis=2)
            np.testing.assert_array_equal(rows[:, :, 0], omlp.bf16(want_cnt / g))
            for a in range(kp):
                np.testing.assert_array_equal(rows[:, :, 1 + a], omlp.bf16((d == a).sum(axis=2) / g),
                                              err_msg="t=%d k'=%d age %d" % (t, kp, a))
            assert np.all(rows[:, :, 1 + kp:65] == 0)
            # the bins add up to the count (before rounding)
            bins = np.stack([(d == a).sum(axis=2) for a in range(kp)]).sum(axis=0)
            np.testing.assert_array_equal(bins, want_cnt)
            P = want_cnt.reshape(o.r, o.frames, -1).sum(axis=2) / (g * (1 << o.c))
            frame = np.arange(o.E) >> o.c
            np.testing.assert_array_equal(rows[:, :, 65], omlp.bf16(P[:, frame]))
            np.testing.assert_array_equal(rows[:, :, 66], omlp.bf16(np.broadcast_to(np.prod(P, axis=0)[frame],
                                                                                    (o.r, o.E))))
            np.testing.assert_array_equal(rows[:, :, 67], omlp.bf16(np.broadcast_to(P.mean(axis=0)[frame],
                                                                                    (o.r, o.E))))
            assert np.all(rows[:, :, 68:] == 0)
        o.advance()


@pytest.mark.parametrize("k,g,mode", [(4, 24, 0), (6, 50, 1), (10, 64, 0)])
def test_candidate_rows_match_last_set_slice(oracle_mod, k, g, mode):
    """Candidate features against the hand-kept last set slice of every AT:
    bin a counts the AT indices active in all r ATVs of the host whose
    oldest last-set slice is a slices ago; bin 0..k'-1 add up to NAT
    (Algorithm 5); the per-row counts and loads are the scan's."""
    o = oracle_mod.Oracle.from_params(_params(k, g), mode=mode)
    last = np.full((o.r, o.E, o.g), -(10 ** 9), dtype=np.int64)
    hosts = synth.random_pairs(5, 0, 12, n_hosts=12)[:, 0]
    for t in range(2 * k + 2):
        n = int(np.random.default_rng(t + 50).integers(0, 400))
        pairs = synth.random_pairs(19, t, n, n_hosts=12, n_bips=200)
        pairs[:, 0] = hosts[pairs[:, 0] % 12]
        o.ingest(pairs)
        for aip, bip in pairs.tolist():
            x, z = o.rrh(aip)
            h = o.bh(bip)
            for i in range(o.r):
                last[i, (z << o.c) | x[i], h] = t
        kp = k if t % 2 else max(1, k // 2)
        rows = ofeat.pool_candidate_rows(o, hosts, kp)
        cnt = o.counts(kp)
        P = o.aat(cnt).astype(np.float64) / (g * (1 << o.c))
        for hi, aip in enumerate(hosts.tolist()):
            x, z = o.rrh(aip)
            d = np.stack([t - last[i, (z << o.c) | x[i]] for i in range(o.r)])     # [r][g]
            act_all = ((d >= 0) & (d < kp)).all(axis=0)
            assert rows[hi, 0] == omlp.bf16(act_all.sum() / g)
            assert int(act_all.sum()) == o.nat(aip, kp)                           # NAT of Algorithm 5
            old = d.max(axis=0)
            for a in range(kp):
                assert rows[hi, 1 + a] == omlp.bf16((act_all & (old == a)).sum() / g), (t, aip, a)
            assert rows[hi, 65] == omlp.bf16(np.prod(P[:, z]))
            assert rows[hi, 66] == omlp.bf16(P[:, z].min()) and rows[hi, 67] == omlp.bf16(P[:, z].max())
            for i in range(o.r):
                assert rows[hi, 68 + i] == omlp.bf16(cnt[i, (z << o.c) | x[i]] / g)
        o.advance()
