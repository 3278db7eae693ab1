"""Pins of the oracle's estimators (Sec. 3, Sec. 4.2, Sec. 4.3):

* the linear-counting closed form: one ATV fed n distinct bips holds on
  average g(1-(1-1/g)^n) active ATs (occupancy of g bins), with the exact
  occupancy variance bounding the sample mean;
* Eq. 2 inverts that expectation (its mean over trials is close to n);
* the super-ATV threshold is exactly "the Eq. 2 estimate of the ATV reaches
  theta";
* Eq. 4 reduces to Eq. 2 when UP = 0, and undoes the Eq. 3 bias of NAT on
  rows with independent background load (Monte Carlo);
* NAT (Algorithm 5) of a lone host is the number of distinct BH values of
  its bips (|BIdx|), and the row-frame loads and UP follow from it;
* end to end on the tiny workload with per-host bip sets: the true super
  points (exact distinct counts over the window) are all reported.
"""
import math

import numpy as np
import pytest

import synth


def _params(g=128, theta=64, k=4, seed=1, **kw):
    p = dict(k=k, theta=theta, g=g, r=4, c=8, u=0, s=8, **synth.method_keys(seed))
    p.update(kw)
    return p


def _occupancy_moments(g, n):
    q1 = (1 - 1 / g) ** n
    q2 = (1 - 2 / g) ** n
    mean = g * (1 - q1)
    # variance of the number of empty bins: g q1 + g(g-1) q2 - g^2 q1^2
    var = g * q1 + g * (g - 1) * q2 - (g * q1) ** 2
    return mean, var


@pytest.mark.parametrize("g,n", [(128, 40), (128, 200), (512, 300), (512, 1500)])
def test_linear_counting_closed_form(oracle_mod, g, n):
    trials = 300
    cnts, ests = [], []
    for t in range(trials):
        o = oracle_mod.Oracle.from_params(_params(g=g, seed=1000 + t))
        aip = 12345 + t
        bips = synth.mix32(np.arange(n, dtype=np.uint32) + np.uint32(7 * t))
        o.ingest(np.stack([np.full(n, aip, dtype=np.uint32), bips], axis=1))
        cnt = o.counts(o.k)
        x, z = o.rrh(aip)
        c0 = int(cnt[0, (z << o.c) | x[0]])
        # every row's ATV of this host holds the same ATs (same BH index in all rows)
        assert all(int(cnt[i, (z << o.c) | x[i]]) == c0 for i in range(o.r))
        assert int(cnt.sum()) == o.r * c0
        cnts.append(c0)
        ests.append(oracle_mod.eq2(g, c0))
        o.close()
    mean, var = _occupancy_moments(g, n)
    assert abs(np.mean(cnts) - mean) < 4.5 * math.sqrt(var / trials), (np.mean(cnts), mean)
    # Eq. 2 is the inverse of the expectation; its mean is within noise of n
    sd_est = math.sqrt(var) * g / (g - mean)
    assert abs(np.mean(ests) - n) < 4.5 * sd_est / math.sqrt(trials) + 0.02 * n


@pytest.mark.parametrize("g,theta", [(128, 64), (512, 1024), (1024, 4096), (4096, 1024), (300, 77)])
def test_threshold_is_eq2_reaching_theta(oracle_mod, g, theta):
    o = oracle_mod.Oracle.from_params(_params(g=g, theta=theta, k=4))
    T = o.threshold()
    assert oracle_mod.eq2(g, T) >= theta > oracle_mod.eq2(g, T - 1)


def test_eq2_and_eq4_special_values(oracle_mod):
    g = 512
    assert oracle_mod.eq2(g, 0) == 0.0
    assert oracle_mod.eq2(g, g) == math.inf
    vals = [oracle_mod.eq2(g, c) for c in range(g)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    for nat in range(0, g, 37):
        assert oracle_mod.eq4(g, nat, 0.0) == oracle_mod.eq2(g, nat)
    assert oracle_mod.eq4(g, g, 0.3) == math.inf
    assert oracle_mod.eq4(g, 10, 1.0) == math.inf
    assert oracle_mod.eq4(g, 51, 0.1) == 0.0            # NAT <= g*UP: ratio >= 1
    assert oracle_mod.eq4(g, 100, 0.1) > 0.0
    # more background load lowers the estimate of the same NAT
    assert oracle_mod.eq4(g, 300, 0.2) < oracle_mod.eq4(g, 300, 0.05) < oracle_mod.eq4(g, 300, 0.0)


@pytest.mark.parametrize("g,n,loads", [(512, 400, (0.2, 0.3, 0.25, 0.35)), (1024, 2000, (0.4, 0.5, 0.45, 0.5)),
                                       (512, 100, (0.6, 0.6, 0.6, 0.6))])
def test_eq4_removes_background_bias(oracle_mod, g, n, loads):
    """Eq. 3: NAT = |BIdx| + UP (g - |BIdx|) on average when each row's other
    ATs are active independently with probability P_i; Eq. 4 then estimates n
    without the upward bias that Eq. 2 on NAT has."""
    rng = np.random.default_rng(g + n)
    trials = 400
    nats, ests, raw, bidx = [], [], [], []
    up = float(np.prod(loads))
    for _ in range(trials):
        hit = np.zeros(g, dtype=bool)
        hit[rng.integers(0, g, n)] = True                # the host's own bips (|BIdx| distinct)
        rows = [hit | (rng.random(g) < p) for p in loads]
        nat = int(np.logical_and.reduce(rows).sum())
        nats.append(nat)
        bidx.append(int(hit.sum()))
        ests.append(oracle_mod.eq4(g, nat, up))
        raw.append(oracle_mod.eq2(g, nat))
    b = np.mean(bidx)
    want_nat = b + up * (g - b)
    assert abs(np.mean(nats) - want_nat) < 0.01 * g
    assert abs(np.mean(ests) - n) < 0.05 * n + 5
    assert np.mean(raw) > np.mean(ests)                  # the bias Eq. 4 removes
    if up * (g - b) > 5:                                 # bias of several ATs: Eq. 4 is much closer
        assert np.mean(raw) - n > 2 * abs(np.mean(ests) - n)


def test_nat_of_lone_host_and_loads(oracle_mod):
    p = _params(g=512, theta=100, k=10, c=12, u=4, s=6)
    o = oracle_mod.Oracle.from_params(p)
    aip = 0xDEADBEEF
    bips = synth.mix32(np.arange(700, dtype=np.uint32))
    o.ingest(np.stack([np.full(700, aip, dtype=np.uint32), bips], axis=1))
    bidx = len({o.bh(b) for b in bips.tolist()})
    assert o.nat(aip, 10) == bidx
    cnt = o.counts(10)
    aat = o.aat(cnt)
    x, z = o.rrh(aip)
    want = np.zeros_like(aat)
    want[:, z] = bidx
    np.testing.assert_array_equal(aat, want)
    assert o.up(aat, z) == pytest.approx((bidx / (512 * 4096)) ** 4, rel=1e-12)
    est, nat = o.estimate(aat, aip, 10)
    assert nat == bidx
    assert est == pytest.approx(oracle_mod.eq2(512, bidx), rel=1e-9)
    # another host shares nothing with it
    assert o.nat(aip ^ 0x1234567, 10) == 0


def _window_truth(w, t, k):
    """Exact |OP(aip)| over slices t-k+1..t: distinct bips per aip (Sec. 2.2)."""
    keys = []
    for s in range(max(0, t - k + 1), t + 1):
        p = w.pairs(s)
        keys.append((p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64))
    keys = np.unique(np.concatenate(keys))
    aip = (keys >> np.uint64(32)).astype(np.uint32)
    u, c = np.unique(aip, return_counts=True)
    return dict(zip(u.tolist(), c.tolist()))


def test_tiny_b_end_to_end_reports_true_super_points(oracle_mod):
    w = synth.workload("tiny_b")
    o = oracle_mod.Oracle.from_params(w.params)
    for t in range(8):
        o.ingest(w.pairs(t))
        res = o.close_report(w.k)
        truth = _window_truth(w, t, w.k)
        true_sp = {a for a, n in truth.items() if n >= w.theta}
        reported = {a for a, _e, _n in res["report"]}
        assert true_sp == set(w.planted_aip.tolist())
        assert true_sp <= reported                     # no false negative
        assert len(reported - true_sp) <= 3
        for a, e, _n in res["report"]:
            if a in true_sp:
                assert 0.6 * truth[a] < e < 1.4 * truth[a]
        o.advance()
