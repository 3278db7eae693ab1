"""The learned estimate of candidate super points, in place of Eq. 4
(include/asse_learn.h): the candidate feature rows of a pool's hosts equal
their definition computed from the oracle's state (oracle/features.py); the
synthetic candidate states the model is trained on are exactly what an oracle
pool holds after ingesting the same host and background pairs; and a model
trained on the GPU beats Eq. 4's relative error on held-out states; and the
report decided by such a model on the device (asse_report_learned) is the
one the oracle's features and FP64 network give."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import mixed_pairs, to_device

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


@pytest.mark.parametrize("k,g,r,c,u,s,counter", [(6, 150, 4, 9, 2, 7, "at"), (10, 512, 4, 8, 0, 8, "at"),
                                                 (5, 77, 5, 7, 1, 6, "ace"), (60, 1024, 4, 8, 1, 8, "at"),
                                                 (12, 200, 8, 6, 2, 4, "at")])
def test_candidate_features_match_definition(mods, k, g, r, c, u, s, counter):
    asse, oracle, torch = mods
    from oracle import features as ofeat
    theta = max(4, g // 3)
    p = dict(k=k, theta=theta, g=g, r=r, c=c, u=u, s=s, **synth.method_keys(k + g))
    pool = asse.Pool(p, counter=counter, restore_cap=1 << 12)
    orc = oracle.Oracle.from_params(p, mode=1 if counter == "ace" else 0)
    for t in range(min(2 * k + 1, 16)):
        pairs = mixed_pairs(13, t, 4001, [theta // 2, theta, 2 * theta, 4 * theta])
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        kp = k if t % 2 else max(1, k - 2)
        if kp > 64:
            kp = 64
        pool.scan(kp)
        pool.restore()
        hosts = np.unique(np.concatenate([pool.candidates()["aip"], pairs[:300, 0]])).astype(np.uint32)
        x = pool.candidate_features(hosts).float().cpu().numpy()
        want = ofeat.pool_candidate_rows(orc, hosts, kp)
        np.testing.assert_allclose(x, want, rtol=0, atol=1e-7, err_msg="t=%d" % t)
        pool.advance()
        orc.advance()


def _twins(orc, aip0, n_rows):
    """For each row i an address whose ATV in row i (and frame) is aip0's and
    whose ATVs in the other rows are not: its bips reach row i only."""
    x0, z0 = orc.rrh(aip0)
    out = [None] * n_rows
    cand = synth.mix32(np.arange(1, 200000, dtype=np.uint32) + np.uint32(0x51ED))
    for a in cand.tolist():
        x, z = orc.rrh(a)
        if z != z0 or a == aip0:
            continue
        same = [x[i] == x0[i] for i in range(n_rows)]
        if sum(same) == 1:
            i = same.index(True)
            if out[i] is None:
                out[i] = a
        if all(o is not None for o in out):
            return out
    raise AssertionError("no twin address found")


@pytest.mark.parametrize("k,g,r,n_max_log2,bg_max", [(10, 512, 4, 16, 0.08), (10, 512, 4, 8, 0.02),
                                                     (30, 256, 3, 12, 0.04)])
def test_synth_candidates_match_oracle_pool(mods, k, g, r, n_max_log2, bg_max):
    """asse_synth_candidates packs each state's r ATVs as ingest would leave
    them: the host's bips go to all r ATVs of RRH(host), each row's
    background to that row alone (through an address that shares only that
    ATV with the host), slice by slice into an oracle pool; the oracle's
    feature row, NAT (Algorithm 5) and Eq. 4 equal the generator's."""
    asse, oracle, torch = mods
    from oracle import features as ofeat
    keys = synth.method_keys(2)
    seed, first, n = 21, 500, 16
    cfg = dict(k=k, g=g, r=r, n_max_log2=n_max_log2, bg_max=bg_max, seed=seed, bh_a=keys["bh_a"],
               bh_b=keys["bh_b"])
    x, ln, e4 = asse.synth_candidates(cfg, first, n)
    x = x.float().cpu().numpy().astype(np.float64)
    ln, e4 = ln.cpu().numpy(), e4.cpu().numpy()
    # an oracle pool of 8 columns per row: twins are easy to find
    p = dict(k=k, theta=g, g=g, r=r, c=3, u=0, s=3, A=keys["A"], bh_a=keys["bh_a"], bh_b=keys["bh_b"])
    probe = oracle.Oracle.from_params(p)
    bip_of_h, b = {}, 0
    while len(bip_of_h) < g:
        bip_of_h.setdefault(probe.bh(b), b)
        b += 1
    aip0 = 0x0A0B0C0D
    twins = _twins(probe, aip0, r)
    act_cache = None
    for si in range(n):
        d = synth.candidate_state_draws(seed, first + si, k, g, r, n_max_log2, bg_max)
        orc = oracle.Oracle.from_params(p)
        for s_ in range(k):
            parts = [np.stack([np.full(d["bips"][s_].size, aip0, dtype=np.uint32), d["bips"][s_]], axis=1)]
            for i in range(r):
                hs = np.nonzero(d["bg"][i][s_])[0]
                bips = np.array([bip_of_h[h] for h in hs], dtype=np.uint32)
                parts.append(np.stack([np.full(bips.size, twins[i], dtype=np.uint32), bips], axis=1))
            orc.ingest(np.concatenate(parts))
            if s_ + 1 < k:
                orc.advance()
        assert ln[si] == np.float32(np.log(d["card"]))
        xs, z = orc.rrh(aip0)
        at = orc.at()
        rows = np.stack([at[i, (z << p["c"]) | xs[i]] for i in range(r)])[None]
        if act_cache is None:
            act_cache = np.array([orc.act(h) for h in range(g)])
        cnt = orc.counts(k)
        cnts = np.array([[cnt[i, (z << p["c"]) | xs[i]] for i in range(r)]])
        pw = np.array([np.float32(1.0) - np.float32(1.0 - pi) ** np.float32(k) for pi in d["p"]], dtype=np.float64)
        want = ofeat.candidate_rows(rows, act_cache, k, k, 0, pw[None], cnts)[0]
        np.testing.assert_array_equal(x[si, :65], want[:65], err_msg="state %d" % si)
        np.testing.assert_array_equal(x[si, 68:], want[68:], err_msg="state %d" % si)
        np.testing.assert_allclose(x[si, 65:68], want[65:68], rtol=2 ** -7, atol=1e-30)
        nat = orc.nat(aip0, k)
        assert round(x[si, 0] * g) == nat or abs(x[si, 0] - nat / g) <= 2 ** -8 * nat / g
        want_e4 = oracle.eq4(g, nat, float(np.prod(pw)))
        if np.isinf(want_e4):
            assert np.isinf(e4[si])
        else:
            assert abs(e4[si] - want_e4) <= 1e-4 * want_e4 + 1e-4, (si, e4[si], want_e4)


def test_candidate_model_beats_eq4(mods):
    """Trained on synthetic candidate states (k = 10, g = 512, r = 4,
    cardinalities up to 2^16, per-row background up to 8 % of the ATs per
    slice) with the relative loss, the model's mean relative error on
    held-out states is below Eq. 4's, overall and around the threshold
    range (2^9 .. 2^12)."""
    asse, oracle, torch = mods
    keys = synth.method_keys(1)
    cfg = dict(k=10, g=512, r=4, n_max_log2=16, bg_max=0.08, seed=31, bh_a=keys["bh_a"], bh_b=keys["bh_b"])
    x, ln, _e4 = asse.synth_candidates(cfg, 0, 400_000)
    xt, lnt, e4t = asse.synth_candidates(cfg, 1 << 40, 40_000)
    m = asse.MLP(seed=4)
    m.set_loss("rel_mse")
    bs = 4096
    perm = torch.randperm(x.shape[0], device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    for step in range(400):
        o = (step * bs) % (x.shape[0] - x.shape[0] % bs)
        i = perm[o:o + bs]
        m.train_step(x[i].contiguous(), ln[i].contiguous(), 2e-3 if step < 300 else 5e-4)
    y = m.forward(xt)
    m.check()
    n_true = torch.exp(lnt.double())
    e4 = torch.where(torch.isinf(e4t), torch.full_like(e4t, 1e12), e4t).double()
    rel_m = torch.abs(torch.exp(y.double()) - n_true) / n_true
    rel_e = torch.abs(e4 - n_true) / n_true
    assert rel_m.mean().item() < rel_e.mean().item(), (rel_m.mean().item(), rel_e.mean().item())
    mid = (lnt >= 9 * np.log(2)) & (lnt < 12 * np.log(2))
    assert rel_m[mid].mean().item() < rel_e[mid].mean().item(), (rel_m[mid].mean().item(), rel_e[mid].mean().item())


@pytest.mark.parametrize("k,g,r,c,u,s,counter", [(10, 512, 4, 8, 0, 8, "at"), (6, 150, 4, 9, 2, 7, "hist")])
def test_learned_report_matches_oracle(mods, k, g, r, c, u, s, counter):
    """asse_report_learned against the oracle, slice by slice over a full 2k
    cycle: the candidates are the oracle's restore (Algorithm 4), their
    feature rows its state's (oracle/features.py), the model the FP64 network
    with the GPU's parameters (oracle/mlp.py).  A candidate whose model output
    lies clearly inside the training range (by more than its error scale) is
    decided by exp(y) >= theta, one clearly outside keeps Eq. 4's decision;
    only outputs within the error scale of ln(theta) or of the range's end
    may go either way.  Estimates: exp(y) within the same scale for model
    decisions, the restore's own record for Eq. 4 ones."""
    asse, oracle, torch = mods
    from oracle import features as ofeat
    from oracle import mlp as omlp
    theta = max(4, g // 3)
    p = dict(k=k, theta=theta, g=g, r=r, c=c, u=u, s=s, **synth.method_keys(3 * k + g))
    pool = asse.Pool(p, counter=counter, restore_cap=1 << 12)
    orc = oracle.Oracle.from_params(p)
    m = asse.MLP(seed=5)
    base = m.params().astype(np.float64)
    seen = {"learned_rep": 0, "learned_not": 0, "eq4": 0}
    for t in range(2 * k + 2):
        pairs = mixed_pairs(17, t, 4001, [theta // 2, theta, 2 * theta, 4 * theta])
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        pool.scan(k)
        pool.restore()
        res = orc.close_report(k, cap=pool.out_cap, limit_extra=0)
        cand = pool.candidates()
        assert sorted(int(a) for a in cand["aip"]) == [a for a, _e, _n in res["candidates"]]
        if cand.size:
            aips = np.sort(cand["aip"]).astype(np.uint32)
            X = ofeat.pool_candidate_rows(orc, aips, k)
            # outputs around ln(theta): a last layer of non-negative weights and
            # no bias (no cancellation, so the error scale is about y itself),
            # scaled so that the median output is ln(theta)
            q = omlp.unpack(base)
            q["w3"] = np.abs(q["w3"])
            q["b3"] = np.zeros(1)
            S = omlp.forward(omlp.pack(q), X)[0]
            q["w3"] = q["w3"] * (np.log(theta) / max(float(np.median(S)), 1e-6))
            m.set_params(omlp.pack(q).astype(np.float32))
            params = m.params().astype(np.float64)
            y = omlp.forward(params, X)[0]
            tol = 2.0 ** -6 * omlp.error_scales(params, X, np.zeros(aips.size))[0]
            max_log_n = float(np.quantile(y, 0.75)) if t % 2 else 40.0
            got = pool.report_learned(m, max_log_n)
            rec = {int(a): (float(e), int(f)) for a, e, f in zip(cand["aip"], cand["est"], cand["flags"])}
            got_by = {int(a): (float(e), int(f)) for a, e, f in zip(got["aip"], got["est"], got["flags"])}
            assert len(got_by) == got.size and set(got_by) <= set(rec)
            for a, yi, ti in zip(aips.tolist(), y, tol):
                if yi + ti <= max_log_n:                       # the model decides
                    if abs(yi - np.log(theta)) <= ti:
                        continue
                    want = yi > np.log(theta)
                    assert (a in got_by) == want, (t, a, yi, ti)
                    seen["learned_rep" if want else "learned_not"] += 1
                    if want:
                        est, fl = got_by[a]
                        assert fl & asse.SP_LEARNED and fl & asse.SP_REPORTED
                        assert abs(np.log(est) - yi) <= ti + 1e-6, (a, est, yi, ti)
                elif yi - ti > max_log_n:                      # Eq. 4 decides, as restored
                    want = bool(rec[a][1] & asse.SP_REPORTED)
                    assert (a in got_by) == want, (t, a)
                    seen["eq4"] += 1
                    if want:
                        assert got_by[a] == rec[a]
            if t == 2 * k + 1:                                 # an output too small for the report
                n = ctypes.c_uint64(0)
                rc = asse.lib().asse_report_learned(pool._h, m._h, ctypes.c_float(max_log_n), None, 0,
                                                    ctypes.byref(n), asse.HOST)
                assert n.value == got.size and rc == (asse.ECAPACITY if got.size else asse.OK)
        pool.advance()
        orc.advance()
    with pytest.raises(asse.AsseError) as ei:          # refreshed since the scan
        pool.report_learned(m, 40.0)
    assert ei.value.status == asse.ESTATE
    assert min(seen.values()) > 0, seen
    m.close()
    pool.close()
