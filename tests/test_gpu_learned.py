"""The learned per-ATV estimator on the GPU (include/asse_learn.h):

* the feature rows of a pool equal the definition computed from the oracle's
  AT values, ACTs and loads;
* forward values and the gradients of every parameter of the GPU kernels
  equal the FP64 CPU reference (oracle/mlp.py, BF16 rounding at the same
  storage points) on the same inputs;
* trained on the GPU on synthetic link-scale states, the model's mean
  relative error on held-out states is below plain linear counting's (Eq. 2)
  at the same pool size.
"""
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
    from oracle import mlp as omlp
    from paper_1807_01527_gb300 import asse, build
    build.build()
    oracle.build()
    return asse, oracle, omlp, torch


def _bf16(x):
    from oracle import mlp as omlp
    return omlp.bf16(x)


@pytest.mark.parametrize("k,g,counter", [(6, 150, "at"), (10, 512, "at"), (5, 77, "ace"), (6, 150, "hist"),
                                         (20, 256, "hist")])
def test_features_match_definition(mods, k, g, counter):
    """Feature rows of a pool against oracle/features.py on the oracle's state
    (slice-count pools build them from their counts, the others from their
    words), every slice of two windows' worth, full and shorter windows."""
    asse, oracle, omlp, torch = mods
    from oracle import features as ofeat
    p = dict(k=k, theta=max(4, g // 3), g=g, r=4, c=9, u=2, s=7, **synth.method_keys(3))
    pool = asse.Pool(p, counter=counter)
    orc = oracle.Oracle.from_params(p, mode=1 if counter == "ace" else 0)
    for t in range(2 * k + 1):
        pairs = mixed_pairs(7, t, 3001, [g // 2, g, 2 * g])
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        kp = k if t % 2 else max(1, k - 2)
        pool.scan(kp)
        x = pool.features().float().cpu().numpy()
        want = ofeat.pool_rows(orc, kp)
        np.testing.assert_allclose(x, want, rtol=0, atol=1e-7, err_msg=f"t={t}")
        pool.advance()
        orc.advance()


@pytest.mark.parametrize("loss_kind", ["log_mse", "rel_mse"])
def test_forward_and_gradients_match_fp64_reference(mods, loss_kind):
    asse, oracle, omlp, torch = mods
    m = asse.MLP(seed=5)
    m.set_loss(loss_kind)
    p = m.params().astype(np.float64)
    rng = np.random.default_rng(0)
    n = 3000                                              # not a multiple of the 64-row tiles
    X = _bf16(np.abs(rng.normal(size=(n, 80))) * 0.3)
    X[:, 68:] = 0.0
    t = rng.normal(loc=5.0, scale=2.0, size=n)
    xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    y = m.forward(xd).cpu().numpy().astype(np.float64)
    m.check()
    y_ref, _h1, _h2 = omlp.forward(p, X)
    ys, gs = omlp.error_scales(p, X, t, loss=loss_kind)
    # entry by entry: within 2^-6 of the sum of the absolute terms (a few
    # BF16 steps where the two sides' FP32 sums round a stored value apart)
    worst = np.max(np.abs(y - y_ref) / ys)
    assert worst <= 2 ** -6, ("forward", worst)
    loss = float(m.backward(xd, td).cpu()[0])
    g = m.grads().astype(np.float64)
    loss_ref, g_ref, _ = omlp.loss_and_grads(p, X, t, loss=loss_kind)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    o = 0
    for name, shape in omlp.SIZES:
        k = int(np.prod(shape))
        a, b, sc = g[o:o + k], g_ref[o:o + k], gs[o:o + k]
        ratio = np.abs(a - b) / (sc + 1e-30)
        i = int(np.argmax(ratio))
        assert ratio[i] <= 2 ** -6, (name, "worst entry", i, a[i], b[i], sc[i], ratio[i])
        o += k


@pytest.mark.parametrize("n", [1, 127, 128, 129, 19456 + 77, 262144 + 77])
def test_tensor_core_inference_matches_fp64_reference(mods, n):
    """The tcgen05 inference kernel on row counts around one 128-row tile,
    one tile per SM plus a ragged tail, and many tiles per SM: every row (or
    a sample of 4096 rows, including the last, for the largest case) against
    the FP64 reference with BF16 rounding at the same points."""
    asse, oracle, omlp, torch = mods
    m = asse.MLP(seed=7)
    rng = np.random.default_rng(n)
    p = m.params().astype(np.float64)
    # non-zero biases so that the bias paths are exercised
    bias = rng.normal(scale=0.1, size=omlp.NPARAMS)
    q = omlp.unpack(p)
    q["b1"] += bias[:256]
    q["b2"] += bias[256:512]
    q["b3"] += 0.3
    p = omlp.pack(q)
    m.set_params(p.astype(np.float32))
    p = m.params().astype(np.float64)
    X = _bf16(np.abs(rng.normal(size=(n, 80))) * 0.3)
    X[:, 68:] = 0.0
    xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    y = m.forward(xd)
    m.check()
    y = y.cpu().numpy().astype(np.float64)
    rows = np.arange(n) if n <= 20000 else np.unique(np.concatenate([rng.integers(0, n, 4095), [n - 1]]))
    y_ref, _h1, _h2 = omlp.forward(p, X[rows])
    ys, _gs = omlp.error_scales(p, X[rows], np.zeros(rows.size))
    worst = np.max(np.abs(y[rows] - y_ref) / ys)
    assert worst <= 2 ** -6, (n, worst)      # row by row, as in the gradient check


@pytest.mark.parametrize("k,g,n_max_log2,bg_max", [(10, 512, 20, 0.08), (10, 512, 12, 0.01), (60, 1024, 16, 0.02)])
def test_synth_states_match_oracle_pool(mods, k, g, n_max_log2, bg_max):
    """asse_synth_states packs each training state as ingest would leave it:
    the same host bips and background ATs, ingested slice by slice into an
    oracle pool (Algorithm 3, with Algorithm 2 between slices), give the same
    feature row (oracle/features.py on the oracle's state), and the labels are
    the exact distinct count of the host's bips (ln n) and Eq. 2 of the
    oracle's active count."""
    asse, oracle, omlp, torch = mods
    from oracle import features as ofeat
    keys = synth.method_keys(1)
    r, seed, first, n = 4, 11, 1000, 24
    cfg = dict(k=k, g=g, r=r, n_max_log2=n_max_log2, bg_max=bg_max, seed=seed, bh_a=keys["bh_a"],
               bh_b=keys["bh_b"])
    x, ln, lc = asse.synth_states(cfg, first, n)
    x = x.float().cpu().numpy().astype(np.float64)
    ln = ln.cpu().numpy()
    lc = lc.cpu().numpy()
    # a one-row oracle pool with the same BH keys; one host address
    p = dict(k=k, theta=g, g=g, r=1, c=1, u=0, s=1, A=keys["A"], bh_a=keys["bh_a"], bh_b=keys["bh_b"])
    probe = oracle.Oracle.from_params(p)
    bip_of_h = {}
    b = 0
    while len(bip_of_h) < g:                       # a bip that lands on each AT index
        bip_of_h.setdefault(probe.bh(b), b)
        b += 1
    aip0 = 0x0A000001
    for si in range(n):
        d = synth.training_state_draws(seed, first + si, k, g, n_max_log2, bg_max)
        orc = oracle.Oracle.from_params(p)
        xs, z = orc.rrh(aip0)
        est = (z << p["c"]) | xs[0]
        distinct = set()
        for s in range(k):
            bg = np.array([bip_of_h[h] for h in np.nonzero(d["bg"][s])[0]], dtype=np.uint32)
            bips = np.concatenate([d["bips"][s], bg])
            pairs = np.stack([np.full(bips.size, aip0, dtype=np.uint32), bips], axis=1)
            orc.ingest(pairs)
            distinct |= set(d["bips"][s].tolist())
            if s + 1 < k:
                orc.advance()
        assert len(distinct) == d["card"]              # the label is an exact distinct count
        assert ln[si] == np.float32(np.log(d["card"])), (si, ln[si], d["card"])
        at = orc.at()[0, est][None, :]
        act = np.array([orc.act(h) for h in range(g)])
        pw = np.float32(1.0) - np.float32(1.0 - d["pbg"]) ** np.float32(k)
        want = ofeat.atv_rows(at, act, k, k, 0, np.array([pw]), np.array([pw ** np.float32(r)]), np.array([pw]))[0]
        np.testing.assert_array_equal(x[si, :65], want[:65], err_msg="state %d" % si)
        # load features: FP32 powf on the device, numpy's here; one BF16 step at most
        np.testing.assert_allclose(x[si, 65:68], want[65:68], rtol=2 ** -7, atol=1e-30)
        assert np.all(x[si, 68:] == 0)
        cnt = int(orc.counts(k)[0, est])
        want_lc = oracle.eq2(g, cnt) if cnt < g else -g * np.log(0.5 / g)
        assert abs(lc[si] - want_lc) <= 1e-6 * want_lc + 1e-6, (si, lc[si], want_lc)


def test_training_beats_linear_counting(mods):
    """Trained on the GPU by the library's kernels on link-shaped states
    (k = 10, g = 512) with cardinalities log-uniform up to 2^20 and
    background at up to 8 % of the ATs per slice, with the relative loss, the
    model's mean relative error on held-out states is below linear
    counting's (Eq. 2) at the same pool size, over the whole range and in
    the range where Eq. 2 is at its best (2^8 to 2^12)."""
    asse, oracle, omlp, torch = mods
    keys = synth.method_keys(1)
    cfg = dict(k=10, g=512, r=4, n_max_log2=20, bg_max=0.08, seed=11, bh_a=keys["bh_a"], bh_b=keys["bh_b"])
    x, ln, lc = asse.synth_states(cfg, 0, 400_000)
    xt, lnt, lct = asse.synth_states(cfg, 1 << 40, 40_000)
    assert torch.all(ln >= 0) and torch.all(ln <= 20 * np.log(2) + 1e-5)
    m = asse.MLP(seed=2)
    m.set_loss("rel_mse")
    bs = 4096
    perm = torch.randperm(x.shape[0], device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    for step in range(400):
        o = (step * bs) % (x.shape[0] - x.shape[0] % bs)
        i = perm[o:o + bs]
        lr = 2e-3 if step < 300 else 5e-4
        m.train_step(x[i].contiguous(), ln[i].contiguous(), lr)
    y = m.forward(xt)
    m.check()
    n_true = torch.exp(lnt.double())
    rel_mlp = torch.abs(torch.exp(y.double()) - n_true) / n_true
    rel_lc = torch.abs(lct.double() - n_true) / n_true
    assert rel_mlp.mean().item() < rel_lc.mean().item(), (rel_mlp.mean().item(), rel_lc.mean().item())
    mid = (lnt >= 8 * np.log(2)) & (lnt < 12 * np.log(2))
    assert rel_mlp[mid].mean().item() < rel_lc[mid].mean().item()


def test_learned_estimate_with_fallback(mods):
    """asse_estimate_learned: exp(max(model, 0)) where the ATV holds an
    active AT and the model is inside its training range, Eq. 2 from the
    ATV's count elsewhere (empty ATVs and outputs above max_log_n), on a pool
    with saturated, light and empty ATVs."""
    asse, oracle, omlp, torch = mods
    g = 128
    p = dict(k=4, theta=40, g=g, r=4, c=8, u=0, s=8, **synth.method_keys(4))
    stream = torch.cuda.current_stream().cuda_stream
    pool = asse.Pool(p, stream=stream)
    m = asse.MLP(seed=3, stream=stream)
    orc = oracle.Oracle.from_params(p)
    for t in range(5):
        pairs = mixed_pairs(11, t, 20001, [20, 60, 400, 5000])
        pool.ingest(to_device(pairs))
        orc.ingest(pairs)
        pool.scan(4)
        # shift the output bias so the model's outputs straddle the training
        # range: some inside, some above, some below
        y0 = m.forward(pool.features()).cpu().numpy().astype(np.float64)
        prm = m.params()
        prm[-1] += np.float32(1.0 - np.median(y0))
        m.set_params(prm)
        y1 = y0 + (1.0 - np.median(y0))
        max_log_n = float(np.quantile(y1, 0.75))
        est, nfb, x = pool.estimate_learned(m, max_log_n)
        y = m.forward(x).cpu().numpy().astype(np.float64)
        cnt = orc.counts(4).reshape(-1).astype(np.float64)
        inside = (cnt > 0) & (y <= max_log_n)
        c = np.where(cnt >= g, g - 0.5, cnt)
        lc = -g * np.log((g - c) / g)
        want = np.where(inside, np.exp(np.maximum(y, 0.0)), lc)
        got = est.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-5)
        assert int(nfb.item()) == int((~inside).sum())
        if t >= 2:
            assert (cnt >= g).any() and inside.any() and (~inside).any()
        pool.restore()
        pool.advance()
        orc.advance()
