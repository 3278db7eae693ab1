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


@pytest.mark.parametrize("k,g,counter", [(6, 150, "at"), (10, 512, "at"), (5, 77, "ace")])
def test_features_match_definition(mods, k, g, counter):
    asse, oracle, omlp, torch = mods
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
        at = orc.at().astype(np.int64)                       # [r][E][g]
        if counter == "ace":
            age = k - at
            active = at >= k - kp + 1
        else:
            act = np.array([orc.act(h) for h in range(g)])[None, None, :]
            age = (act - at) % (2 * k)
            active = (at != 2 * k) & (age < kp)
        cnt = active.sum(axis=2)
        want = np.zeros((orc.r * orc.E, 80))
        want[:, 0] = (cnt / g).reshape(-1)
        for a in range(min(kp, 64)):
            want[:, 1 + a] = ((active & (age == a)).sum(axis=2) / g).reshape(-1)
        aat = orc.aat(orc.counts(kp)).astype(np.float64) / (g * (1 << orc.c))     # [r][frames]
        frame = (np.arange(orc.E) >> orc.c)
        for i in range(orc.r):
            rows = slice(i * orc.E, (i + 1) * orc.E)
            want[rows, 65] = aat[i, frame]
            want[rows, 66] = np.prod(aat, axis=0)[frame]
            want[rows, 67] = aat.mean(axis=0)[frame]
        np.testing.assert_allclose(x, _bf16(want), rtol=0, atol=1e-7, err_msg=f"t={t}")
        pool.advance()
        orc.advance()


def test_forward_and_gradients_match_fp64_reference(mods):
    asse, oracle, omlp, torch = mods
    m = asse.MLP(seed=5)
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
    assert np.max(np.abs(y - y_ref)) <= 2e-3 * (1 + np.max(np.abs(y_ref)))
    loss = float(m.backward(xd, td).cpu()[0])
    g = m.grads().astype(np.float64)
    loss_ref, g_ref, _ = omlp.loss_and_grads(p, X, t)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    o = 0
    for name, shape in omlp.SIZES:
        k = int(np.prod(shape))
        a, b = g[o:o + k], g_ref[o:o + k]
        # FP32 accumulation over up to n rows and the rare BF16 rounding tie:
        # a relative error of the whole block well under 1 %
        assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b) + 1e-7, (name, np.linalg.norm(a - b),
                                                                          np.linalg.norm(b))
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
    tol = 2e-3 * (1 + np.max(np.abs(y_ref)))
    assert np.max(np.abs(y[rows] - y_ref)) <= tol, (n, np.max(np.abs(y[rows] - y_ref)))


def test_training_beats_linear_counting(mods):
    asse, oracle, omlp, torch = mods
    keys = synth.method_keys(1)
    cfg = dict(k=10, g=512, r=4, n_max_log2=14, bg_max=0.01, seed=11, bh_a=keys["bh_a"], bh_b=keys["bh_b"])
    x, ln, lc = asse.synth_states(cfg, 0, 200_000)
    xt, lnt, lct = asse.synth_states(cfg, 10_000_000, 20_000)
    assert torch.all(ln >= 0) and torch.all(ln <= 14 * np.log(2) + 1e-5)
    m = asse.MLP(seed=2)
    bs = 4096
    perm = torch.randperm(x.shape[0], device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    for step in range(600):
        i = perm[(step * bs) % x.shape[0]:(step * bs) % x.shape[0] + bs]
        lr = 2e-3 if step < 400 else 5e-4
        m.train_step(x[i].contiguous(), ln[i].contiguous(), lr)
    y = m.forward(xt)
    n_true = torch.exp(lnt)
    mre_mlp = torch.mean(torch.abs(torch.exp(y) - n_true) / n_true).item()
    mre_lc = torch.mean(torch.abs(lct - n_true) / n_true).item()
    assert mre_mlp < mre_lc, (mre_mlp, mre_lc)


def test_learned_estimate_with_fallback(mods):
    """asse_estimate_learned: the model's output where it is inside its
    training range, Eq. 2 from the ATV's count elsewhere (saturated ATVs and
    outputs above max_log_n), on a pool with saturated and light ATVs."""
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
        inside = (cnt < g) & (y >= 0.0) & (y <= max_log_n)
        c = np.where(cnt >= g, g - 0.5, cnt)
        lc = -g * np.log((g - c) / g)
        want = np.where(inside, np.exp(y), lc)
        got = est.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-5)
        assert int(nfb.item()) == int((~inside).sum())
        if t >= 2:
            assert (cnt >= g).any() and inside.any()
        pool.restore()
        pool.advance()
        orc.advance()
