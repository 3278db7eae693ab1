"""Pins of the FP64 MLP reference used to check the GPU training kernels:
BF16 rounding agrees with torch's BF16 conversion (round to nearest even),
and the analytic gradients of the unrounded network agree with central
finite differences of its loss."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -2.5, 65504.0]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)


def _params(seed):
    rng = np.random.default_rng(seed)
    q = {name: rng.normal(scale=0.2, size=shape) for name, shape in mlp.SIZES}
    return mlp.pack(q)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradients_match_finite_differences(seed):
    rng = np.random.default_rng(seed + 10)
    p = _params(seed)
    X = rng.normal(size=(12, mlp.FEAT))
    t = rng.normal(size=12)
    loss, g, _y = mlp.loss_and_grads(p, X, t, rounding=False)
    idx = np.concatenate([rng.integers(0, mlp.NPARAMS, 60), [mlp.NPARAMS - 1]])
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        lp = mlp.loss_and_grads(p + e, X, t, rounding=False)[0]
        lm = mlp.loss_and_grads(p - e, X, t, rounding=False)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # with rounding the loss moves by at most the BF16 perturbation of the activations
    loss_r = mlp.loss_and_grads(p, X, t, rounding=True)[0]
    assert abs(loss_r - loss) < 0.05 * max(1.0, loss)
