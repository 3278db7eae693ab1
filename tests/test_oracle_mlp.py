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


@pytest.mark.parametrize("seed,loss_kind", [(1, "log_mse"), (2, "log_mse"), (3, "rel_mse"), (4, "rel_mse")])
def test_gradients_match_finite_differences(seed, loss_kind):
    rng = np.random.default_rng(seed + 10)
    p = _params(seed)
    X = rng.normal(size=(12, mlp.FEAT))
    t = rng.normal(size=12)
    if loss_kind == "rel_mse":
        # targets near the outputs: relative errors of order one, away from the clamp
        t = mlp.forward(p, X, rounding=False)[0] + rng.normal(scale=0.7, size=12)
    loss, g, _y = mlp.loss_and_grads(p, X, t, rounding=False, loss=loss_kind)
    idx = np.concatenate([rng.integers(0, mlp.NPARAMS, 60), [mlp.NPARAMS - 1]])
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        lp = mlp.loss_and_grads(p + e, X, t, rounding=False, loss=loss_kind)[0]
        lm = mlp.loss_and_grads(p - e, X, t, rounding=False, loss=loss_kind)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # with rounding the loss moves by at most the BF16 perturbation of the activations
    loss_r = mlp.loss_and_grads(p, X, t, rounding=True, loss=loss_kind)[0]
    assert abs(loss_r - loss) < (0.05 if loss_kind == "log_mse" else 0.15) * max(1.0, loss)


def test_rel_mse_is_the_squared_relative_error():
    """The relative loss is the mean squared relative error of exp(y)
    against exp(t), computed here from the estimates themselves."""
    rng = np.random.default_rng(7)
    p = _params(5)
    X = rng.normal(size=(20, mlp.FEAT))
    t = rng.normal(size=20) + 3.0
    loss, _g, y = mlp.loss_and_grads(p, X, t, rounding=False, loss="rel_mse")
    n_hat, n_true = np.exp(y), np.exp(t)
    assert abs(loss - np.mean(((n_hat - n_true) / n_true) ** 2)) <= 1e-12 * max(1.0, loss)
