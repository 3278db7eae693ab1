"""FP64 CPU reference of the learned per-ATV estimator -- TEST
INFRASTRUCTURE ONLY (gradient checks of the GPU kernels).

The model of include/asse_learn.h: y = w3 . H2 + b3, H2 = relu(H1 W2^T + b2),
H1 = relu(X W1^T + b1), loss = mean (y - t)^2, and its exact gradients.  The
arithmetic is float64; the values the GPU stores in BF16 (the inputs, the
weight copies W1, W2, the activations H1, H2 and the back-propagated
pre-activations dZ2, dZ1) are rounded to BF16 at the same points, so the two
differ only by FP32 accumulation order and the rare rounding tie."""
from __future__ import annotations

import numpy as np

FEAT, HID = 80, 256
SIZES = [("W1", (HID, FEAT)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("w3", (HID,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _n, s in SIZES)


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    b = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _s in SIZES])


def _id(x):
    return np.asarray(x, dtype=np.float64)


def forward(p: np.ndarray, X: np.ndarray, rounding: bool = True):
    """y and the stored activations for inputs X (already BF16 values).
    rounding=False gives the plain float64 network."""
    r = bf16 if rounding else _id
    q = unpack(p)
    H1 = r(np.maximum(X @ r(q["W1"]).T + q["b1"], 0.0))
    H2 = r(np.maximum(H1 @ r(q["W2"]).T + q["b2"], 0.0))
    y = H2 @ q["w3"] + q["b3"][0]
    return y, H1, H2


def loss_and_grads(p: np.ndarray, X: np.ndarray, t: np.ndarray, rounding: bool = True, loss: str = "log_mse"):
    """Loss and gradients: 'log_mse' = mean (y - t)^2; 'rel_mse' = mean
    (exp(y - t) - 1)^2 (y - t clamped at 20), the squared relative error of
    exp(y) against exp(t)."""
    r = bf16 if rounding else _id
    q = unpack(p)
    n = X.shape[0]
    y, H1, H2 = forward(p, X, rounding)
    d = y - t
    if loss == "rel_mse":
        e = np.exp(np.minimum(d, 20.0))
        dy = 2.0 * (e - 1.0) * e / n
        loss = float(np.mean((e - 1.0) ** 2))
    else:
        dy = 2.0 * d / n
        loss = float(np.mean(d * d))
    g = {"w3": H2.T @ dy, "b3": np.array([dy.sum()])}
    dZ2 = r(dy[:, None] * q["w3"][None, :] * (H2 > 0))
    g["b2"] = dZ2.sum(axis=0)
    g["W2"] = dZ2.T @ H1
    dZ1 = r((dZ2 @ r(q["W2"])) * (H1 > 0))
    g["b1"] = dZ1.sum(axis=0)
    g["W1"] = dZ1.T @ X
    return loss, pack(g), y


def error_scales(p: np.ndarray, X: np.ndarray, t: np.ndarray, loss: str = "log_mse"):
    """Per-entry scales for comparing a BF16-in / FP32-accumulate computation
    of the network with this reference: for y and for every gradient entry,
    the sum of the absolute values of the terms that make it up (with the
    absolute values of the upstream factors).  Two implementations that
    round the same BF16 storage points differ by at most a few BF16 steps
    (2^-8 relative) of some of those terms, so |gpu - reference| stays
    within a small multiple of 2^-8 times the scale, entry by entry.
    Returns (scale of y [n], scale of the gradients [NPARAMS])."""
    q = unpack(p)
    n = X.shape[0]
    y, H1, H2 = forward(p, X)
    ys = np.abs(H2) @ np.abs(q["w3"]) + abs(q["b3"][0])
    d = y - t
    if loss == "rel_mse":
        e = np.exp(np.minimum(d, 20.0))
        ady = np.abs(2.0 * (e - 1.0) * e / n)
    else:
        ady = np.abs(2.0 * d / n)
    s = {"w3": np.abs(H2).T @ ady, "b3": np.array([ady.sum()])}
    A2 = ady[:, None] * np.abs(q["w3"])[None, :] * (H2 > 0)
    s["b2"] = A2.sum(axis=0)
    s["W2"] = A2.T @ np.abs(H1)
    A1 = (A2 @ np.abs(bf16(q["W2"]))) * (H1 > 0)
    s["b1"] = A1.sum(axis=0)
    s["W1"] = A1.T @ np.abs(X)
    return ys, pack(s)
