"""Float64 reference of the join-size network — TEST INFRASTRUCTURE.

Only tests import this module.  It shares no code with the GPU library.

The network (not in the paper, which has no learned part)
maps 16 join features to a prediction of log2(1 + join output size):
    h1 = relu(W1 x + b1)      W1: 64 x 16
    h2 = relu(W2 h1 + b2)     W2: 64 x 64
    y' = w3 . h2 + b3         w3: 64
trained with the pinball (quantile) loss at level tau,
    L = mean_n max(tau (y_n - y'_n), (tau - 1)(y_n - y'_n)),
whose derivative in y'_n is -tau/N where y_n > y'_n and (1 - tau)/N
elsewhere (the value 0 at the kink is taken on the second branch), and the
Adam update (Kingma & Ba, 2015) with bias correction.

Parameters are one flat vector in the order W1 (row-major), b1, W2
(row-major), b2, w3, b3: 64*16 + 64 + 64*64 + 64 + 64 + 1 = 5313 values.
"""
from __future__ import annotations

import numpy as np

D_IN, H = 16, 64
SIZES = [("W1", (H, D_IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(theta, X):
    """Returns (prediction, cache) for inputs X (N x 16)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["w3"] + p["b3"][0]
    return out, (X, z1, h1, z2, h2)


def to_bf16(a) -> np.ndarray:
    """Rounds float32 values to bfloat16 (round to nearest, ties to even),
    returned as float64: the upper 16 bits of the float32 pattern after
    adding 0x7FFF plus the lowest kept bit."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, X):
    """The prediction path: weights, inputs and hidden activations rounded
    to bfloat16, sums in float64 (the kernel sums in float32)."""
    p = {k: to_bf16(v) for k, v in unpack(theta).items()}
    x = to_bf16(np.asarray(X, dtype=np.float32))
    h1 = to_bf16(np.maximum(x @ p["W1"].T + p["b1"], 0.0).astype(np.float32))
    h2 = to_bf16(np.maximum(h1 @ p["W2"].T + p["b2"], 0.0).astype(np.float32))
    return h2 @ p["w3"] + p["b3"][0]


def pinball(pred, y, tau):
    r = np.asarray(y, dtype=np.float64) - pred
    return float(np.mean(np.maximum(tau * r, (tau - 1.0) * r)))


def gradient(theta, X, y, tau):
    """Loss and its gradient with respect to the flat parameter vector."""
    pred, (X, z1, h1, z2, h2) = forward(theta, X)
    p = unpack(theta)
    n = X.shape[0]
    y = np.asarray(y, dtype=np.float64)
    g = np.where(y > pred, -tau, 1.0 - tau) / n           # dL/dpred
    grads = {"w3": h2.T @ g, "b3": np.array([g.sum()])}
    gh2 = np.outer(g, p["w3"]) * (z2 > 0)                  # N x 64
    grads["W2"] = gh2.T @ h1
    grads["b2"] = gh2.sum(axis=0)
    gh1 = (gh2 @ p["W2"]) * (z1 > 0)
    grads["W1"] = gh1.T @ X
    grads["b1"] = gh1.sum(axis=0)
    return pinball(pred, y, tau), pack(grads)


def adam(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init(seed: int) -> np.ndarray:
    """He-uniform initial weights from a seeded numpy generator (zero biases)."""
    rng = np.random.default_rng(seed)
    parts = {"W1": rng.uniform(-1, 1, (H, D_IN)) * np.sqrt(6.0 / D_IN),
             "b1": np.zeros(H),
             "W2": rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H),
             "b2": np.zeros(H),
             "w3": rng.uniform(-1, 1, H) * np.sqrt(6.0 / H),
             "b3": np.zeros(1)}
    return pack(parts)
