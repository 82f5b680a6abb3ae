"""CPU reference of the troubled-cell indicator network (FP64 numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network 32 -> 64 -> 64 -> 1: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
z = w3 . h2 + b3, p = sigmoid(z).  Loss: class-weighted binary cross-entropy
averaged over the batch, L = (1/n) sum_i c(y_i) [-y log p - (1-y) log(1-p)],
with c(1) = w_pos, c(0) = w_neg.  Gradients by hand-written backpropagation,
pinned by finite differences in the tests.

``bf16=True`` rounds, as the GPU kernels do, the inputs x, the weights W1, W2,
w3, the hidden activation h1 fed to the second layer, and the back-propagated
dh2 and dh1 fed to the gradient products, to bfloat16 (round to nearest
even); everything else stays FP64.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 32, 64
SHAPES = {"W1": (N_H, N_IN), "b1": (N_H,), "W2": (N_H, N_H), "b2": (N_H,), "w3": (N_H,), "b3": (1,)}
ORDER = ("W1", "b1", "W2", "b2", "w3", "b3")
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())


def bf16(a) -> np.ndarray:
    """Round to bfloat16 (nearest even) and return as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(theta) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name in ORDER:
        n = int(np.prod(SHAPES[name]))
        out[name] = theta[k:k + n].reshape(SHAPES[name])
        k += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[n], dtype=np.float64).ravel() for n in ORDER])


def forward(theta, X, bf16_round: bool = False, h1=None):
    """Logits z [n] and the activations needed by backward.  h1, if given,
    replaces the rounded first hidden layer fed to the second layer (e.g. a
    device's own BF16 rounding of it)."""
    p = unflatten(theta)
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(X)
    a1 = x @ r(p["W1"]).T + p["b1"]
    h1r = r(np.maximum(a1, 0.0)) if h1 is None else np.asarray(h1, dtype=np.float64)
    a2 = h1r @ r(p["W2"]).T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ r(p["w3"]) + p["b3"][0]
    return z, {"x": x, "a1": a1, "h1r": h1r, "a2": a2, "h2": h2}


def loss(theta, X, y, w_pos=1.0, w_neg=1.0, bf16_round=False) -> float:
    z, _ = forward(theta, X, bf16_round)
    c = np.where(y > 0.5, w_pos, w_neg)
    # -y log s(z) - (1-y) log(1-s(z)) = softplus(z) - y z, evaluated stably
    sp = np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))
    return float(np.mean(c * (sp - y * z)))


def grad(theta, X, y, w_pos=1.0, w_neg=1.0, bf16_round=False, h1=None, terms=False) -> np.ndarray:
    """Gradient of loss() with respect to the flat parameter vector (h1 as in
    forward()).  terms=True returns instead, per parameter, the sum of the
    magnitudes of the per-sample terms whose signed sum is that gradient
    entry (the scale of its rounding error)."""
    p = unflatten(theta)
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    z, a = forward(theta, X, bf16_round, h1)
    n = X.shape[0]
    c = np.where(y > 0.5, w_pos, w_neg)
    s = 1.0 / (1.0 + np.exp(-z))
    dz = c * (s - y) / n
    f = np.abs if terms else (lambda v: v)
    g = {}
    g["w3"] = f(a["h2"]).T @ f(dz)
    g["b3"] = np.array([f(dz).sum()])
    dh2 = np.outer(dz, r(p["w3"])) * (a["a2"] > 0)
    dh2r = r(dh2)
    g["W2"] = f(dh2r).T @ f(a["h1r"])
    g["b2"] = f(dh2).sum(axis=0)
    dh1 = (dh2r @ r(p["W2"])) * (a["a1"] > 0)
    dh1r = r(dh1)
    g["W1"] = f(dh1r).T @ f(a["x"])
    g["b1"] = f(dh1).sum(axis=0)
    return flatten(g)


def init(seed: int) -> np.ndarray:
    """He-normal initial weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.normal(0.0, np.sqrt(2.0 / N_IN), SHAPES["W1"]),
        "b1": np.zeros(N_H),
        "W2": rng.normal(0.0, np.sqrt(2.0 / N_H), SHAPES["W2"]),
        "b2": np.zeros(N_H),
        "w3": rng.normal(0.0, np.sqrt(1.0 / N_H), SHAPES["w3"]),
        "b3": np.zeros(1),
    }
    return flatten(p)


def adam_step(theta, g, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
