"""FP64 NumPy reference of the candidate-scoring network (test infrastructure only).

The network scores a candidate conditioning variable k for an edge side (i, j)
at level l from five features and is used only to reorder subset enumeration:

    x  = (|rho_ik|, |rho_jk|, |rho_ij|, l / 8, |rho_ij.k|)          (5)
    h1 = relu(W1 x + b1)                                            (64)
    h2 = relu(W2 h1 + b2)                                           (64)
    y  = w3 . h2 + b3                                               (logit)

Training minimises the mean binary cross-entropy with logits,
    L = mean( log(1 + exp(y)) - t * y ),
with t = 1 when k belongs to the separating set the plain method stored.
Parameters are updated with Adam (Kingma and Ba, 2015):
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
    theta <- theta - lr * (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps).

The paper has no learned component; this module is the plain definition the
GPU forward, backward and update kernels are compared against. Parity is
pinned by central finite differences and closed forms in the tests.
"""
from __future__ import annotations

import numpy as np

IN, H1, H2 = 5, 64, 64
PARAM_SHAPES = (("W1", (H1, IN)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)),
                ("w3", (H2,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in PARAM_SHAPES)


def init_params(seed: int = 0) -> dict:
    """He-uniform initialisation (seeded); biases zero."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, shape in PARAM_SHAPES:
        if name.startswith("b"):
            P[name] = np.zeros(shape)
        else:
            fan_in = shape[-1] if len(shape) > 1 else shape[0]
            bound = np.sqrt(6.0 / fan_in)
            P[name] = rng.uniform(-bound, bound, size=shape)
    return P


def flatten(P: dict) -> np.ndarray:
    """Parameters packed in the fixed order W1, b1, W2, b2, w3, b3 (row-major)."""
    return np.concatenate([np.asarray(P[name], dtype=np.float64).reshape(-1) for name, _ in PARAM_SHAPES])


def unflatten(v: np.ndarray) -> dict:
    P, k = {}, 0
    for name, shape in PARAM_SHAPES:
        size = int(np.prod(shape))
        P[name] = np.asarray(v[k:k + size], dtype=np.float64).reshape(shape)
        k += size
    return P


def forward(P: dict, X: np.ndarray):
    """Returns (logits, cache). X is B x 5."""
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (X, a1, h1, a2, h2)


def softplus(y):
    return np.where(y > 0, y + np.log1p(np.exp(-np.abs(y))), np.log1p(np.exp(-np.abs(y))))


def loss(P: dict, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(P, X)
    return float(np.mean(softplus(y) - t * y))


def backward(P: dict, X: np.ndarray, t: np.ndarray):
    """Returns (loss, grads dict) for the mean BCE-with-logits loss."""
    y, (X, a1, h1, a2, h2) = forward(P, X)
    B = X.shape[0]
    L = float(np.mean(softplus(y) - t * y))
    sig = 1.0 / (1.0 + np.exp(-y))
    dy = (sig - t) / B                       # B
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, P["w3"]) * (a2 > 0)   # B x H2
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ P["W2"]) * (a1 > 0)         # B x H1
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return L, g


def adam_step(P: dict, g: dict, m: dict, v: dict, step: int, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update in place; ``step`` counts from 1."""
    for name, _ in PARAM_SHAPES:
        m[name] = beta1 * m[name] + (1 - beta1) * g[name]
        v[name] = beta2 * v[name] + (1 - beta2) * g[name] ** 2
        mhat = m[name] / (1 - beta1 ** step)
        vhat = v[name] / (1 - beta2 ** step)
        P[name] = P[name] - lr * mhat / (np.sqrt(vhat) + eps)
    return P, m, v


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
