"""Training data and training driver for the candidate-scoring network.

The network (5 -> 64 -> 64 -> 1, kernels in csrc/k_mlp.cu) scores each
candidate k of a row i of A'_G at level l >= 1; the level kernel enumerates the
row's subsets in the order of descending score. The examples come from the
separating sets the plain method stores (cupc_mlp_examples: the side whose
frozen neighbourhood holds S, one example per candidate of that row other than
the other endpoint, labelled 1 iff the candidate is in S, features computed on
the device by the kernels' own feature code).

This module only marshals: it runs the library calls per problem, concatenates
their device tensors, shuffles them with a seeded permutation and seeds the
initial weights; the forward, backward and Adam updates run in the library's
kernels (Context.mlp_train).
"""
from __future__ import annotations

import numpy as np

HIDDEN, FEATURES = 64, 5
PARAMS = HIDDEN * FEATURES + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def init_weights(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, packed W1, b1, W2, b2, w3, b3."""
    rng = np.random.default_rng(seed)
    w1 = rng.uniform(-1, 1, (HIDDEN, FEATURES)) * np.sqrt(6.0 / FEATURES)
    w2 = rng.uniform(-1, 1, (HIDDEN, HIDDEN)) * np.sqrt(6.0 / HIDDEN)
    w3 = rng.uniform(-1, 1, HIDDEN) * np.sqrt(6.0 / HIDDEN)
    return np.concatenate([w1.ravel(), np.zeros(HIDDEN), w2.ravel(), np.zeros(HIDDEN), w3, [0.0]]).astype(np.float32)


def collect(ctx, problems, mode=None, per_problem=None, seed=0):
    """Examples (device tensors X [m x 5], t [m]) from the plain method's
    canonical SepSets on each problem; with per_problem, a seeded sample of at
    most that many examples of each problem."""
    import torch

    import paper_1812_08491_gb300 as cupc
    mode = cupc.MODE_PLAIN_FP64 if mode is None else mode
    rng = np.random.default_rng(seed)
    xs, ts = [], []
    for s in problems:
        X = torch.from_numpy(np.ascontiguousarray(s.Xt)).cuda().T
        res = ctx.skeleton(X, s.alpha, mode=mode, canonical=True)
        C32 = ctx.correlation(X, cupc.F32)
        Xe, te = res.mlp_examples(C32)
        res.free()
        if per_problem is not None and Xe.shape[0] > per_problem:
            pick = torch.from_numpy(np.sort(rng.choice(Xe.shape[0], per_problem, replace=False))).cuda()
            Xe, te = Xe[pick], te[pick]
        xs.append(Xe)
        ts.append(te)
    return torch.cat(xs), torch.cat(ts)


def train(ctx, X, t, epochs: int = 6, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Seeded shuffle, then Adam in the library's kernels. X, t: numpy arrays or
    CUDA tensors. Returns per-epoch losses."""
    import torch
    Xd = torch.as_tensor(X).cuda()
    td = torch.as_tensor(t).cuda()
    order = torch.from_numpy(np.random.default_rng(seed).permutation(Xd.shape[0])).cuda()
    Xd = Xd[order].contiguous()
    td = td[order].contiguous()
    ctx.mlp_set_weights(init_weights(seed))
    return ctx.mlp_train(Xd, td, batch=batch, epochs=epochs, lr=lr)
