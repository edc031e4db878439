"""Training data and training driver for the candidate-scoring network.

The network (5 -> 64 -> 64 -> 1, kernels in csrc/k_mlp.cu) scores a candidate
conditioning variable k for an edge side (i, j) at level l >= 2; the level
kernel enumerates each side's subsets in the order of descending score. The
examples come from separating sets the plain method stores: for a pair (x, y)
removed at level l with set S, the side whose frozen neighbourhood adj'_l
contains S (the smaller endpoint first, as the serial order) contributes one
example per candidate k in adj'_l(side) minus the other endpoint, labelled 1
iff k is in S. Features match the kernel's: (|C_ik|, |C_jk|, |C_ij|, l/8,
|rho_ij.k|) on the FP32 correlation the kernels read.

Host-side work here is data plumbing only: gathering examples from results
and seeding the initial weights; the forward, backward and Adam updates run in
the library's kernels (Context.mlp_train).
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


def features(C: np.ndarray, i: int, j: int, ks: np.ndarray, level: int) -> np.ndarray:
    """Feature rows of candidates ks for side (i, j) (same formulas as the kernel)."""
    C = C.astype(np.float32, copy=False)
    cij = np.float32(C[i, j])
    cik = C[i, ks]
    cjk = C[j, ks]
    den = (np.float32(1) - cik * cik) * (np.float32(1) - cjk * cjk)
    rho = np.where(den > 1e-12, np.abs((cij - cik * cjk) / np.sqrt(np.maximum(den, 1e-30))), 1.0)
    out = np.empty((ks.size, FEATURES), dtype=np.float32)
    out[:, 0] = np.abs(cik)
    out[:, 1] = np.abs(cjk)
    out[:, 2] = abs(cij)
    out[:, 3] = level * 0.125
    out[:, 4] = rho
    return out


def examples_from_result(C32: np.ndarray, sep_levels: np.ndarray, sepsets: dict):
    """(X, t) examples from one skeleton result (levels >= 2)."""
    p = sep_levels.shape[0]
    xs, ts = [], []
    for (x, y), (level, S) in sepsets.items():
        if level < 2:
            continue
        frozen = (sep_levels < 0) | (sep_levels >= level)
        np.fill_diagonal(frozen, False)
        Sset = set(S)
        for a, b in ((x, y), (y, x)):
            nb = np.nonzero(frozen[a])[0]
            if not Sset.issubset(set(nb.tolist())):
                continue
            ks = nb[nb != b]
            xs.append(features(C32, a, b, ks, level))
            ts.append(np.isin(ks, list(Sset)).astype(np.float32))
            break
    if not xs:
        return np.zeros((0, FEATURES), np.float32), np.zeros(0, np.float32)
    return np.concatenate(xs), np.concatenate(ts)


def collect(ctx, problems, mode=None):
    """Examples from the plain method's canonical SepSets on each problem."""
    import paper_1812_08491_gb300 as cupc
    import torch
    mode = cupc.MODE_PLAIN_FP64 if mode is None else mode
    xs, ts = [], []
    for s in problems:
        X = torch.from_numpy(s.Xt).cuda().T
        res = ctx.skeleton(X, s.alpha, mode=mode, canonical=True)
        C32 = ctx.correlation(X, cupc.F32).cpu().numpy()
        Xe, te = examples_from_result(C32, res.sep_levels(), res.sepsets())
        res.free()
        xs.append(Xe)
        ts.append(te)
    return np.concatenate(xs), np.concatenate(ts)


def train(ctx, X: np.ndarray, t: np.ndarray, epochs: int = 6, batch: int = 4096, lr: float = 2e-3,
          seed: int = 0):
    """Seeded shuffle, then Adam in the library's kernels. Returns per-epoch losses."""
    import torch
    rng = np.random.default_rng(seed)
    order = rng.permutation(X.shape[0])
    Xd = torch.from_numpy(np.ascontiguousarray(X[order])).cuda()
    td = torch.from_numpy(np.ascontiguousarray(t[order])).cuda()
    ctx.mlp_set_weights(init_weights(seed))
    return ctx.mlp_train(Xd, td, batch=batch, epochs=epochs, lr=lr)
