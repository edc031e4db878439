"""Pins of the FP64 MLP reference: finite differences, closed forms, Adam."""
import numpy as np
import pytest

from oracle import mlp


def _batch(seed, B=33):
    rng = np.random.default_rng(seed)
    X = np.column_stack([rng.uniform(0, 1, B), rng.uniform(0, 1, B), rng.uniform(0, 1, B),
                         rng.integers(2, 7, B) / 8.0, rng.uniform(0, 1, B)])
    t = (rng.random(B) < 0.3).astype(np.float64)
    return X, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_central_differences(seed):
    P = mlp.init_params(seed)
    for name in P:                         # nonzero biases so every term is exercised
        if name.startswith("b"):
            P[name] = np.random.default_rng(seed + 50).normal(0, 0.1, P[name].shape)
    X, t = _batch(seed)
    L, g = mlp.backward(P, X, t)
    v = mlp.flatten(P)
    gv = mlp.flatten(g)
    rng = np.random.default_rng(seed + 100)
    h = 1e-6
    for k in rng.choice(v.size, size=80, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[k] += h
        vm[k] -= h
        fd = (mlp.loss(mlp.unflatten(vp), X, t) - mlp.loss(mlp.unflatten(vm), X, t)) / (2 * h)
        assert abs(fd - gv[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gv[k])


def test_zero_network_closed_form():
    P = {name: np.zeros(shape) for name, shape in mlp.PARAM_SHAPES}
    P["b3"] = np.array([0.7])
    X, t = _batch(3)
    L, g = mlp.backward(P, X, t)
    sp = np.log1p(np.exp(0.7))
    assert L == pytest.approx(sp - t.mean() * 0.7, rel=1e-14)
    # only the output bias has a gradient: mean(sigmoid(b3) - t)
    assert g["b3"][0] == pytest.approx(1 / (1 + np.exp(-0.7)) - t.mean(), rel=1e-13)
    for name in ("W1", "b1", "W2", "b2", "w3"):
        assert np.all(g[name] == 0)


def test_adam_first_step_is_signed_lr():
    P = mlp.init_params(4)
    X, t = _batch(4)
    _, g = mlp.backward(P, X, t)
    m = {k: np.zeros_like(a) for k, a in P.items()}
    v = {k: np.zeros_like(a) for k, a in P.items()}
    P2, _, _ = mlp.adam_step({k: a.copy() for k, a in P.items()}, g, m, v, step=1, lr=1e-3, eps=0.0)
    for name in P:
        d = P2[name] - P[name]
        nz = g[name] != 0
        assert np.allclose(d[nz], -1e-3 * np.sign(g[name][nz]), rtol=1e-12, atol=0)


def test_bf16_round():
    vals = np.array([1.0, 1.00390625, 1.0 + 2**-9, 1.0 + 3 * 2**-9, -3.14159, 0.0])
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0  # 1 + 2**-8 is a tie: to even
    assert r[3] == 1.0 + 2**-7
    assert abs(r[4] - (-3.140625)) < 1e-12
