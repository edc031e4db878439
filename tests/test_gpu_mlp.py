"""GPU kernels of the candidate-scoring network against the FP64 reference
(oracle/mlp.py), and learned subset ordering against the skeleton oracle.

Tolerances: the GPU computes in FP32, the reference in FP64 on the same
(FP32-rounded) weights and data: gradients within 1e-4 relative of the largest
entry plus 1e-3 of each entry; scores (bf16 weights, FP32 accumulation) within
1e-4 relative. The learned order changes only the enumeration order, so the
skeleton must equal the oracle's exactly and every stored SepSet must test
independent under the oracle's CI test.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as mref
from synth import sem

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")
from paper_1812_08491_gb300 import learned  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    cupc.build_library()
    c = cupc.Context(0)
    yield c
    c.close()


def _params(seed):
    P = mref.init_params(seed)
    rng = np.random.default_rng(seed + 7)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(0, 0.2, P[k].shape)
    v = mref.flatten(P).astype(np.float32)
    return v, mref.unflatten(v.astype(np.float64))


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = np.column_stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.uniform(0, 1, n),
                         rng.integers(2, 9, n) / 8.0, rng.uniform(0, 1, n)]).astype(np.float32)
    t = (rng.random(n) < 0.25).astype(np.float32)
    return X, t


@pytest.mark.parametrize("n", [1, 37, 1000, 5000])
def test_gradient_matches_reference(ctx, n):
    v, P = _params(1)
    X, t = _data(2, n)
    ctx.mlp_set_weights(v)
    g, loss = ctx.mlp_grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    L, gr = mref.backward(P, X.astype(np.float64), t.astype(np.float64))
    ref = mref.flatten(gr)
    scale = np.max(np.abs(ref))
    assert np.all(np.abs(g - ref) <= 1e-4 * scale + 1e-3 * np.abs(ref)), np.max(np.abs(g - ref))
    assert loss == pytest.approx(L, rel=1e-5)


def test_forward_matches_reference_with_bf16_weights(ctx):
    v, _ = _params(3)
    X, _ = _data(4, 3000)
    ctx.mlp_set_weights(v)
    y = ctx.mlp_forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Pb = mref.unflatten(mref.bf16_round(v))
    ref, _ = mref.forward(Pb, X.astype(np.float64))
    assert np.max(np.abs(y - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


def test_adam_step_matches_reference(ctx):
    v, P = _params(5)
    X, t = _data(6, 2048)
    ctx.mlp_set_weights(v)
    lr = 1e-3
    ctx.mlp_train(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), batch=2048, epochs=1, lr=lr)
    w = ctx.mlp_get_weights()
    L, gr = mref.backward(P, X.astype(np.float64), t.astype(np.float64))
    m = {k: np.zeros_like(a) for k, a in P.items()}
    vv = {k: np.zeros_like(a) for k, a in P.items()}
    P2, _, _ = mref.adam_step({k: a.copy() for k, a in P.items()}, gr, m, vv, step=1, lr=lr)
    ref = mref.flatten(P2)
    gflat = np.abs(mref.flatten(gr))
    sure = gflat > 1e-4 * gflat.max()          # the first step is lr * sign(g): skip g ~ 0
    assert np.max(np.abs(w[sure] - ref[sure])) <= 1e-6


def test_training_reduces_loss(ctx):
    X, _ = _data(8, 20000)
    t = (X[:, 4] < 0.2).astype(np.float32)     # a learnable rule
    losses = learned.train(ctx, X, t, epochs=5, batch=2048, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]


def _host_examples(C32, sep_levels, sepsets):
    """The examples' definition written out on the host (test reference): for a
    removal (x, y) at level l >= 1 with set S, the endpoint a whose neighbours
    N at the start of level l contain S (x first) gives one row per neighbour
    k != y of N: (|C_ak|, mean |C_jk|, mean |C_aj|, l/8, mean |rho_aj.k|), the
    means over j in N \\ {k} (the C_jk terms 0 at level 1), label k in S."""
    rows, labels = [], []
    for (x, y), (level, S) in sorted(sepsets.items()):
        if level < 1:
            continue
        G = (sep_levels < 0) | (sep_levels >= level)
        np.fill_diagonal(G, False)
        for a, b in ((x, y), (y, x)):
            nb = np.nonzero(G[a])[0]
            if not set(S) <= set(nb.tolist()):
                continue
            for k in nb[nb != b]:
                others = nb[nb != k]
                cik = np.float64(C32[a, k])
                mij = np.mean(np.abs(C32[a, others].astype(np.float64))) if others.size else 0.0
                mjk = mrho = 0.0
                if level >= 2 and others.size:
                    cjk = C32[others, k].astype(np.float64)
                    cij = C32[a, others].astype(np.float64)
                    den = (1 - cik * cik) * (1 - cjk * cjk)
                    rho = np.where(den > 1e-12, np.abs(cij - cik * cjk) / np.sqrt(np.maximum(den, 1e-300)), 1.0)
                    mjk, mrho = np.mean(np.abs(cjk)), np.mean(rho)
                rows.append([abs(cik), mjk, mij, level / 8.0, mrho])
                labels.append(1.0 if k in S else 0.0)
            break
    return np.array(rows).reshape(-1, 5), np.array(labels)


def test_examples_match_host_definition(ctx):
    s = sem.generate(300, 400, 31500, "scale_free", m=2, w_min=0.2)
    X = torch.from_numpy(s.Xt).cuda().T
    res = ctx.skeleton(X, s.alpha, mode=cupc.MODE_PLAIN_FP64)
    C32 = ctx.correlation(X, cupc.F32)
    Xe, te = res.mlp_examples(C32)
    Xr, tr = _host_examples(C32.cpu().numpy(), res.sep_levels(), res.sepsets())
    assert Xe.shape[0] == Xr.shape[0] > 100
    assert np.array_equal(te.cpu().numpy(), tr.astype(np.float32))
    assert np.max(np.abs(Xe.cpu().numpy() - Xr)) <= 1e-5
    lv = np.round(Xr[:, 3] * 8).astype(int)
    assert (lv == 1).any() and (lv >= 2).any()


N_TRAIN = 200        # seeded p = 500 preferential-attachment instances


@pytest.fixture(scope="module")
def trained(ctx):
    probs = [sem.mlp_training_instance(k) for k in range(N_TRAIN)]
    X, t = learned.collect(ctx, probs)
    assert X.shape[0] > 10000 and 0 < float(t.mean()) < 0.5
    losses = learned.train(ctx, X, t, epochs=4, batch=4096, lr=2e-3)
    assert losses[-1] < losses[0]
    return ctx.mlp_get_weights()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_learned_order_skeleton_parity(ctx, trained, seed):
    s = sem.generate(300, 500, 32000 + seed, "scale_free", m=2, w_min=0.2)
    C = oracle.correlation(s.X, nthreads=8)
    ref = oracle.pc_stable(C, s.n, s.alpha, nthreads=8)
    ctx.mlp_set_weights(trained)
    res = ctx.skeleton(s.X, s.alpha, mode=cupc.MODE_FP32_RECHECK, learned_order=True)
    assert np.array_equal(res.adjacency(), ref.adj)
    assert np.array_equal(res.sep_levels(), ref.sep_level)
    got = res.sepsets()
    assert set(got) == set(ref.sepsets)
    for (i, j), (l, S) in got.items():
        ind, rho, z = oracle.ci_gauss(C, s.n, s.alpha, i, j, S)
        assert ind, ((i, j), S, rho, z)


def test_learned_order_recovery_paths(ctx, trained):
    """The learned order through the rebuilt-A'_G paths: a CSR capacity rerun
    (A'_G rebuilt from A_G at a level >= 2, rows scored there) and recheck
    queue reruns; skeleton and removal levels as the oracle's, every SepSet
    separating."""
    s = sem.generate(400, 500, 32100, "scale_free", m=2, w_min=0.2)
    C = oracle.correlation(s.X, nthreads=8)
    ref = oracle.pc_stable(C, s.n, s.alpha, nthreads=8)
    ctx.mlp_set_weights(trained)
    for kw in ({"test_nnz_cap": 64}, {"test_qcap": 1}, {"test_nnz_cap": 16, "test_qcap": 1, "test_rec_cap": 8}):
        res = ctx.skeleton(s.X, s.alpha, mode=cupc.MODE_FP32_RECHECK, learned_order=True, **kw)
        assert sum(res.stats()["reruns"]) >= 1, kw
        assert np.array_equal(res.adjacency(), ref.adj), kw
        assert np.array_equal(res.sep_levels(), ref.sep_level), kw
        for (i, j), (l, S) in res.sepsets().items():
            assert oracle.ci_gauss(C, s.n, s.alpha, i, j, S)[0], (kw, (i, j), S)
        res.free()


def test_learned_order_gain(ctx, trained):
    """What the trained network gains: serial-order CI tests at levels >= 1
    (the tests the serial algorithm performs before each edge's first
    separating set, in the enumeration order used) on held-out instances of
    the training family, against lexicographic order (the method without the
    network) and against the same network untrained. The skeleton never
    changes; the trained order must cost fewer tests than lexicographic order
    and than the untrained network."""
    probs = [sem.generate(500, 500, 39000 + k, "scale_free", m=2, w_min=0.2) for k in range(8)]

    def count(weights):
        per_level, adjs = np.zeros(16, np.int64), []
        for s in probs:
            if weights is None:
                r = ctx.skeleton(s.X, s.alpha, mode=cupc.MODE_FP32_RECHECK)
            else:
                ctx.mlp_set_weights(weights)
                r = ctx.skeleton(s.X, s.alpha, mode=cupc.MODE_FP32_RECHECK, learned_order=True)
            st = r.stats()["serial_tests"]
            per_level[:len(st)] += np.array(st, np.int64)
            adjs.append(r.adjacency())
            r.free()
        return per_level, adjs

    lex, a_lex = count(None)
    untrained, a_un = count(learned.init_weights(5).astype(np.float32))
    tr, a_tr = count(trained)
    for x, y, z in zip(a_lex, a_un, a_tr):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    L, U, T = int(lex[1:].sum()), int(untrained[1:].sum()), int(tr[1:].sum())
    print(f"serial tests at l >= 1: lexicographic {L}, untrained {U}, trained {T} "
          f"(gain vs lexicographic {100.0 * (L - T) / max(L, 1):.2f} %); per level "
          f"lex {lex[1:6].tolist()} trained {tr[1:6].tolist()}")
    assert T < L and T < U


def test_learned_order_full_size_c3(ctx, trained):
    """C3 at full size with the learned order: same skeleton and removal levels
    as the oracle, and every stored SepSet separates (re-verified one by one by
    the oracle's CI test)."""
    s = sem.workload("scalefree2500")
    C = oracle.correlation(s.X, nthreads=16)
    ref = oracle.pc_stable(C, s.n, s.alpha, max_level=s.max_level, nthreads=16)
    ctx.mlp_set_weights(trained)
    res = ctx.skeleton(torch.from_numpy(s.Xt).cuda().T, s.alpha, mode=cupc.MODE_FP32_RECHECK,
                       learned_order=True, max_level=s.max_level)
    assert np.array_equal(res.adjacency(), ref.adj)
    assert np.array_equal(res.sep_levels(), ref.sep_level)
    got = res.sepsets()
    assert set(got) == set(ref.sepsets)
    for (i, j), (l, S) in got.items():                     # every stored set separates
        ind, rho, z = oracle.ci_gauss(C, s.n, s.alpha, i, j, S)
        assert ind, ((i, j), S, rho, z)
