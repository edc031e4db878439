"""Batched skeletons (many independent problems in one pass, CUDA graph) against
the FP64 CPU oracle, problem by problem, and against single-problem calls.

PC-stable on a batch must give every problem exactly its own result: the same
skeleton, removal levels and canonical SepSets as the oracle, and the same
serial-order test counts per level. Launch configurations (chunk, CTAs per SM,
product K-steps) and graph replay versus direct launches must not change any
of it.
"""
import numpy as np
import pytest

import oracle
from synth import sem

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    cupc.build_library()
    c = cupc.Context(0)
    yield c
    c.close()


def _oracle(s):
    C = oracle.correlation(s.X, nthreads=8)
    return oracle.pc_stable(C, s.n, s.alpha, max_level=s.max_level, nthreads=8)


def _assert_problem(res, ref, bstats_ok=True):
    assert np.array_equal(res.adjacency(), ref.adj)
    assert np.array_equal(res.sep_levels(), ref.sep_level)
    assert res.sepsets() == ref.sepsets
    st = res.stats()
    L = ref.levels_run
    assert st["serial_tests"][:L] == list(ref.tests)[:L]
    assert all(t == 0 for t in st["serial_tests"][L:])
    assert st["removed"][:L] == list(ref.removed)[:L]


def _trim(v):
    v = list(v)
    while v and v[-1] == 0:
        v.pop()
    return v


def _mixed_batch(seed, count=7):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        p = int(rng.integers(20, 160))
        n = int(rng.integers(200, 1500))
        d = float(rng.uniform(2.0, 6.0))
        out.append(sem.generate(p, n, 91000 + 100 * seed + k, "random", degree=d, w_min=0.1,
                                dtype=np.float64, alpha=0.05))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_batch_matches_oracle(ctx, seed):
    probs = _mixed_batch(seed)
    res, bst = ctx.skeleton_batch([s.X for s in probs], [s.alpha for s in probs])
    assert bst["cuda_graph"] in (0, 1)
    for s, r in zip(probs, res):
        _assert_problem(r, _oracle(s))
    # batch totals are the sums of the problems' counts
    tot = sum(sum(r.stats()["serial_tests"]) for r in res)
    assert tot == sum(bst["serial_tests"])


def test_graph_replay_new_data(ctx):
    # same shapes, new data: the second call replays the recorded graph
    a = _mixed_batch(3, 5)
    b = [sem.generate(s.p, s.n, s.seed + 500, "random", degree=3.0, w_min=0.1, dtype=np.float64, alpha=0.05)
         for s in a]
    ctx.skeleton_batch([s.X for s in a], [s.alpha for s in a])
    res, bst = ctx.skeleton_batch([s.X for s in b], [s.alpha for s in b])
    assert bst["cuda_graph"] == 1
    for s, r in zip(b, res):
        _assert_problem(r, _oracle(s))


def test_direct_launch_equals_graph(ctx):
    probs = _mixed_batch(4, 6)
    Xs, al = [s.X for s in probs], [s.alpha for s in probs]
    g, _ = ctx.skeleton_batch(Xs, al)
    d, bst = ctx.skeleton_batch(Xs, al, batch_direct=True)
    assert bst["cuda_graph"] == 0
    for x, y in zip(g, d):
        assert np.array_equal(x.adjacency(), y.adjacency())
        assert x.sepsets() == y.sepsets()


def test_batch_equals_single_calls_and_layouts(ctx):
    probs = _mixed_batch(5, 6)
    res, _ = ctx.skeleton_batch([np.ascontiguousarray(s.X, dtype=np.float32) for s in probs],
                                [s.alpha for s in probs])
    res_vm, _ = ctx.skeleton_batch([s.Xt.astype(np.float32).T for s in probs], [s.alpha for s in probs])
    for s, r, rv in zip(probs, res, res_vm):
        one = ctx.skeleton(np.ascontiguousarray(s.X, dtype=np.float32), s.alpha)
        assert np.array_equal(r.adjacency(), one.adjacency())
        assert np.array_equal(rv.adjacency(), one.adjacency())
        assert r.sepsets() == one.sepsets() == rv.sepsets()
        # records in (i, j) order, int for int, and the per-level removal counts
        assert np.array_equal(r.records_raw(), one.records_raw())
        assert np.array_equal(rv.records_raw(), one.records_raw())
        assert _trim(r.stats()["removed"]) == _trim(one.stats()["removed"])
        for (i, j), (l, S) in list(one.sepsets().items())[:25]:
            assert r.sepset(j, i) == S


def test_device_inputs(ctx):
    probs = _mixed_batch(6, 4)
    Xd = [torch.from_numpy(np.ascontiguousarray(s.X)).cuda() for s in probs]
    res, bst = ctx.skeleton_batch(Xd, [s.alpha for s in probs])
    assert bst["h2d_bytes"] == 0
    for s, r in zip(probs, res):
        _assert_problem(r, _oracle(s))


def test_edge_cases(ctx):
    rng = np.random.default_rng(7)
    tiny = sem.generate(2, 50, 92001, "random", degree=1.0, dtype=np.float64, alpha=0.05)
    few = sem.generate(33, 5, 92002, "random", degree=2.0, dtype=np.float64, alpha=0.05)  # n = 5: level <= 1
    odd = sem.generate(97, 700, 92003, "random", degree=4.0, dtype=np.float64, alpha=0.05)
    capped = sem.generate(64, 900, 92004, "random", degree=5.0, dtype=np.float64, alpha=0.05)
    probs = [tiny, few, odd, capped]
    res, _ = ctx.skeleton_batch([s.X for s in probs], [s.alpha for s in probs])
    for s, r in zip(probs, res):
        _assert_problem(r, _oracle(s))
    # max_level applies to every problem
    res, _ = ctx.skeleton_batch([s.X for s in probs], [s.alpha for s in probs], max_level=1)
    for s, r in zip(probs, res):
        C = oracle.correlation(s.X, nthreads=8)
        ref = oracle.pc_stable(C, s.n, s.alpha, max_level=1, nthreads=8)
        _assert_problem(r, ref)
    # a zero-variance variable in one problem fails the call
    bad = np.array(odd.X, copy=True)
    bad[:, 5] = 3.0
    with pytest.raises(cupc.CupcError) as ei:
        ctx.skeleton_batch([tiny.X, bad], [0.05, 0.05])
    assert "CUPC_E_NUMERIC" in str(ei.value)
    _ = rng


def test_invalid_arguments(ctx):
    s = _mixed_batch(8, 2)
    with pytest.raises(cupc.CupcError):
        ctx.skeleton_batch([x.X for x in s], [0.05, 1.5])
    with pytest.raises(cupc.CupcError):
        ctx.skeleton_batch([x.X for x in s], [0.05, 0.05], mode=cupc.MODE_PLAIN_FP64)


def test_autotuner_consistent(ctx):
    probs = _mixed_batch(9, 6)
    table = ctx.autotune_batch([s.X for s in probs], [s.alpha for s in probs], reps=1)
    assert len(table) == 30
    assert all(table[q]["ms"] <= table[q + 1]["ms"] for q in range(len(table) - 1))
    best = table[0]
    res, _ = ctx.skeleton_batch([s.X for s in probs], [s.alpha for s in probs], chunk=best["chunk"],
                                ctas_per_sm=best["ctas_per_sm"], corr_kps=best["corr_kps"])
    for s, r in zip(probs, res):
        _assert_problem(r, _oracle(s))


def test_full_batch_workload(ctx):
    """The 64-problem workload (p ~ U[50, 800], n ~ U[200, 5000], degree ~ U[2, 6],
    alpha 0.05) as the benchmark runs it: every problem against the oracle and
    against its single-problem run."""
    probs = sem.batch_workload(64, 0)
    Xs = [np.ascontiguousarray(s.X, dtype=np.float32) for s in probs]
    res, bst = ctx.skeleton_batch(Xs, [s.alpha for s in probs])
    assert bst["cuda_graph"] == 1 or bst["cuda_graph"] == 0
    for X, s, r in zip(Xs, probs, res):
        one = ctx.skeleton(X, s.alpha)
        assert np.array_equal(r.adjacency(), one.adjacency())
        assert r.sepsets() == one.sepsets()
        assert _trim(r.stats()["serial_tests"]) == _trim(one.stats()["serial_tests"])
    refs = []
    for k, s in enumerate(probs):
        C = oracle.correlation(Xs[k].astype(np.float64), nthreads=16)
        refs.append(oracle.pc_stable(C, s.n, s.alpha, nthreads=16))
        _assert_problem(res[k], refs[k])
    # both level-1 forms, explicitly, give the same results
    for form in (cupc.L1_BY_PIVOT, cupc.L1_BY_ROW):
        res_f, _ = ctx.skeleton_batch(Xs, [s.alpha for s in probs], level1_form=form)
        for k in range(len(probs)):
            _assert_problem(res_f[k], refs[k])
