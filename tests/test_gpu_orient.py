"""GPU parity of the orientation step (second step of PC-stable, Sec. 2.4).

The device orientation of a skeleton result (cupc_result_orient, through the
C ABI) must give exactly the oracle's edge marks, computed by the oracle from
its own skeleton and SepSets of the same data (which the skeleton tests show
equal to the GPU's), and the same number of rule rounds.
"""
import numpy as np
import pytest

import oracle
from synth import sem

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MODES = {"plain": cupc.MODE_PLAIN_FP64, "fp32": cupc.MODE_FP32_RECHECK}


@pytest.fixture(scope="module")
def ctx(cuda_device):
    cupc.build_library()
    c = cupc.Context(0)
    yield c
    c.close()


def _oracle(X, alpha, max_level=-1, nthreads=8):
    C = oracle.correlation(X, nthreads=nthreads)
    return oracle.pc_stable(C, X.shape[0], alpha, max_level=max_level, nthreads=nthreads)


def _counts(mark):
    up = np.triu(np.ones_like(mark, dtype=bool), 1)
    a, b = mark, mark.T
    edge = (a > 0) & up
    heads = (a == 1).astype(int) + (b == 1).astype(int)
    return (int((edge & (heads == 1)).sum()), int((edge & (heads == 0)).sum()), int((edge & (heads == 2)).sum()))


def _check(res, ref):
    want, rounds = oracle.orient(ref)
    got, st = res.orient()
    assert np.array_equal(got, want), f"{int((got != want).sum())} marks differ"
    assert st["rounds"] == rounds
    assert (st["directed"], st["undirected"], st["bidirected"]) == _counts(want)
    return st


@pytest.mark.parametrize("mode", ["plain", "fp32"])
@pytest.mark.parametrize("seed", range(5))
def test_orient_small20(ctx, mode, seed):
    s = sem.workload("small20", seed)
    ref = _oracle(s.X, s.alpha)
    _check(ctx.skeleton(s.X, s.alpha, mode=MODES[mode]), ref)


@pytest.mark.parametrize("p,n,fam,deg,alpha", [(150, 2000, "random", 3.0, 0.01), (300, 500, "scale_free", 0, 0.01),
                                               (97, 300, "random", 5.0, 0.05), (40, 120, "random", 6.0, 0.2),
                                               (24, 3000, "random", 10.0, 0.01)])
def test_orient_medium(ctx, p, n, fam, deg, alpha):
    s = sem.generate(p, n, 7 * p + n, fam, degree=deg, w_min=0.2)
    ref = _oracle(s.X, alpha)
    for mode in MODES.values():
        _check(ctx.skeleton(s.X, alpha, mode=mode), ref)


def test_orient_edge_cases(ctx):
    rng = np.random.default_rng(5)
    # no edges at all
    X = rng.standard_normal((2000, 45))
    st = _check(ctx.skeleton(X, 1e-4), _oracle(X, 1e-4))
    assert st["directed"] == 0
    # two variables, dependent: one undirected edge
    a = rng.standard_normal(500)
    X = np.column_stack([a, a + 0.5 * rng.standard_normal(500)])
    st = _check(ctx.skeleton(X, 0.01), _oracle(X, 0.01))
    assert st["undirected"] == 1
    # a complete graph (every pair dependent given everything): nothing to orient
    Z = rng.standard_normal((4000, 1))
    X = Z + 0.3 * rng.standard_normal((4000, 6))
    st = _check(ctx.skeleton(X, 0.01), _oracle(X, 0.01))
    assert st["undirected"] == 15 and st["directed"] == 0


def test_orient_batch_results(ctx):
    probs = [sem.generate(p, n, 31 * p + n, "random", degree=d, w_min=0.2)
             for p, n, d in ((60, 800, 3.0), (130, 400, 4.0), (33, 2000, 2.0), (90, 300, 5.0))]
    res, _ = ctx.skeleton_batch([s.X for s in probs], [s.alpha for s in probs])
    for r, s in zip(res, probs):
        _check(r, _oracle(s.X, s.alpha))


def _full(name):
    s = sem.workload(name)
    ref = _oracle(s.X, s.alpha, s.max_level, nthreads=16)
    Xd = torch.from_numpy(s.Xt).cuda().T
    return s, ref, Xd


def test_orient_medium1000_full_size(ctx):
    s, ref, Xd = _full("medium1000")
    st = _check(ctx.skeleton(Xd, s.alpha, mode=MODES["fp32"], max_level=s.max_level), ref)
    assert st["directed"] > 0 and st["rounds"] >= 2


def test_orient_scalefree2500_full_size(ctx):
    s, ref, Xd = _full("scalefree2500")
    _check(ctx.skeleton(Xd, s.alpha, mode=MODES["fp32"], max_level=s.max_level), ref)


def test_orient_large10000_full_size(ctx):
    s, ref, Xd = _full("large10000")
    st = _check(ctx.skeleton(Xd, s.alpha, mode=MODES["fp32"], max_level=s.max_level), ref)
    assert st["directed"] > 0
