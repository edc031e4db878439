"""Recovery paths of single-problem calls, against the oracle.

A level whose buffer would overflow reports it; the host enlarges the buffer
and runs the affected levels again: level 0's recheck queue (level 0 again),
the A'_G slots and the SepSet record pool (the whole call again), and a level
>= 1 recheck queue (that level and the later ones again; the level stopped
before its removals, so A_G is as at its start and A'_G is rebuilt from it).
The test capacities in the options make each path run; the skeleton,
removal levels, canonical SepSets and serial test counts must still be the
oracle's, and cupc_stats.reruns shows which path ran.
"""
import numpy as np
import pytest

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")

import oracle
from synth import sem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = cupc.Context(0)
    yield c
    c.close()


def _ref(X, n, alpha, max_level=-1):
    C = oracle.correlation(X, nthreads=8)
    return oracle.pc_stable(C, n, alpha, max_level=max_level, nthreads=8)


def _assert_same(res, ref):
    assert np.array_equal(res.adjacency(), ref.adj)
    assert np.array_equal(res.sep_levels(), ref.sep_level)
    assert res.sepsets() == ref.sepsets
    assert res.stats()["serial_tests"][:ref.levels_run] == list(ref.tests)


@pytest.fixture(scope="module")
def medium():
    s = sem.generate(800, 3000, 7101, "random", degree=3.0)
    return s, _ref(s.X, s.n, s.alpha)


def test_level0_queue_overflow(ctx, medium):
    s, ref = medium
    base = ctx.skeleton(s.X, s.alpha)
    q0 = base.stats()["rechecks_queued"][0]
    base.free()
    assert q0 >= 2, q0                      # the level-0 FP32 band holds some pairs here
    res = ctx.skeleton(s.X, s.alpha, test_qcap=q0 // 2)
    assert res.stats()["reruns"][0] >= 1
    _assert_same(res, ref)


def test_level1_queue_overflow(ctx, medium):
    s, ref = medium
    base = ctx.skeleton(s.X, s.alpha)
    q = base.stats()["rechecks_queued"]
    base.free()
    assert q[1] > q[0], q[:2]
    res = ctx.skeleton(s.X, s.alpha, test_qcap=max(q[0], 1))
    st = res.stats()
    assert st["reruns"][3] >= 1 and st["reruns"][0] == 0, st["reruns"]
    _assert_same(res, ref)


def test_csr_capacity_rerun(ctx, medium):
    s, ref = medium
    res = ctx.skeleton(s.X, s.alpha, test_nnz_cap=64)
    assert res.stats()["reruns"][1] >= 1
    _assert_same(res, ref)
    res = ctx.skeleton(s.X, s.alpha, mode=cupc.MODE_PLAIN_FP64, test_nnz_cap=64)
    assert res.stats()["reruns"][1] >= 1
    _assert_same(res, ref)


def test_sepset_pool_rerun(ctx, medium):
    s, ref = medium
    res = ctx.skeleton(s.X, s.alpha, test_rec_cap=16)
    assert res.stats()["reruns"][2] >= 1
    _assert_same(res, ref)


def test_all_capacities_small(ctx, medium):
    s, ref = medium
    res = ctx.skeleton(s.X, s.alpha, test_qcap=1, test_nnz_cap=16, test_rec_cap=8)
    rr = res.stats()["reruns"]
    assert rr[1] >= 1 and rr[2] >= 1 and rr[0] + rr[3] >= 1, rr
    _assert_same(res, ref)


def test_level_queue_overflow_after_quiet_level(ctx):
    """A recheck-queue overflow at level 2 right after a level that removed
    nothing (A'_G reused at level 2). Data: twelve indicators of one latent
    factor, so no edge is ever removed and every level's test count grows;
    with the FP32 band widened to the whole range every test goes to the FP64
    queue, whose length per level is then the level's full enumeration."""
    rng = np.random.default_rng(4242)
    p, n = 12, 2000
    z = rng.standard_normal(n)
    a = rng.uniform(0.6, 0.9, p)
    X = np.outer(z, a) + 0.6 * rng.standard_normal((n, p))
    ref = _ref(X, n, 0.05, max_level=3)
    assert ref.levels_run == 4 and int(ref.adj.sum()) == p * (p - 1)
    base = ctx.skeleton(X, 0.05, max_level=3, recheck_margin=1.0)
    st = base.stats()
    base.free()
    q, removed = st["rechecks_queued"], st["removed"]
    assert removed[1] == 0 and q[2] > max(q[0], q[1]), (q, removed)
    res = ctx.skeleton(X, 0.05, max_level=3, recheck_margin=1.0, test_qcap=max(q[0], q[1]))
    st = res.stats()
    assert st["reruns"][3] >= 1 and st["reruns"][0] == 0, st["reruns"]
    _assert_same(res, ref)
