"""Global sharing of conditioning sets (Sec. 5.5, Fig. 9) on the GPU, against
the oracle's histogram of the same frozen graph.

The device histogram (cupc_result_sshare: a hash table over every (row, S)
pair of A'_G at a level) must equal oracle.sshare_histogram's count for count,
with the same pair, distinct-set, redundant-set and largest-row counts. The
GPU's skeleton and removal levels equal the oracle's (other tests), so both
see the same A'_G. The numbers are printed (pytest -s).
"""
import numpy as np
import pytest

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")

import oracle
from synth import sem

pytestmark = pytest.mark.gpu

BINS = [1, 2, 3, 5, 9, 17, 33, 41, 65, 129]


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = cupc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["medium1000", "scalefree2500", "large10000"])
def test_sshare_matches_oracle(ctx, name):
    s = sem.workload(name)
    C = oracle.correlation(s.X, nthreads=16)
    ref = oracle.pc_stable(C, s.n, s.alpha, max_level=s.max_level, nthreads=16)
    res = ctx.skeleton(torch.from_numpy(s.Xt).cuda().T, s.alpha, max_level=s.max_level)
    assert np.array_equal(res.sep_levels(), ref.sep_level)
    for level in (1, 2, 3):
        if level >= ref.levels_run:
            continue
        got, st = res.sshare(level, BINS)
        want, wst = oracle.sshare_histogram(oracle.frozen_adjacency(ref, level), level, BINS)
        assert got == want, (level, got, want)
        for k in ("pairs", "distinct", "redundant", "max_rows"):
            assert st[k] == wst[k], (level, k, st[k], wst[k])
        print(f"{name} level {level}: pairs {st['pairs']} distinct {st['distinct']} redundant {st['redundant']} "
              f"max rows {st['max_rows']} search {st['search_ms']:.3f} ms histogram {got}")


def test_sshare_arguments(ctx):
    s = sem.workload("small20")
    res = ctx.skeleton(s.X, s.alpha)
    with pytest.raises(cupc.CupcError):
        res.sshare(0, BINS)
    with pytest.raises(cupc.CupcError):
        res.sshare(2, [2, 1])
    counts, st = res.sshare(4, [1])                 # a level with no tests: all zero
    assert counts == [0] and st["pairs"] == 0
