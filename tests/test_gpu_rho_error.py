"""Partial-correlation error against the FP64 oracle, per workload and level.

For each workload the oracle runs PC-stable; at every level it ran, tests of
that level are drawn from its frozen graph G' (a slot (i, j) of a row with
enough neighbours and an l-subset S of adj(i) without j), and rho(i, j | S)
is evaluated by the oracle (Sec. 4.3, Cholesky / Algorithm 7) and on the GPU
three ways:
  * FP32 bulk: the tensor-core correlation and the CI kernels' FP32 factor;
  * FP64 recheck: the recheck arithmetic from the data (moments, Gram sums of
    the centred data, FP64 elimination);
  * plain FP64: the FP64 correlation and the CI kernels' FP64 factor.
The error of a result is |rho_gpu - rho_oracle| / max(|rho_oracle|, r_tau(l))
(the scale of the decision |rho| <= r_tau). Bounds, per workload over all its
sampled tests: FP32 bulk p99 <= 1e-5 and max <= 1e-4 (the FP32 band sends any
test whose FP32 value could be this far off near the threshold to the FP64
recheck), FP64 paths <= 1e-10 for every sampled test. The max and p99 are
printed per workload and level (pytest -s).
"""
import math

import numpy as np
import pytest

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")

import oracle
from synth import sem

pytestmark = pytest.mark.gpu

PER_LEVEL = 1500


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = cupc.Context(0)
    yield c
    c.close()


def _frozen(sep, l):
    G = (sep < 0) | (sep >= l)
    np.fill_diagonal(G, False)
    return G


def _sample(ref, l, rng, k):
    """Up to k tests (i, j, S) of level l of the oracle's run."""
    G = _frozen(ref.sep_level, l)
    nb = [np.nonzero(G[a])[0] for a in range(G.shape[0])]
    slots = [(a, b) for a in range(G.shape[0]) if len(nb[a]) - 1 >= l for b in nb[a]]
    if not slots:
        return np.zeros((0, 2 + l), np.int32)
    pick = rng.choice(len(slots), size=min(k, len(slots)), replace=len(slots) < k)
    rows = []
    for t in pick:
        a, b = slots[t]
        cand = nb[a][nb[a] != b]
        S = np.sort(rng.choice(cand, size=l, replace=False)) if l else np.zeros(0, np.int64)
        rows.append([a, b] + S.tolist())
    return np.unique(np.array(rows, dtype=np.int32), axis=0)


def _errors(ctx, name, X, n, alpha, max_level=-1):
    Xh = np.asarray(X)
    C = oracle.correlation(Xh.astype(np.float64), nthreads=16)
    ref = oracle.pc_stable(C, n, alpha, max_level=max_level, nthreads=16)
    Xd = torch.from_numpy(np.ascontiguousarray(Xh.T)).cuda().T      # device, variable-major
    C32 = ctx.correlation(Xd, cupc.F32)
    C64 = ctx.correlation(Xd, cupc.F64)
    rng = np.random.default_rng(12345)
    out = []
    for l in range(ref.levels_run):
        Q = _sample(ref, l, rng, PER_LEVEL)
        if Q.shape[0] == 0:
            continue
        rho = np.array([oracle.pcor(C, int(q[0]), int(q[1]), q[2:].tolist())[0] for q in Q])
        ok = np.isfinite(rho)
        r = math.tanh(oracle.tau(alpha, n, l))
        scale = np.maximum(np.abs(rho), r)
        q = torch.from_numpy(Q).cuda()
        e32 = np.abs(ctx.pcor_batch(C32, q, l).cpu().numpy() - rho) / scale
        erc = np.abs(ctx.pcor_data(Xd, q, l).cpu().numpy() - rho) / scale
        e64 = np.abs(ctx.pcor_batch(C64, q, l).cpu().numpy() - rho) / scale
        e32, erc, e64 = e32[ok], erc[ok], e64[ok]
        out.append((l, e32, erc, e64))
        print(f"{name} l={l} tests={int(ok.sum())} fp32 max={e32.max():.2e} p99={np.percentile(e32, 99):.2e} "
              f"recheck max={erc.max():.2e} p99={np.percentile(erc, 99):.2e} plain max={e64.max():.2e}")
    e32 = np.concatenate([r[1] for r in out])
    erc = np.concatenate([r[2] for r in out])
    e64 = np.concatenate([r[3] for r in out])
    print(f"{name} all levels: tests={e32.size} fp32 max={e32.max():.2e} p99={np.percentile(e32, 99):.2e} "
          f"recheck max={erc.max():.2e} plain max={e64.max():.2e}")
    return e32, erc, e64


def _check(errs):
    e32, erc, e64 = errs
    assert e32.size > 0
    assert np.percentile(e32, 99) <= 1e-5 and e32.max() <= 1e-4, (np.percentile(e32, 99), e32.max())
    assert erc.max() <= 1e-10, erc.max()
    assert e64.max() <= 1e-10, e64.max()


@pytest.mark.parametrize("name", ["small20", "medium1000", "scalefree2500", "large10000"])
def test_rho_error_workload(ctx, name):
    s = sem.workload(name)
    _check(_errors(ctx, name, s.X, s.n, s.alpha, s.max_level))


def test_rho_error_batch_problems(ctx):
    """Four problems of the 64-problem workload: the largest p, the largest and
    the smallest n, and the first."""
    probs = sem.batch_workload(64, 0)
    pick = {int(np.argmax([s.p for s in probs])), int(np.argmax([s.n for s in probs])),
            int(np.argmin([s.n for s in probs])), 0}
    parts = [_errors(ctx, f"batch64[{k}]", probs[k].X.astype(np.float32), probs[k].n, probs[k].alpha)
             for k in sorted(pick)]
    _check(tuple(np.concatenate([p[q] for p in parts]) for q in range(3)))
