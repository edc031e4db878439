"""Brute-force definition checks of a PC-stable skeleton result (test helper).

Independent of the oracle's arithmetic: the CI test here uses the precision
matrix of the (l+2) block (numpy.linalg.inv), rho = -P12 / sqrt(P11 P22), the
inverse hyperbolic tangent and scipy's normal quantile. The enumeration uses
itertools, whose combinations come out in lexicographic order.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.special import ndtri

NEAR_TIE = 1e-9


def ci_precision(C, n, alpha, a, b, S):
    """(independent, |z| - tau) by the precision-matrix route."""
    idx = [a, b] + list(S)
    P = np.linalg.inv(C[np.ix_(idx, idx)])
    rho = -P[0, 1] / np.sqrt(P[0, 0] * P[1, 1])
    z = abs(np.arctanh(np.clip(rho, -1.0, 1.0)))
    tau = ndtri(1.0 - alpha / 2.0) / np.sqrt(n - len(S) - 3)
    return bool(z <= tau), float(z - tau)


def frozen_graph(sep_level: np.ndarray, level: int) -> np.ndarray:
    """G' at the start of a level: present edges plus those removed at >= level."""
    p = sep_level.shape[0]
    G = (sep_level < 0) | (sep_level >= level)
    G[np.arange(p), np.arange(p)] = False
    return G


def check_result(res, C, n, alpha, max_level=-1, ci=None):
    """Assert that ``res`` is exactly PC-stable's output with canonical SepSets.

    ``ci(a, b, S) -> (independent, margin)``; defaults to the Gaussian test.
    Returns the recomputed serial test counts per level.
    """
    if ci is None:
        ci = lambda a, b, S: ci_precision(C, n, alpha, a, b, S)
    p = res.adj.shape[0]
    counts = []
    for level in range(res.levels_run):
        G = frozen_graph(res.sep_level, level)
        nb = [list(np.nonzero(G[a])[0]) for a in range(p)]
        tests = 0
        for x in range(p):
            for y in nb[x]:
                if y <= x:
                    continue
                removed_here = int(res.sep_level[x, y]) == level
                if level == 0:
                    tests += 1
                    ind, m = ci(x, y, [])
                    if abs(m) > NEAR_TIE:
                        assert ind == removed_here, (x, y, level)
                    continue
                first = None
                for side_a, side_b in ((x, y), (y, x)):
                    cand = [v for v in nb[side_a] if v != side_b]
                    for S in itertools.combinations(cand, level):
                        tests += 1
                        ind, m = ci(side_a, side_b, list(S))
                        if abs(m) <= NEAR_TIE:
                            continue
                        if ind:
                            first = tuple(int(v) for v in S)
                            break
                    if first is not None:
                        break
                assert removed_here == (first is not None), (x, y, level)
                if removed_here:
                    assert res.sepsets[(x, y)] == (level, first), (x, y, level)
        counts.append(tests)
        if level >= 1:
            maxdeg = max(len(v) for v in nb)
            assert maxdeg - 1 >= level
    # the level after the last one run must not be due
    nxt = res.levels_run
    if max_level < 0 or nxt <= max_level:
        G = frozen_graph(res.sep_level, nxt)
        assert G.sum(axis=1).max(initial=0) - 1 < nxt
    return counts
