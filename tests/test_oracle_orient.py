"""Pins of the oracle's orientation step (second step of PC-stable, Sec. 2.4).

Sec. 2.2 defines the target: two DAGs are Markov equivalent when they share
the skeleton and the v-structures, and the CPDAG has a -> b exactly when every
DAG of the class has that edge in that direction, a - b otherwise. The main pin
computes that definition by brute force -- every orientation of a small DAG's
skeleton, kept when acyclic with the same v-structures -- and compares it with
the oracle's orientation of PC-stable driven by d-separation in the DAG (a
perfect CI oracle). It shares nothing with the oracle's rules. The other pins
are textbook graphs for each rule, a conflict between two v-structures, and
relabelling invariance.
"""
import itertools

import numpy as np

import oracle

NONE, ARROW, TAIL = 0, 1, 2


def _vstructs(D):
    p = D.shape[0]
    out = set()
    for k in range(p):
        par = [i for i in range(p) if D[i, k]]
        for i, j in itertools.combinations(par, 2):
            if not D[i, j] and not D[j, i]:
                out.add((min(i, j), k, max(i, j)))
    return out


def _acyclic(D):
    p = D.shape[0]
    indeg = D.sum(axis=0).astype(int)
    stack = [v for v in range(p) if indeg[v] == 0]
    seen = 0
    while stack:
        v = stack.pop()
        seen += 1
        for w in range(p):
            if D[v, w]:
                indeg[w] -= 1
                if indeg[w] == 0:
                    stack.append(w)
    return seen == p


def cpdag_brute_force(D):
    """CPDAG marks of DAG D by the definition of Sec. 2.2 (enumeration)."""
    p = D.shape[0]
    edges = [(i, j) for i in range(p) for j in range(p) if D[i, j]]
    target = _vstructs(D)
    members = []
    for bits in range(1 << len(edges)):
        E = np.zeros_like(D)
        for q, (i, j) in enumerate(edges):
            if bits >> q & 1:
                E[j, i] = 1
            else:
                E[i, j] = 1
        if _acyclic(E) and _vstructs(E) == target:
            members.append(E)
    mark = np.zeros((p, p), dtype=np.uint8)
    for (i, j) in edges:
        fwd = all(E[i, j] for E in members)
        bwd = all(E[j, i] for E in members)
        if fwd:
            mark[i, j], mark[j, i] = ARROW, TAIL
        elif bwd:
            mark[j, i], mark[i, j] = ARROW, TAIL
        else:
            mark[i, j] = mark[j, i] = TAIL
    return mark


def _orient_dag(D):
    res = oracle.pc_stable_dsep(D)
    return oracle.orient(res)


def test_orient_equals_cpdag_definition_on_random_dags():
    rng = np.random.default_rng(20240)
    checked = directed = undirected = 0
    for t in range(160):
        p = int(rng.integers(3, 8))
        prob = float(rng.uniform(0.25, 0.7))
        order = rng.permutation(p)
        D = np.zeros((p, p), dtype=np.uint8)
        for a in range(p):
            for b in range(a + 1, p):
                if rng.random() < prob:
                    D[order[a], order[b]] = 1
        if D.sum() > 11:
            continue
        mark, rounds = _orient_dag(D)
        expect = cpdag_brute_force(D)
        assert np.array_equal(mark, expect), (t, D.tolist(), mark.tolist(), expect.tolist())
        assert rounds >= 1
        checked += 1
        directed += int(((mark == ARROW) & (mark.T == TAIL)).sum())
        undirected += int(((mark == TAIL) & (mark.T == TAIL)).sum()) // 2
    assert checked >= 100 and directed > 50 and undirected > 50


def test_collider_and_chain():
    D = np.zeros((3, 3), dtype=np.uint8)
    D[0, 2] = D[1, 2] = 1                       # 0 -> 2 <- 1
    mark, _ = _orient_dag(D)
    assert mark[0, 2] == ARROW and mark[2, 0] == TAIL and mark[1, 2] == ARROW and mark[2, 1] == TAIL
    assert mark[0, 1] == NONE
    D = np.zeros((3, 3), dtype=np.uint8)
    D[0, 1] = D[1, 2] = 1                       # chain: no v-structure, nothing oriented
    mark, _ = _orient_dag(D)
    assert mark[0, 1] == mark[1, 0] == mark[1, 2] == mark[2, 1] == TAIL


def test_rule_r1():
    # 0 -> 2 <- 1 and 2 - 3 with 0, 3 not adjacent: R1 orients 2 -> 3
    # (0 _||_ 3 | {2} is a level-1 removal whose SepSet contains 2: no v-structure there)
    D = np.zeros((4, 4), dtype=np.uint8)
    D[0, 2] = D[1, 2] = D[2, 3] = 1
    res = oracle.pc_stable_dsep(D)
    assert res.sepset(0, 3) == (1, (2,))
    mark, rounds = oracle.orient(res)
    assert mark[2, 3] == ARROW and mark[3, 2] == TAIL and rounds == 2


def test_rule_r2():
    # d -> c <- a (v-structure), c -> b by R1, then a -> c -> b with a - b: R2 gives a -> b
    a, b, c, d = 0, 1, 2, 3
    D = np.zeros((4, 4), dtype=np.uint8)
    D[a, b] = D[a, c] = D[c, b] = D[d, c] = 1
    mark, _ = _orient_dag(D)
    assert mark[a, b] == ARROW and mark[b, a] == TAIL
    assert mark[c, b] == ARROW and mark[a, c] == ARROW
    assert np.array_equal(mark, cpdag_brute_force(D))


def test_rule_r3():
    # a - c1 -> b <- c2 - a, c1 and c2 not adjacent, a - b: R3 gives a -> b
    a, b, c1, c2 = 0, 1, 2, 3
    D = np.zeros((4, 4), dtype=np.uint8)
    D[a, c1] = D[a, c2] = D[c1, b] = D[c2, b] = D[a, b] = 1
    mark, _ = _orient_dag(D)
    assert mark[a, b] == ARROW and mark[b, a] == TAIL
    assert mark[a, c1] == TAIL and mark[c1, a] == TAIL and mark[a, c2] == TAIL
    assert np.array_equal(mark, cpdag_brute_force(D))


def test_conflicting_v_structures_leave_both_arrowheads():
    # path 0 - 1 - 2 - 3 with 0 _||_ 2, 1 _||_ 3, 0 _||_ 3 (all with S empty):
    # the triples give 0 -> 1 <- 2 and 1 -> 2 <- 3, which disagree on 1 - 2
    res = oracle.pc_stable_table(4, [(0, 2, ()), (1, 3, ()), (0, 3, ())])
    assert res.adj[0, 1] and res.adj[1, 2] and res.adj[2, 3] and not res.adj[0, 2]
    mark, _ = oracle.orient(res)
    assert mark[1, 2] == ARROW and mark[2, 1] == ARROW
    assert mark[0, 1] == ARROW and mark[1, 0] == TAIL and mark[3, 2] == ARROW and mark[2, 3] == TAIL


def test_orientation_is_invariant_under_relabelling():
    rng = np.random.default_rng(77)
    for _ in range(10):
        p = 9
        D = np.triu((rng.random((p, p)) < 0.35).astype(np.uint8), 1)
        perm = rng.permutation(p)
        Dp = np.zeros_like(D)
        Dp[np.ix_(perm, perm)] = D
        m1, _ = _orient_dag(D)
        m2, _ = _orient_dag(Dp)
        assert np.array_equal(m2[np.ix_(perm, perm)], m1)
