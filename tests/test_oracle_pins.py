"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: printed worked
examples, closed forms, library routines that compute the same quantity by a
different route, brute force on tiny inputs, and invariants.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.special import ndtri

import oracle
from synth import sem
from tests.pc_check import check_result, ci_precision

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Sec. 4.2 / Algorithm 6: combinations
# --------------------------------------------------------------------------

def _golden_comb():
    rows = []
    for line in open(os.path.join(GOLDEN, "comb_examples.txt")):
        line = line.split("#")[0].strip()
        if line:
            rows.append(line)
    return rows


def test_comb_paper_examples():
    rows = _golden_comb()
    assert len(rows) == 7
    for line in rows:
        lhs, rhs = line.split(":")
        expected = [int(v) for v in rhs.split()]
        row_entries = None
        if lhs.startswith("set"):
            head, lhs = lhs.split("|")
            row_entries = [int(v) for v in head.split()[1:]]
        kind, *args = lhs.split()
        args = [int(v) for v in args]
        if kind == "comb":
            got = oracle.comb(*args)
        elif kind == "row":
            got = oracle.comb_row(*args)
        elif kind == "skip":
            got = oracle.comb_skip(*args)
        else:
            raise AssertionError(kind)
        if row_entries is not None:
            got = [row_entries[k] for k in got]
        assert got == expected, line


@pytest.mark.parametrize("n", range(0, 13))
def test_comb_matches_itertools(n):
    for l in range(0, min(n, 6) + 1):
        combos = list(itertools.combinations(range(1, n + 1), l))
        assert oracle.binom(n, l) == len(combos)
        for t, c in enumerate(combos):
            assert oracle.comb(n, l, t) == list(c)
            assert oracle.comb_row(n, l, t) == [v - 1 for v in c]
        with pytest.raises(ValueError):
            oracle.comb(n, l, len(combos))


@pytest.mark.parametrize("nrow", range(1, 11))
def test_comb_skip_matches_filtered_lex_order(nrow):
    for pos in range(nrow):
        others = [k for k in range(nrow) if k != pos]
        for l in range(0, min(nrow - 1, 5) + 1):
            combos = list(itertools.combinations(others, l))
            for t, c in enumerate(combos):
                assert oracle.comb_skip(nrow, l, t, pos) == list(c)


def test_binom_exact_and_saturating():
    for n in range(0, 70):
        for k in range(0, n + 1):
            expect = math.comb(n, k)
            got = oracle.binom(n, k)
            assert got == (expect if expect < 2**64 - 1 else 2**64 - 1)
    assert oracle.binom(10000, 5) == math.comb(10000, 5)
    assert oracle.binom(10000, 6) == 2**64 - 1  # 1.4e21 exceeds 64 bits
    assert oracle.binom(3, 5) == 0


# --------------------------------------------------------------------------
# Eq. (threshold)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q", [1e-12, 1e-6, 0.005, 0.025, 0.1, 0.3, 0.5, 0.7, 0.975, 0.995, 1 - 1e-9])
def test_norm_quantile_vs_scipy(q):
    got = oracle.norm_quantile(q)
    ref = ndtri(q)
    assert abs(got - ref) <= 2e-15 * max(1.0, abs(ref))


@pytest.mark.parametrize("alpha,n,l", [(0.01, 1000, 0), (0.01, 1000, 3), (0.05, 200, 1),
                                       (0.01, 10000, 6), (1e-4, 50, 2)])
def test_tau_formula(alpha, n, l):
    ref = ndtri(1.0 - alpha / 2.0) / math.sqrt(n - l - 3)
    assert oracle.tau(alpha, n, l) == pytest.approx(ref, rel=1e-14)
    assert math.isnan(oracle.tau(0.01, 5, 2))  # m - |S| - 3 = 0 is undefined


# --------------------------------------------------------------------------
# Correlation matrix
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order,dtype", [("C", np.float64), ("F", np.float64), ("C", np.float32)])
def test_correlation_vs_numpy(order, dtype):
    rng = np.random.default_rng(7)
    n, p = 1500, 37
    A = rng.standard_normal((n, p)) @ rng.standard_normal((p, p)) + 3.0
    X = np.asarray(A, dtype=dtype, order=order)
    C = oracle.correlation(X)
    R = np.corrcoef(X.astype(np.float64).T)
    assert np.max(np.abs(C - R)) < 1e-13
    assert np.all(np.diag(C) == 1.0)
    assert np.array_equal(C, C.T)


# --------------------------------------------------------------------------
# Sec. 4.3: partial correlation
# --------------------------------------------------------------------------

def _random_corr(rng, p, n=400):
    X = rng.standard_normal((n, p)) @ rng.standard_normal((p, p))
    return np.corrcoef(X.T)


def test_pcor_level0_is_the_correlation():
    C = _random_corr(np.random.default_rng(1), 6)
    for i, j in itertools.combinations(range(6), 2):
        rho, deg, _ = oracle.pcor(C, i, j, [])
        assert not deg
        assert rho == pytest.approx(C[i, j], abs=1e-15)


def test_pcor_level1_textbook_formula():
    C = _random_corr(np.random.default_rng(2), 7)
    for i, j, k in itertools.permutations(range(7), 3):
        rho, deg, _ = oracle.pcor(C, i, j, [k])
        ref = (C[i, j] - C[i, k] * C[j, k]) / math.sqrt((1 - C[i, k] ** 2) * (1 - C[j, k] ** 2))
        assert abs(rho - ref) < 1e-13


@pytest.mark.parametrize("l", [1, 2, 3, 4, 6])
def test_pcor_matches_precision_matrix(l):
    rng = np.random.default_rng(10 + l)
    p = l + 5
    C = _random_corr(rng, p)
    for trial in range(30):
        idx = rng.permutation(p)[: l + 2]
        i, j, S = int(idx[0]), int(idx[1]), [int(v) for v in idx[2:]]
        rho, deg, used = oracle.pcor(C, i, j, S)
        P = np.linalg.inv(C[np.ix_(idx, idx)])
        ref = -P[0, 1] / math.sqrt(P[0, 0] * P[1, 1])
        assert not deg and not used
        assert abs(rho - ref) < 1e-12
        # the ordering of S does not matter
        rho2, _, _ = oracle.pcor(C, i, j, S[::-1])
        assert abs(rho - rho2) < 1e-13
        # symmetric in i and j
        rho3, _, _ = oracle.pcor(C, j, i, S)
        assert abs(rho - rho3) < 1e-13


def test_pcor_rank_deficient_uses_pinv_and_projection():
    # duplicate a conditioning variable: the projection onto span(S) is unchanged,
    # so the pseudo-inverse path must give the same rho as the reduced set.
    rng = np.random.default_rng(3)
    n = 500
    Z = rng.standard_normal((n, 5))
    X = np.column_stack([Z[:, 0] + Z[:, 2], Z[:, 1] - Z[:, 2] + 0.5 * Z[:, 3], Z[:, 2], Z[:, 3], Z[:, 2]])
    C = np.corrcoef(X.T)
    C[2, 4] = C[4, 2] = 1.0  # columns 2 and 4 are identical
    rho_dup, deg, used = oracle.pcor(C, 0, 1, [2, 3, 4])
    rho_red, _, used_red = oracle.pcor(C, 0, 1, [2, 3])
    assert used and not used_red and not deg
    assert abs(rho_dup - rho_red) < 1e-9


def test_pcor_degenerate_conditional_variance():
    # C[0,2] = 1: V0 is a function of V2, so Var(V0 | V2) = 0 exactly.
    C = np.array([[1.0, 0.3, 1.0], [0.3, 1.0, 0.3], [1.0, 0.3, 1.0]])
    rho, deg, _ = oracle.pcor(C, 0, 1, [2])
    assert deg and math.isnan(rho)


@pytest.mark.parametrize("h, degenerate", [(5e-11, True), (9e-11, True), (1e-9, False), (5e-9, False)])
def test_pcor_near_zero_conditional_variance(h, degenerate):
    # Var(V0 | V2) = 1 - C02^2 = h > 0. A conditional variance at or below 1e-10 is
    # the rounding level of C's unit diagonal, where V0 is treated as a linear
    # function of S (zero variance, independent); above it the test is an
    # ordinary one and rho follows the level-1 textbook formula.
    # Unit-variance V2 = Z2, V0 = c Z2 + sqrt(h) Z0, V1 = 0.3 Z2 + 0.4 Z0 + sqrt(0.75) Z1
    # with independent standard Z: C02 = c = sqrt(1 - h), C12 = 0.3, C01 = 0.3 c + 0.4 sqrt(h),
    # and rho(V0, V1 | V2) = 0.4 / sqrt(0.91) whatever h is.
    c02 = math.sqrt(1.0 - h)
    c01 = 0.3 * c02 + 0.4 * math.sqrt(h)
    C = np.array([[1.0, c01, c02], [c01, 1.0, 0.3], [c02, 0.3, 1.0]])
    rho, deg, _ = oracle.pcor(C, 0, 1, [2])
    assert deg == degenerate
    if degenerate:
        assert math.isnan(rho)
    else:
        ref = (c01 - c02 * 0.3) / math.sqrt((1.0 - c02 * c02) * (1.0 - 0.09))
        assert abs(ref - 0.4 / math.sqrt(0.91)) < 1e-5
        assert abs(abs(rho) - ref) <= 1e-6 * ref, (rho, ref)


# --------------------------------------------------------------------------
# Sec. 4.4 / Algorithm 7
# --------------------------------------------------------------------------

@pytest.mark.parametrize("l", [1, 2, 3, 5, 8])
def test_pinv_alg7_full_rank_equals_inverse(l):
    rng = np.random.default_rng(20 + l)
    A = rng.standard_normal((l, l))
    M = A @ A.T + l * np.eye(l)
    Mp, r = oracle.pinv_alg7(M)
    assert r == l
    assert np.max(np.abs(Mp - np.linalg.inv(M))) < 1e-11
    Mi = oracle.inverse_spd(M)
    assert np.max(np.abs(Mi - np.linalg.inv(M))) < 1e-12
    # a non-symmetric nonsingular matrix as well
    B = rng.standard_normal((l, l)) + 2 * np.eye(l)
    Bp, rb = oracle.pinv_alg7(B)
    assert rb == l
    assert np.max(np.abs(Bp - np.linalg.inv(B))) < 1e-8


@pytest.mark.parametrize("l,rank", [(2, 1), (3, 2), (5, 3), (6, 1), (8, 5)])
def test_pinv_alg7_rank_deficient_vs_numpy(l, rank):
    rng = np.random.default_rng(100 + 10 * l + rank)
    A = rng.standard_normal((l, rank))
    M = A @ A.T
    Mp, r = oracle.pinv_alg7(M)
    assert r == rank
    ref = np.linalg.pinv(M)
    assert np.max(np.abs(Mp - ref)) < 1e-8 * max(1.0, np.max(np.abs(ref)))
    assert oracle.inverse_spd(M) is None
    # Moore-Penrose conditions
    assert np.allclose(M @ Mp @ M, M, atol=1e-9)
    assert np.allclose(Mp @ M @ Mp, Mp, atol=1e-9)


def test_pinv_alg7_zero_matrix():
    Mp, r = oracle.pinv_alg7(np.zeros((3, 3)))
    assert r == 0 and np.all(Mp == 0)


# --------------------------------------------------------------------------
# Eq. (FisherZTransform) and the decision rule
# --------------------------------------------------------------------------

def test_level0_decisions_follow_pearson_closed_form():
    s = sem.workload("small20")
    C = oracle.correlation(s.X)
    res = oracle.pc_stable(C, s.n, s.alpha, max_level=0)
    crit = ndtri(1 - s.alpha / 2)
    for i, j in itertools.combinations(range(s.p), 2):
        z = abs(np.arctanh(C[i, j])) * math.sqrt(s.n - 3)
        if abs(z - crit) > 1e-9:
            assert (res.sep_level[i, j] == 0) == (z <= crit)
    assert res.tests == [s.p * (s.p - 1) // 2]


def test_fisher_decision_edges():
    C = np.array([[1.0, 1.0], [1.0, 1.0]])
    ind, rho, z = oracle.ci_gauss(C, 100, 0.01, 0, 1, [])
    assert not ind and math.isinf(z)          # |rho| = 1 is dependent
    t = oracle.tau(0.01, 100, 0)
    for r, expect in ((math.tanh(t) * (1 - 1e-9), True), (math.tanh(t) * (1 + 1e-9), False)):
        C = np.array([[1.0, r], [r, 1.0]])
        assert oracle.ci_gauss(C, 100, 0.01, 0, 1, [])[0] == expect


# --------------------------------------------------------------------------
# Algorithm 1: test counts, brute force, invariants
# --------------------------------------------------------------------------

def _golden_fig2():
    stmts, levels, p = [], {}, None
    for line in open(os.path.join(GOLDEN, "fig2_counts.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("p "):
            p = int(line.split()[1])
        elif line.startswith("ind"):
            lhs, rhs = line.split(":")
            _, i, j = lhs.split()
            stmts.append((int(i), int(j), [int(v) for v in rhs.split()]))
        elif line.startswith("level"):
            _, l, _, t, _, r = line.split()
            levels[int(l)] = (int(t), int(r))
    return p, stmts, levels


def test_fig2_test_counts():
    p, stmts, levels = _golden_fig2()
    res = oracle.pc_stable_table(p, stmts)
    for l, (t, r) in levels.items():
        assert res.tests[l] == t
        assert res.removed[l] == r
    assert res.sepset(1, 2) == (0, ())
    assert res.sepset(1, 3) == (1, (0,))
    assert res.sepset(3, 2) == (1, (0,))
    expect = np.zeros((4, 4), np.uint8)
    for a, b in ((0, 1), (0, 2), (0, 3)):
        expect[a, b] = expect[b, a] = 1
    assert np.array_equal(res.adj, expect)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_definition_tiny_gaussian(seed):
    p = 7 + seed % 2
    s = sem.generate(p, 150 + 50 * seed, 900 + seed, "random", degree=3.0, w_min=0.3)
    C = oracle.correlation(s.X)
    res = oracle.pc_stable(C, s.n, 0.05)
    assert res.status == 0
    counts = check_result(res, C, s.n, 0.05)
    assert counts == res.tests
    assert sum(res.removed[1:]) > 0 or seed > 3  # most seeds exercise level >= 1


def test_bruteforce_with_max_level():
    s = sem.generate(8, 300, 77, "random", degree=4.0, w_min=0.3)
    C = oracle.correlation(s.X)
    res = oracle.pc_stable(C, s.n, 0.05, max_level=1)
    assert res.levels_run <= 2
    check_result(res, C, s.n, 0.05, max_level=1)


@pytest.mark.parametrize("family,p,seed,degree", [("random", 20, 1, 3.0), ("random", 30, 2, 3.0),
                                                  ("random", 40, 3, 2.0), ("random", 60, 7, 2.0),
                                                  ("scale_free", 20, 4, 0), ("scale_free", 16, 8, 0)])
def test_dsep_oracle_recovers_true_skeleton(family, p, seed, degree):
    # Spirtes et al.: under a perfect CI oracle PC returns the true skeleton.
    s = sem.generate(p, 10, seed, family, degree=degree)
    D = s.dag_matrix()
    res = oracle.pc_stable_dsep(D, nthreads=4)
    assert np.array_equal(res.adj, s.skeleton())
    # every stored SepSet d-separates its pair
    for (i, j), (l, S) in res.sepsets.items():
        assert oracle.dsep(D, i, j, S)


def test_dsep_bruteforce_small():
    s = sem.generate(8, 10, 11, "random", degree=3.0)
    D = s.dag_matrix()
    res = oracle.pc_stable_dsep(D)
    ci = lambda a, b, S: (oracle.dsep(D, a, b, S), 1.0)
    counts = check_result(res, None, None, None, ci=ci)
    assert counts == res.tests


def test_order_independence_under_relabelling():
    s = sem.workload("small20")
    C = oracle.correlation(s.X)
    base = oracle.pc_stable(C, s.n, s.alpha)
    rng = np.random.default_rng(5)
    for _ in range(3):
        perm = rng.permutation(s.p)
        res = oracle.pc_stable(C[np.ix_(perm, perm)], s.n, s.alpha)
        assert np.array_equal(res.adj, base.adj[np.ix_(perm, perm)])
        assert np.array_equal(res.sep_level, base.sep_level[np.ix_(perm, perm)])


def test_threads_give_identical_results():
    s = sem.generate(60, 400, 31, "random", degree=4.0)
    C = oracle.correlation(s.X)
    a = oracle.pc_stable(C, s.n, 0.05, nthreads=1)
    b = oracle.pc_stable(C, s.n, 0.05, nthreads=4)
    assert np.array_equal(a.adj, b.adj)
    assert np.array_equal(a.sep_level, b.sep_level)
    assert a.sepsets == b.sepsets
    assert a.tests == b.tests


def test_precision_route_agrees_on_small_workload():
    s = sem.workload("small20")
    C = oracle.correlation(s.X)
    res = oracle.pc_stable(C, s.n, s.alpha)
    check_result(res, C, s.n, s.alpha)
    assert res.min_margin > 1e-9


def test_paper_density_workload_is_ill_posed_in_fp64():
    """The paper's scalability generator (Sec. 5.6: positive weights, Bernoulli(d)
    lower triangle) grows the data geometrically along the topological order, so
    correlations reach 1 - 1e-11 and the skeleton is decided by rounding: the
    oracle's own skeleton changes under a 1e-15 perturbation of C. Exact parity
    is therefore not defined on it (the configs' workloads are well conditioned)."""
    s = sem.paper_density(300, 10000, 0.1, 17310)
    C = oracle.correlation(s.X, nthreads=8)
    ref = oracle.pc_stable(C, s.n, s.alpha, nthreads=8)
    assert np.abs(C - np.eye(s.p)).max() > 1 - 1e-9
    rng = np.random.default_rng(1)
    E = rng.standard_normal(C.shape) * 1e-15
    E = (E + E.T) / 2
    np.fill_diagonal(E, 0)
    r2 = oracle.pc_stable(C + E, s.n, s.alpha, nthreads=8)
    assert int((r2.adj != ref.adj).sum()) > 0


# --------------------------------------------------------------------------
# Sec. 5.5 / Fig. 9: global sharing of conditioning sets
# --------------------------------------------------------------------------

def test_sshare_histogram_hand_built_graph():
    """Rows 0: {1, 2, 3}, 1: {0, 2, 3}, 2: {0, 1}, 3: {0, 1}, 4: {5}, 5: {4}.
    At level 2 only rows 0 and 1 run tests (degree >= 3): row 0 uses {1,2}, {1,3},
    {2,3}; row 1 uses {0,2}, {0,3}, {2,3}. So {2,3} appears in two rows and the
    other four sets in one; at level 1 rows 0-3 run tests (degree >= 2) with S = {v}
    for every neighbour v: {0} and {1} in three rows, {2} and {3} in two."""
    adj = np.zeros((6, 6), bool)
    for a, b in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (4, 5)]:
        adj[a, b] = adj[b, a] = True
    counts, st = oracle.sshare_histogram(adj, 2, [1, 2, 3])
    assert counts == [4, 1, 0]
    assert st == {"pairs": 6, "distinct": 5, "redundant": 1, "max_rows": 2}
    counts, st = oracle.sshare_histogram(adj, 1, [1, 2, 3, 4])
    assert counts == [0, 2, 2, 0]
    assert st == {"pairs": 10, "distinct": 4, "redundant": 4, "max_rows": 3}
    counts, st = oracle.sshare_histogram(adj, 3, [1])
    assert counts == [0] and st["pairs"] == 0


def test_paper_density_signed_generator():
    """Sec. 5.6's structure: edges only from lower to higher index (V_j -> V_i,
    j < i), density d, weights of magnitude in [0.1, 1] with both signs, and every
    variable at unit sample variance."""
    from synth import sem
    s = sem.paper_density_signed(120, 500, 0.2, 7)
    assert np.all(s.src < s.dst)
    assert abs(len(s.src) / (120 * 119 / 2) - 0.2) < 0.03
    assert np.all((np.abs(s.weight) >= 0.1) & (np.abs(s.weight) <= 1.0))
    assert (s.weight > 0).any() and (s.weight < 0).any()
    assert np.allclose(s.Xt.std(axis=1), 1.0, atol=1e-12)
