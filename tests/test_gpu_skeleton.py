"""GPU parity of the CUDA skeleton path against the FP64 CPU oracle.

All calls go through the C ABI (the ctypes binding). Tolerances:
  * correlation: FP64 product within 1e-13 absolute; FP32 (split) product within
    2e-5 absolute (FP32 accumulation over n terms);
  * partial correlations: |d rho| <= 1e-10 * max(|rho|, r_tau) in FP64 and
    <= 1e-5 * max(|rho|, r_tau) in FP32 (the FP32 band is wider than that error);
  * skeletons and canonical SepSets: exactly equal.
"""
import itertools
import math

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


def _oracle_run(X, alpha, max_level=-1):
    C = oracle.correlation(X, nthreads=8)
    return C, oracle.pc_stable(C, X.shape[0], alpha, max_level=max_level, nthreads=8)


def _assert_same(res, ref, canonical=True, C=None, n=None, alpha=None):
    adj = res.adjacency()
    assert np.array_equal(adj, ref.adj), f"skeleton differs in {int((adj != ref.adj).sum()) // 2} pairs"
    lev = res.sep_levels()
    assert np.array_equal(lev, ref.sep_level)
    got = res.sepsets()
    if canonical:
        assert got == ref.sepsets
    else:
        assert set(got) == set(ref.sepsets)
        for (i, j), (l, S) in got.items():
            ind, rho, z = oracle.ci_gauss(C, n, alpha, i, j, S)
            assert ind, ((i, j), S, rho, z)


# --------------------------------------------------------------------------
# correlation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p,n", [(70, 333), (129, 1000), (257, 64)])
def test_correlation_f64_parity(ctx, p, n):
    s = sem.generate(p, n, 11 + p, "random", degree=3.0)
    ref = oracle.correlation(s.X, nthreads=8)
    for X in (s.X, np.ascontiguousarray(s.X), torch.from_numpy(np.ascontiguousarray(s.X)).cuda(),
              torch.from_numpy(s.Xt).cuda().T):
        C = ctx.correlation(X, cupc.F64).cpu().numpy()
        assert np.max(np.abs(C - ref)) < 1e-13
        assert np.array_equal(C, C.T) and np.all(np.diag(C) == 1.0)


def test_correlation_f32_parity(ctx):
    s = sem.generate(300, 2000, 5, "random", degree=3.0)
    ref = oracle.correlation(s.X, nthreads=8)
    C = ctx.correlation(s.X, cupc.F32).cpu().numpy().astype(np.float64)
    err = np.max(np.abs(C - ref))
    assert err < 2e-5, err
    assert np.array_equal(C, C.T)


@pytest.mark.parametrize("p,n", [(130, 200), (1500, 200), (1501, 150), (700, 5000)])
def test_correlation_f32_tile_shapes(ctx, p, n):
    """Short sample counts make every tile one whole-K unit that writes C itself
    (row segments and mirrored columns, vector or scalar stores by p mod 4); the
    long one splits K and goes through the partial-sum reduction. Both must give
    the same bound against the FP64 definition, exact symmetry and a unit
    diagonal, ragged row and column blocks included."""
    s = sem.generate(p, n, 700 + p, "random", degree=3.0)
    ref = oracle.correlation(s.X, nthreads=8)
    C = ctx.correlation(s.X, cupc.F32).cpu().numpy().astype(np.float64)
    err = np.max(np.abs(C - ref))
    assert err < 2e-5, err
    assert np.array_equal(C, C.T)
    assert np.all(np.diag(C) == 1.0)


def test_correlation_float32_input(ctx):
    s = sem.generate(90, 500, 6, "random", degree=3.0, dtype=np.float32)
    ref = oracle.correlation(s.X.astype(np.float64))
    C = ctx.correlation(s.X, cupc.F64).cpu().numpy()
    assert np.max(np.abs(C - ref)) < 1e-13


# --------------------------------------------------------------------------
# partial correlations
# --------------------------------------------------------------------------

@pytest.mark.parametrize("l", [1, 2, 3, 4, 6, 9])
def test_pcor_parity(ctx, l):
    s = sem.generate(40, 800, 100 + l, "random", degree=4.0)
    C = oracle.correlation(s.X)
    rng = np.random.default_rng(l)
    Q = np.array([rng.permutation(s.p)[: l + 2] for _ in range(400)], dtype=np.int32)
    ref = np.array([oracle.pcor(C, int(q[0]), int(q[1]), q[2:].tolist())[0] for q in Q])
    r = math.tanh(oracle.tau(0.01, s.n, l))
    Ct = torch.from_numpy(C).cuda()
    q = torch.from_numpy(Q).cuda()
    got64 = ctx.pcor_batch(Ct, q, l).cpu().numpy()
    scale = np.maximum(np.abs(ref), r)
    err64 = np.abs(got64 - ref) / scale
    assert err64.max() <= 1e-10, err64.max()
    got32 = ctx.pcor_batch(Ct.float(), q, l).cpu().numpy()
    err32 = np.abs(got32 - ref) / scale
    assert np.percentile(err32, 99) <= 1e-5 and err32.max() <= 1e-4, (np.percentile(err32, 99), err32.max())


# --------------------------------------------------------------------------
# whole skeleton
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["plain", "fp32"])
@pytest.mark.parametrize("seed", range(5))
def test_skeleton_small20(ctx, mode, seed):
    s = sem.workload("small20", seed)
    C, ref = _oracle_run(s.X, s.alpha)
    res = ctx.skeleton(s.X, s.alpha, mode=MODES[mode])
    _assert_same(res, ref)
    st = res.stats()
    assert st["levels"] == ref.levels_run
    assert st["serial_tests"] == ref.tests
    assert st["removed"] == ref.removed


@pytest.mark.parametrize("mode", ["plain", "fp32"])
@pytest.mark.parametrize("p,n,fam,deg,alpha", [(150, 2000, "random", 3.0, 0.01), (300, 500, "scale_free", 0, 0.01),
                                               (97, 300, "random", 5.0, 0.05), (40, 120, "random", 6.0, 0.2)])
def test_skeleton_medium(ctx, mode, p, n, fam, deg, alpha):
    s = sem.generate(p, n, 7 * p + n, fam, degree=deg, w_min=0.2)
    C, ref = _oracle_run(s.X, alpha)
    res = ctx.skeleton(s.X, alpha, mode=MODES[mode])
    _assert_same(res, ref)
    assert res.stats()["serial_tests"] == ref.tests


@pytest.mark.parametrize("p,n,deg,alpha", [(150, 2000, 3.0, 0.01), (97, 300, 5.0, 0.05), (40, 120, 6.0, 0.2),
                                          (200, 60, 8.0, 0.3)])
def test_skeleton_float32_data(ctx, p, n, deg, alpha):
    """FP32 data: the rechecks near the threshold form their Gram sums from the
    data in compensated FP32 pairs; the skeleton, SepSets and serial counts must
    still be the FP64 definition's (the oracle runs on the same float32 values)."""
    s = sem.generate(p, n, 11 * p + n, "random", degree=deg, w_min=0.2, dtype=np.float32)
    C, ref = _oracle_run(s.X.astype(np.float64), alpha)
    res = ctx.skeleton(s.X, alpha)
    _assert_same(res, ref)
    assert res.stats()["serial_tests"] == ref.tests


@pytest.mark.parametrize("mode", ["plain", "fp32"])
def test_skeleton_free_sepsets_reverify(ctx, mode):
    s = sem.generate(120, 400, 77, "random", degree=5.0, w_min=0.2)
    C, ref = _oracle_run(s.X, 0.05)
    res = ctx.skeleton(s.X, 0.05, mode=MODES[mode], canonical=False)
    _assert_same(res, ref, canonical=False, C=C, n=s.n, alpha=0.05)


@pytest.mark.parametrize("max_level", [0, 1, 2])
def test_skeleton_max_level(ctx, max_level):
    s = sem.generate(60, 300, 21, "random", degree=5.0, w_min=0.2)
    C, ref = _oracle_run(s.X, 0.05, max_level=max_level)
    for mode in MODES.values():
        res = ctx.skeleton(s.X, 0.05, mode=mode, max_level=max_level)
        _assert_same(res, ref)
        assert res.stats()["levels"] == ref.levels_run


def test_skeleton_input_forms(ctx):
    s = sem.generate(64, 700, 3, "random", degree=3.0)
    C, ref = _oracle_run(s.X, 0.01)
    forms = [s.X, np.ascontiguousarray(s.X), torch.from_numpy(np.ascontiguousarray(s.X)).cuda(),
             torch.from_numpy(s.Xt).cuda().T]
    for X in forms:
        _assert_same(ctx.skeleton(X, 0.01), ref)
    # padded leading dimension
    big = np.zeros((s.n, s.p + 13))
    big[:, : s.p] = s.X
    _assert_same(ctx.skeleton(big[:, : s.p], 0.01), ref)


def test_skeleton_corr_entry(ctx):
    s = sem.generate(80, 900, 4, "random", degree=3.0)
    C, ref = _oracle_run(s.X, 0.01)
    for mode in MODES.values():
        _assert_same(ctx.skeleton_corr(C, s.n, 0.01, mode=mode), ref)
        _assert_same(ctx.skeleton_corr(torch.from_numpy(C).cuda(), s.n, 0.01, mode=mode), ref)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_two_variables(ctx):
    rng = np.random.default_rng(0)
    a = rng.standard_normal(500)
    for b, expect in ((rng.standard_normal(500), 0), (a + 0.5 * rng.standard_normal(500), 1)):
        X = np.column_stack([a, b])
        ref = _oracle_run(X, 0.01)[1]
        assert ref.adj[0, 1] == expect
        for mode in MODES.values():
            _assert_same(ctx.skeleton(X, 0.01, mode=mode), ref)


def test_independent_variables_empty_graph(ctx):
    X = np.random.default_rng(1).standard_normal((2000, 45))
    ref = _oracle_run(X, 1e-4)[1]
    for mode in MODES.values():
        res = ctx.skeleton(X, 1e-4, mode=mode)
        _assert_same(res, ref)


def test_duplicated_column_pinv_path(ctx):
    s = sem.generate(30, 400, 9, "random", degree=4.0, w_min=0.3)
    X = np.column_stack([s.X, s.X[:, 3]])
    C, ref = _oracle_run(X, 0.05)
    for mode in MODES.values():
        _assert_same(ctx.skeleton(X, 0.05, mode=mode), ref)


def test_complete_dependence_dense_levels(ctx):
    # a strongly connected dense DAG drives many levels
    s = sem.generate(24, 3000, 12, "random", degree=10.0, w_min=0.5)
    C, ref = _oracle_run(s.X, 0.01)
    assert ref.levels_run >= 3
    for mode in MODES.values():
        _assert_same(ctx.skeleton(s.X, 0.01, mode=mode), ref)


def test_zero_variance_is_an_error(ctx):
    X = np.random.default_rng(2).standard_normal((100, 5))
    X[:, 2] = 1.5
    with pytest.raises(cupc.CupcError) as e:
        ctx.skeleton(X, 0.01)
    assert e.value.status == -6
    # the context stays usable
    ctx.skeleton(np.random.default_rng(3).standard_normal((100, 5)), 0.01)


def test_invalid_arguments(ctx):
    X = np.random.default_rng(2).standard_normal((100, 5))
    for alpha in (0.0, 1.0, -1.0):
        with pytest.raises(cupc.CupcError):
            ctx.skeleton(X, alpha)
    with pytest.raises(cupc.CupcError):
        ctx.skeleton(X[:, :1], 0.01)


# --------------------------------------------------------------------------
# full-size workload in the benchmark configuration
# --------------------------------------------------------------------------

def test_medium1000_full_size_parity(ctx):
    s = sem.workload("medium1000")
    C, ref = _oracle_run(s.X, s.alpha)
    Xd = torch.from_numpy(s.Xt).cuda().T          # device-resident, variable-major
    for mode in ("fp32", "plain"):
        res = ctx.skeleton(Xd, s.alpha, mode=MODES[mode])
        _assert_same(res, ref)
        assert res.stats()["serial_tests"] == ref.tests


@pytest.mark.parametrize("name", ["medium1000", "scalefree2500", "large10000"])
def test_level1_forms_full_size(ctx, name):
    """Level 1 by conditioning variable (a staged C row per pivot) and by row
    (each {k} shared across the row's j) run the same tests: both give the
    oracle's skeleton, removal levels, canonical SepSets and serial counts, in
    both arithmetic modes (plain mode at p = 10^4 is left out: its FP64 product
    alone takes ~90 ms per call and the FP32 run covers the level-1 forms)."""
    s = sem.workload(name)
    ref = _oracle_full(s)
    Xd = torch.from_numpy(s.Xt).cuda().T
    modes = ("fp32",) if name == "large10000" else ("fp32", "plain")
    for mode in modes:
        for form in (cupc.L1_BY_PIVOT, cupc.L1_BY_ROW):
            res = ctx.skeleton(Xd, s.alpha, mode=MODES[mode], max_level=s.max_level, level1_form=form)
            _assert_same(res, ref)
            assert res.stats()["serial_tests"] == ref.tests, (mode, form)
            res.free()


def _oracle_full(s, nthreads=16):
    C = oracle.correlation(s.X, nthreads=nthreads)
    return oracle.pc_stable(C, s.n, s.alpha, max_level=s.max_level, nthreads=nthreads)


def test_scalefree2500_full_size_parity(ctx):
    """C3 (p = 2500, n = 500, scale-free hubs), both forms, against the oracle."""
    s = sem.workload("scalefree2500")
    ref = _oracle_full(s)
    Xd = torch.from_numpy(s.Xt).cuda().T
    for mode in ("fp32", "plain"):
        res = ctx.skeleton(Xd, s.alpha, mode=MODES[mode], max_level=s.max_level)
        _assert_same(res, ref)
        assert res.stats()["serial_tests"] == ref.tests


def test_large10000_full_size_parity(ctx):
    """C5 (p = 10^4, n = 1000, levels up to 6) in both forms: the benchmarked
    FP32 + recheck form and the plain FP64 form."""
    s = sem.workload("large10000")
    ref = _oracle_full(s)
    Xd = torch.from_numpy(s.Xt).cuda().T
    for mode in ("fp32", "plain"):
        res = ctx.skeleton(Xd, s.alpha, mode=MODES[mode], max_level=s.max_level)
        assert np.array_equal(res.adjacency(), ref.adj), mode
        assert np.array_equal(res.sep_levels(), ref.sep_level), mode
        assert res.sepsets() == ref.sepsets, mode
        assert res.stats()["serial_tests"][:ref.levels_run] == list(ref.tests), mode
        res.free()


def test_device_peaks(ctx):
    pk = ctx.device_peaks()
    # GB300: FP32 FMA throughput is tens of times the FP64 rate; both positive
    assert pk["fp64_tflops"] > 0.1 and pk["fp32_tflops"] > 10 * pk["fp64_tflops"]


def test_edge_list_matches_adjacency(ctx):
    """cupc_result_edges: the pairs (i, j), i < j, of the skeleton in increasing order."""
    for seed in range(3):
        s = sem.workload("small20", seed)
        res = ctx.skeleton(s.X, s.alpha)
        adj = res.adjacency()
        want = np.argwhere(np.triu(adj, 1)).astype(np.int32)
        assert np.array_equal(res.edges(), want)
        assert np.array_equal(res.edges(), want)          # cached on the second call
    s = sem.generate(300, 500, 2100, "scale_free", w_min=0.2)
    res = ctx.skeleton(s.X, s.alpha)
    assert np.array_equal(res.edges(), np.argwhere(np.triu(res.adjacency(), 1)).astype(np.int32))
    probs = [sem.generate(p, 600, 40 + p, "random", degree=3.0) for p in (33, 70)]
    for r in ctx.skeleton_batch([q.X for q in probs], [q.alpha for q in probs])[0]:
        assert np.array_equal(r.edges(), np.argwhere(np.triu(r.adjacency(), 1)).astype(np.int32))


def test_host_input_chunked_upload(ctx):
    """A variable-major host input of 8 MB or more is uploaded in variable chunks,
    each standardised on arrival: the result equals the device-input call's
    (FP32 data in the FP32 form; FP64 data in both forms, against the oracle)."""
    s = sem.workload("medium1000")                         # 40 MB of float32
    Xh = s.Xt.T                                            # variable-major host view
    assert Xh.nbytes >= 8 << 20 and Xh.strides[0] == Xh.itemsize
    rh = ctx.skeleton(Xh, s.alpha, max_level=s.max_level)
    rd = ctx.skeleton(torch.from_numpy(s.Xt).cuda().T, s.alpha, max_level=s.max_level)
    assert np.array_equal(rh.adjacency(), rd.adjacency())
    assert np.array_equal(rh.records_raw(), rd.records_raw())
    assert rh.stats()["serial_tests"] == rd.stats()["serial_tests"]
    assert rh.stats()["kernel_count"]["standardize"] == 4
    s2 = sem.generate(300, 5000, 31, "random", degree=3.0)  # 12 MB of float64
    _, ref = _oracle_run(s2.X, s2.alpha)
    for mode in ("fp32", "plain"):
        res = ctx.skeleton(np.ascontiguousarray(s2.Xt).T, s2.alpha, mode=MODES[mode])
        _assert_same(res, ref)


def _records_sorted(seps):
    out = []
    for (i, j) in sorted(seps):
        l, S = seps[(i, j)]
        out += [i, j, l, *S]
    return np.array(out, dtype=np.int32)


def test_records_in_pair_order(ctx):
    """cupc_result_sepset_records: the records (i, j, l, S) of the removals at
    levels >= 1 in increasing (i, j), int for int the oracle's in that order;
    single lookups by cupc_result_sepset (either order of the pair) agree."""
    cases = [sem.workload("small20", seed) for seed in range(3)]
    cases.append(sem.generate(300, 500, 2100, "scale_free", w_min=0.2))
    cases.append(sem.generate(150, 2000, 7, "random", degree=3.0))
    for s in cases:
        _, ref = _oracle_run(s.X, s.alpha)
        want = _records_sorted(ref.sepsets)
        edges = np.argwhere(np.triu(ref.adj, 1)).astype(np.int32)
        for mode in ("fp32", "plain"):
            for host_lists in (False, True):        # built on request, or with the call
                res = ctx.skeleton(s.X, s.alpha, mode=MODES[mode], host_lists=host_lists)
                assert np.array_equal(res.records_raw(), want), (mode, host_lists)
                assert np.array_equal(res.records_raw(), want), (mode, host_lists)     # cached
                assert np.array_equal(res.edges(), edges), (mode, host_lists)
                for (i, j), (l, S) in list(ref.sepsets.items())[:40]:
                    assert res.sepset(j, i) == tuple(S)
                assert np.array_equal(res.sep_levels(), ref.sep_level)
                res.free()


@pytest.mark.parametrize("d", [0.1, 0.3])
def test_sweep_generator_parity(ctx, d):
    """The scalability workload's generator (dense lower-triangular DAG, signed
    weights, unit variance) at a small size, levels 0-2, both forms, against the
    oracle."""
    s = sem.paper_density_signed(250, 3000, d, 6100 + int(100 * d), max_level=2)
    C = oracle.correlation(s.X, nthreads=8)
    ref = oracle.pc_stable(C, s.n, s.alpha, max_level=2, nthreads=8)
    for mode in ("fp32", "plain"):
        res = ctx.skeleton(s.X, s.alpha, mode=MODES[mode], max_level=2)
        _assert_same(res, ref)
        assert res.stats()["serial_tests"][:ref.levels_run] == list(ref.tests)
