"""CPU FP64 oracle for the PC-stable skeleton (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
import this package. The product library never loads it, and it shares no code
with the CUDA path: it is a ctypes wrapper around ``pc_oracle.c`` (plain C,
compiled with gcc) plus the NumPy MLP reference in ``mlp.py``.

Functions mirror the paper's definitions (Zarebavani et al., TPDS 2019):
``comb`` (Sec. 4.2, Eq. comb / Algorithm 6), ``pcor`` (Sec. 4.3, Eqs.
PartialCorMat and RhoCal), ``tau`` (Eq. threshold), ``pinv_alg7`` (Sec. 4.4,
Algorithm 7), ``pc_stable`` (Algorithm 1 with the readings in the C file's
header) and ``orient`` (the second step of PC-stable, Sec. 2.4: v-structures
and Meek's rules, giving the CPDAG of Sec. 2.2).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None


def lib_path() -> str:
    return os.path.join(_BUILD, f"liborc_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile pc_oracle.c with gcc (-O2, no FMA contraction, OpenMP)."""
    out = lib_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    L = ctypes.CDLL(build())
    i64, u64, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    vp = ctypes.c_void_p
    L.orc_binom.restype = u64
    L.orc_binom.argtypes = [i64, i64]
    for name in ("orc_comb", "orc_comb_row"):
        getattr(L, name).restype = i32
        getattr(L, name).argtypes = [i32, i32, u64, vp]
    L.orc_comb_skip.restype = i32
    L.orc_comb_skip.argtypes = [i32, i32, u64, i32, vp]
    L.orc_correlation.restype = i32
    L.orc_correlation.argtypes = [vp, i64, i64, i64, i64, vp, i32]
    L.orc_norm_quantile.restype = dbl
    L.orc_norm_quantile.argtypes = [dbl]
    L.orc_tau.restype = dbl
    L.orc_tau.argtypes = [dbl, i64, i32]
    L.orc_inverse_spd.restype = i32
    L.orc_inverse_spd.argtypes = [vp, i32, vp]
    L.orc_pinv_alg7.restype = i32
    L.orc_pinv_alg7.argtypes = [vp, i32, vp]
    L.orc_pcor.restype = i32
    L.orc_pcor.argtypes = [vp, i64, i32, i32, vp, i32, vp, vp]
    L.orc_fisher_decide.restype = i32
    L.orc_fisher_decide.argtypes = [dbl, i32, dbl, vp]
    L.orc_dsep.restype = i32
    L.orc_dsep.argtypes = [vp, i32, i32, i32, vp, i32]
    L.orc_ci_gauss.restype = i32
    L.orc_ci_gauss.argtypes = [vp, i64, i64, dbl, i32, i32, vp, i32, vp, vp]
    for name in ("orc_pc_gauss", "orc_pc_dsep", "orc_pc_table"):
        getattr(L, name).restype = vp
    L.orc_pc_gauss.argtypes = [vp, i32, i64, dbl, i32, i32]
    L.orc_pc_dsep.argtypes = [vp, i32, i32, i32]
    L.orc_pc_table.argtypes = [i32, vp, i32, i32, i32]
    L.orc_run_free.argtypes = [vp]
    L.orc_run_free.restype = None
    for name, rt in (("orc_run_p", i32), ("orc_run_levels", i32), ("orc_run_status", i32),
                     ("orc_run_min_margin", dbl), ("orc_run_degenerate", i64),
                     ("orc_run_pinv_used", i64), ("orc_run_rec_len", i64), ("orc_run_n_rec", i64)):
        getattr(L, name).restype = rt
        getattr(L, name).argtypes = [vp]
    L.orc_orient.restype = i64
    L.orc_orient.argtypes = [i32, vp, vp, vp, vp, vp, i64, vp]
    L.orc_run_copy.restype = None
    L.orc_run_copy.argtypes = [vp, vp, vp, vp, vp, vp]
    _LIB = L
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Scalar / small-matrix functions
# --------------------------------------------------------------------------

def binom(n: int, k: int) -> int:
    return int(_lib().orc_binom(n, k))


def comb(n: int, l: int, t: int) -> list[int]:
    """Algorithm 6: the t-th l-combination of {1..n} in lex order (1-based)."""
    O = np.zeros(max(l, 1), dtype=np.int32)
    if _lib().orc_comb(n, l, t, _ptr(O)) != 0:
        raise ValueError("rank out of range")
    return O[:l].tolist()


def comb_row(nrow: int, l: int, t: int) -> list[int]:
    """Sec. 4.2 cuPC-S form: 0-based positions within a row of nrow entries."""
    P = np.zeros(max(l, 1), dtype=np.int32)
    if _lib().orc_comb_row(nrow, l, t, _ptr(P)) != 0:
        raise ValueError("rank out of range")
    return P[:l].tolist()


def comb_skip(nrow: int, l: int, t: int, pos: int) -> list[int]:
    """Sec. 4.2 cuPC-E form: 0-based positions skipping position ``pos``."""
    P = np.zeros(max(l, 1), dtype=np.int32)
    if _lib().orc_comb_skip(nrow, l, t, pos, _ptr(P)) != 0:
        raise ValueError("rank out of range")
    return P[:l].tolist()


def norm_quantile(q: float) -> float:
    return float(_lib().orc_norm_quantile(q))


def tau(alpha: float, n_samples: int, l: int) -> float:
    """Eq. (threshold)."""
    return float(_lib().orc_tau(alpha, n_samples, l))


def inverse_spd(M: np.ndarray):
    M = np.ascontiguousarray(M, dtype=np.float64)
    l = M.shape[0]
    out = np.zeros((l, l))
    rc = _lib().orc_inverse_spd(_ptr(M), l, _ptr(out))
    return (out if rc == 0 else None)


def pinv_alg7(M: np.ndarray):
    """Algorithm 7; returns (pseudo-inverse, numerical rank)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    l = M.shape[0]
    out = np.zeros((l, l))
    r = _lib().orc_pinv_alg7(_ptr(M), l, _ptr(out))
    return out, int(r)


def correlation(X: np.ndarray, nthreads: int = 1) -> np.ndarray:
    """Correlation matrix of X (n x p, any memory order), FP64, unit diagonal."""
    X = np.asarray(X)
    if X.dtype != np.float64:
        X = X.astype(np.float64)
    n, p = X.shape
    s_stride, v_stride = (X.strides[0] // 8, X.strides[1] // 8)
    if X.strides[0] % 8 or X.strides[1] % 8:
        X = np.ascontiguousarray(X)
        s_stride, v_stride = p, 1
    C = np.empty((p, p), dtype=np.float64)
    rc = _lib().orc_correlation(_ptr(X), n, p, s_stride, v_stride, _ptr(C), nthreads)
    if rc != 0:
        raise RuntimeError(f"orc_correlation failed ({rc})")
    return C


def pcor(C: np.ndarray, i: int, j: int, S) -> tuple[float, bool, bool]:
    """Sec. 4.3: (rho, degenerate, used_pinv) for V_i, V_j given S."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    Sa = np.ascontiguousarray(np.asarray(list(S), dtype=np.int32).reshape(-1))
    rho = ctypes.c_double()
    used = ctypes.c_int()
    deg = _lib().orc_pcor(_ptr(C), C.shape[0], i, j,
                          _ptr(Sa) if Sa.size else None, int(Sa.size),
                          ctypes.byref(rho), ctypes.byref(used))
    return rho.value, bool(deg), bool(used.value)


def ci_gauss(C: np.ndarray, n_samples: int, alpha: float, i: int, j: int, S):
    """One Gaussian CI test: (independent, rho, z)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    Sa = np.ascontiguousarray(np.asarray(list(S), dtype=np.int32).reshape(-1))
    rho = ctypes.c_double()
    z = ctypes.c_double()
    ind = _lib().orc_ci_gauss(_ptr(C), C.shape[0], n_samples, alpha, i, j,
                              _ptr(Sa) if Sa.size else None, int(Sa.size),
                              ctypes.byref(rho), ctypes.byref(z))
    return bool(ind), rho.value, z.value


def dsep(dag: np.ndarray, i: int, j: int, S) -> bool:
    D = np.ascontiguousarray(dag, dtype=np.uint8)
    Sa = np.ascontiguousarray(np.asarray(list(S), dtype=np.int32).reshape(-1))
    return bool(_lib().orc_dsep(_ptr(D), D.shape[0], i, j, _ptr(Sa) if Sa.size else None, int(Sa.size)))


# --------------------------------------------------------------------------
# Skeleton driver
# --------------------------------------------------------------------------

@dataclass
class OracleResult:
    adj: np.ndarray           # p x p uint8
    sep_level: np.ndarray     # p x p int16, -1 where the edge is present
    sepsets: dict             # (i, j) with i < j -> (level, tuple(S)) for removals at level >= 1
    tests: list               # serial-order tests per level
    removed: list             # removals per level
    levels_run: int
    min_margin: float         # min |Z - tau| over all Gaussian tests
    degenerate: int
    pinv_used: int
    status: int

    def sepset(self, i: int, j: int):
        """(level, S) for a removed pair, None if the edge is present."""
        a, b = min(i, j), max(i, j)
        lv = int(self.sep_level[a, b])
        if lv < 0:
            return None
        if lv == 0:
            return (0, ())
        return self.sepsets[(a, b)]

    @property
    def total_tests(self) -> int:
        return int(sum(self.tests))


def _collect(handle) -> OracleResult:
    L = _lib()
    try:
        p = L.orc_run_p(handle)
        adj = np.empty((p, p), dtype=np.uint8)
        sep = np.empty((p, p), dtype=np.int16)
        rl = L.orc_run_rec_len(handle)
        rec = np.empty(max(rl, 1), dtype=np.int32)
        tests = np.zeros(256, dtype=np.int64)
        removed = np.zeros(256, dtype=np.int64)
        L.orc_run_copy(handle, _ptr(adj), _ptr(sep), _ptr(rec), _ptr(tests), _ptr(removed))
        levels = L.orc_run_levels(handle)
        sepsets = {}
        k = 0
        while k < rl:
            i, j, l = int(rec[k]), int(rec[k + 1]), int(rec[k + 2])
            sepsets[(i, j)] = (l, tuple(int(v) for v in rec[k + 3:k + 3 + l]))
            k += 3 + l
        return OracleResult(adj=adj, sep_level=sep, sepsets=sepsets,
                            tests=tests[:levels].tolist(), removed=removed[:levels].tolist(),
                            levels_run=levels, min_margin=L.orc_run_min_margin(handle),
                            degenerate=int(L.orc_run_degenerate(handle)),
                            pinv_used=int(L.orc_run_pinv_used(handle)),
                            status=int(L.orc_run_status(handle)))
    finally:
        L.orc_run_free(handle)


def pc_stable(C: np.ndarray, n_samples: int, alpha: float, max_level: int = -1,
              nthreads: int = 1) -> OracleResult:
    """Algorithm 1 with Gaussian CI tests on the correlation matrix C."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    h = _lib().orc_pc_gauss(_ptr(C), C.shape[0], n_samples, alpha, max_level, nthreads)
    return _collect(h)


def pc_stable_data(X: np.ndarray, alpha: float, max_level: int = -1, nthreads: int = 1) -> OracleResult:
    """Correlation of X (n x p) followed by Algorithm 1."""
    C = correlation(X, nthreads=nthreads)
    return pc_stable(C, X.shape[0], alpha, max_level, nthreads)


def pc_stable_dsep(dag: np.ndarray, max_level: int = -1, nthreads: int = 1) -> OracleResult:
    """Algorithm 1 driven by d-separation in the DAG (a perfect CI oracle)."""
    D = np.ascontiguousarray(dag, dtype=np.uint8)
    h = _lib().orc_pc_dsep(_ptr(D), D.shape[0], max_level, nthreads)
    return _collect(h)


def pc_stable_table(p: int, statements, max_level: int = -1) -> OracleResult:
    """Algorithm 1 driven by a fixed list of independence statements (i, j, S)."""
    width = 3 + max([len(S) for (_, _, S) in statements] + [0])
    T = np.full((max(len(statements), 1), width), -1, dtype=np.int32)
    for r, (i, j, S) in enumerate(statements):
        T[r, 0], T[r, 1], T[r, 2] = i, j, len(S)
        T[r, 3:3 + len(S)] = sorted(S)
    h = _lib().orc_pc_table(p, _ptr(T), len(statements), width, max_level)
    return _collect(h)


# --------------------------------------------------------------------------
# Second step of PC-stable: orientation
# --------------------------------------------------------------------------

MARK_NONE, MARK_ARROW, MARK_TAIL = 0, 1, 2


def orient(res: OracleResult):
    """Sec. 2.4, second step: v-structures from the SepSets of ``res``, then
    Meek's rules R1-R3 in rounds (readings in pc_oracle.c). Returns
    (mark, rounds): mark[a, b] = 0 no edge, 1 arrowhead at b, 2 tail at b."""
    p = res.adj.shape[0]
    items = sorted(res.sepsets.items())
    keys = np.array([i * p + j for (i, j), _ in items] or [0], dtype=np.int64)
    off = np.zeros(max(len(items), 1), dtype=np.int64)
    mem = []
    for r, (_, (l, S)) in enumerate(items):
        off[r] = len(mem)
        mem.extend(S)
    members = np.array(mem or [0], dtype=np.int32)
    adj = np.ascontiguousarray(res.adj, dtype=np.uint8)
    sep = np.ascontiguousarray(res.sep_level, dtype=np.int16)
    mark = np.zeros((p, p), dtype=np.uint8)
    rounds = _lib().orc_orient(p, _ptr(adj), _ptr(sep), _ptr(keys), _ptr(off), _ptr(members), len(items),
                               _ptr(mark))
    if rounds < 0:
        raise ValueError("a removed pair has no SepSet record")
    return mark, int(rounds)


def frozen_adjacency(res: OracleResult, level: int) -> np.ndarray:
    """A'_G at the start of `level` (>= 1): the final skeleton plus the pairs
    removed at that level or later (Algorithm 1 freezes adj at level start)."""
    G = (res.sep_level < 0) | (res.sep_level >= level)
    np.fill_diagonal(G, False)
    return G


def sshare_histogram(adj: np.ndarray, level: int, bins):
    """Global sharing of conditioning sets at one level (Sec. 5.5, Fig. 9): every
    l-subset S of adj(i) in a row i that runs tests at this level (|adj(i)| >= l + 1)
    is counted once per such row. Returns (counts per bin [bins[k], bins[k+1]),
    the last bin open-ended; stats) with stats = pairs (row, S), distinct S,
    redundant S (in two rows or more), the largest number of rows of one S.
    Plain Python over itertools.combinations (lexicographic subsets)."""
    import itertools
    from collections import Counter
    rows = Counter()
    p = adj.shape[0]
    pairs = 0
    for i in range(p):
        nb = np.nonzero(adj[i])[0].tolist()
        if len(nb) < level + 1:
            continue
        for S in itertools.combinations(nb, level):
            rows[S] += 1
            pairs += 1
    counts = [0] * len(bins)
    for c in rows.values():
        ks = [q for q in range(len(bins)) if bins[q] <= c]
        if ks:                                  # (fewer rows than bins[0]: in no bin)
            counts[ks[-1]] += 1
    stats = {"pairs": pairs, "distinct": len(rows), "redundant": sum(1 for c in rows.values() if c >= 2),
             "max_rows": max(rows.values(), default=0)}
    return counts, stats
