"""Seeded synthetic linear-Gaussian SEM data for the PC-stable skeleton workloads.

This module is the one input source shared by the tests, the benchmark and the
oracle checks. It holds none of the skeleton method's arithmetic: it only draws
a DAG, its edge weights and samples from the structural equations.

Model (Sec. 5.6 describes the paper's own generator; the workloads here use the
signed-weight variant):

    x_v = sum_{u -> v} w_uv * x_u + e_v,   e_v ~ N(0, 1),

evaluated in a topological order. Weights have magnitude U[w_min, 1] and a
random sign. Two DAG families are provided:

* ``random``: a random topological order; every ordered pair (earlier, later)
  receives an edge independently with probability ``degree / (p - 1)``, so the
  expected total degree of a node is ``degree``.
* ``scale_free``: preferential attachment. Nodes arrive one at a time and each
  new node draws ``m`` distinct earlier nodes with probability proportional to
  (current degree + 1). Edges point from the new node to the earlier node, so
  the early nodes become collider hubs with power-law in-degree. Node labels are
  then permuted at random.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class SEM:
    """A generated problem: data X (n x p, samples x variables) and its DAG."""

    Xt: np.ndarray              # p x n, C-contiguous: one row of samples per variable
    src: np.ndarray             # edge tails (int64)
    dst: np.ndarray             # edge heads (int64)
    weight: np.ndarray          # edge weights (float64)
    p: int
    n: int
    seed: int
    family: str
    alpha: float = 0.01
    max_level: int = -1
    meta: dict = field(default_factory=dict)

    @property
    def X(self) -> np.ndarray:
        """n x p view (samples x variables) of the same data, column-major in memory."""
        return self.Xt.T

    def dag_matrix(self) -> np.ndarray:
        """p x p uint8 matrix with D[u, v] = 1 iff u -> v."""
        D = np.zeros((self.p, self.p), dtype=np.uint8)
        D[self.src, self.dst] = 1
        return D

    def skeleton(self) -> np.ndarray:
        """p x p uint8 symmetric adjacency of the DAG's skeleton."""
        D = self.dag_matrix()
        return (D | D.T).astype(np.uint8)


def random_dag(rng: np.random.Generator, p: int, degree: float):
    """Random DAG over a random topological order, edge prob degree/(p-1)."""
    order = rng.permutation(p)
    q = 0.0 if p < 2 else min(1.0, degree / (p - 1))
    src, dst = [], []
    for b in range(1, p):
        hits = np.nonzero(rng.random(b) < q)[0]
        if hits.size:
            src.append(order[hits])
            dst.append(np.full(hits.size, order[b], dtype=np.int64))
    if src:
        return np.concatenate(src).astype(np.int64), np.concatenate(dst).astype(np.int64), order
    return np.zeros(0, np.int64), np.zeros(0, np.int64), order


def scale_free_dag(rng: np.random.Generator, p: int, m: int = 2):
    """Preferential-attachment DAG, edges new -> old, labels permuted."""
    deg = np.zeros(p, dtype=np.float64)
    src, dst = [], []
    for t in range(1, p):
        k = min(m, t)
        w = deg[:t] + 1.0
        chosen = rng.choice(t, size=k, replace=False, p=w / w.sum())
        for c in chosen:
            src.append(t)
            dst.append(int(c))
            deg[t] += 1
            deg[c] += 1
    perm = rng.permutation(p)
    src = perm[np.asarray(src, dtype=np.int64)]
    dst = perm[np.asarray(dst, dtype=np.int64)]
    # topological order in the new labels: arrival order reversed (new -> old)
    order = perm[np.arange(p - 1, -1, -1)]
    return src.astype(np.int64), dst.astype(np.int64), order


def sample_sem(rng: np.random.Generator, p: int, n: int, src, dst, weight, order) -> np.ndarray:
    """Draw n samples of the linear SEM in topological order (float64, p x n)."""
    Xt = rng.standard_normal((p, n))            # noise; one contiguous row per variable
    if src.size:
        key = np.argsort(dst, kind="stable")
        s_sorted, d_sorted, w_sorted = src[key], dst[key], weight[key]
        starts = np.searchsorted(d_sorted, np.arange(p + 1))
    for v in order.tolist():
        if src.size and starts[v + 1] > starts[v]:
            a, b = starts[v], starts[v + 1]
            Xt[v] += w_sorted[a:b] @ Xt[s_sorted[a:b]]
    return Xt


def generate(p: int, n: int, seed: int, family: str = "random", degree: float = 2.0,
             m: int = 2, w_min: float = 0.1, dtype=np.float64, alpha: float = 0.01,
             max_level: int = -1) -> SEM:
    """Generate one seeded SEM problem."""
    rng = np.random.default_rng(seed)
    if family == "random":
        src, dst, order = random_dag(rng, p, degree)
    elif family == "scale_free":
        src, dst, order = scale_free_dag(rng, p, m)
    else:
        raise ValueError(f"unknown family {family!r}")
    mag = rng.uniform(w_min, 1.0, size=src.size)
    sign = np.where(rng.random(src.size) < 0.5, -1.0, 1.0)
    weight = mag * sign
    Xt = sample_sem(rng, p, n, src, dst, weight, order)
    if np.dtype(dtype) != Xt.dtype:
        Xt = Xt.astype(dtype)
    return SEM(Xt=Xt, src=src, dst=dst, weight=weight, p=p, n=n, seed=seed, family=family,
               alpha=alpha, max_level=max_level,
               meta={"degree": degree, "m": m, "w_min": w_min, "dtype": np.dtype(dtype).name})


# ---------------------------------------------------------------------------
# The five workloads. seed = 1000 * workload number + instance.
# ---------------------------------------------------------------------------

def workload(name: str, instance: int = 0) -> SEM:
    """Named workloads: small20, medium1000, scalefree2500, large10000."""
    if name == "small20":        # p=20 n=1000 random DAG, edge prob 2/(p-1), float64
        return generate(20, 1000, 1000 + instance, "random", degree=2.0, w_min=0.1,
                        dtype=np.float64, alpha=0.01)
    if name == "medium1000":     # p=1000 n=10000 expected degree 3, float32 input
        return generate(1000, 10000, 2000 + instance, "random", degree=3.0, w_min=0.1,
                        dtype=np.float32, alpha=0.01)
    if name == "scalefree2500":  # p=2500 n=500 preferential attachment m=2
        return generate(2500, 500, 3000 + instance, "scale_free", m=2, w_min=0.2,
                        dtype=np.float64, alpha=0.01)
    if name == "large10000":     # p=10000 n=1000 expected degree 5, levels <= 6
        return generate(10000, 1000, 5000 + instance, "random", degree=5.0, w_min=0.1,
                        dtype=np.float64, alpha=0.01, max_level=6)
    raise ValueError(f"unknown workload {name!r}")


def mlp_training_instance(k: int) -> SEM:
    """Training problems for the ordering network: p=500 preferential attachment."""
    return generate(500, 500, 30000 + k, "scale_free", m=2, w_min=0.2,
                    dtype=np.float64, alpha=0.01)


def batch_workload(count: int = 64, instance: int = 0):
    """64 independent problems of uneven size: p~U[50,800], n~U[200,5000], degree~U[2,6]."""
    rng = np.random.default_rng(4000 + instance)
    ps = rng.integers(50, 801, size=count)
    ns = rng.integers(200, 5001, size=count)
    ds = rng.uniform(2.0, 6.0, size=count)
    return [generate(int(ps[k]), int(ns[k]), 4000 * 1000 + 1000 * instance + k, "random",
                     degree=float(ds[k]), w_min=0.1, dtype=np.float64, alpha=0.05)
            for k in range(count)]


def paper_density(p: int, n: int, d: float, seed: int, alpha: float = 0.01) -> SEM:
    """The paper's scalability generator (Sec. 5.6): a lower-triangular random
    weight matrix A with Bernoulli(d) support and U[0.1, 1] entries (all
    positive), V_j -> V_i for A[i, j] != 0, and V_i = N_i + sum_{j < i} A[i, j] V_j
    for i = 0 .. p - 1 with N_i ~ N(0, 1). The variables are labelled in
    topological order. With positive weights the magnitudes grow
    geometrically along that order, so the data is FP64."""
    rng = np.random.default_rng(seed)
    sup = rng.random((p, p)) < d
    A = np.tril(sup, -1) * rng.uniform(0.1, 1.0, size=(p, p))
    N = rng.standard_normal((p, n))
    Xt = np.empty((p, n))
    for i in range(p):
        Xt[i] = N[i] + A[i, :i] @ Xt[:i]
    dst, src = np.nonzero(A)
    return SEM(Xt=Xt, src=src.astype(np.int64), dst=dst.astype(np.int64), weight=A[dst, src], p=p, n=n, seed=seed,
               family="paper_density", alpha=alpha, meta={"density": d, "w_min": 0.1, "dtype": "float64"})


def paper_density_signed(p: int, n: int, d: float, seed: int, alpha: float = 0.01, max_level: int = 2) -> SEM:
    """The scalability workload's structure (Sec. 5.6: a lower-triangular matrix
    A with Bernoulli(d) support, V_j -> V_i for A[i, j] != 0, generated from i = 0
    to p - 1) with signed weights +-U[0.1, 1], and each variable rescaled to unit
    sample variance as soon as it is generated, so that later variables do not
    grow geometrically with the number of parents (at d = 0.1 and p = 1000 a
    variable has about 50 parents). The graph, the order and the sample draws
    follow the paper's recipe; only the signs and the rescaling differ.
    max_level caps the level loop (dense graphs make every level's subset count
    grow as C(degree, l))."""
    rng = np.random.default_rng(seed)
    sup = rng.random((p, p)) < d
    mag = rng.uniform(0.1, 1.0, size=(p, p))
    sign = np.where(rng.random((p, p)) < 0.5, -1.0, 1.0)
    A = np.tril(sup, -1) * mag * sign
    N = rng.standard_normal((p, n))
    Xt = np.empty((p, n))
    # in blocks of rows: the parents in earlier blocks by one matrix product,
    # then row by row within the block
    blk = 256
    for b0 in range(0, p, blk):
        b1 = min(p, b0 + blk)
        acc = N[b0:b1] + (A[b0:b1, :b0] @ Xt[:b0] if b0 else 0.0)
        for i in range(b0, b1):
            v = acc[i - b0] + A[i, b0:i] @ Xt[b0:i]
            Xt[i] = v / v.std()
    dst, src = np.nonzero(A)
    return SEM(Xt=Xt, src=src.astype(np.int64), dst=dst.astype(np.int64), weight=A[dst, src], p=p, n=n, seed=seed,
               family="paper_density_signed", alpha=alpha, max_level=max_level,
               meta={"density": d, "w_min": 0.1, "dtype": "float64"})
