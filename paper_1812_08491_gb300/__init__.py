"""GB300 (sm_103a) PC-stable skeleton library -- Python binding.

A thin ctypes layer over the C ABI declared in ``include/cupc.h``: it only
marshals arguments (pointers, sizes, options) and copies results out. Every
step of the skeleton runs in the library's CUDA kernels; there is no Python or
CPU fallback. If the shared library has not been built, every call raises.

PyTorch is used only to hand over device memory and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["CupcError", "Context", "Result", "load", "lib_path", "build_library", "MODE_PLAIN_FP64",
           "MODE_FP32_RECHECK", "F32", "F64", "SAMPLE_MAJOR", "VARIABLE_MAJOR", "MAX_LEVEL",
           "fisher_threshold", "exported_symbols"]

F32, F64 = 0, 1
FAIL_NONE, FAIL_ALLOC, FAIL_LAUNCH, FAIL_BARRIER = 0, 1, 2, 3
SAMPLE_MAJOR, VARIABLE_MAJOR = 0, 1
MODE_PLAIN_FP64, MODE_FP32_RECHECK = 0, 1
L1_AUTO, L1_BY_PIVOT, L1_BY_ROW = 0, 1, 2          # cupc_options.level1_form
MAX_LEVEL = 16
STATS_LEVELS = 24
KERNEL_CLASSES = ("upload", "standardize", "correlation", "level0", "compact", "ci", "recheck", "finalize")

_STATUS = {0: "CUPC_OK", -1: "CUPC_E_INVALID", -2: "CUPC_E_NOMEM", -3: "CUPC_E_CUDA", -4: "CUPC_E_TIMEOUT",
           -5: "CUPC_E_RANGE", -6: "CUPC_E_NUMERIC", -7: "CUPC_E_CANCELLED", -8: "CUPC_E_STATE"}

# Every entry point declared in include/cupc.h (kept in sync by a CPU test).
_SIGNATURES = {
    "cupc_options_default": (None, ["opts_p"]),
    "cupc_create": ("status", ["pp", "int", "vp"]),
    "cupc_set_stream": ("status", ["vp", "vp"]),
    "cupc_destroy": (None, ["vp"]),
    "cupc_last_error": ("str", ["vp"]),
    "cupc_cancel": ("status", ["vp"]),
    "cupc_debug_fail": ("status", ["vp", "int", "i64"]),
    "cupc_skeleton": ("status", ["vp", "vp", "int", "int", "int", "i64", "i64", "i64", "dbl", "opts_p", "pp"]),
    "cupc_skeleton_corr": ("status", ["vp", "vp", "int", "int", "i64", "i64", "i64", "dbl", "opts_p", "pp"]),
    "cupc_result_p": ("status", ["vp", "vp"]),
    "cupc_result_adjacency": ("status", ["vp", "vp"]),
    "cupc_result_sep_levels": ("status", ["vp", "vp"]),
    "cupc_result_edges": ("status", ["vp", "vp", "i64", "vp"]),
    "cupc_result_sepset": ("status", ["vp", "i64", "i64", "vp", "vp"]),
    "cupc_result_sepset_records": ("status", ["vp", "vp", "i64", "vp"]),
    "cupc_result_stats": ("status", ["vp", "vp"]),
    "cupc_result_checkpoint": ("status", ["vp", "vp", "i64", "vp"]),
    "cupc_result_sshare": ("status", ["vp", "int", "vp", "int", "vp", "vp"]),
    "cupc_skeleton_resume": ("status", ["vp", "vp", "int", "int", "int", "i64", "i64", "i64", "dbl", "opts_p", "vp",
                                        "i64", "pp"]),
    "cupc_result_orient": ("status", ["vp", "vp", "vp"]),
    "cupc_result_free": (None, ["vp"]),
    "cupc_correlation": ("status", ["vp", "vp", "int", "int", "int", "i64", "i64", "i64", "int", "vp"]),
    "cupc_pcor_batch": ("status", ["vp", "vp", "int", "i64", "vp", "i64", "int", "vp"]),
    "cupc_pcor_data": ("status", ["vp", "vp", "int", "int", "int", "i64", "i64", "i64", "vp", "i64", "int", "vp"]),
    "cupc_fisher_threshold": ("status", ["dbl", "i64", "int", "vp", "vp"]),
    "cupc_correlation_noalloc": ("status", ["vp", "int", "int", "i64", "i64", "i64", "vp", "vp"]),
    "cupc_skeleton_batch": ("status", ["vp", "int", "vp", "int", "int", "int", "vp", "vp", "vp", "opts_p", "vp",
                                       "vp"]),
    "cupc_device_peaks": ("status", ["vp", "vp", "vp"]),
    "cupc_batch_autotune": ("status", ["vp", "int", "vp", "int", "int", "int", "vp", "vp", "vp", "opts_p", "int",
                                       "vp", "int", "vp"]),
    "cupc_mlp_set_weights": ("status", ["vp", "vp"]),
    "cupc_mlp_get_weights": ("status", ["vp", "vp"]),
    "cupc_mlp_grad": ("status", ["vp", "vp", "vp", "i64", "vp", "vp"]),
    "cupc_mlp_forward": ("status", ["vp", "vp", "i64", "vp"]),
    "cupc_mlp_train": ("status", ["vp", "vp", "vp", "i64", "i64", "int", "dbl", "vp"]),
    "cupc_mlp_examples": ("status", ["vp", "vp", "vp", "vp", "i64", "vp"]),
}
MLP_PARAMS = 4609
MLP_FEATURES = 5


class CupcError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        super().__init__(f"{where}: {_STATUS.get(status, status)}" + (f" ({message})" if message else ""))


class Options(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("canonical_sepset", ctypes.c_int), ("learned_order", ctypes.c_int),
                ("max_level", ctypes.c_int), ("recheck_margin", ctypes.c_double),
                ("threads_per_block", ctypes.c_int), ("chunk", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("corr_kps", ctypes.c_int), ("batch_direct", ctypes.c_int), ("test_qcap", ctypes.c_int),
                ("test_nnz_cap", ctypes.c_int), ("test_rec_cap", ctypes.c_int), ("level1_form", ctypes.c_int),
                ("host_lists", ctypes.c_int)]


class Stats(ctypes.Structure):
    L = STATS_LEVELS
    _fields_ = [("levels", ctypes.c_int), ("tests", ctypes.c_int64 * L), ("serial_tests", ctypes.c_int64 * L),
                ("removed", ctypes.c_int64 * L), ("rechecks", ctypes.c_int64 * L),
                ("edges_start", ctypes.c_int64 * L), ("max_degree", ctypes.c_int32 * L),
                ("level_ms", ctypes.c_float * L), ("prep_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("edges_final", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("kernel_ms", ctypes.c_float * 8), ("kernel_count", ctypes.c_int32 * 8),
                ("ci_block_entries", ctypes.c_int64 * L), ("phase_ms", (ctypes.c_float * 4) * L),
                ("cuda_graph", ctypes.c_int32), ("recheck_ms", (ctypes.c_float * 3) * L),
                ("rechecks_queued", ctypes.c_int64 * L), ("reruns", ctypes.c_int32 * 4),
                ("order_ms", (ctypes.c_float * 2) * L), ("host_ms", ctypes.c_float * 2)]


class OrientStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("directed", ctypes.c_int64), ("undirected", ctypes.c_int64),
                ("bidirected", ctypes.c_int64), ("rule_conflicts", ctypes.c_int64), ("ms", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class SShareStats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int64), ("distinct", ctypes.c_int64), ("redundant", ctypes.c_int64),
                ("max_rows", ctypes.c_int64), ("rows", ctypes.c_int64), ("search_ms", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("corr_kps", ctypes.c_int),
                ("ms", ctypes.c_float)]


_LIB = None


def lib_path() -> str:
    return _build.lib_path()


def build_library(force: bool = False) -> str:
    return _build.build(force=force)


def load():
    """Loads the shared library; raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built ({path}); call paper_1812_08491_gb300.build_library()")
    L = ctypes.CDLL(path)
    types = {"status": ctypes.c_int, "int": ctypes.c_int, "i64": ctypes.c_int64, "dbl": ctypes.c_double,
             "vp": ctypes.c_void_p, "pp": ctypes.POINTER(ctypes.c_void_p), "str": ctypes.c_char_p,
             "opts_p": ctypes.POINTER(Options), None: None}
    for name, (rt, args) in _SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = types[rt]
        fn.argtypes = [types[a] for a in args]
    _LIB = L
    return L


def exported_symbols():
    return list(_SIGNATURES)


def fisher_threshold(alpha: float, n_samples: int, l: int):
    """(tau, tanh(tau)) of Eq. (threshold) as the library computes it."""
    L = load()
    tau, r = ctypes.c_double(), ctypes.c_double()
    st = L.cupc_fisher_threshold(alpha, n_samples, l, ctypes.byref(tau), ctypes.byref(r))
    if st != 0:
        raise CupcError(st, "cupc_fisher_threshold")
    return tau.value, r.value


def _torch():
    import torch
    return torch


def _describe(X):
    """(pointer, dtype code, layout, on_device, n, p, ld, keepalive) for an n x p array/tensor."""
    if isinstance(X, np.ndarray):
        if X.dtype not in (np.float32, np.float64) or X.ndim != 2:
            raise ValueError("X must be a 2-D float32/float64 array")
        es = X.itemsize
        n, p = X.shape
        if X.strides[1] == es and X.strides[0] % es == 0:
            layout, ld = SAMPLE_MAJOR, X.strides[0] // es
        elif X.strides[0] == es and X.strides[1] % es == 0:
            layout, ld = VARIABLE_MAJOR, X.strides[1] // es
        else:
            X = np.ascontiguousarray(X)
            layout, ld = SAMPLE_MAJOR, p
        return X.ctypes.data, (F64 if X.dtype == np.float64 else F32), layout, 0, n, p, ld, X
    torch = _torch()
    if isinstance(X, torch.Tensor):
        if X.dtype not in (torch.float32, torch.float64) or X.dim() != 2:
            raise ValueError("X must be a 2-D float32/float64 tensor")
        n, p = X.shape
        s0, s1 = X.stride()
        if s1 == 1:
            layout, ld = SAMPLE_MAJOR, s0
        elif s0 == 1:
            layout, ld = VARIABLE_MAJOR, s1
        else:
            X = X.contiguous()
            layout, ld = SAMPLE_MAJOR, p
        return (X.data_ptr(), F64 if X.dtype == torch.float64 else F32, layout, 1 if X.is_cuda else 0,
                n, p, ld, X)
    raise TypeError("X must be a numpy array or a torch tensor")


def _stats_dict(s: Stats) -> dict:
    L = s.levels
    return {"levels": L, "tests": list(s.tests[:L]), "serial_tests": list(s.serial_tests[:L]),
            "removed": list(s.removed[:L]), "rechecks": list(s.rechecks[:L]),
            "edges_start": list(s.edges_start[:L]), "max_degree": list(s.max_degree[:L]),
            "level_ms": list(s.level_ms[:L]), "prep_ms": s.prep_ms, "total_ms": s.total_ms,
            "edges_final": s.edges_final, "kernel_launches": s.kernel_launches,
            "h2d_bytes": s.h2d_bytes, "d2h_bytes": s.d2h_bytes,
            "kernel_ms": dict(zip(KERNEL_CLASSES, list(s.kernel_ms))),
            "kernel_count": dict(zip(KERNEL_CLASSES, list(s.kernel_count))),
            "ci_block_entries": list(s.ci_block_entries[:L]),
            "phase_ms": [list(s.phase_ms[q]) for q in range(L)], "cuda_graph": s.cuda_graph,
            "recheck_ms": [list(s.recheck_ms[q]) for q in range(L)],
            "rechecks_queued": list(s.rechecks_queued[:L]), "reruns": list(s.reruns),
            "order_ms": [list(s.order_ms[q]) for q in range(L)], "host_ms": list(s.host_ms)}


class Result:
    """Skeleton and SepSets of one call; owns library memory until free()."""

    def __init__(self, ctx: "Context", handle: int):
        self._ctx = ctx
        self._h = ctypes.c_void_p(handle)
        p = ctypes.c_int64()
        self._check(load().cupc_result_p(self._h, ctypes.byref(p)), "cupc_result_p")
        self.p = p.value

    def _check(self, st, where):
        if st != 0:
            raise CupcError(st, where, self._ctx.last_error())

    def adjacency(self) -> np.ndarray:
        out = np.empty((self.p, self.p), dtype=np.uint8)
        self._check(load().cupc_result_adjacency(self._h, out.ctypes.data), "cupc_result_adjacency")
        return out

    def edges(self) -> np.ndarray:
        """The skeleton's edges as an (m, 2) int32 array of pairs (i, j), i < j."""
        L = load()
        n = ctypes.c_int64()
        self._check(L.cupc_result_edges(self._h, None, 0, ctypes.byref(n)), "cupc_result_edges")
        out = np.empty((n.value, 2), dtype=np.int32)
        self._check(L.cupc_result_edges(self._h, out.ctypes.data, n.value, ctypes.byref(n)), "cupc_result_edges")
        return out

    def sep_levels(self) -> np.ndarray:
        out = np.empty((self.p, self.p), dtype=np.int16)
        self._check(load().cupc_result_sep_levels(self._h, out.ctypes.data), "cupc_result_sep_levels")
        return out

    def sepset(self, i: int, j: int):
        """Tuple S of a removed pair, () for level 0, None when the edge is present."""
        buf = (ctypes.c_int32 * MAX_LEVEL)()
        ln = ctypes.c_int()
        self._check(load().cupc_result_sepset(self._h, i, j, buf, ctypes.byref(ln)), "cupc_result_sepset")
        return None if ln.value < 0 else tuple(buf[k] for k in range(ln.value))

    def records_raw(self) -> np.ndarray:
        n = ctypes.c_int64()
        L = load()
        self._check(L.cupc_result_sepset_records(self._h, None, 0, ctypes.byref(n)), "records")
        out = np.empty(max(n.value, 1), dtype=np.int32)
        self._check(L.cupc_result_sepset_records(self._h, out.ctypes.data, n.value, ctypes.byref(n)), "records")
        return out[:n.value]

    def sepsets(self) -> dict:
        """{(i, j): (level, S)} for removals at level >= 1 (i < j)."""
        raw = self.records_raw()
        out, k = {}, 0
        while k < raw.size:
            i, j, l = int(raw[k]), int(raw[k + 1]), int(raw[k + 2])
            out[(i, j)] = (l, tuple(int(v) for v in raw[k + 3:k + 3 + l]))
            k += 3 + l
        return out

    def orient(self, marks: bool = True):
        """Second step of PC-stable on the device: (marks, stats). marks[a, b] = 0 no
        edge, 1 arrowhead at b, 2 tail at b (None when marks=False)."""
        out = np.empty((self.p, self.p), dtype=np.uint8) if marks else None
        s = OrientStats()
        self._check(load().cupc_result_orient(self._h, out.ctypes.data if marks else None, ctypes.byref(s)),
                    "cupc_result_orient")
        return out, {"rounds": s.rounds, "directed": s.directed, "undirected": s.undirected,
                     "bidirected": s.bidirected, "rule_conflicts": s.rule_conflicts, "ms": s.ms}

    def sshare(self, level: int, bins):
        """Global-sharing histogram of conditioning sets at `level` (Sec. 5.5):
        (counts per bin, stats dict)."""
        b = (ctypes.c_int64 * len(bins))(*[int(x) for x in bins])
        c = (ctypes.c_int64 * len(bins))()
        st = SShareStats()
        self._check(load().cupc_result_sshare(self._h, level, b, len(bins), c, ctypes.byref(st)),
                    "cupc_result_sshare")
        return list(c), {"pairs": st.pairs, "distinct": st.distinct, "redundant": st.redundant,
                         "max_rows": st.max_rows, "rows": st.rows, "search_ms": st.search_ms}

    def mlp_examples(self, C):
        """Training examples (X [m x 5], t [m]) of the network from this result's
        SepSets, features from the CUDA float32 correlation C; CUDA tensors."""
        torch = _torch()
        L = load()
        n = ctypes.c_int64()
        Cc = C.to(torch.float32).contiguous()
        self._check(L.cupc_mlp_examples(self._h, ctypes.c_void_p(Cc.data_ptr()), None, None, 0, ctypes.byref(n)),
                    "cupc_mlp_examples")
        X = torch.empty((n.value, MLP_FEATURES), dtype=torch.float32, device=Cc.device)
        t = torch.empty(n.value, dtype=torch.float32, device=Cc.device)
        if n.value:
            self._check(L.cupc_mlp_examples(self._h, ctypes.c_void_p(Cc.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                            ctypes.c_void_p(t.data_ptr()), n.value, ctypes.byref(n)),
                        "cupc_mlp_examples")
        return X, t

    def checkpoint(self) -> bytes:
        """Level-boundary checkpoint of this result (opaque bytes)."""
        L = load()
        n = ctypes.c_int64()
        self._check(L.cupc_result_checkpoint(self._h, None, 0, ctypes.byref(n)), "cupc_result_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        self._check(L.cupc_result_checkpoint(self._h, buf, n.value, ctypes.byref(n)), "cupc_result_checkpoint")
        return buf.raw

    def stats(self) -> dict:
        s = Stats()
        self._check(load().cupc_result_stats(self._h, ctypes.byref(s)), "cupc_result_stats")
        return _stats_dict(s)

    def free(self):
        if self._h:
            load().cupc_result_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A library context bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None, level1_form: int = L1_AUTO):
        """level1_form: the default of options(level1_form=...) for this context."""
        self.level1_form = level1_form
        L = load()
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        st = L.cupc_create(ctypes.byref(h), device, ctypes.c_void_p(stream))
        if st != 0:
            raise CupcError(st, "cupc_create", "device must be an sm_103 GPU")
        self._h = h
        self.device = device

    def cancel(self):
        """Stops the running (other thread) or next call between levels."""
        self._check(load().cupc_cancel(self._h), "cupc_cancel")

    def debug_fail(self, kind: int, k: int = 1):
        """Arms a host-side failure (FAIL_ALLOC / FAIL_LAUNCH on the k-th next event,
        FAIL_BARRIER with a k-ns grid-barrier limit for the next call; FAIL_NONE disarms)."""
        self._check(load().cupc_debug_fail(self._h, kind, k), "cupc_debug_fail")

    def last_error(self) -> str:
        if not self._h:
            return ""
        return (load().cupc_last_error(self._h) or b"").decode()

    def _check(self, st, where):
        if st != 0:
            raise CupcError(st, where, self.last_error())

    def options(self, mode=MODE_FP32_RECHECK, canonical=True, max_level=-1, recheck_margin=0.0,
                threads_per_block=0, chunk=0, learned_order=False, ctas_per_sm=0, corr_kps=0,
                batch_direct=False, test_qcap=0, test_nnz_cap=0, test_rec_cap=0, level1_form=None,
                host_lists=False) -> Options:
        o = Options()
        load().cupc_options_default(ctypes.byref(o))
        o.mode = mode
        o.canonical_sepset = 1 if canonical else 0
        o.max_level = max_level
        o.recheck_margin = recheck_margin
        o.threads_per_block = threads_per_block
        o.chunk = chunk
        o.learned_order = 1 if learned_order else 0
        o.ctas_per_sm = ctas_per_sm
        o.corr_kps = corr_kps
        o.batch_direct = 1 if batch_direct else 0
        o.test_qcap = test_qcap
        o.test_nnz_cap = test_nnz_cap
        o.test_rec_cap = test_rec_cap
        o.level1_form = self.level1_form if level1_form is None else level1_form
        o.host_lists = 1 if host_lists else 0
        return o

    @staticmethod
    def _batch_args(Xs, alphas):
        """Pointer, size and alpha arrays for a list of dense n x p arrays/tensors."""
        if len(Xs) == 0:
            raise ValueError("empty batch")
        descs = [_describe(X) for X in Xs]
        dts = {d[1] for d in descs}
        lays = {d[2] for d in descs}
        devs = {d[3] for d in descs}
        if len(dts) != 1 or len(lays) != 1 or len(devs) != 1:
            raise ValueError("all problems of a batch share dtype, layout and location")
        layout = lays.pop()
        for d in descs:
            dense = d[6] == (d[5] if layout == SAMPLE_MAJOR else d[4])
            if not dense:
                raise ValueError("batch inputs must be dense (ld = row length)")
        k = len(descs)
        ptrs = (ctypes.c_void_p * k)(*[d[0] for d in descs])
        ns = (ctypes.c_int64 * k)(*[d[4] for d in descs])
        ps = (ctypes.c_int64 * k)(*[d[5] for d in descs])
        if np.isscalar(alphas):
            alphas = [float(alphas)] * k
        al = (ctypes.c_double * k)(*[float(a) for a in alphas])
        keep = [d[7] for d in descs]
        return k, ptrs, dts.pop(), layout, devs.pop(), ns, ps, al, keep

    def device_peaks(self) -> dict:
        """Measured FP64 / FP32 FMA throughput of the device (TFLOP/s)."""
        f64, f32 = ctypes.c_double(), ctypes.c_double()
        self._check(load().cupc_device_peaks(self._h, ctypes.byref(f64), ctypes.byref(f32)), "cupc_device_peaks")
        return {"fp64_tflops": f64.value, "fp32_tflops": f32.value}

    def skeleton_batch(self, Xs, alphas, opts: Options | None = None, **kw):
        """Skeletons of independent problems (list of n_k x p_k arrays or tensors,
        all host or all device, one dtype and layout) in one batched pass.
        Returns (list of Result, batch stats dict)."""
        k, ptrs, dt, layout, on_dev, ns, ps, al, keep = self._batch_args(Xs, alphas)
        o = opts if opts is not None else self.options(**kw)
        outs = (ctypes.c_void_p * k)()
        bst = Stats()
        st = load().cupc_skeleton_batch(self._h, k, ptrs, dt, layout, on_dev, ns, ps, al, ctypes.byref(o), outs,
                                        ctypes.byref(bst))
        self._check(st, "cupc_skeleton_batch")
        del keep
        return [Result(self, outs[q]) for q in range(k)], _stats_dict(bst)

    def autotune_batch(self, Xs, alphas, opts: Options | None = None, reps: int = 2, **kw):
        """Launch configurations of a batch, fastest first:
        [{"chunk", "ctas_per_sm", "corr_kps", "ms"}, ...]."""
        k, ptrs, dt, layout, on_dev, ns, ps, al, keep = self._batch_args(Xs, alphas)
        o = opts if opts is not None else self.options(**kw)
        cap = 64
        ents = (TuneEntry * cap)()
        cnt = ctypes.c_int()
        st = load().cupc_batch_autotune(self._h, k, ptrs, dt, layout, on_dev, ns, ps, al, ctypes.byref(o), reps,
                                        ents, cap, ctypes.byref(cnt))
        self._check(st, "cupc_batch_autotune")
        del keep
        return [{"chunk": e.chunk, "ctas_per_sm": e.ctas_per_sm, "corr_kps": e.corr_kps, "ms": e.ms}
                for e in ents[:cnt.value]]

    def skeleton(self, X, alpha: float, opts: Options | None = None, **kw) -> Result:
        """Algorithm 1 on data X (n x p numpy array or torch tensor, host or device)."""
        ptr, dt, layout, on_dev, n, p, ld, keep = _describe(X)
        o = opts if opts is not None else self.options(**kw)
        out = ctypes.c_void_p()
        st = load().cupc_skeleton(self._h, ctypes.c_void_p(ptr), dt, layout, on_dev, n, p, ld, alpha,
                                  ctypes.byref(o), ctypes.byref(out))
        self._check(st, "cupc_skeleton")
        del keep
        return Result(self, out.value)

    def skeleton_resume(self, X, alpha: float, checkpoint: bytes, opts: Options | None = None, **kw) -> Result:
        """Continues a run from Result.checkpoint() on the same data X and alpha."""
        ptr, dt, layout, on_dev, n, p, ld, keep = _describe(X)
        o = opts if opts is not None else self.options(**kw)
        out = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(bytes(checkpoint), len(checkpoint))
        st = load().cupc_skeleton_resume(self._h, ctypes.c_void_p(ptr), dt, layout, on_dev, n, p, ld, alpha,
                                         ctypes.byref(o), buf, len(checkpoint), ctypes.byref(out))
        self._check(st, "cupc_skeleton_resume")
        del keep
        return Result(self, out.value)

    def skeleton_corr(self, C, n_samples: int, alpha: float, opts: Options | None = None, **kw) -> Result:
        """Algorithm 1 from a p x p correlation matrix (row-major, host or device)."""
        ptr, dt, layout, on_dev, p0, p1, ld, keep = _describe(C)
        if layout != SAMPLE_MAJOR or p0 != p1:
            raise ValueError("C must be a square row-major matrix")
        o = opts if opts is not None else self.options(**kw)
        out = ctypes.c_void_p()
        st = load().cupc_skeleton_corr(self._h, ctypes.c_void_p(ptr), dt, on_dev, p0, ld, n_samples, alpha,
                                       ctypes.byref(o), ctypes.byref(out))
        self._check(st, "cupc_skeleton_corr")
        del keep
        return Result(self, out.value)

    def correlation(self, X, precision: int = F64):
        """Correlation matrix of X as a CUDA tensor (float64 or float32)."""
        torch = _torch()
        ptr, dt, layout, on_dev, n, p, ld, keep = _describe(X)
        C = torch.empty((p, p), dtype=torch.float64 if precision == F64 else torch.float32,
                        device=f"cuda:{self.device}")
        st = load().cupc_correlation(self._h, ctypes.c_void_p(ptr), dt, layout, on_dev, n, p, ld, precision,
                                     ctypes.c_void_p(C.data_ptr()))
        self._check(st, "cupc_correlation")
        del keep
        return C

    def pcor_batch(self, C, queries, l: int):
        """rho(i, j | S) for rows (i, j, S...) of an int32 CUDA tensor, on CUDA matrix C."""
        torch = _torch()
        q = queries.to(device=C.device, dtype=torch.int32).contiguous()
        rho = torch.empty(q.shape[0], dtype=torch.float64, device=C.device)
        st = load().cupc_pcor_batch(self._h, ctypes.c_void_p(C.data_ptr()),
                                    F32 if C.dtype == torch.float32 else F64, C.shape[0],
                                    ctypes.c_void_p(q.data_ptr()), q.shape[0], l, ctypes.c_void_p(rho.data_ptr()))
        self._check(st, "cupc_pcor_batch")
        return rho

    def pcor_data(self, X, queries, l: int):
        """rho(i, j | S) from the data X with the FP64 recheck arithmetic, for rows
        (i, j, S...) of an int32 tensor; a CUDA float64 tensor."""
        torch = _torch()
        ptr, dt, layout, on_dev, n, p, ld, keep = _describe(X)
        q = queries.to(device=f"cuda:{self.device}", dtype=torch.int32).contiguous()
        rho = torch.empty(q.shape[0], dtype=torch.float64, device=q.device)
        st = load().cupc_pcor_data(self._h, ctypes.c_void_p(ptr), dt, layout, on_dev, n, p, ld,
                                   ctypes.c_void_p(q.data_ptr()), q.shape[0], l, ctypes.c_void_p(rho.data_ptr()))
        self._check(st, "cupc_pcor_data")
        del keep
        return rho

    # ---- candidate-scoring network -------------------------------------------
    def mlp_set_weights(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if p.size != MLP_PARAMS:
            raise ValueError(f"expected {MLP_PARAMS} parameters")
        self._check(load().cupc_mlp_set_weights(self._h, p.ctypes.data), "cupc_mlp_set_weights")

    def mlp_get_weights(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        self._check(load().cupc_mlp_get_weights(self._h, out.ctypes.data), "cupc_mlp_get_weights")
        return out

    def mlp_grad(self, X, t):
        """(gradient, mean loss) over device feature rows X [n x 5] and labels t [n]."""
        torch = _torch()
        X = X.to(torch.float32).contiguous()
        t = t.to(torch.float32).contiguous()
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(load().cupc_mlp_grad(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                         X.shape[0], g.ctypes.data, ctypes.byref(loss)), "cupc_mlp_grad")
        return g, loss.value

    def mlp_forward(self, X):
        torch = _torch()
        X = X.to(torch.float32).contiguous()
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        self._check(load().cupc_mlp_forward(self._h, ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                            ctypes.c_void_p(y.data_ptr())), "cupc_mlp_forward")
        return y

    def mlp_train(self, X, t, batch=4096, epochs=4, lr=1e-3):
        torch = _torch()
        X = X.to(torch.float32).contiguous()
        t = t.to(torch.float32).contiguous()
        losses = np.zeros(max(epochs, 1), dtype=np.float64)
        self._check(load().cupc_mlp_train(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                          X.shape[0], batch, epochs, lr, losses.ctypes.data), "cupc_mlp_train")
        return losses[:epochs]

    def close(self):
        if getattr(self, "_h", None):
            load().cupc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
