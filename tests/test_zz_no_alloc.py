"""The allocation-free correlation entry point against the allocating one.

cupc_correlation_noalloc serves callers that may not allocate device memory
(frameworks that own all GPU memory, latency-critical pipelines where a
cudaMalloc is not acceptable). Its scratch is a fixed device array inside the
library, shared by all calls. This test calls it twice in a row through the C
ABI, with different shapes and layouts, and compares each output with
cupc_correlation's (FP64) and with the FP64 CPU oracle's correlation, within
the correlation tolerance of the other tests (1e-13). It also checks that
oversized inputs are refused. This file is collected last so a failure here
never hides the other tests' results.
"""
import ctypes

import numpy as np
import pytest

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")

import oracle
from synth import sem

pytestmark = pytest.mark.gpu


def _call(L, X, layout, n, p, ld, out, stream):
    dt = cupc.F64 if X.dtype == torch.float64 else cupc.F32
    return L.cupc_correlation_noalloc(ctypes.c_void_p(X.data_ptr()), dt, layout, n, p, ld,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_allocating_entry_point(cuda_device):
    cupc.build_library()
    L = cupc.load()
    ctx = cupc.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(700, 90, "variable", np.float64), (333, 257, "sample", np.float32)]
    for n, p, layout, dt in cases:            # two calls in a row, different shapes
        s = sem.generate(p, n, 4242 + p, "random", degree=3.0, dtype=dt)
        if layout == "variable":
            Xd = torch.from_numpy(s.Xt).cuda()          # p x n rows
            X = Xd.T
            code, ld = cupc.VARIABLE_MAJOR, n
        else:
            X = torch.from_numpy(np.ascontiguousarray(s.X)).cuda()
            code, ld = cupc.SAMPLE_MAJOR, p
        ref = ctx.correlation(X, cupc.F64)
        out = torch.full((p, p), float("nan"), dtype=torch.float64, device="cuda")
        st = _call(L, X, code, n, p, ld, out, stream)
        assert st == 0, st
        err = (out - ref).abs().max().item()
        assert err <= 1e-13, err
        # and against the FP64 oracle on the same values (float32 data widened)
        C_or = oracle.correlation(np.asarray(s.X, dtype=np.float64))
        err_or = np.max(np.abs(out.cpu().numpy() - C_or))
        assert err_or <= 1e-13, err_or
    ctx.close()


def test_noalloc_refuses_oversized_input(cuda_device):
    L = cupc.load()
    stream = torch.cuda.current_stream().cuda_stream
    X = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    # n * p beyond 2^21: refused before any GPU work (the pointers are not read)
    st = L.cupc_correlation_noalloc(ctypes.c_void_p(X.data_ptr()), cupc.F64, cupc.VARIABLE_MAJOR,
                                    1 << 12, 1 << 10, 1 << 12, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream))
    assert st == -5
