"""CPU-side checks of the C-ABI library: it loads, exports every declared
entry point, and its host-only functions behave (no GPU compute here)."""
import ctypes
import math
import os
import re

import pytest
from scipy.special import ndtri

import paper_1812_08491_gb300 as cupc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cupc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cupc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    cupc.build_library()
    return cupc.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(cupc.exported_symbols()) == declared


def test_library_is_sm103a_only():
    # the build requests only sm_103a code
    from paper_1812_08491_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_options_default(lib):
    o = cupc.Options()
    lib.cupc_options_default(ctypes.byref(o))
    assert o.mode == cupc.MODE_FP32_RECHECK and o.canonical_sepset == 1 and o.max_level == -1


@pytest.mark.parametrize("alpha,n,l", [(0.01, 1000, 0), (0.01, 10000, 1), (0.05, 200, 3), (1e-6, 50, 5)])
def test_fisher_threshold_vs_scipy(lib, alpha, n, l):
    tau, r = cupc.fisher_threshold(alpha, n, l)
    ref = -ndtri(alpha / 2) / math.sqrt(n - l - 3)  # same value; avoids rounding 1 - alpha/2
    assert tau == pytest.approx(ref, rel=2e-15)
    assert r == pytest.approx(math.tanh(ref), rel=2e-15)


def test_fisher_threshold_rejects_bad_args(lib):
    with pytest.raises(cupc.CupcError):
        cupc.fisher_threshold(0.0, 100, 0)
    with pytest.raises(cupc.CupcError):
        cupc.fisher_threshold(0.01, 5, 2)


def test_create_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.cupc_create(ctypes.byref(h), 0, None)
    assert st == -3 and not h.value


def test_result_entry_points_reject_null_results(lib):
    """The result accessors and the orientation step check their arguments
    before any CUDA work (CUPC_E_INVALID = -1)."""
    n = ctypes.c_int64()
    assert lib.cupc_result_orient(None, None, None) == -1
    assert lib.cupc_result_edges(None, None, 0, ctypes.byref(n)) == -1
    assert lib.cupc_result_sepset_records(None, None, 0, ctypes.byref(n)) == -1
    assert lib.cupc_result_adjacency(None, None) == -1


def test_control_entry_points_reject_null(lib):
    """Cancellation, fault injection, checkpoint and resume check their
    arguments before any CUDA work."""
    n = ctypes.c_int64()
    assert lib.cupc_cancel(None) == -1
    assert lib.cupc_debug_fail(None, cupc.FAIL_ALLOC, 1) == -1
    assert lib.cupc_result_checkpoint(None, None, 0, ctypes.byref(n)) == -1
    out = ctypes.c_void_p()
    assert lib.cupc_skeleton_resume(None, None, 0, 0, 0, 10, 2, 2, 0.01, None, None, 0, ctypes.byref(out)) == -1
