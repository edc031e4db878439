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


@pytest.mark.parametrize("cname,pyname", [("cupc_options", "Options"), ("cupc_stats", "Stats"),
                                          ("cupc_tune_entry", "TuneEntry"), ("cupc_orient_stats", "OrientStats"),
                                          ("cupc_sshare_stats", "SShareStats")])
def test_binding_structs_match_the_header(tmp_path, cname, pyname):
    """The ctypes structures of the binding have the C header's size and field
    offsets (a field added on one side only would shift every later one)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    cls = getattr(cupc, pyname)
    names = [f[0] for f in cls._fields_]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cupc.h"', "int main(void) {",
             '    printf("%%zu\\n", sizeof(%s));' % cname]
    lines += ['    printf("%%zu\\n", offsetof(%s, %s));' % (cname, nm) for nm in names]
    lines += ["    return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(cls)] + [getattr(cls, nm).offset for nm in names]
    assert got == want, (cname, list(zip(["sizeof"] + names, got, want)))
