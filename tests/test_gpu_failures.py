"""Failure handling and level-boundary checkpoints, on the GPU.

Every failure here is made on the host or by a bounded device wait that runs
out; none faults, traps or hangs the GPU:
  * cancellation (cupc_cancel): the call stops between levels with
    CUPC_E_CANCELLED;
  * an injected allocation or launch failure (cupc_debug_fail): the call
    returns CUPC_E_NOMEM / CUPC_E_CUDA without doing that allocation or launch;
  * a grid-barrier wait that nothing ends: in the first level kernel of the
    call CTA 0 never arrives at the first grid barrier, the other CTAs give up
    after 50 us (their bounded wait runs out) and the call returns
    CUPC_E_TIMEOUT.
After each, the same context runs the skeleton again and matches the oracle.
Checkpoints: a run stopped after level k and resumed from its checkpoint gives
the skeleton, removal levels, SepSets and serial counts of the oracle's
uninterrupted run.
"""
import numpy as np
import pytest

cupc = pytest.importorskip("paper_1812_08491_gb300")
torch = pytest.importorskip("torch")

import oracle
from synth import sem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(cuda_device):
    c = cupc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def prob():
    s = sem.generate(400, 2000, 7301, "random", degree=3.0)
    C = oracle.correlation(s.X, nthreads=8)
    return s, oracle.pc_stable(C, s.n, s.alpha, nthreads=8)


def _assert_same(res, ref):
    assert np.array_equal(res.adjacency(), ref.adj)
    assert np.array_equal(res.sep_levels(), ref.sep_level)
    assert res.sepsets() == ref.sepsets
    assert res.stats()["serial_tests"][:ref.levels_run] == list(ref.tests)


def _status(exc):
    return exc.value.status


def test_cancel_between_levels(ctx, prob):
    s, ref = prob
    ctx.cancel()
    with pytest.raises(cupc.CupcError) as e:
        ctx.skeleton(s.X, s.alpha)
    assert _status(e) == -7
    assert "cancelled" in ctx.last_error()
    _assert_same(ctx.skeleton(s.X, s.alpha), ref)       # the request was consumed


@pytest.mark.parametrize("k", [1, 2, 3])
def test_injected_allocation_failure(ctx, prob, k):
    s, ref = prob
    ctx.skeleton(s.X, s.alpha).free()                    # workspace already sized
    ctx.debug_fail(cupc.FAIL_ALLOC, k)
    with pytest.raises(cupc.CupcError) as e:
        ctx.skeleton(s.X, s.alpha)
    assert _status(e) == -2 and "injected" in ctx.last_error()
    _assert_same(ctx.skeleton(s.X, s.alpha), ref)


@pytest.mark.parametrize("k", [1, 3, 5, 6])
def test_injected_launch_failure(ctx, prob, k):
    s, ref = prob
    ctx.debug_fail(cupc.FAIL_LAUNCH, k)
    with pytest.raises(cupc.CupcError) as e:
        ctx.skeleton(s.X, s.alpha)
    assert _status(e) == -3 and "injected" in ctx.last_error()
    _assert_same(ctx.skeleton(s.X, s.alpha), ref)


@pytest.mark.parametrize("mode", [cupc.MODE_FP32_RECHECK, cupc.MODE_PLAIN_FP64])
def test_barrier_wait_expiry(ctx, prob, mode):
    s, ref = prob
    ctx.debug_fail(cupc.FAIL_BARRIER, 50000)
    with pytest.raises(cupc.CupcError) as e:
        ctx.skeleton(s.X, s.alpha, mode=mode)
    assert _status(e) == -4, ctx.last_error()
    _assert_same(ctx.skeleton(s.X, s.alpha, mode=mode), ref)


def test_debug_fail_arguments(ctx):
    with pytest.raises(cupc.CupcError):
        ctx.debug_fail(7, 1)
    with pytest.raises(cupc.CupcError):
        ctx.debug_fail(cupc.FAIL_ALLOC, 0)
    with pytest.raises(cupc.CupcError):
        ctx.debug_fail(cupc.FAIL_BARRIER, 10)              # below the 1 us floor
    ctx.debug_fail(cupc.FAIL_LAUNCH, 5)
    ctx.debug_fail(cupc.FAIL_NONE, 0)                     # disarmed: the next call runs
    ctx.skeleton(sem.workload("small20").X, 0.01).free()


@pytest.mark.parametrize("mode", [cupc.MODE_FP32_RECHECK, cupc.MODE_PLAIN_FP64])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_checkpoint_resume(ctx, prob, mode, k):
    s, ref = prob
    part = ctx.skeleton(s.X, s.alpha, mode=mode, max_level=k)
    assert part.stats()["levels"] == min(k + 1, ref.levels_run)
    ck = part.checkpoint()
    part.free()
    res = ctx.skeleton_resume(s.X, s.alpha, ck, mode=mode)
    _assert_same(res, ref)
    assert res.stats()["levels"] == ref.levels_run
    # resuming a finished run changes nothing
    ck2 = res.checkpoint()
    again = ctx.skeleton_resume(s.X, s.alpha, ck2, mode=mode)
    _assert_same(again, ref)


def test_checkpoint_resume_device_input_and_max_level(ctx, prob):
    """Device-resident data, and a resume that itself stops at a level and is
    resumed again (levels 0-1, 2-3, then to the end)."""
    s, ref = prob
    Xd = torch.from_numpy(s.Xt).cuda().T
    a = ctx.skeleton(Xd, s.alpha, max_level=1)
    b = ctx.skeleton_resume(Xd, s.alpha, a.checkpoint(), max_level=3)
    assert b.stats()["levels"] == min(4, ref.levels_run)
    c = ctx.skeleton_resume(Xd, s.alpha, b.checkpoint())
    _assert_same(c, ref)


def test_checkpoint_rejected(ctx, prob):
    s, ref = prob
    ck = ctx.skeleton(s.X, s.alpha, max_level=1).checkpoint()
    bad = [b"", ck[:100], b"X" + ck[1:], ck + b"\0"]
    for blob in bad:
        with pytest.raises(cupc.CupcError) as e:
            ctx.skeleton_resume(s.X, s.alpha, blob)
        assert _status(e) == -1
    with pytest.raises(cupc.CupcError):
        ctx.skeleton_resume(s.X, s.alpha * 2, ck)             # another alpha
    with pytest.raises(cupc.CupcError):
        ctx.skeleton_resume(s.X, s.alpha, ck, mode=cupc.MODE_PLAIN_FP64)   # other options
    with pytest.raises(cupc.CupcError):
        ctx.skeleton_resume(s.X, s.alpha, ck, max_level=0)   # below the checkpoint's level
