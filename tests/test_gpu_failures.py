"""Failure detection without a GPU fault, through the C ABI.

  * A device wait that runs out: LSE_TEST_STALL_NS at context creation makes
    the next evolution's first tile-form step wait on an mbarrier that
    nothing completes.  The bounded wait must give up after the given time,
    drain the copies in flight, report LSE_ERR_TIMEOUT in the statistics,
    and leave the context usable for the next call.
  * A failed allocation: LSE_TEST_FAIL_ALLOC makes the next scratch growth
    fail as a failed cudaMalloc would; the call must return LSE_ERR_OOM and
    the next one succeed.

Neither traps, faults or hangs the GPU: the stalled wait is bounded by a
50 ms clock limit, and the allocation failure happens on the host.
"""
import os
import time

import numpy as np
import pytest

import oracle
from paper_1409_7474_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def lse():
    import paper_1409_7474_gb300.lse as m
    return m


def context_with(lse, var, value, **kw):
    os.environ[var] = value
    try:
        return lse.Context(0, **kw)
    finally:
        del os.environ[var]


def test_device_wait_that_runs_out_reports_timeout(torch, lse):
    img, _, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    x = torch.from_numpy(img).cuda()
    p = torch.from_numpy(phi0).cuda()
    ctx = context_with(lse, "LSE_TEST_STALL_NS", "50000000", max_pixels=256 * 256, max_bands=1)
    try:
        t0 = time.perf_counter()
        _, _, st = ctx.evolve(x, p, iterations=5)
        torch.cuda.synchronize()
        assert st["status"] == "LSE_ERR_TIMEOUT"
        assert time.perf_counter() - t0 < 10.0
        # the hook is spent: the same context evolves normally afterwards
        v, _, st = ctx.evolve(x, p, iterations=1)
        torch.cuda.synchronize()
        assert st["status"] == "LSE_OK"
        v_ref, *_ = oracle.step(img, phi0)
        assert np.abs(v.cpu().numpy() - v_ref).max() <= 1e-5
    finally:
        ctx.destroy()


def test_failed_allocation_reports_oom_and_the_next_call_succeeds(torch, lse):
    img, _, _ = scenes.rect_scene(128, 160, 60, 40)
    phi0 = scenes.circle_phi(128, 160, radius=40)
    # host buffers: the first call must grow the context's staging buffers
    ctx = context_with(lse, "LSE_TEST_FAIL_ALLOC", "1", max_pixels=128 * 160, max_bands=1)
    try:
        with pytest.raises(lse.LseError) as e:
            ctx.evolve(img, phi0, iterations=2)
        assert e.value.status == lse.LSE_ERR_OOM
        assert b"cudaMalloc" in lse.raw_library().lse_last_error(ctx._h)
        v, _, st = ctx.evolve(img, phi0, iterations=1)
        assert st["status"] == "LSE_OK"
        v_ref, *_ = oracle.step(img, phi0)
        assert np.abs(v - v_ref).max() <= 1e-5
    finally:
        ctx.destroy()
