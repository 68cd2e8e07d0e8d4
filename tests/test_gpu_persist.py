"""The persistent evolution against one launch per step, through the C ABI.

lse_evolve runs every iteration of a one-band or edge-term evolution on the
tile form in one cooperative launch whose CTAs meet at a grid barrier after
each step; LSE_PERSIST=0 (read at every call) makes it launch one kernel per
step instead, as batches and the server do.  Both take tiles in the same way
and add the statistics as exact integers, so they must give the same bits:
v, mask and every statistic, for both terms, both tile heights, 16-bit
storage, re-initialisation periods and early stops.  The oracle comparison of
the default (persistent) path is in the other parity tests.
"""
import os

import numpy as np
import pytest

import oracle
from _parity import assert_mask_parity
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


def run_both(torch, ctx, img, phi0, **kw):
    out = {}
    for mode in ("1", "0"):
        os.environ["LSE_PERSIST"] = mode
        try:
            v, m, st = ctx.evolve(img, phi0, **kw)
            torch.cuda.synchronize()
        finally:
            os.environ.pop("LSE_PERSIST", None)
        out[mode] = (v.cpu().numpy(), m.cpu().numpy(), st)
    return out["1"], out["0"]


def assert_same(a, b):
    va, ma, sa = a
    vb, mb, sb = b
    assert np.array_equal(va.view(np.uint32), vb.view(np.uint32))
    assert np.array_equal(ma, mb)
    for k in ("iterations_run", "last_flips", "area_plus", "c_plus", "c_minus", "norm",
              "status"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])


@pytest.mark.parametrize("rows", ["32", "64"])
@pytest.mark.parametrize("H,W", [(256, 256), (300, 412), (1030, 770)])
@pytest.mark.parametrize("term", ["region", "edge"])
def test_persistent_equals_one_launch_per_step(torch, lse, rows, H, W, term):
    os.environ["LSE_TILE_ROWS"] = rows
    try:
        ctx = lse.Context(0, max_pixels=H * W, max_bands=1)
    finally:
        os.environ.pop("LSE_TILE_ROWS", None)
    with ctx:
        img, _, _ = scenes.rect_scene(H, W, W // 3, H // 4, noise=0.05)
        x = torch.from_numpy(img).cuda()
        if term == "region":
            phi0 = torch.from_numpy(scenes.circle_phi(H, W, radius=min(H, W) / 3)).cuda()
            a, b = run_both(torch, ctx, x, phi0, term="region", iterations=37)
        else:
            g = ctx.precompute_edge(x, 1.0, 9, 255.0)
            phi0 = torch.from_numpy(scenes.box_phi(H, W, [(8, 8, H - 8, W - 8)])).cuda()
            a, b = run_both(torch, ctx, None, phi0, term="edge", g=g, iterations=37)
        assert_same(a, b)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_persistent_16bit_storage(torch, lse, storage):
    with lse.Context(0, max_pixels=600 * 500, max_bands=1) as ctx:
        img, _, _ = scenes.rect_scene(600, 500, 200, 90, noise=0.05)
        x = torch.from_numpy(img).cuda()
        phi0 = torch.from_numpy(scenes.circle_phi(600, 500, radius=150)).cuda()
        a, b = run_both(torch, ctx, x, phi0, term="region", iterations=25, storage=storage)
        assert_same(a, b)


@pytest.mark.parametrize("period", [0, 3])
def test_persistent_reinit_period(torch, lse, period):
    with lse.Context(0, max_pixels=256 * 256, max_bands=1) as ctx:
        img, _, _ = scenes.rect_scene()
        x = torch.from_numpy(img).cuda()
        phi0 = torch.from_numpy(scenes.circle_phi(256, 256)).cuda()
        a, b = run_both(torch, ctx, x, phi0, term="region", iterations=20,
                        reinit_period=period)
        assert_same(a, b)
        v_ref, m_ref, _ = oracle.evolve(img, scenes.circle_phi(256, 256), iterations=20,
                                        reinit_period=period)
        assert_mask_parity(a[1], m_ref)


def test_persistent_early_stop(torch, lse):
    # the noiseless truth is a fixed point: the evolution stops after one
    # iteration on both paths, with no sign change
    img, truth, _ = scenes.rect_scene(noise=0.0)
    phi_t = np.where(truth, 1.0, -1.0).astype(np.float32)
    with lse.Context(0, max_pixels=256 * 256, max_bands=1) as ctx:
        x = torch.from_numpy(img).cuda()
        p = torch.from_numpy(phi_t).cuda()
        a, b = run_both(torch, ctx, x, p, term="region", iterations=50, early_stop_frac=1e-4)
        assert_same(a, b)
        assert a[2]["iterations_run"] == 1 and a[2]["last_flips"] == 0
        # a run that stops later: on the noisy scene the sign changes per
        # iteration fall from about 590 to a plateau near 460 (oracle), so a
        # threshold of 500 is reached after a dozen or more iterations
        img, _, _ = scenes.rect_scene(noise=0.05)
        x = torch.from_numpy(img).cuda()
        p = torch.from_numpy(scenes.circle_phi(256, 256)).cuda()
        frac = 500.0 / (256 * 256)
        a, b = run_both(torch, ctx, x, p, term="region", iterations=300, early_stop_frac=frac)
        assert_same(a, b)
        assert 1 < a[2]["iterations_run"] < 300
        assert a[2]["last_flips"] < 500


def test_kernel_launch_count(torch, lse):
    # the persistent path enqueues the prologue, one kernel for every
    # iteration and the output; one launch per step enqueues one per iteration
    img, _, _ = scenes.rect_scene()
    with lse.Context(0, max_pixels=256 * 256, max_bands=1) as ctx:
        x = torch.from_numpy(img).cuda()
        p = torch.from_numpy(scenes.circle_phi(256, 256)).cuda()
        n0 = ctx.kernel_launches()
        ctx.evolve(x, p, "region", iterations=40)
        n1 = ctx.kernel_launches()
        os.environ["LSE_PERSIST"] = "0"
        try:
            ctx.evolve(x, p, "region", iterations=40)
        finally:
            os.environ.pop("LSE_PERSIST", None)
        n2 = ctx.kernel_launches()
        g = ctx.precompute_edge(x, 1.0, 9, 255.0)
        n3 = ctx.kernel_launches()
        assert (n1 - n0, n2 - n1, n3 - n2) == (3, 42, 1)
