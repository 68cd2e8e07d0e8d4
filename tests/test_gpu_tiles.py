"""The tile-form step with 32-row tiles (4 warps per CTA) and the tile-height
autotuner, through the C ABI.

Tile height only regroups the work: every pixel's u, h and v are computed by
the same arithmetic whichever tile holds it, so one step gives the same bits
with 32- and 64-row tiles; the region statistics are summed per tile, so
later steps may differ in the last bits of c+ / c-.  32-row tiles are held
to the oracle with the parity tests' bars (|v - v_oracle| <= 1e-5 after one
step; masks within 0.05 % and 1 px of the oracle's contour), and an
autotuned context must still give batched and served images the bits
lse_evolve gives them.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from _parity import assert_mask_parity, is_vector_region, mask_report, step_launches
from paper_1409_7474_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V = 1e-5
SHAPES = [(1, 17), (17, 1), (37, 53), (64, 129), (130, 250), (300, 121), (241, 360)]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def lse():
    import paper_1409_7474_gb300.lse as m
    return m


@pytest.fixture(scope="module")
def ctx64(torch, lse):
    # 64-row tiles even for images the automatic choice gives 32-row tiles
    os.environ["LSE_TILE_ROWS"] = "64"
    try:
        c = lse.Context(0, max_pixels=1024 * 1024, max_bands=4)
    finally:
        del os.environ["LSE_TILE_ROWS"]
    yield c
    c.destroy()


@pytest.fixture(scope="module")
def ctx32(torch, lse):
    # LSE_TILE_ROWS is read once, at context creation
    os.environ["LSE_TILE_ROWS"] = "32"
    try:
        c = lse.Context(0, max_pixels=1024 * 1024, max_bands=4)
    finally:
        del os.environ["LSE_TILE_ROWS"]
    yield c
    c.destroy()


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rng_scene(H, W, seed):
    r = np.random.default_rng(seed)
    img = 0.3 + 0.4 * (r.random((1, H, W)) < 0.3) + 0.05 * r.standard_normal((1, H, W))
    return img.astype(np.float32)


def run(torch, ctx, img, phi0, g=None, **kw):
    x = dev(torch, img) if kw.get("term", "region") == "region" else None
    v, m, st = ctx.evolve(x, dev(torch, phi0), g=g, **kw)
    torch.cuda.synchronize()
    return v.cpu().numpy(), m.cpu().numpy(), st


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("term", ["region", "edge"])
@pytest.mark.parametrize("H,W", SHAPES)
def test_32_row_tiles_match_64_row_tiles_and_the_oracle(torch, ctx32, ctx64, storage, term,
                                                        H, W):
    img = rng_scene(H, W, 3 * H + W)
    phi0 = np.where(np.random.default_rng(H * W).random((H, W)) < 0.5,
                    1.0, -1.0).astype(np.float32)
    g = g_ref = None
    if term == "edge":
        g = ctx64.precompute_edge(dev(torch, img), 1.0, 9, 255.0)
        g_ref = oracle.edge_indicator(img, 1.0, 9, 255.0)
    kw = dict(term=term, storage=storage)
    v32, _, _ = run(torch, ctx32, img, phi0, g=g, iterations=1, **kw)
    v64, _, _ = run(torch, ctx64, img, phi0, g=g, iterations=1, **kw)
    assert same_bits(v32, v64)
    if storage == "f32":
        v_ref, *_ = oracle.step(img, phi0, term, g_ref)
        assert np.abs(v32 - v_ref).max() <= TOL_V
    # several steps run the +-1 steady-state kernels; statistics are summed
    # per tile, so allow the parity bar between the two tilings
    _, m32, st32 = run(torch, ctx32, img, phi0, g=g, iterations=6, **kw)
    _, m64, st64 = run(torch, ctx64, img, phi0, g=g, iterations=6, **kw)
    rep = mask_report(m32, m64)
    assert rep["far"] == 0 and rep["disagree"] <= max(2, int(5e-4 * H * W)), rep
    assert st32["status"] == "LSE_OK"


@pytest.mark.parametrize("ts", [3, 5, 7, 9, 11, 13, 15])
def test_32_row_tiles_template_sizes(torch, ctx32, ts):
    img = rng_scene(200, 300, ts)
    phi0 = scenes.circle_phi(200, 300, radius=60)
    v, _, _ = run(torch, ctx32, img, phi0, sigma=2.0, ts=ts, iterations=1)
    v_ref, *_ = oracle.step(img, phi0, sigma=2.0, ts=ts)
    assert np.abs(v - v_ref).max() <= TOL_V


@pytest.mark.parametrize("term", ["region", "edge"])
def test_32_row_tiles_rectangle_200_iterations(torch, ctx32, term):
    img, _, _ = scenes.rect_scene()
    if term == "region":
        phi0 = scenes.circle_phi(256, 256)
        _, m, st = run(torch, ctx32, img, phi0, iterations=200)
        _, m_ref, _ = oracle.evolve(img, phi0, iterations=200)
    else:
        phi0 = scenes.box_phi(256, 256, [(20, 20, 236, 236)])
        g = ctx32.precompute_edge(dev(torch, img), 1.0, 9, 255.0)
        _, m, st = run(torch, ctx32, img, phi0, g=g, term="edge", iterations=200)
        g_ref = oracle.edge_indicator(img, 1.0, 9, 255.0)
        _, m_ref, _ = oracle.evolve(img, phi0, "edge", g=g_ref, iterations=200)
    assert st["iterations_run"] == 200
    assert_mask_parity(m, m_ref)


def device_items(torch, ctx, probs):
    items = []
    for q in probs:
        img = torch.from_numpy(q["image"]).cuda()
        it = {"phi0": torch.from_numpy(q["phi0"]).cuda(), "term": q["term"],
              "iterations": q["iterations"], "early_stop_frac": q["early_stop_frac"],
              "storage": q.get("storage", "f32")}
        if q["term"] == "region":
            it["image"] = img
        else:
            it["g"] = ctx.precompute_edge(img, 1.0, 9, 255.0)
        items.append(it)
    torch.cuda.synchronize()
    return items


def test_autotuned_context_keeps_batch_and_server_equal_to_evolve(torch, lse):
    probs = scenes.batch_problems(14, seed=31, min_side=40, max_side=600, cap_range=(3, 30))
    for k, q in enumerate(probs):
        if q["term"] == "edge" or q["image"].shape[0] == 1:
            q["storage"] = ("f32", "bf16")[k % 2]
    with lse.Context(0, max_pixels=1024 * 1024, max_bands=4) as ctx:
        items = device_items(torch, ctx, probs)
        rows = ctx.autotune(items, iterations=6)
        for q, r in zip(probs, rows):
            # every problem here has at most 4 bands and TS 9: all tile form
            assert r in (32, 64), (q["term"], q["image"].shape, r)
        # the tuner wrote to scratch, not to the problems' outputs
        res = ctx.evolve_batch(items, use_graph=True)
        sv = lse.Server(ctx, 256 << 20)
        ids = [sv.submit(it) for it in items]
        served = {}
        for _ in range(200):
            for rid in ids:
                if rid not in served:
                    out = sv.poll(rid)
                    if out is not None:
                        served[rid] = out
            if len(served) == len(ids):
                break
            sv.advance(8)
        sv.destroy()
        assert len(served) == len(ids)
        def alone(it, per_step):
            with step_launches(per_step):
                v1, m1, st1 = ctx.evolve(it.get("image"), it["phi0"], it["term"],
                                         g=it.get("g"), iterations=it["iterations"],
                                         early_stop_frac=it["early_stop_frac"],
                                         storage=it["storage"])
            torch.cuda.synchronize()
            return v1.cpu().numpy(), st1

        for it, (v, m, st), rid in zip(items, res, ids):
            # batches and the server give every image lse_evolve's bits
            v1, st1 = alone(it, False)
            assert same_bits(v.cpu().numpy(), v1)
            assert st["iterations_run"] == st1["iterations_run"]
            assert st["c_plus"] == st1["c_plus"]
            assert same_bits(served[rid][0].cpu().numpy(), v1)


def test_autotune_rejects_bad_arguments(torch, lse, ctx64):
    lib = lse.raw_library()
    probs = (lse.Problem * 1)()
    rows = (ctypes.c_int * 1)()
    assert lib.lse_autotune(ctx64._h, 0, probs, 4, rows, None) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_autotune(ctx64._h, 1, probs, 0, rows, None) == lse.LSE_ERR_INVALID_ARG
    assert lib.lse_autotune(None, 1, probs, 4, rows, None) == lse.LSE_ERR_INVALID_ARG
    x = torch.rand((1, 64, 64), device="cuda")
    phi = torch.ones((64, 64))                  # host memory: refused by the batch checks
    with pytest.raises(lse.LseError, match="device memory"):
        ctx64.autotune([{"image": x, "phi0": phi, "iterations": 3}])
