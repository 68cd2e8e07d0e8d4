"""lse_evolve_batch: uneven images advanced together, vs lse_evolve alone and
vs the FP64 oracle.

Every image of a batch keeps its own planes, statistics, CTA count,
iteration cap and early stop, so its results must equal lse_evolve's on the
same image bit for bit, with and without CUDA-graph capture (for vector
images: lse_evolve on the band passes, which batches take too).  lse_evolve is
itself held to the oracle by the parity tests; a few small batch images are
also compared with the oracle directly (mask parity, the early stop's
iteration count).
"""
import ctypes

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


@pytest.fixture(scope="module")
def ctx(lse, torch):
    c = lse.Context(0, max_pixels=1024 * 1024, max_bands=4)
    yield c
    c.destroy()


def device_items(torch, ctx, probs):
    """The work list on the device; the edge images get g from the library."""
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


def single(torch, ctx, it):
    # vector images in a batch run as a group of persistent evolutions, each
    # with its own share of the CTAs: the bits of one call alone
    v, m, st = ctx.evolve(it.get("image"), it["phi0"], it["term"], g=it.get("g"),
                          iterations=it["iterations"],
                          early_stop_frac=it["early_stop_frac"], storage=it["storage"])
    torch.cuda.synchronize()
    return v.cpu().numpy(), m.cpu().numpy(), st


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_single_calls(torch, ctx, use_graph):
    probs = scenes.batch_problems(24, seed=11, min_side=40, max_side=400, cap_range=(3, 40))
    for k, q in enumerate(probs):        # half with the early stop, half without
        if k % 2:
            q["early_stop_frac"] = 0.0
    items = device_items(torch, ctx, probs)
    res = ctx.evolve_batch(items, use_graph=use_graph)
    torch.cuda.synchronize()
    for it, (v, m, st) in zip(items, res):
        v1, m1, st1 = single(torch, ctx, it)
        assert same_bits(v.cpu().numpy(), v1)
        assert np.array_equal(m.cpu().numpy(), m1)
        for key in ("iterations_run", "last_flips", "area_plus", "status"):
            assert st[key] == st1[key], key
        assert st["c_plus"] == st1["c_plus"] and st["c_minus"] == st1["c_minus"]


def with_16bit_storage(probs):
    """BF16 and F16 storage, alternating, for the images 16-bit storage
    serves (one band, or the edge term); FP32 for the 4-band region images."""
    k = 0
    for q in probs:
        if q["term"] == "edge" or q["image"].shape[0] == 1:
            q["storage"] = ("bf16", "f16")[k % 2]
            k += 1
    return probs


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_16bit_storage_equals_single_calls(torch, ctx, use_graph):
    probs = with_16bit_storage(scenes.batch_problems(20, seed=13, min_side=40, max_side=400,
                                                     cap_range=(3, 40)))
    assert sum(q.get("storage", "f32") != "f32" for q in probs) >= 8
    items = device_items(torch, ctx, probs)
    res = ctx.evolve_batch(items, use_graph=use_graph)
    torch.cuda.synchronize()
    for it, (v, m, st) in zip(items, res):
        v1, m1, st1 = single(torch, ctx, it)
        assert same_bits(v.cpu().numpy(), v1), it["storage"]
        assert np.array_equal(m.cpu().numpy(), m1)
        for key in ("iterations_run", "last_flips", "area_plus", "status"):
            assert st[key] == st1[key], key
        assert st["c_plus"] == st1["c_plus"] and st["c_minus"] == st1["c_minus"]


def test_batch_against_oracle(torch, ctx):
    probs = scenes.batch_problems(6, seed=5, min_side=48, max_side=160, cap_range=(10, 30))
    items = device_items(torch, ctx, probs)
    res = ctx.evolve_batch(items, use_graph=True)
    torch.cuda.synchronize()
    for q, (v, m, st) in zip(probs, res):
        if q["term"] == "region":
            _, m_ref, st_ref = oracle.evolve(q["image"], q["phi0"], iterations=q["iterations"],
                                             early_stop_frac=q["early_stop_frac"])
        else:
            g = oracle.edge_indicator(q["image"], 1.0, 9, 255.0)
            _, m_ref, st_ref = oracle.evolve(q["image"], q["phi0"], term="edge", g=g,
                                             iterations=q["iterations"],
                                             early_stop_frac=q["early_stop_frac"])
        assert st["iterations_run"] == st_ref["iterations_run"]
        assert_mask_parity(m.cpu().numpy(), m_ref)


def test_uneven_caps_and_early_stop(torch, ctx):
    """Images stop at their own caps; a converged image stops early while the
    others go on."""
    img, truth, _ = scenes.rect_scene(noise=0.0)
    phi_t = np.where(truth, 1.0, -1.0).astype(np.float32)
    img2, _, _ = scenes.rect_scene(96, 128, 40, 30)
    x, x2 = torch.from_numpy(img).cuda(), torch.from_numpy(img2).cuda()
    items = [
        {"image": x, "phi0": torch.from_numpy(phi_t).cuda(), "iterations": 50,
         "early_stop_frac": 1e-4},
        {"image": x2, "phi0": torch.from_numpy(scenes.circle_phi(96, 128, radius=30)).cuda(),
         "iterations": 7},
        {"image": x2, "phi0": torch.from_numpy(scenes.circle_phi(96, 128, radius=30)).cuda(),
         "iterations": 13},
    ]
    res = ctx.evolve_batch(items)
    torch.cuda.synchronize()
    assert [r[2]["iterations_run"] for r in res] == [1, 7, 13]
    assert np.array_equal(res[0][1].cpu().numpy().astype(bool), truth)
    _, m7, _ = oracle.evolve(img2, scenes.circle_phi(96, 128, radius=30), iterations=7)
    assert_mask_parity(res[1][1].cpu().numpy(), m7)


def test_batch_rejections(torch, lse, ctx):
    lib = lse.raw_library()
    x = torch.rand((1, 64, 64), device="cuda")
    phi = torch.ones((64, 64), device="cuda")
    out = torch.empty_like(phi)

    def run(image, params, phi0=phi):
        probs = (lse.Problem * 1)()
        probs[0] = lse.Problem(ctypes.c_void_p(image.data_ptr()), lse.F32, 64, 64, 1, None,
                               ctypes.c_void_p(phi0.data_ptr()), params,
                               ctypes.c_void_p(out.data_ptr()), None)
        return lib.lse_evolve_batch(ctx._h, 1, probs, 1, None, None)

    ok = lse.Params(lse.TERM_REGION, 15.0, 1.0, 9, 3, 1, 0.0, lse.F32)
    assert run(x, ok) == lse.LSE_OK
    big_ts = lse.Params(lse.TERM_REGION, 15.0, 1.0, 17, 3, 1, 0.0, lse.F32)
    assert run(x, big_ts) == lse.LSE_ERR_INVALID_ARG
    assert b"plain step kernel" in lib.lse_last_error(ctx._h)
    half = lse.Params(lse.TERM_REGION, 15.0, 1.0, 9, 3, 1, 0.0, lse.BF16)
    assert run(x, half) == lse.LSE_OK
    table1 = lse.Params(lse.TERM_REGION, 15.0, 1.0, 9, 3, 1, 0.0, lse.F32, 1, 0)
    assert run(x, table1) == lse.LSE_ERR_INVALID_ARG
    assert b"order" in lib.lse_last_error(ctx._h)
    host_phi = torch.ones((64, 64))
    assert run(x, ok, phi0=host_phi) == lse.LSE_ERR_INVALID_ARG
    assert b"device memory" in lib.lse_last_error(ctx._h)


@pytest.mark.parametrize("use_graph", [True, False])
def test_vector_images_beyond_one_group_launch(torch, ctx, use_graph):
    # 320 small 4-band images: more than one cooperative launch holds (two
    # CTAs per SM), so they run as several group launches; each image's
    # bits are those of one call alone, and a batch of vector images only
    # has no per-iteration launches at all
    probs = scenes.batch_problems(320, seed=17, min_side=24, max_side=72, cap_range=(2, 9))
    for q in probs:
        q["image"] = np.ascontiguousarray(np.repeat(q["image"][:1], 4, axis=0) *
                                          np.array([1.0, 0.9, 0.8, 0.7], np.float32)[:, None, None])
        q["term"] = "region"
        q["early_stop_frac"] = 0.0
    items = device_items(torch, ctx, probs)
    res = ctx.evolve_batch(items, use_graph=use_graph)
    torch.cuda.synchronize()
    for k in range(0, len(items), 23):
        v, m, st = res[k]
        v1, m1, st1 = single(torch, ctx, items[k])
        assert same_bits(v.cpu().numpy(), v1)
        assert np.array_equal(m.cpu().numpy(), m1)
        assert st["iterations_run"] == st1["iterations_run"] == items[k]["iterations"]
        assert st["c_plus"] == st1["c_plus"]


def test_vector_groups_by_band_count_and_radius(torch, ctx):
    # 2, 3 and 4 bands at two template sizes, with and without the early
    # stop: one group launch per (bands, radius), every image lse_evolve's bits
    probs = scenes.batch_problems(18, seed=29, min_side=40, max_side=180, cap_range=(5, 30))
    for k, q in enumerate(probs):
        B = 2 + k % 3
        q["image"] = np.ascontiguousarray(np.repeat(q["image"][:1], B, axis=0) *
                                          np.linspace(1.0, 0.6, B, dtype=np.float32)[:, None, None])
        q["term"] = "region"
        q["early_stop_frac"] = 0.0 if k % 2 else 2e-3
    items = device_items(torch, ctx, probs)
    for k, it in enumerate(items):
        it["ts"] = 9 if k % 4 < 2 else 7
    res = ctx.evolve_batch(items, use_graph=False)
    torch.cuda.synchronize()
    for it, (v, m, st) in zip(items, res):
        v1, m1, st1 = ctx.evolve(it["image"], it["phi0"], "region", ts=it["ts"],
                                 iterations=it["iterations"],
                                 early_stop_frac=it["early_stop_frac"])
        torch.cuda.synchronize()
        assert same_bits(v.cpu().numpy(), v1.cpu().numpy())
        assert st["iterations_run"] == st1["iterations_run"]
        assert st["last_flips"] == st1["last_flips"]
