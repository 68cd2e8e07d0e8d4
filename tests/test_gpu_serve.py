"""lse_server: continuous batching of requests within a memory budget.

Requests join a running mix at different launch indices, share its batched
launches, and leave when they reach their cap or stop early.  Each keeps the
CTA count, statistics and reductions lse_evolve gives it alone, so every
served result must equal lse_evolve's on the same image bit for bit,
whatever else ran beside it.
"""
import ctypes

import numpy as np
import pytest

from _parity import is_vector_region, step_launches
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


def alone(torch, ctx, it):
    # vector images on the server take the band passes: so does the call alone
    with step_launches(is_vector_region(it)):
        v, m, st = ctx.evolve(it.get("image"), it["phi0"], it["term"], g=it.get("g"),
                              iterations=it["iterations"],
                              early_stop_frac=it["early_stop_frac"], storage=it["storage"])
    torch.cuda.synchronize()
    return v.cpu().numpy(), m.cpu().numpy(), st


def drain(server, ids, results, max_rounds=500, ticks=10):
    for _ in range(max_rounds):
        for rid in ids:
            if rid not in results:
                r = server.poll(rid)
                if r is not None:
                    results[rid] = r
        if len(results) == len(ids):
            return
        server.advance(ticks)
    raise AssertionError("requests did not finish")


def test_served_results_equal_alone(torch, lse, ctx):
    probs = scenes.batch_problems(16, seed=21, min_side=40, max_side=300, cap_range=(4, 60))
    for k, q in enumerate(probs):
        if k % 3 == 0:
            q["early_stop_frac"] = 0.0
    items = device_items(torch, ctx, probs)
    sv = lse.Server(ctx, 512 << 20)
    ids, results = [], {}
    # requests arrive in three waves while earlier ones are mid-evolution
    for it in items[:6]:
        ids.append(sv.submit(it))
    sv.advance(7)
    for it in items[6:11]:
        ids.append(sv.submit(it))
    sv.advance(3)
    for it in items[11:]:
        ids.append(sv.submit(it))
    drain(sv, ids, results)
    sv.destroy()
    for rid, it in zip(ids, items):
        v, m, st = results[rid]
        v1, m1, st1 = alone(torch, ctx, it)
        assert np.array_equal(v.cpu().numpy().view(np.uint32), v1.view(np.uint32))
        assert np.array_equal(m.cpu().numpy(), m1)
        for key in ("iterations_run", "last_flips", "area_plus", "status"):
            assert st[key] == st1[key], key
        assert st["c_plus"] == st1["c_plus"]


def test_served_16bit_results_equal_alone(torch, lse, ctx):
    # BF16 / F16 storage where it applies (one band or the edge term), FP32
    # for the 4-band region images, all in one mix
    probs = scenes.batch_problems(14, seed=23, min_side=40, max_side=300, cap_range=(4, 50))
    k = 0
    for q in probs:
        if q["term"] == "edge" or q["image"].shape[0] == 1:
            q["storage"] = ("bf16", "f16")[k % 2]
            k += 1
    items = device_items(torch, ctx, probs)
    sv = lse.Server(ctx, 512 << 20)
    ids, results = [], {}
    for it in items[:7]:
        ids.append(sv.submit(it))
    sv.advance(5)
    for it in items[7:]:
        ids.append(sv.submit(it))
    drain(sv, ids, results)
    sv.destroy()
    for rid, it in zip(ids, items):
        v, m, st = results[rid]
        v1, m1, st1 = alone(torch, ctx, it)
        assert np.array_equal(v.cpu().numpy().view(np.uint32), v1.view(np.uint32)), it["storage"]
        assert np.array_equal(m.cpu().numpy(), m1)
        for key in ("iterations_run", "last_flips", "area_plus", "status"):
            assert st[key] == st1[key], key


def test_16bit_requests_take_half_the_plane_memory(torch, lse, ctx):
    # a 256 x 256 single-band request holds 3 planes: 768 KiB in FP32,
    # 384 KiB in BF16, plus the same partial sums; a 3 MiB budget admits at
    # most three FP32 requests, and more BF16 ones
    probs = scenes.batch_problems(8, seed=4, min_side=256, max_side=256, cap_range=(6, 12))
    counts = {}
    for storage in ("f32", "bf16"):
        for q in probs:
            q["image"] = q["image"][:1]
            q["term"] = "region"
            q["early_stop_frac"] = 0.0
            q["storage"] = storage
        items = device_items(torch, ctx, probs)
        sv = lse.Server(ctx, 3 << 20)
        ids = [sv.submit(it) for it in items]
        counts[storage] = sv.advance(1)
        results = {}
        drain(sv, ids, results, ticks=4)
        sv.destroy()
        for rid, it in zip(ids, items):
            v, m, st = results[rid]
            v1, m1, _ = alone(torch, ctx, it)
            assert np.array_equal(v.cpu().numpy().view(np.uint32), v1.view(np.uint32))
    assert 1 <= counts["f32"] <= 3 and counts["bf16"] > counts["f32"], counts


def test_budget_queues_and_reuses_memory(torch, lse, ctx):
    # each 256 x 256 single-band request needs 3 planes of 256 x 256 floats
    # (768 KiB) plus its partials: a 3 MiB budget holds at most three
    probs = scenes.batch_problems(8, seed=4, min_side=256, max_side=256, cap_range=(6, 12))
    for q in probs:
        q["image"] = q["image"][:1]
        q["term"] = "region"
        q["early_stop_frac"] = 0.0
    items = device_items(torch, ctx, probs)
    sv = lse.Server(ctx, 3 << 20)
    ids = [sv.submit(it) for it in items]
    running = sv.advance(1)
    assert 1 <= running <= 3
    states = []
    for rid in ids:
        st = ctypes.c_int()
        assert lse.raw_library().lse_server_poll(sv._h, rid, ctypes.byref(st), None) == 0
        states.append(st.value)
    assert states.count(0) >= 5            # the rest wait in the queue
    results = {}
    drain(sv, ids, results, ticks=4)
    sv.destroy()
    for rid, it in zip(ids, items):
        v, m, st = results[rid]
        v1, m1, _ = alone(torch, ctx, it)
        assert np.array_equal(v.cpu().numpy().view(np.uint32), v1.view(np.uint32))
        assert st["iterations_run"] == it["iterations"]


def test_server_rejections(torch, lse, ctx):
    lib = lse.raw_library()
    sv = lse.Server(ctx, 2 << 20)
    x = torch.rand((1, 1024, 1024), device="cuda")
    phi = torch.ones((1024, 1024), device="cuda")
    with pytest.raises(lse.LseError, match="more than the budget"):
        sv.submit({"image": x, "phi0": phi, "iterations": 3})
    small = torch.rand((1, 32, 32), device="cuda")
    with pytest.raises(lse.LseError, match="ts <= 15"):
        sv.submit({"image": small, "phi0": torch.ones((32, 32), device="cuda"), "ts": 17})
    with pytest.raises(lse.LseError, match="device memory"):
        sv.submit({"image": small, "phi0": torch.ones((32, 32)), "iterations": 3})
    st = ctypes.c_int()
    assert lib.lse_server_poll(sv._h, 12345, ctypes.byref(st), None) == lse.LSE_ERR_INVALID_ARG
    rid = sv.submit({"image": small, "phi0": torch.ones((32, 32), device="cuda"),
                     "iterations": 2})
    results = {}
    drain(sv, [rid], results)
    assert results[rid][2]["iterations_run"] == 2
    # reported once, then forgotten
    assert lib.lse_server_poll(sv._h, rid, ctypes.byref(st), None) == lse.LSE_ERR_INVALID_ARG
    sv.destroy()
