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


def test_a_lone_request_runs_to_its_end_in_one_advance(torch, lse, ctx):
    # one band or the edge term alone, and a vector image always: lse_evolve's
    # persistent path inside the advance, the same bits
    probs = scenes.batch_problems(6, seed=31, min_side=64, max_side=200, cap_range=(30, 40))
    probs[0]["image"] = probs[0]["image"][:1]
    probs[0]["term"] = "region"
    probs[1]["term"] = "edge"
    probs[2]["image"] = np.ascontiguousarray(np.repeat(probs[2]["image"][:1], 3, axis=0))
    probs[2]["term"] = "region"
    for q in probs[:3]:
        q["early_stop_frac"] = 0.0
    items = device_items(torch, ctx, probs[:3])
    for k, it in enumerate(items):
        sv = lse.Server(ctx, 512 << 20)
        rid = sv.submit(it)
        left = sv.advance(1)
        r = sv.poll(rid)
        assert left == 0 and r is not None
        v, m, st = r
        v1, m1, st1 = alone(torch, ctx, it)
        assert np.array_equal(v.cpu().numpy().view(np.uint32), v1.view(np.uint32))
        assert np.array_equal(m.cpu().numpy(), m1)
        assert st["iterations_run"] == it["iterations"] and st["elapsed_ms"] == -1.0
        sv.destroy()


def test_vector_and_large_requests_run_alone_beside_the_mix(torch, lse, ctx):
    # small single-band requests join the mix and advance `ticks` iterations
    # per call; a vector image and an image of 2^21 pixels or more each run
    # alone, to their end, one per advance, oldest first
    probs = scenes.batch_problems(5, seed=41, min_side=64, max_side=128, cap_range=(40, 50))
    for q in probs:
        q["image"] = q["image"][:1]
        q["term"] = "region"
        q["early_stop_frac"] = 0.0
    big = scenes.batch_problems(1, seed=42, min_side=1449, max_side=1449, cap_range=(20, 21))[0]
    big["image"] = big["image"][:1]
    big["term"], big["early_stop_frac"] = "region", 0.0
    vec = scenes.batch_problems(1, seed=43, min_side=100, max_side=100, cap_range=(30, 31))[0]
    vec["image"] = np.ascontiguousarray(np.repeat(vec["image"][:1], 4, axis=0))
    vec["term"], vec["early_stop_frac"] = "region", 0.0
    assert big["phi0"].size >= 1 << 21
    ctx = lse.Context(0, max_pixels=1 << 22, max_bands=4)
    items = device_items(torch, ctx, probs[:3] + [big, vec] + probs[3:])
    sv = lse.Server(ctx, 512 << 20)
    ids = [sv.submit(it) for it in items]
    running = sv.advance(4)            # the big image alone; the small ones join the mix
    assert running == 5
    assert sv.poll(ids[3]) is not None and sv.poll(ids[4]) is None
    running = sv.advance(4)            # the vector image alone
    assert sv.poll(ids[4]) is not None and running == 5
    results = {}
    drain(sv, [ids[k] for k in (0, 1, 2, 5, 6)], results)
    sv.destroy()
    for k in (0, 1, 2, 5, 6):
        v, m, st = results[ids[k]]
        v1, m1, _ = alone(torch, ctx, items[k])
        assert np.array_equal(v.cpu().numpy().view(np.uint32), v1.view(np.uint32))
    ctx.destroy()


def test_light_load_runs_one_request_per_advance_in_arrival_order(torch, lse, ctx):
    # at most four waiting and nothing in the mix: each advance runs the
    # oldest request alone, to its end; five waiting start the mix
    probs = scenes.batch_problems(5, seed=51, min_side=48, max_side=96, cap_range=(20, 30))
    for q in probs:
        q["image"] = q["image"][:1]
        q["early_stop_frac"] = 0.0
    items = device_items(torch, ctx, probs)
    sv = lse.Server(ctx, 512 << 20)
    ids = [sv.submit(it) for it in items[:3]]
    for k in range(3):
        assert sv.advance(2) == 0
        assert sv.poll(ids[k]) is not None
        assert all(sv.poll(r) is None for r in ids[k + 1:])
    ids = [sv.submit(it) for it in items]
    assert sv.advance(2) == 5
    results = {}
    drain(sv, ids, results)
    sv.destroy()


def test_queued_vector_images_run_together(torch, lse, ctx):
    # three vector images queued behind small requests: one advance runs
    # them together (one batch, each on its own CTAs) and admits the rest
    # into the mix; every result keeps lse_evolve's bits
    probs = scenes.batch_problems(8, seed=61, min_side=48, max_side=160, cap_range=(20, 40))
    for k, q in enumerate(probs):
        q["early_stop_frac"] = 0.0
        if k < 5:
            q["image"] = q["image"][:1]
        else:
            q["image"] = np.ascontiguousarray(np.repeat(q["image"][:1], 3, axis=0) *
                                              np.array([1.0, 0.8, 0.6], np.float32)[:, None, None])
            q["term"] = "region"
    items = device_items(torch, ctx, probs)
    sv = lse.Server(ctx, 512 << 20)
    ids = [sv.submit(it) for it in items]
    running = sv.advance(1)
    assert running == 5
    for k in (5, 6, 7):
        r = sv.poll(ids[k])
        assert r is not None
        v1, m1, st1 = alone(torch, ctx, items[k])
        assert np.array_equal(r[0].cpu().numpy().view(np.uint32), v1.view(np.uint32))
        assert r[2]["iterations_run"] == st1["iterations_run"]
    results = {}
    drain(sv, ids[:5], results)
    sv.destroy()
