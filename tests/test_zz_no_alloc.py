"""lse_evolve_static: the evolution for callers that cannot allocate.

Callers inside a framework or memory pool that owns all device memory, or a
serving loop that must not call cudaMalloc, use lse_evolve_static, whose
scratch is a fixed array in the library.  These tests call it through the C
ABI and check that its outputs and statistics match lse_evolve's on the same
inputs, on two calls in a row (the second call reuses the array the first one
left behind, and leaves the device memory in use unchanged), that it agrees
with the FP64 oracle directly, and that sizes beyond its limit are refused
with a message.

The file is named to be collected last, and passes alone in a fresh process
as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1409_7474_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1409_7474_gb300.lse as lse
    torch.cuda.set_device(0)
    ctx = lse.Context(0, max_pixels=512 * 512, max_bands=4)
    yield torch, lse, ctx
    ctx.destroy()


def call_static(torch, lse, image, phi0, term, g=None, iterations=20, ts=9, sigma=1.0,
                out=None):
    """One lse_evolve_static call through the C ABI; returns (v, mask, stats).

    `out` = (phi_out, mask) lets a caller allocate the outputs beforehand;
    the device memory in use is then compared around the raw call, which
    must leave it unchanged."""
    H, W = phi0.shape
    B = 1 if image is None else image.shape[0]
    if out is None:
        out = (torch.empty((H, W), dtype=torch.float32, device="cuda"),
               torch.empty((H, W), dtype=torch.uint8, device="cuda"))
    phi_out, mask = out
    params = lse.Params(lse.TERM_REGION if term == "region" else lse.TERM_EDGE, 15.0,
                        sigma, ts, iterations, 1, 0.0, lse.F32)
    st = lse.Stats()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    alloc_before = torch.cuda.memory_allocated()
    rc = lse.raw_library().lse_evolve_static(
        ctypes.c_void_p(image.data_ptr()) if image is not None else None, H, W, B,
        ctypes.c_void_p(g.data_ptr()) if g is not None else None,
        ctypes.c_void_p(phi0.data_ptr()), ctypes.byref(params),
        ctypes.c_void_p(phi_out.data_ptr()), ctypes.c_void_p(mask.data_ptr()),
        ctypes.byref(st), stream)
    assert rc == lse.LSE_OK, lse.raw_library().lse_last_error(None).decode()
    torch.cuda.synchronize()
    moved = (torch.cuda.mem_get_info()[0] - free_before,
             torch.cuda.memory_allocated() - alloc_before)
    return phi_out.cpu().numpy(), mask.cpu().numpy(), st.to_dict(B), moved


def outputs(torch, H, W):
    return (torch.empty((H, W), dtype=torch.float32, device="cuda"),
            torch.empty((H, W), dtype=torch.uint8, device="cuda"))


def test_region_matches_lse_evolve_twice(env):
    torch, lse, ctx = env
    img, _, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    x = torch.from_numpy(img).cuda()
    p = torch.from_numpy(phi0).cuda()
    v_ref, m_ref, st_ref = ctx.evolve(x, p, "region", iterations=20)
    v_ref, m_ref = v_ref.cpu().numpy(), m_ref.cpu().numpy()
    out = outputs(torch, 256, 256)
    for call in range(2):
        v, m, st, moved = call_static(torch, lse, x, p, "region", iterations=20, out=out)
        assert np.abs(v - v_ref).max() <= TOL_V
        assert np.array_equal(m, m_ref)
        assert st["iterations_run"] == 20 and st["status"] == "LSE_OK"
        assert st["area_plus"] == st_ref["area_plus"]
        assert np.allclose(st["c_plus"], st_ref["c_plus"], rtol=1e-12)
        if call == 1:
            # the device code is loaded by now: the call reserves nothing
            assert moved == (0, 0), moved


def test_region_matches_the_oracle(env):
    # the same evolution directly against the FP64 oracle: one step within
    # 1e-5, and after 60 iterations the mask within 0.05 % and 1 px
    import oracle
    from _parity import assert_mask_parity
    torch, lse, ctx = env
    img, _, _ = scenes.rect_scene(noise=0.05)
    phi0 = scenes.circle_phi(256, 256)
    x = torch.from_numpy(img).cuda()
    p = torch.from_numpy(phi0).cuda()
    v, m, st, _ = call_static(torch, lse, x, p, "region", iterations=1)
    v_ref, norm, *_ = oracle.step(img, phi0)
    assert np.abs(v - v_ref).max() <= TOL_V
    assert abs(st["norm"] - norm) <= 1e-6 * norm
    v, m, st, _ = call_static(torch, lse, x, p, "region", iterations=60)
    v_ref, m_ref, st_ref = oracle.evolve(img, phi0, iterations=60)
    assert_mask_parity(m, m_ref)
    assert st["iterations_run"] == st_ref["iterations_run"] == 60


def test_multiband_and_edge_match_lse_evolve_twice(env):
    torch, lse, ctx = env
    sc = scenes.multiband_scene(200, 240, 4, seed=5, n_roofs=5)
    img = torch.from_numpy(sc["image"].astype(np.float32) / np.float32(65535.0)).cuda()
    phi0 = torch.from_numpy(scenes.circle_phi(200, 240, radius=60)).cuda()
    v_ref, m_ref, st_ref = ctx.evolve(img, phi0, "region", iterations=12)
    v_ref, m_ref = v_ref.cpu().numpy(), m_ref.cpu().numpy()
    g = ctx.precompute_edge(img, 1.0, 9, 255.0)
    torch.cuda.synchronize()
    pe = torch.from_numpy(-scenes.circle_phi(200, 240, radius=80)).cuda()
    ve_ref, me_ref, ste_ref = ctx.evolve(None, pe, "edge", g=g, iterations=12)
    ve_ref, me_ref = ve_ref.cpu().numpy(), me_ref.cpu().numpy()
    out = outputs(torch, 200, 240)
    out_e = outputs(torch, 200, 240)
    for call in range(2):
        v, m, st, moved = call_static(torch, lse, img, phi0, "region", iterations=12,
                                      out=out)
        assert np.abs(v - v_ref).max() <= TOL_V and np.array_equal(m, m_ref)
        # the statistics the header promises are lse_evolve's too
        assert st["area_plus"] == st_ref["area_plus"]
        assert np.allclose(st["c_plus"], st_ref["c_plus"], rtol=1e-6)
        assert np.allclose(st["c_minus"], st_ref["c_minus"], rtol=1e-6)
        ve, me, ste, moved_e = call_static(torch, lse, None, pe, "edge", g=g,
                                           iterations=12, out=out_e)
        assert np.abs(ve - ve_ref).max() <= TOL_V and np.array_equal(me, me_ref)
        assert ste["area_plus"] == ste_ref["area_plus"]
        if call == 1:
            assert moved == (0, 0) and moved_e == (0, 0), (moved, moved_e)


def test_limits_are_refused_with_a_message(env):
    torch, lse, ctx = env
    lib = lse.raw_library()
    big = torch.zeros((1, 600, 600), dtype=torch.float32, device="cuda")
    phi = torch.ones((600, 600), dtype=torch.float32, device="cuda")
    out = torch.empty_like(phi)
    params = lse.Params(lse.TERM_REGION, 15.0, 1.0, 9, 3, 1, 0.0, lse.F32)
    rc = lib.lse_evolve_static(ctypes.c_void_p(big.data_ptr()), 600, 600, 1, None,
                               ctypes.c_void_p(phi.data_ptr()), ctypes.byref(params),
                               ctypes.c_void_p(out.data_ptr()), None, None, None)
    assert rc == lse.LSE_ERR_INVALID_ARG
    assert b"LSE_STATIC_MAX_PIXELS" in lib.lse_last_error(None)
    host = np.zeros((64, 64), np.float32)
    rc = lib.lse_evolve_static(ctypes.c_void_p(host.ctypes.data), 64, 64, 1, None,
                               ctypes.c_void_p(host.ctypes.data), ctypes.byref(params),
                               ctypes.c_void_p(host.ctypes.data), None, None, None)
    assert rc == lse.LSE_ERR_INVALID_ARG
    assert b"device memory" in lib.lse_last_error(None)
