"""The Table I step order and replicate padding on the GPU, against the FP64
oracle's variants, through the C ABI.

Table I (steps 2-4) re-initialises the updated LSF u before smoothing it;
the MATLAB listing smooths first and re-initialises v.  Replicate padding
lets the convolution see the nearest image value outside the image instead
of the listing's zeros.  Both run on the plain shared-memory step kernel.
Tolerances as in the main parity tests: |v - v_oracle| <= 1e-5 after one
step; after several steps at most 0.05 % of the mask differs and none of it
more than 1 px from the oracle's contour.
"""
import ctypes

import numpy as np
import pytest

import oracle
from _parity import assert_mask_parity, mask_report
from paper_1409_7474_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V = 1e-5
TOL_C = 1e-6
VARIANTS = [("table1", "zero"), ("listing", "replicate"), ("table1", "replicate")]
SHAPES = [(1, 17), (17, 1), (8, 8), (37, 53), (64, 129), (130, 250)]


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
def ctx(torch, lse):
    c = lse.Context(0, max_pixels=512 * 512, max_bands=4)
    yield c
    c.destroy()


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rng_scene(B, H, W, seed):
    r = np.random.default_rng(seed)
    img = (0.3 + 0.4 * (r.random((B, H, W)) < 0.3) + 0.05 * r.standard_normal((B, H, W)))
    return img.astype(np.float32)


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def run(torch, ctx, img, phi0, g=None, **kw):
    x = dev(torch, img) if img is not None else None
    v, m, st = ctx.evolve(x, dev(torch, phi0), g=g, **kw)
    torch.cuda.synchronize()
    return v.cpu().numpy(), m.cpu().numpy(), st


@pytest.mark.parametrize("order,padding", VARIANTS)
@pytest.mark.parametrize("term", ["region", "edge"])
@pytest.mark.parametrize("H,W", SHAPES)
def test_one_and_five_steps(torch, ctx, order, padding, term, H, W):
    img = rng_scene(1, H, W, 7 * H + W)
    phi0 = np.where(np.random.default_rng(H + 3 * W).random((H, W)) < 0.5,
                    1.0, -1.0).astype(np.float32)
    g_gpu = g_ref = None
    if term == "edge":
        g_gpu = ctx.precompute_edge(dev(torch, img), 1.0, 9, 255.0)
        torch.cuda.synchronize()
        g_ref = oracle.edge_indicator(img, 1.0, 9, 255.0)
    for iters in (1, 5):
        kw = dict(term=term, dt=15.0, sigma=1.0, ts=9, iterations=iters)
        if term == "edge":
            v, m, st = run(torch, ctx, None, phi0, g=g_gpu, order=order, padding=padding, **kw)
            v_ref, m_ref, _ = oracle.evolve(img, phi0, g=g_ref, order=order, padding=padding,
                                            **kw)
        else:
            v, m, st = run(torch, ctx, img, phi0, order=order, padding=padding, **kw)
            v_ref, m_ref, _ = oracle.evolve(img, phi0, order=order, padding=padding, **kw)
        if iters == 1:
            v1, *_ = oracle.step(img, phi0, term, g_ref, order=order, padding=padding)
            assert np.abs(v_ref - v1).max() == 0.0      # the oracle agrees with itself
            assert np.abs(v - v_ref).max() <= TOL_V, (H, W, term, order, padding)
        else:
            rep = mask_report(m, m_ref)
            assert rep["far"] == 0 and rep["disagree"] <= max(2, int(5e-4 * H * W)), rep
        assert st["status"] == "LSE_OK"


@pytest.mark.parametrize("order,padding", VARIANTS)
def test_rectangle_256_200_iterations(torch, ctx, order, padding):
    img, _, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    v, m, st = run(torch, ctx, img, phi0, iterations=200, order=order, padding=padding)
    v_ref, m_ref, st_ref = oracle.evolve(img, phi0, iterations=200, order=order,
                                         padding=padding)
    assert st["iterations_run"] == 200
    assert_mask_parity(m, m_ref)
    cp1, cm1, n1 = oracle.region_stats(img, v)
    assert st["area_plus"] == n1
    assert rel(st["c_plus"][:1], cp1) <= TOL_C and rel(st["c_minus"][:1], cm1) <= TOL_C


@pytest.mark.parametrize("order,padding", VARIANTS)
@pytest.mark.parametrize("B", [2, 4])
def test_multiband_one_step(torch, ctx, order, padding, B):
    img = rng_scene(B, 90, 140, B)
    phi0 = scenes.circle_phi(90, 140, radius=30)
    v, m, st = run(torch, ctx, img, phi0, iterations=1, order=order, padding=padding)
    v_ref, norm, *_ = oracle.step(img, phi0, order=order, padding=padding)
    assert np.abs(v - v_ref).max() <= TOL_V
    assert rel(st["norm"], norm) <= TOL_C


@pytest.mark.parametrize("period", [0, 3])
@pytest.mark.parametrize("padding", ["zero", "replicate"])
def test_table1_order_reinit_period(torch, ctx, period, padding):
    img, _, _ = scenes.rect_scene(96, 128, 40, 30)
    phi0 = scenes.circle_phi(96, 128, radius=30)
    v, m, st = run(torch, ctx, img, phi0, iterations=6, reinit_period=period,
                   order="table1", padding=padding)
    v_ref, m_ref, _ = oracle.evolve(img, phi0, iterations=6, reinit_period=period,
                                    order="table1", padding=padding)
    assert np.abs(v - v_ref).max() <= TOL_V * max(1.0, np.abs(v_ref).max())


@pytest.mark.parametrize("ts", [1, 5, 15, 31])
def test_replicate_padding_template_sizes(torch, ctx, ts):
    img = rng_scene(1, 70, 90, ts)
    phi0 = scenes.circle_phi(70, 90, radius=25)
    v, m, st = run(torch, ctx, img, phi0, sigma=2.0, ts=ts, iterations=1, padding="replicate")
    v_ref, *_ = oracle.step(img, phi0, sigma=2.0, ts=ts, padding="replicate")
    assert np.abs(v - v_ref).max() <= TOL_V


def test_variants_are_rejected_where_unsupported(torch, lse, ctx):
    img = rng_scene(1, 32, 32, 1)
    phi0 = scenes.circle_phi(32, 32, radius=8)
    for kw in (dict(order="table1", storage="bf16"), dict(padding="replicate", storage="f16")):
        with pytest.raises(lse.LseError) as e:
            ctx.evolve(dev(torch, img), dev(torch, phi0), iterations=2, **kw)
        assert e.value.status == lse.LSE_ERR_INVALID_ARG
    lib = lse.raw_library()
    x, p0 = dev(torch, img), dev(torch, phi0)
    out = torch.empty((32, 32), dtype=torch.float32, device="cuda")
    for order, padding in ((2, 0), (0, 5), (1, 0), (0, 1)):
        p = lse.Params(lse.TERM_REGION, 15.0, 1.0, 9, 2, 1, 0.0, lse.F32, order, padding)
        if order > 1 or padding > 1:
            rc = lib.lse_evolve(ctx._h, ctypes.c_void_p(x.data_ptr()), lse.F32, 32, 32, 1, None,
                                ctypes.c_void_p(p0.data_ptr()), ctypes.byref(p),
                                ctypes.c_void_p(out.data_ptr()), None, None, None)
            assert rc == lse.LSE_ERR_INVALID_ARG
        else:
            rc = lib.lse_evolve_static(ctypes.c_void_p(x.data_ptr()), 32, 32, 1, None,
                                       ctypes.c_void_p(p0.data_ptr()), ctypes.byref(p),
                                       ctypes.c_void_p(out.data_ptr()), None, None, None)
            assert rc == lse.LSE_ERR_INVALID_ARG
            assert b"order" in lib.lse_last_error(None)
    torch.cuda.synchronize()
