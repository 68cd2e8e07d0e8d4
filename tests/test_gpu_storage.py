"""16-bit storage (lse_params.storage = LSE_F16 / LSE_BF16) vs the FP64 oracle.

The library rounds the data term (I or g) to the storage type once, keeps the
LSF planes in it, and computes in FP32 with FP64 sums.  A re-initialised LSF
is +-1, exact in both 16-bit types, so with re-initialisation every
iteration the method runs on the rounded data term and nothing else is
rounded until the final v.  The tests therefore compare with the oracle run
on the same rounded data term (rounded here with PyTorch's CPU conversion,
round to nearest even):
  * one step: |v_gpu - v_oracle| <= half an ulp of the type at v plus the
    FP32 bound 1e-5;
  * 200 iterations: masks within the FP32 bar (0.05 %, none more than 1 px
    from the oracle's contour), and within 0.5 % of the oracle on the
    unrounded image;
  * without re-initialisation every v is rounded: a few steps stay within a
    bound that grows by one rounding per step.
"""
import ctypes

import numpy as np
import pytest

import oracle
from _parity import assert_mask_parity, mask_report
from paper_1409_7474_gb300 import scenes

pytestmark = pytest.mark.gpu

STORAGES = ["bf16", "f16"]
# half an ulp relative to |v|: 2^-8 (bfloat16, 8 significant bits), 2^-11 (half)
HALF_ULP = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    import paper_1409_7474_gb300.lse as lse
    c = lse.Context(0, max_pixels=2048 * 2048, max_bands=4)
    yield c
    c.destroy()


def rounded(torch, a, storage):
    """a rounded to the storage type (RNE), back as float32."""
    ty = torch.bfloat16 if storage == "bf16" else torch.float16
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(ty).float().numpy()


def gpu(torch, ctx, img, phi0, g=None, **kw):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    v, m, st = ctx.evolve(d(img) if img is not None else None, d(phi0),
                          g=d(g) if g is not None else None, **kw)
    torch.cuda.synchronize()
    return v.cpu().numpy(), m.cpu().numpy(), st


def noise_scene(H, W, seed):
    r = np.random.default_rng(seed)
    img = 0.3 + 0.4 * (r.random((1, H, W)) < 0.3) + 0.05 * r.standard_normal((1, H, W))
    return img.astype(np.float32)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("term", ["region", "edge"])
@pytest.mark.parametrize("H,W", [(37, 53), (130, 250), (300, 121), (1, 17), (256, 256)])
def test_one_step(torch, ctx, storage, term, H, W):
    img = noise_scene(H, W, H * 7 + W)
    phi0 = np.where(np.random.default_rng(W).random((H, W)) < 0.5, 1.0, -1.0).astype(np.float32)
    if term == "region":
        v, m, st = gpu(torch, ctx, img, phi0, term="region", iterations=1, storage=storage)
        v_ref, *_ = oracle.step(rounded(torch, img, storage), phi0)
    else:
        # the same g on both sides (the oracle's), so both round identical values
        g = oracle.edge_indicator(img, 1.0, 9, 255.0).astype(np.float32)
        v, m, st = gpu(torch, ctx, None, phi0, g=g, term="edge", iterations=1, storage=storage)
        v_ref, *_ = oracle.step(img, phi0, term="edge", g=rounded(torch, g, storage))
    err = np.abs(v - v_ref)
    bound = HALF_ULP[storage] * np.abs(v_ref) + 1e-5
    assert (err <= bound).all(), float((err - bound).max())
    assert st["status"] in ("LSE_OK", "LSE_WARN_DEGENERATE")


@pytest.mark.parametrize("storage", STORAGES)
def test_rectangle_200_iterations(torch, ctx, storage):
    img, truth, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    v, m, st = gpu(torch, ctx, img, phi0, iterations=200, storage=storage)
    _, m_q, _ = oracle.evolve(rounded(torch, img, storage), phi0, iterations=200)
    assert st["iterations_run"] == 200
    assert_mask_parity(m, m_q)
    _, m_full, _ = oracle.evolve(img, phi0, iterations=200)
    rep = mask_report(m, m_full)
    assert rep["frac"] <= 5e-3, rep


@pytest.mark.parametrize("storage", STORAGES)
def test_edge_term_multiband_scene(torch, ctx, storage):
    sc = scenes.multiband_scene(512, 512, 4, seed=3, n_roofs=8)
    img = (sc["image"].astype(np.float32) / np.float32(65535.0))
    g = oracle.edge_indicator(img, 1.0, 9, 255.0).astype(np.float32)
    phi0 = -scenes.circle_phi(512, 512, radius=200)
    v, m, st = gpu(torch, ctx, None, phi0, g=g, term="edge", iterations=60, storage=storage)
    _, m_q, _ = oracle.evolve(img, phi0, term="edge", g=rounded(torch, g, storage),
                              iterations=60)
    assert_mask_parity(m, m_q)


@pytest.mark.parametrize("storage", STORAGES)
def test_without_reinitialisation(torch, ctx, storage):
    img, _, _ = scenes.rect_scene(96, 128, 40, 30)
    phi0 = scenes.circle_phi(96, 128, radius=30)
    steps = 5
    v, m, st = gpu(torch, ctx, img, phi0, iterations=steps, reinit_period=0, storage=storage)
    v_ref, m_ref, _ = oracle.evolve(rounded(torch, img, storage), phi0, iterations=steps,
                                    reinit_period=0)
    # each step rounds v once more; smoothing does not amplify an error
    bound = (steps + 1) * HALF_ULP[storage] * np.abs(v_ref).max() + 1e-4
    assert np.abs(v - v_ref).max() <= bound
    assert (m != m_ref).mean() <= 5e-3


def test_storage_limits(torch, ctx):
    import paper_1409_7474_gb300.lse as lse
    img4 = np.zeros((4, 32, 32), np.float32)
    phi = np.ones((32, 32), np.float32)
    with pytest.raises(lse.LseError, match="16-bit storage"):
        gpu(torch, ctx, img4, phi, iterations=1, storage="bf16")
    img1 = np.zeros((1, 32, 32), np.float32)
    # radius 5..7 would start the tile's 16-bit TMA boxes off 16 bytes: the
    # argument check refuses them before anything reaches the GPU
    for ts in (11, 13, 15, 17):
        for sto in ("f16", "bf16"):
            with pytest.raises(lse.LseError, match="16-bit storage"):
                gpu(torch, ctx, img1, phi, iterations=1, ts=ts, storage=sto)
    gpu(torch, ctx, img1, phi, iterations=1, ts=9, storage="bf16")
    p = lse.Params(lse.TERM_REGION, 15.0, 1.0, 9, 1, 1, 0.0, lse.U16)
    st = lse.Stats()
    x = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    o = torch.empty_like(x)
    rc = lse.raw_library().lse_evolve(ctx._h, ctypes.c_void_p(x.data_ptr()), lse.F32, 32, 32, 1,
                                      None, ctypes.c_void_p(x.data_ptr()), ctypes.byref(p),
                                      ctypes.c_void_p(o.data_ptr()), None, ctypes.byref(st), None)
    assert rc == lse.LSE_ERR_INVALID_ARG


def test_storage_is_deterministic(torch, ctx):
    img, _, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    a = gpu(torch, ctx, img, phi0, iterations=30, storage="bf16")
    b = gpu(torch, ctx, img, phi0, iterations=30, storage="bf16")
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert a[2]["c_plus"] == b[2]["c_plus"]
