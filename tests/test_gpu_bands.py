"""Statistics of vector images (2-4 bands) on both of their paths, through
the C ABI.

lse_evolve runs a vector image as one persistent launch whose step stages
the bands and sums them over phi >= 0 exactly (fixed point); with
LSE_PERSIST=0, and in batches, it takes the band passes, whose statistics
pass keeps running FP64 band sums over phi >= 0 and phi < 0 (Eq. 15) and
updates them, each iteration, from the pixels whose sign the step changed.
After hundreds of iterations, with and without an early stop, the c+ / c-
and |{phi >= 0}| the library reports must still be those of the LSF it
returns, as the oracle computes them directly from that LSF: the count
exactly, c+- within 1e-7 relative (rounding of the sums is orders of
magnitude below; a lost or double-counted update is not).  The two paths
agree with each other within the parity tolerance.
"""
import numpy as np
import pytest

import oracle
from _parity import assert_mask_parity, step_launches
from paper_1409_7474_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_REL = 1e-7


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    import paper_1409_7474_gb300.lse as lse
    c = lse.Context(0, max_pixels=1024 * 1024, max_bands=4)
    yield c
    c.destroy()


@pytest.fixture(scope="module")
def scene():
    sc = scenes.multiband_scene(768, 1024, 4, seed=11, n_roofs=25)
    return (sc["image"].astype(np.float32) / np.float32(65535.0)).astype(np.float32)


def check_stats(img, v, st):
    B = img.shape[0]
    cp, cm, n = oracle.region_stats(img, v)
    assert st["area_plus"] == n
    for b in range(B):
        assert abs(st["c_plus"][b] - cp[b]) <= TOL_REL * abs(cp[b]), (b, st["c_plus"][b], cp[b])
        assert abs(st["c_minus"][b] - cm[b]) <= TOL_REL * abs(cm[b]), (b, st["c_minus"][b], cm[b])


@pytest.mark.parametrize("path", ["persistent", "band passes"])
@pytest.mark.parametrize("B", [2, 3, 4])
@pytest.mark.parametrize("iterations", [1, 2, 37, 400])
def test_statistics_are_those_of_the_returned_lsf(torch, ctx, scene, B, iterations, path):
    img = np.ascontiguousarray(scene[:B])
    phi0 = scenes.circle_phi(768, 1024, radius=300)
    with step_launches(path == "band passes"):
        v, m, st = ctx.evolve(torch.from_numpy(img).cuda(), torch.from_numpy(phi0).cuda(),
                              "region", iterations=iterations)
    torch.cuda.synchronize()
    assert st["status"] == "LSE_OK"
    assert st["iterations_run"] == iterations
    check_stats(img, v.cpu().numpy(), st)


@pytest.mark.parametrize("path", ["persistent", "band passes"])
@pytest.mark.parametrize("B", [2, 4])
def test_statistics_after_an_early_stop(torch, ctx, scene, B, path):
    # the statistics pass after the stopping step updates the sums once; the
    # passes scheduled after it (and the closing one) must change nothing
    img = np.ascontiguousarray(scene[:B])
    phi0 = scenes.circle_phi(768, 1024, radius=300)
    with step_launches(path == "band passes"):
        v, m, st = ctx.evolve(torch.from_numpy(img).cuda(), torch.from_numpy(phi0).cuda(),
                              "region", iterations=600, early_stop_frac=1e-2)
    torch.cuda.synchronize()
    assert st["status"] == "LSE_OK"
    assert st["iterations_run"] < 600
    check_stats(img, v.cpu().numpy(), st)


def test_batched_vector_images_report_their_own_statistics(torch, ctx, scene):
    # two vector images of different sizes and caps in one batch: each one's
    # running sums follow its own steps
    imgs = [np.ascontiguousarray(scene[:4, :512, :640]), np.ascontiguousarray(scene[:3])]
    phis = [scenes.circle_phi(512, 640, radius=200), scenes.circle_phi(768, 1024, radius=300)]
    items = [{"image": torch.from_numpy(i).cuda(), "phi0": torch.from_numpy(p).cuda(),
              "term": "region", "iterations": it, "early_stop_frac": 0.0}
             for i, p, it in zip(imgs, phis, (150, 61))]
    res = ctx.evolve_batch(items, use_graph=True)
    torch.cuda.synchronize()
    for img, (v, m, st) in zip(imgs, res):
        assert st["status"] == "LSE_OK"
        check_stats(img, v.cpu().numpy(), st)


@pytest.mark.parametrize("B", [2, 3, 4])
def test_persistent_path_agrees_with_the_band_passes_and_the_oracle(torch, ctx, scene, B):
    img = np.ascontiguousarray(scene[:B, :300, :412])
    phi0 = scenes.circle_phi(300, 412, radius=110)
    x = torch.from_numpy(img).cuda()
    p = torch.from_numpy(phi0).cuda()
    # one step: v within 1e-5 of the oracle, the normaliser within 1e-6
    v, m, st = ctx.evolve(x, p, "region", iterations=1)
    torch.cuda.synchronize()
    v_ref, norm, cp, cm, _ = oracle.step(img, phi0)
    assert np.abs(v.cpu().numpy() - v_ref).max() <= 1e-5
    assert abs(st["norm"] - norm) <= 1e-6 * norm
    # many steps: masks within the parity bar of the oracle and of the
    # band passes
    v, m, st = ctx.evolve(x, p, "region", iterations=120)
    with step_launches():
        v2, m2, st2 = ctx.evolve(x, p, "region", iterations=120)
    torch.cuda.synchronize()
    v_ref, m_ref, st_ref = oracle.evolve(img, phi0, iterations=120)
    assert_mask_parity(m.cpu().numpy(), m_ref)
    assert_mask_parity(m.cpu().numpy(), m2.cpu().numpy())
    assert abs(st["norm"] - st_ref["norm"]) <= 1e-6 * st_ref["norm"]


@pytest.fixture(scope="module")
def scene_u16():
    sc = scenes.multiband_scene(768, 1024, 4, seed=11, n_roofs=25)
    return np.ascontiguousarray(sc["image"])


@pytest.mark.parametrize("B", [2, 3, 4])
def test_u16_bands_against_the_oracle(torch, ctx, scene_u16, B):
    # a uint16 vector image (the library reads it as k / 65535, as the
    # oracle does): the same bars against the oracle
    img16 = np.ascontiguousarray(scene_u16[:B, :300, :412])
    img = img16.astype(np.float32) / np.float32(65535.0)
    phi0 = scenes.circle_phi(300, 412, radius=110)
    x16 = torch.from_numpy(img16).cuda()
    p = torch.from_numpy(phi0).cuda()
    n0 = ctx.kernel_launches()
    v, m, st = ctx.evolve(x16, p, "region", iterations=1)
    torch.cuda.synchronize()
    # conversion, prologue, candidates (2), the persistent evolution, output
    assert ctx.kernel_launches() - n0 == 6
    v_ref, norm, cp, cm, _ = oracle.step(img, phi0)
    assert np.abs(v.cpu().numpy() - v_ref).max() <= 1e-5
    assert abs(st["norm"] - norm) <= 1e-6 * norm
    check_stats(img, v.cpu().numpy(), st)
    v, m, st = ctx.evolve(x16, p, "region", iterations=150)
    x32 = torch.from_numpy(img).cuda()
    v2, m2, st2 = ctx.evolve(x32, p, "region", iterations=150)
    torch.cuda.synchronize()
    v_ref, m_ref, st_ref = oracle.evolve(img, phi0, iterations=150)
    assert st["status"] == "LSE_OK" and st["iterations_run"] == 150
    assert_mask_parity(m.cpu().numpy(), m_ref)
    assert np.array_equal(m.cpu().numpy(), m2.cpu().numpy())
    check_stats(img, v.cpu().numpy(), st)


def test_u16_bands_from_host_memory_and_ragged_width(torch, ctx, scene_u16):
    # host input and a width that is no multiple of the pitch: the library
    # converts the planes into its pitched FP32 buffer
    img16 = np.ascontiguousarray(scene_u16[:3, :211, :333])
    img = img16.astype(np.float32) / np.float32(65535.0)
    phi0 = scenes.circle_phi(211, 333, radius=70)
    v, m, st = ctx.evolve(img16, phi0, "region", iterations=40)
    v_ref, m_ref, st_ref = oracle.evolve(img, phi0, iterations=40)
    assert_mask_parity(np.asarray(m), m_ref)
    check_stats(img, np.asarray(v), st)
