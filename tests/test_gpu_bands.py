"""Statistics of vector images (2-4 bands) on the band-pass path, through
the C ABI.

The band statistics pass keeps running FP64 band sums over phi >= 0 and
phi < 0 (Eq. 15) and updates them, each iteration, from the pixels whose
sign the step changed.  After hundreds of iterations, with and without an
early stop, the c+ / c- and |{phi >= 0}| the library reports must still be
those of the LSF it returns, as the oracle computes them directly from that
LSF: the count exactly, c+- within 1e-7 relative (rounding of the sums is
orders of magnitude below; a lost or double-counted update is not).
"""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("B", [2, 3, 4])
@pytest.mark.parametrize("iterations", [1, 2, 37, 400])
def test_statistics_are_those_of_the_returned_lsf(torch, ctx, scene, B, iterations):
    img = np.ascontiguousarray(scene[:B])
    phi0 = scenes.circle_phi(768, 1024, radius=300)
    v, m, st = ctx.evolve(torch.from_numpy(img).cuda(), torch.from_numpy(phi0).cuda(),
                          "region", iterations=iterations)
    torch.cuda.synchronize()
    assert st["status"] == "LSE_OK"
    assert st["iterations_run"] == iterations
    check_stats(img, v.cpu().numpy(), st)


@pytest.mark.parametrize("B", [2, 4])
def test_statistics_after_an_early_stop(torch, ctx, scene, B):
    # the statistics pass after the stopping step updates the sums once; the
    # passes scheduled after it (and the closing one) must change nothing
    img = np.ascontiguousarray(scene[:B])
    phi0 = scenes.circle_phi(768, 1024, radius=300)
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
