"""Checkpoint and resume: an evolution stopped after k iterations continues
from its result.

With re-initialisation every iteration the LSF between iterations is the
binary function of the last mask (Table I step 3), so the state to keep is
that mask: resuming from phi0 = +1 where mask, -1 elsewhere, runs the same
recurrence as the uninterrupted evolution.  Only the grouping of the region
sums differs (the resumed call sums them in its prologue, the uninterrupted
one in the step kernel), so the results must agree to the parity tests'
one-step bar, with identical masks.
"""
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
def ctx(torch):
    import paper_1409_7474_gb300.lse as lse
    c = lse.Context(0, max_pixels=1024 * 1024, max_bands=4)
    yield c
    c.destroy()


def evolve(torch, ctx, img, phi0, term, g, iterations):
    x = torch.from_numpy(img).cuda() if term == "region" else None
    v, m, st = ctx.evolve(x, torch.from_numpy(np.ascontiguousarray(phi0)).cuda(), term,
                          g=g, iterations=iterations)
    torch.cuda.synchronize()
    return v.cpu().numpy(), m.cpu().numpy(), st


@pytest.mark.parametrize("term", ["region", "edge"])
@pytest.mark.parametrize("side", [256, 1000])
def test_resume_from_the_mask_continues_the_evolution(torch, ctx, term, side):
    img, _, _ = scenes.rect_scene(side, side, side // 3, side // 4)
    if term == "region":
        phi0 = scenes.circle_phi(side, side, radius=side / 4)
        g = None
    else:
        phi0 = scenes.box_phi(side, side, [(side // 10, side // 10, side - side // 10,
                                            side - side // 10)])
        g = ctx.precompute_edge(torch.from_numpy(img).cuda(), 1.0, 9, 255.0)
    v_all, m_all, st_all = evolve(torch, ctx, img, phi0, term, g, 40)
    _, m_k, _ = evolve(torch, ctx, img, phi0, term, g, 15)
    phi_k = np.where(m_k.astype(bool), 1.0, -1.0).astype(np.float32)
    v_res, m_res, st_res = evolve(torch, ctx, img, phi_k, term, g, 25)
    assert np.array_equal(m_res, m_all)
    assert np.abs(v_res - v_all).max() <= 1e-5
    assert st_res["area_plus"] == st_all["area_plus"]
