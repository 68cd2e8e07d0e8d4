"""GPU path vs the FP64 oracle, through the C ABI.

Tolerances (from the project's stated bar):
  * the smoothed LSF v after one step: max |v_gpu - v_oracle| <= 1e-5;
  * region means c+/c-: within 1e-6 relative;
  * final masks after many iterations: at most 0.05 % of pixels differ and
    none lies more than 1 px from the oracle's contour.
Sizes span several warp strips (120 columns) and row blocks, ragged tails,
unaligned widths, single rows/columns, every template size, 1-8 bands, and
the full benchmark scene in the benchmark's launch configuration.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from _parity import assert_mask_parity, mask_report
from paper_1409_7474_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V = 1e-5
TOL_C = 1e-6


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    import paper_1409_7474_gb300.lse as lse
    c = lse.Context(0, max_pixels=8192 * 8192, max_bands=8)
    yield c
    c.destroy()


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_evolve(torch, ctx, img, phi0, **kw):
    x = dev(torch, img) if img is not None else None
    g = kw.pop("g", None)
    if g is not None and not isinstance(g, torch.Tensor):
        g = dev(torch, g)
    v, m, st = ctx.evolve(x, dev(torch, phi0), g=g, **kw)
    torch.cuda.synchronize()
    return v.cpu().numpy(), m.cpu().numpy(), st


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def rng_scene(B, H, W, seed):
    r = np.random.default_rng(seed)
    img = (0.3 + 0.4 * (r.random((B, H, W)) < 0.3) + 0.05 * r.standard_normal((B, H, W)))
    return img.astype(np.float32)


# ------------------------------------------------ 256 x 256 rectangle scene
@pytest.mark.parametrize("sigma", [1.0, 3.0])
def test_rectangle_256_one_step(torch, ctx, sigma):
    img, truth, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, dt=15.0, sigma=sigma, ts=9, iterations=1)
    v_ref, norm, cp, cm, _ = oracle.step(img, phi0, dt=15.0, sigma=sigma, ts=9)
    assert np.abs(v - v_ref).max() <= TOL_V
    assert rel(st["norm"], norm) <= TOL_C
    # c+/c- the library reports are those of its own new LSF
    cp1, cm1, n1 = oracle.region_stats(img, v)
    assert st["area_plus"] == n1
    assert rel(st["c_plus"][:1], cp1) <= TOL_C and rel(st["c_minus"][:1], cm1) <= TOL_C
    assert st["status"] == "LSE_OK"


@pytest.mark.parametrize("sigma", [1.0, 3.0])
def test_rectangle_256_200_iterations(torch, ctx, sigma):
    img, truth, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, dt=15.0, sigma=sigma, ts=9, iterations=200)
    v_ref, m_ref, st_ref = oracle.evolve(img, phi0, dt=15.0, sigma=sigma, ts=9, iterations=200)
    assert st["iterations_run"] == 200
    assert_mask_parity(m, m_ref)
    cp1, cm1, _ = oracle.region_stats(img, v)
    assert rel(st["c_plus"][:1], cp1) <= TOL_C and rel(st["c_minus"][:1], cm1) <= TOL_C


# ---------------------------------------------------------------- shapes
SHAPES = [(8, 8), (1, 17), (17, 1), (1, 1), (2, 3), (37, 53), (130, 250),
          (64, 129), (300, 121), (241, 360), (16, 1000)]


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("term", ["region", "edge"])
def test_shapes_one_and_five_steps(torch, ctx, H, W, term):
    img = rng_scene(1, H, W, H * 1000 + W)
    phi0 = np.where(np.random.default_rng(W).random((H, W)) < 0.5, 1.0, -1.0).astype(np.float32)
    g_gpu = g_ref = None
    if term == "edge":
        g_gpu = ctx.precompute_edge(dev(torch, img), 1.0, 9, 255.0)
        torch.cuda.synchronize()
        g_ref = oracle.edge_indicator(img, 1.0, 9, 255.0)
        assert np.abs(g_gpu.cpu().numpy() - g_ref).max() <= 2e-7
    for iters in (1, 5):
        kw = dict(term=term, dt=15.0, sigma=1.0, ts=9, iterations=iters)
        if term == "edge":
            # each side uses its own g: the GPU's float32 g, the oracle's FP64 g
            v, m, st = gpu_evolve(torch, ctx, None, phi0, g=g_gpu, **kw)
            v_ref, m_ref, _ = oracle.evolve(img, phi0, term="edge", g=g_ref, iterations=iters)
        else:
            v, m, st = gpu_evolve(torch, ctx, img, phi0, **kw)
            v_ref, m_ref, _ = oracle.evolve(img, phi0, iterations=iters)
        if iters == 1:
            assert np.abs(v - v_ref).max() <= TOL_V, (H, W, term)
        else:
            rep = mask_report(m, m_ref)
            assert rep["far"] == 0 and rep["disagree"] <= max(2, int(5e-4 * H * W)), rep


# ---------------------------------------------------------------- template sizes
@pytest.mark.parametrize("ts", [1, 3, 5, 7, 9, 11, 13, 15, 17, 21, 31])
def test_template_sizes(torch, ctx, ts):
    img = rng_scene(1, 200, 300, ts)
    phi0 = scenes.circle_phi(200, 300, radius=60)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, sigma=2.0, ts=ts, iterations=1)
    v_ref, *_ = oracle.step(img, phi0, sigma=2.0, ts=ts)
    assert np.abs(v - v_ref).max() <= TOL_V


# ---------------------------------------------------------------- bands
@pytest.mark.parametrize("B", [2, 3, 4, 5, 8])
def test_multiband_region(torch, ctx, B):
    img = rng_scene(B, 150, 260, 40 + B)
    phi0 = scenes.circle_phi(150, 260, radius=50)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, iterations=1)
    v_ref, norm, cp, cm, _ = oracle.step(img, phi0)
    assert np.abs(v - v_ref).max() <= TOL_V
    assert rel(st["norm"], norm) <= 1e-5
    cp1, cm1, _ = oracle.region_stats(img, v)
    assert rel(st["c_plus"][:B], cp1) <= TOL_C and rel(st["c_minus"][:B], cm1) <= TOL_C
    v, m, st = gpu_evolve(torch, ctx, img, phi0, iterations=30)
    v_ref, m_ref, _ = oracle.evolve(img, phi0, iterations=30)
    assert_mask_parity(m, m_ref)


# ---------------------------------------------------------------- input types
@pytest.mark.parametrize("kind", ["u16", "f16", "bf16"])
def test_input_dtypes(torch, ctx, kind):
    sc = scenes.multiband_scene(256, 320, 4, seed=3, n_roofs=6)
    u16 = sc["image"]
    ref = u16.astype(np.float32) / np.float32(65535.0)
    if kind == "u16":
        x = torch.from_numpy(u16.astype(np.int32)).to(torch.uint16).cuda()
        as_f32 = ref
    elif kind == "f16":
        h = torch.from_numpy(ref).half()           # rounding done on the CPU
        x, as_f32 = h.cuda(), h.float().numpy()
    else:
        h = torch.from_numpy(ref).bfloat16()
        x, as_f32 = h.cuda(), h.float().numpy()
    phi0 = scenes.circle_phi(256, 320, radius=80)
    v, m, st = ctx.evolve(x, dev(torch, phi0), iterations=1)
    torch.cuda.synchronize()
    v_ref, *_ = oracle.step(as_f32, phi0)
    assert np.abs(v.cpu().numpy() - v_ref).max() <= TOL_V


# ---------------------------------------------------------------- host buffers, determinism
@pytest.mark.parametrize("W", [230, 232])
def test_host_buffers_match_device_buffers_bitwise(torch, ctx, W):
    # W = 232: a host FP32 image is copied straight into the kernels' layout
    # (pitch W); W = 230 goes through the conversion kernel (pitch 256)
    img, _, _ = scenes.rect_scene(190, W, 70, 40)
    phi0 = scenes.circle_phi(190, W, radius=50)
    v_d, m_d, st_d = gpu_evolve(torch, ctx, img, phi0, iterations=7)
    v_h, m_h, st_h = ctx.evolve(img, phi0, iterations=7)   # numpy: host pointers
    assert isinstance(v_h, np.ndarray)
    assert np.array_equal(v_h.view(np.uint32), v_d.view(np.uint32))
    assert np.array_equal(m_h, m_d)
    pinned = torch.from_numpy(img).pin_memory()
    v_p, m_p, _ = ctx.evolve(pinned, torch.from_numpy(phi0).pin_memory(), iterations=7)
    assert np.array_equal(v_p.numpy().view(np.uint32), v_d.view(np.uint32))


def test_runs_are_bitwise_deterministic(torch, ctx):
    sc = scenes.large_scene(1024, 1536, n_roofs=60, n_roads=8, seed=5)
    phi0 = scenes.circle_phi(1024, 1536, radius=400)
    a = gpu_evolve(torch, ctx, sc["image"], phi0, iterations=25)
    b = gpu_evolve(torch, ctx, sc["image"], phi0, iterations=25)
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert a[2]["c_plus"] == b[2]["c_plus"] and a[2]["last_flips"] == b[2]["last_flips"]


@pytest.mark.parametrize("term", ["region", "edge"])
def test_step_forms_agree(torch, term):
    """The tile form, the streaming form and the plain shared-memory kernel
    (LSE_STEP_KERNEL selects them) compute the same step: the two TMA forms
    sum in the same order, so one iteration agrees bit for bit; the plain
    kernel agrees to rounding.  Four iterations with re-initialisation run
    the +-1 input and output variants."""
    code = r"""
import numpy as np, torch, sys
sys.path.insert(0, %r)
import paper_1409_7474_gb300.lse as lse
from paper_1409_7474_gb300 import scenes
img, _, _ = scenes.rect_scene(300, 412, 120, 70)
phi0 = scenes.circle_phi(300, 412, radius=90)
x = torch.from_numpy(img).cuda()
p = torch.from_numpy(phi0).cuda()
out = {}
with lse.Context(0, 300 * 412, 1) as c:
    g = c.precompute_edge(x) if sys.argv[2] == "edge" else None
    for it in (1, 4):
        v, m, st = c.evolve(x, p, sys.argv[2], g=g, iterations=it)
        out["v%%d" %% it] = v.cpu().numpy()
        out["m%%d" %% it] = m.cpu().numpy()
np.savez(sys.argv[1], **out)
""" % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = {}
    for kern in ("tile", "stream", "generic"):
        path = f"/tmp/lse_kernel_{kern}_{os.getpid()}.npz"
        env = dict(os.environ, LSE_STEP_KERNEL=kern)
        subprocess.run([sys.executable, "-c", code, path, term], env=env, check=True,
                       timeout=300)
        with np.load(path) as z:
            outs[kern] = {k: z[k] for k in z.files}
        os.remove(path)
    t, s_, g = outs["tile"], outs["stream"], outs["generic"]
    assert np.array_equal(t["v1"].view(np.uint32), s_["v1"].view(np.uint32))
    assert np.abs(t["v1"] - g["v1"]).max() <= 4e-6
    for other in (s_, g):
        assert (t["m4"] != other["m4"]).mean() <= 1e-4


# ---------------------------------------------------------------- options
@pytest.mark.parametrize("period", [0, 3])
def test_reinit_period(torch, ctx, period):
    img, _, _ = scenes.rect_scene(96, 128, 40, 30)
    phi0 = scenes.circle_phi(96, 128, radius=30)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, iterations=6, reinit_period=period)
    v_ref, m_ref, _ = oracle.evolve(img, phi0, iterations=6, reinit_period=period)
    assert np.abs(v - v_ref).max() <= TOL_V * max(1.0, np.abs(v_ref).max())


def test_early_stop(torch, ctx):
    img, truth, _ = scenes.rect_scene(noise=0.0)
    phi_t = np.where(truth, 1.0, -1.0).astype(np.float32)
    v, m, st = gpu_evolve(torch, ctx, img, phi_t, iterations=50, early_stop_frac=1e-4)
    assert st["iterations_run"] == 1 and st["last_flips"] == 0
    assert np.array_equal(m.astype(bool), truth)
    img, _, _ = scenes.rect_scene()
    phi0 = scenes.circle_phi(256, 256)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, iterations=100, early_stop_frac=2e-2)
    _, m_ref, st_ref = oracle.evolve(img, phi0, iterations=100, early_stop_frac=2e-2)
    assert st["iterations_run"] == st_ref["iterations_run"] < 100
    assert_mask_parity(m, m_ref)


def test_constant_image_is_degenerate(torch, ctx):
    img = np.full((1, 40, 50), 0.37, np.float32)
    phi0 = scenes.circle_phi(40, 50, radius=12)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, iterations=1)
    v_ref, *_ = oracle.step(img, phi0)
    assert st["status"] == "LSE_WARN_DEGENERATE"
    assert np.abs(v - v_ref).max() <= TOL_V


def test_nonfinite_input_is_reported(torch, ctx):
    img = rng_scene(1, 30, 40, 9)
    img[0, 5, 7] = np.nan
    phi0 = scenes.circle_phi(30, 40, radius=10)
    _, _, st = gpu_evolve(torch, ctx, img, phi0, iterations=3)
    assert st["status"] == "LSE_ERR_NONFINITE"
    # the context stays usable
    img[0, 5, 7] = 0.3
    _, _, st = gpu_evolve(torch, ctx, img, phi0, iterations=3)
    assert st["status"] == "LSE_OK"


def test_bad_arguments_are_rejected(torch, ctx):
    import paper_1409_7474_gb300.lse as lse
    img = rng_scene(1, 16, 16, 1)
    phi0 = scenes.circle_phi(16, 16, radius=4)
    for kw in (dict(ts=8), dict(ts=33), dict(dt=0.0), dict(sigma=-1.0), dict(iterations=0)):
        with pytest.raises(lse.LseError) as e:
            ctx.evolve(dev(torch, img), dev(torch, phi0), **kw)
        assert e.value.status == lse.LSE_ERR_INVALID_ARG
    with pytest.raises(lse.LseError):
        ctx.evolve(dev(torch, np.zeros((9, 16, 16), np.float32)), dev(torch, phi0))


# ---------------------------------------------------------------- edge indicator
@pytest.mark.parametrize("B,sigma1,ts1", [(1, 1.0, 9), (1, 3.0, 15), (4, 1.0, 9), (3, 1.7, 31)])
def test_edge_indicator(torch, ctx, B, sigma1, ts1):
    # the C ABI takes sigma1 as float32: give the oracle the same value
    sigma1 = float(np.float32(sigma1))
    img = rng_scene(B, 140, 210, B + ts1)
    g = ctx.precompute_edge(dev(torch, img), sigma1, ts1, 255.0)
    torch.cuda.synchronize()
    g_ref = oracle.edge_indicator(img, sigma1, ts1, 255.0)
    assert np.abs(g.cpu().numpy() - g_ref).max() <= 2e-7
    g_h = ctx.precompute_edge(img, sigma1, ts1, 255.0)       # host in, host out
    assert np.array_equal(g_h, g.cpu().numpy())


# ---------------------------------------------------------------- multi-band scene (2048^2 x 4, uint16)
@pytest.fixture(scope="module")
def scene2048():
    return scenes.multiband_scene(2048, 2048, 4, seed=7)


def test_multiband_2048_region_vector_term(torch, ctx, scene2048):
    u16 = scene2048["image"]
    img = u16.astype(np.float32) / np.float32(65535.0)
    phi0 = scenes.circle_phi(2048, 2048, radius=512)
    x = torch.from_numpy(u16.astype(np.int32)).to(torch.uint16).cuda()
    v, m, st = ctx.evolve(x, dev(torch, phi0), iterations=1)
    torch.cuda.synchronize()
    v_ref, norm, *_ = oracle.step(img, phi0)
    assert np.abs(v.cpu().numpy() - v_ref).max() <= TOL_V
    v, m, st = ctx.evolve(x, dev(torch, phi0), iterations=20)
    torch.cuda.synchronize()
    _, m_ref, _ = oracle.evolve(img, phi0, iterations=20)
    assert_mask_parity(m.cpu().numpy(), m_ref)


def test_multiband_2048_edge_term(torch, ctx, scene2048):
    u16 = scene2048["image"]
    img = u16.astype(np.float32) / np.float32(65535.0)
    y0, x0, y1, x1 = scene2048["runway_box"]
    phi0 = scenes.box_phi(2048, 2048, [(y0 - 20, x0 - 20, y1 + 20, x1 + 20)])
    x = torch.from_numpy(u16.astype(np.int32)).to(torch.uint16).cuda()
    g = ctx.precompute_edge(x, 1.0, 9, 255.0)
    torch.cuda.synchronize()
    g_np = g.cpu().numpy()
    g_ref = oracle.edge_indicator(img, 1.0, 9, 255.0)
    assert np.abs(g_np - g_ref).max() <= 2e-7
    v, m, st = ctx.evolve(None, dev(torch, phi0), "edge", g=g, iterations=20)
    torch.cuda.synchronize()
    _, m_ref, _ = oracle.evolve(img, phi0, "edge", g=g_ref, iterations=20)
    assert_mask_parity(m.cpu().numpy(), m_ref)


# ---------------------------------------------------------------- full benchmark scene
def sample_points(H, W, n, seed):
    r = np.random.default_rng(seed)
    ys = list(r.integers(0, H, n))
    xs = list(r.integers(0, W, n))
    # borders, corners, strip and row-block seams
    for y in (0, 1, H - 2, H - 1):
        for x in (0, 1, 119, 120, 121, W // 2, W - 2, W - 1):
            ys.append(y)
            xs.append(x)
    for k in range(1, 8):
        ys += [int(r.integers(0, H))] * 3
        xs += [k * 120 - 1, k * 120, k * 120 + 1]
    return np.array(ys), np.array(xs)


def test_full_size_bench_scene_one_step_sampled(torch, ctx):
    sc = scenes.large_scene()
    img = sc["image"]
    H, W = img.shape[1:]
    phi0 = scenes.circle_phi(H, W, radius=H / 4)
    v, m, st = gpu_evolve(torch, ctx, img, phi0, iterations=1)
    ys, xs = sample_points(H, W, 3000, 1)
    vs, norm, cp, cm, _ = oracle.step_sampled(img, phi0, ys, xs)
    assert np.abs(v[ys, xs] - vs).max() <= TOL_V
    assert rel(st["norm"], norm) <= TOL_C
    cp1, cm1, n1 = oracle.region_stats(img, v)
    assert st["area_plus"] == n1
    assert rel(st["c_plus"][:1], cp1) <= TOL_C and rel(st["c_minus"][:1], cm1) <= TOL_C
