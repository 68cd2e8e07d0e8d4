"""Pins of the FP64 oracle to things other than itself.

Each test checks the oracle against a closed form, an invariant the paper
states or the mathematics fixes, an independent library routine (numpy,
scipy), a brute-force formulation on tiny inputs, or a qualitative outcome
the paper reports for its synthetic examples (Sec. III-E, Figs. 2-4).  They
are chosen so that a dropped term, a wrong sign or index, or a transposed
operand anywhere in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import ndimage, signal

import oracle
from paper_1409_7474_gb300 import scenes


# ---------------------------------------------------------------- helpers
def gauss_1d(sigma, ts):
    r = (ts - 1) // 2
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return w / w.sum()


def np_gradient(f):
    """(f_x, f_y) from numpy.gradient; zero along a dimension of size 1."""
    H, W = f.shape
    fx = np.gradient(f, axis=1) if W > 1 else np.zeros_like(f)
    fy = np.gradient(f, axis=0) if H > 1 else np.zeros_like(f)
    return fx, fy


def conv_matrix(H, W, G):
    """The 'same' zero-padded convolution as an (HW x HW) matrix, built from
    scipy's response to unit impulses."""
    cols = []
    for p in range(H * W):
        e = np.zeros(H * W)
        e[p] = 1.0
        cols.append(signal.convolve2d(e.reshape(H, W), G, mode="same",
                                      boundary="fill").ravel())
    return np.stack(cols, axis=1)


def independent_step(I, phi, term, g=None, dt=15.0, sigma=1.0, ts=9):
    """One iteration written independently of the oracle:
    gradient by numpy, region force from the squared form of Eq. 15 (with
    lambda = 1) summed over bands, normalised by its maximum magnitude
    (Eq. 17), smoothing as a matrix product with scipy impulse responses."""
    B, H, W = I.shape
    fx, fy = np_gradient(phi)
    s = np.hypot(fx, fy)
    if term == "region":
        P = phi >= 0
        if P.all() or not P.any():
            R = np.zeros_like(phi)
        else:
            D = np.zeros_like(phi)
            for b in range(B):
                cp = I[b][P].mean()
                cm = I[b][~P].mean()
                D += -(I[b] - cp) ** 2 + (I[b] - cm) ** 2
            M = np.abs(D).max()
            R = D / M if M > 0 else np.zeros_like(D)
    else:
        R = g
    u = phi + dt * R * s
    g1 = gauss_1d(sigma, ts)
    K = conv_matrix(H, W, np.outer(g1, g1))
    return (K @ u.ravel()).reshape(H, W)


def rng_image(shape, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, shape)


def rng_phi(H, W, seed):
    r = np.random.default_rng(seed)
    return np.where(r.random((H, W)) < 0.45, 1.0, -1.0)


# ---------------------------------------------------------------- taps
@pytest.mark.parametrize("sigma,ts", [(1.0, 9), (2.0, 15), (0.5, 3), (3.0, 9),
                                      (1.5, 31), (4.0, 9)])
def test_taps_sum_to_one_and_separate(sigma, ts):
    G = oracle.gaussian_taps(sigma, ts)
    assert abs(G.sum() - 1.0) < 1e-14
    g1 = gauss_1d(sigma, ts)
    np.testing.assert_allclose(G, np.outer(g1, g1), rtol=1e-13, atol=1e-17)
    assert np.array_equal(G, G.T) and np.array_equal(G, G[::-1, ::-1])


def test_tap_closed_forms():
    # sigma = 1, TS = 9: centre = (1 / sum_{k=-4..4} e^{-k^2/2})^2
    S1 = sum(math.exp(-k * k / 2.0) for k in range(-4, 5))
    G = oracle.gaussian_taps(1.0, 9)
    assert abs(G[4, 4] - 1.0 / (S1 * S1)) < 1e-15
    assert abs(1.0 / S1 - 0.3989434) < 1e-6
    # wide window: the normaliser tends to 2 pi sigma^2 (the Gaussian pdf);
    # the lattice sum differs from it by a relative 2 e^{-2 pi^2 sigma^2}
    G = oracle.gaussian_taps(1.0, 31)
    assert abs(G[15, 15] * 2.0 * math.pi - 1.0) < 1e-7


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("H,W", [(7, 11), (11, 7), (2, 5), (5, 2), (1, 6),
                                 (6, 1), (1, 1)])
def test_gradient_matches_numpy(H, W):
    f = rng_image((H, W), 3)
    fx, fy = oracle.gradient(f)
    ex, ey = np_gradient(f)
    np.testing.assert_array_equal(fx, ex)
    np.testing.assert_array_equal(fy, ey)


def test_gradient_single_pixel_by_hand():
    phi = -np.ones((8, 8))
    phi[3, 4] = 1.0
    fx, fy = oracle.gradient(phi)
    s = np.hypot(fx, fy)
    for (y, x) in [(2, 4), (4, 4), (3, 3), (3, 5)]:
        assert s[y, x] == 1.0
    assert s[3, 4] == 0.0
    for (y, x) in [(2, 3), (2, 5), (4, 3), (4, 5), (0, 0)]:
        assert s[y, x] == 0.0
    # corner pixel: one-sided differences of 2 in both directions
    phi = -np.ones((5, 6))
    phi[0, 0] = 1.0
    fx, fy = oracle.gradient(phi)
    assert fx[0, 0] == -2.0 and fy[0, 0] == -2.0
    assert fx[0, 1] == -1.0 and fy[1, 0] == -1.0
    # constant field: no gradient
    fx, fy = oracle.gradient(np.full((4, 9), 0.7))
    assert not fx.any() and not fy.any()


# ---------------------------------------------------------------- convolution
def test_conv_matches_scipy_with_asymmetric_kernel():
    f = rng_image((13, 17), 4)
    G = rng_image((5, 5), 5)   # asymmetric: pins the flip convention
    out = oracle.conv_same(f, G)
    ref = signal.convolve2d(f, G, mode="same", boundary="fill")
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-14)


def test_conv_small_image_smaller_than_kernel():
    f = rng_image((3, 2), 6)
    G = oracle.gaussian_taps(2.0, 9)
    np.testing.assert_allclose(
        oracle.conv_same(f, G),
        signal.convolve2d(f, G, mode="same", boundary="fill"), rtol=1e-13)


# ---------------------------------------------------------------- edge indicator
@pytest.mark.parametrize("B", [1, 3])
def test_edge_indicator_matches_scipy(B):
    I = rng_image((B, 12, 15), 7)
    g = oracle.edge_indicator(I, sigma1=1.5, ts1=7, edge_scale=255.0)
    J = 255.0 * I.mean(axis=0)
    g1 = gauss_1d(1.5, 7)
    S = signal.convolve2d(J, np.outer(g1, g1), mode="same", boundary="fill")
    sx, sy = np_gradient(S)
    ref = 1.0 / (1.0 + sx ** 2 + sy ** 2)
    np.testing.assert_allclose(g, ref, rtol=1e-12)
    assert (g > 0).all() and (g <= 1).all()


def test_edge_indicator_band_mean():
    I = rng_image((1, 10, 10), 8)
    g1 = oracle.edge_indicator(I)
    g3 = oracle.edge_indicator(np.repeat(I, 3, axis=0))
    np.testing.assert_allclose(g1, g3, rtol=1e-13)


# ---------------------------------------------------------------- region statistics
def test_region_means_are_masked_means():
    I = rng_image((2, 9, 14), 9)
    phi = rng_phi(9, 14, 10)
    phi[0, 0] = 0.0   # a zero belongs to the phi >= 0 side (Eq. 15)
    cp, cm, n = oracle.region_stats(I, phi)
    P = phi >= 0
    assert n == P.sum()
    for b in range(2):
        assert abs(cp[b] - I[b][P].mean()) < 1e-15
        assert abs(cm[b] - I[b][~P].mean()) < 1e-15


def test_normaliser_closed_form_single_band():
    I = rng_image((1, 16, 12), 11)
    phi = rng_phi(16, 12, 12)
    R, norm, cp, cm, z = oracle.region_force(I, phi)
    assert not z
    s = cp[0] + cm[0]
    closed = abs(cp[0] - cm[0]) * max(abs(2 * I.max() - s), abs(2 * I.min() - s))
    assert abs(norm - closed) <= 1e-14 * closed
    assert abs(np.abs(R).max() - 1.0) < 1e-15


def test_region_force_sign_and_squared_form():
    # Eq. 15 with lambda = 1: -(I - c+)^2 + (I - c-)^2 equals
    # (c+ - c-)(2I - c+ - c-), the numerator of Eq. 17 (not Eq. 16's plus).
    I = rng_image((1, 10, 10), 13)
    phi = rng_phi(10, 10, 14)
    R, norm, cp, cm, _ = oracle.region_force(I, phi)
    D = -(I[0] - cp[0]) ** 2 + (I[0] - cm[0]) ** 2
    np.testing.assert_allclose(R, D / np.abs(D).max(), rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- one step, by an independent formulation
@pytest.mark.parametrize("term,B,H,W,sigma,ts", [
    ("region", 1, 8, 8, 1.0, 9),
    ("region", 3, 8, 11, 1.5, 5),
    ("region", 2, 11, 8, 2.0, 9),
    ("edge", 1, 8, 8, 1.0, 9),
    ("edge", 4, 9, 12, 1.0, 7),
    ("region", 1, 1, 9, 1.0, 5),
    ("region", 1, 9, 1, 1.0, 3),
])
def test_step_against_independent_formulation(term, B, H, W, sigma, ts):
    I = rng_image((B, H, W), 20 + B)
    phi = rng_phi(H, W, 30 + H)
    if phi.min() == phi.max():
        phi[0, 0] = -phi[0, 0]
    g = oracle.edge_indicator(I) if term == "edge" else None
    v, norm, cp, cm, z = oracle.step(I, phi, term=term, g=g, dt=15.0,
                                     sigma=sigma, ts=ts)
    ref = independent_step(I, phi, term, g=g, dt=15.0, sigma=sigma, ts=ts)
    np.testing.assert_allclose(v, ref, rtol=1e-11, atol=1e-12)


def test_five_iterations_against_independent_formulation():
    I = rng_image((2, 8, 8), 40)
    phi0 = rng_phi(8, 8, 41)
    phi = phi0.copy()
    for _ in range(5):
        v_ref = independent_step(I, phi, "region", dt=15.0, sigma=1.0, ts=9)
        phi = np.where(v_ref >= 0, 1.0, -1.0)
    v, mask, st = oracle.evolve(I, phi0, iterations=5)
    np.testing.assert_allclose(v, v_ref, rtol=1e-11, atol=1e-12)
    assert np.array_equal(mask.astype(bool), v_ref >= 0)


def test_sampled_step_equals_full_step():
    I = rng_image((1, 20, 23), 42)
    phi = rng_phi(20, 23, 43)
    v, *_ = oracle.step(I, phi, sigma=2.0, ts=9)
    ys = np.array([0, 19, 5, 0, 19, 10])
    xs = np.array([0, 22, 7, 22, 0, 11])
    vs, *_ = oracle.step_sampled(I, phi, ys, xs, sigma=2.0, ts=9)
    np.testing.assert_array_equal(vs, v[ys, xs])


# ---------------------------------------------------------------- invariants
def test_constant_image_gives_no_data_motion():
    H, W = 24, 31
    I = np.full((1, H, W), 0.42)
    phi0 = rng_phi(H, W, 50)
    R, norm, cp, cm, z = oracle.region_force(I, phi0)
    # the two means agree to rounding; the contrast rule makes R exactly 0
    assert abs(cp[0] - cm[0]) < 1e-14 and norm == 0.0 and z and not R.any()
    v, mask, st = oracle.evolve(I, phi0, iterations=1)
    ref = signal.convolve2d(phi0, np.outer(gauss_1d(1.0, 9), gauss_1d(1.0, 9)),
                            mode="same", boundary="fill")
    np.testing.assert_allclose(v, ref, rtol=1e-12, atol=1e-14)
    assert st["degenerate"]


def test_small_real_contrast_is_not_degenerate():
    I = np.full((1, 12, 12), 0.5)
    I[0, :6] += 1e-3
    phi = np.where(np.arange(12)[:, None] < 6, 1.0, -1.0) * np.ones((12, 12))
    R, norm, cp, cm, z = oracle.region_force(I, phi)
    assert not z and abs(np.abs(R).max() - 1.0) < 1e-12


def test_affine_intensity_invariance():
    img, truth, _ = scenes.rect_scene(64, 64, 30, 20, noise=0.05)
    phi0 = scenes.circle_phi(64, 64, radius=16)
    v1, m1, _ = oracle.evolve(img, phi0, iterations=8)
    v2, m2, _ = oracle.evolve(3.7 * img.astype(np.float64) - 1.2, phi0,
                              iterations=8)
    np.testing.assert_allclose(v1, v2, rtol=1e-9, atol=1e-9)
    assert np.array_equal(m1, m2)


def test_sign_antisymmetry_of_region_term():
    img, truth, _ = scenes.rect_scene(64, 64, 30, 20, noise=0.05)
    phi0 = scenes.circle_phi(64, 64, radius=16)
    v1, m1, s1 = oracle.evolve(img, phi0, iterations=8)
    v2, m2, s2 = oracle.evolve(img, -phi0, iterations=8)
    assert (v1 != 0).all()
    np.testing.assert_allclose(v2, -v1, rtol=1e-12, atol=1e-12)
    assert np.array_equal(m1, 1 - m2)
    np.testing.assert_allclose(s1["c_plus"], s2["c_minus"], rtol=1e-13)


def test_duplicated_and_constant_bands_change_nothing():
    img, truth, _ = scenes.rect_scene(48, 40, 20, 12, noise=0.05)
    phi0 = scenes.circle_phi(48, 40, radius=12)
    v1, m1, _ = oracle.evolve(img, phi0, iterations=6)
    v3, m3, _ = oracle.evolve(np.repeat(img, 3, axis=0), phi0, iterations=6)
    np.testing.assert_allclose(v1, v3, rtol=1e-10, atol=1e-10)
    with_const = np.concatenate([img, np.full_like(img, 0.5)], axis=0)
    vc, mc, _ = oracle.evolve(with_const, phi0, iterations=6)
    np.testing.assert_allclose(v1, vc, rtol=1e-10, atol=1e-10)


def test_edge_update_never_decreases_phi():
    # E_Td = g > 0 and |grad phi| >= 0, so u >= phi (Sec. III-D, Step 3)
    img, truth, _ = scenes.rect_scene(40, 40, 16, 10, noise=0.1)
    g = oracle.edge_indicator(img)
    phi = rng_phi(40, 40, 60)
    u, _ = oracle.update(img, phi, term="edge", g=g)
    assert (u >= phi).all() and (u > phi).any()


def test_degenerate_all_positive_lsf():
    I = rng_image((1, 10, 10), 61)
    phi = np.ones((10, 10))
    R, norm, cp, cm, z = oracle.region_force(I, phi)
    assert z and not R.any() and cm[0] == 0.0
    assert abs(cp[0] - I.mean()) < 1e-15


# ---------------------------------------------------------------- the paper's synthetic experiments
def test_noiseless_truth_is_exact_fixed_point():
    img, truth, _ = scenes.rect_scene(noise=0.0)
    phi_t = np.where(truth, 1.0, -1.0)
    for it in (1, 2, 25):
        v, mask, st = oracle.evolve(img, phi_t, dt=15.0, sigma=1.0, ts=9,
                                    iterations=it)
        assert st["last_flips"] == 0
        assert np.array_equal(mask.astype(bool), truth)
    # the scene is stored in FP32: the exact means are the FP32 levels
    assert abs(st["c_plus"][0] - float(np.float32(0.7))) < 1e-12
    assert abs(st["c_minus"][0] - float(np.float32(0.3))) < 1e-12


def test_noiseless_circle_start_ends_on_the_true_contour():
    img, truth, _ = scenes.rect_scene(noise=0.0)
    phi0 = scenes.circle_phi(256, 256)
    _, m200, _ = oracle.evolve(img, phi0, iterations=200)
    _, m204, _ = oracle.evolve(img, phi0, iterations=204)
    # settled: with dt = 15 the straight edges overshoot by one pixel each
    # way (period 2) and the corners cycle with period 4
    assert np.array_equal(m200, m204)
    m = m200.astype(bool)
    ring = ndimage.binary_dilation(truth) & ~ndimage.binary_erosion(truth)
    near = ndimage.binary_dilation(ring)
    bad = m != truth
    assert bad.sum() < 400 and not (bad & ~near).any()


def test_edge_term_stops_one_pixel_outside_the_object():
    # Fig. 2(a) / 3(a): phi < 0 inside a curve around the object moves in and
    # stops where g is small, i.e. on the pixel ring just outside the object.
    img, truth, (y0, x0, y1, x1) = scenes.rect_scene(noise=0.0)
    g = oracle.edge_indicator(img)
    phi0 = scenes.box_phi(256, 256, [(y0 - 20, x0 - 20, y1 + 20, x1 + 20)])
    v, mask, st = oracle.evolve(img, phi0, term="edge", g=g, iterations=100)
    cross = ndimage.generate_binary_structure(2, 1)
    assert st["last_flips"] == 0
    assert np.array_equal(~mask.astype(bool), ndimage.binary_dilation(truth, cross))


def test_edge_term_vanishes_when_the_curve_crosses_the_object():
    # Fig. 2(b): the negative region only shrinks and disappears.
    img, truth, (y0, x0, y1, x1) = scenes.rect_scene(noise=0.0)
    g = oracle.edge_indicator(img)
    cy = (y0 + y1) // 2
    phi0 = scenes.box_phi(256, 256, [(cy - 10, x0 - 30, cy + 80, x0 + 40)])
    v, mask, st = oracle.evolve(img, phi0, term="edge", g=g, iterations=200)
    assert mask.all()
    # Fig. 2(c): the region term extracts the object from the same start
    v, mask, st = oracle.evolve(img, phi0, term="region", iterations=200)
    m = mask.astype(bool)
    assert min((m != truth).sum(), (m == truth).sum()) < 400


def test_noise_defeats_the_edge_term_not_the_region_term():
    # Fig. 4: additive noise of standard deviation 0.2.
    img, truth, (y0, x0, y1, x1) = scenes.rect_scene(noise=0.2)
    g = oracle.edge_indicator(img)
    phi_e = scenes.box_phi(256, 256, [(y0 - 20, x0 - 20, y1 + 20, x1 + 20)])
    _, mask, _ = oracle.evolve(img, phi_e, term="edge", g=g, iterations=200)
    assert ((~mask.astype(bool)) != truth).sum() > truth.sum() // 2
    _, mask, _ = oracle.evolve(img, scenes.circle_phi(256, 256), iterations=200)
    m = mask.astype(bool)
    assert min((m != truth).sum(), (m == truth).sum()) < 300


def test_tie_goes_to_plus():
    # Table I step 3 / the listing: a zero of the smoothed LSF becomes +1.
    # TS = 1 makes the smoothing the identity and a constant image makes R = 0,
    # so v = phi exactly and a zero in phi0 is a tie.
    I = np.full((1, 5, 6), 0.25)
    phi0 = -np.ones((5, 6))
    phi0[:, :2] = 1.0
    phi0[2, 4] = 0.0
    v, mask, st = oracle.evolve(I, phi0, ts=1, iterations=1)
    assert v[2, 4] == 0.0 and mask[2, 4] == 1
    v, mask, st = oracle.evolve(I, phi0, ts=1, iterations=2)
    assert v[2, 4] == 1.0 and mask[2, 4] == 1


def test_early_stop_rule():
    img, truth, _ = scenes.rect_scene(noise=0.0)
    phi_t = np.where(truth, 1.0, -1.0)
    _, _, st = oracle.evolve(img, phi_t, iterations=50, early_stop_frac=1e-4)
    assert st["iterations_run"] == 1 and st["last_flips"] == 0


def test_reinit_period_zero_keeps_real_lsf():
    img, truth, _ = scenes.rect_scene(32, 32, 12, 8, noise=0.05)
    phi0 = scenes.circle_phi(32, 32, radius=8)
    v1, _, _ = oracle.evolve(img, phi0, iterations=1)
    v2, _, _ = oracle.evolve(img, phi0, iterations=2, reinit_period=0)
    ref, *_ = oracle.step(img, v1)
    np.testing.assert_allclose(v2, ref, rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------- variants: Table I order, replicate padding
def replicate_conv(f, G):
    """'same' convolution with the nearest image value outside (scipy)."""
    return ndimage.convolve(f, G, mode="nearest")


def independent_variant_step(I, phi, term, g=None, dt=15.0, sigma=1.0, ts=9,
                             order="listing", reinit=True, padding="zero"):
    """independent_step's update, then Table I's re-initialisation of u when
    asked, then the smoothing with zero (scipy impulse matrix) or replicate
    (scipy 'nearest') padding."""
    B, H, W = I.shape
    fx, fy = np_gradient(phi)
    s = np.hypot(fx, fy)
    if term == "region":
        P = phi >= 0
        D = np.zeros_like(phi)
        for b in range(B):
            cp = I[b][P].mean()
            cm = I[b][~P].mean()
            D += -(I[b] - cp) ** 2 + (I[b] - cm) ** 2
        R = D / np.abs(D).max()
    else:
        R = g
    u = phi + dt * R * s
    if order == "table1" and reinit:
        u = np.where(u >= 0, 1.0, -1.0)
    g1 = gauss_1d(sigma, ts)
    G = np.outer(g1, g1)
    if padding == "zero":
        return (conv_matrix(H, W, G) @ u.ravel()).reshape(H, W)
    return replicate_conv(u, G)


def test_replicate_convolution_matches_scipy_nearest():
    f = rng_image((13, 17), 70)
    G = np.random.default_rng(71).uniform(0.0, 1.0, (5, 5))   # asymmetric
    np.testing.assert_allclose(oracle.conv_same(f, G, "replicate"), replicate_conv(f, G),
                               rtol=1e-12, atol=1e-14)
    # a 1-pixel-wide image: every outside value is that column's
    f1 = rng_image((9, 1), 72)
    np.testing.assert_allclose(oracle.conv_same(f1, G, "replicate"), replicate_conv(f1, G),
                               rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("term,B,H,W,order,reinit,padding", [
    ("region", 1, 9, 11, "table1", True, "zero"),
    ("region", 3, 8, 10, "table1", True, "replicate"),
    ("region", 1, 10, 9, "listing", True, "replicate"),
    ("edge", 1, 9, 9, "table1", True, "zero"),
    ("edge", 4, 8, 12, "listing", True, "replicate"),
    ("region", 2, 9, 9, "table1", False, "zero"),
])
def test_variant_step_against_independent_formulation(term, B, H, W, order, reinit, padding):
    I = rng_image((B, H, W), 80 + B)
    phi = rng_phi(H, W, 81 + H)
    g = oracle.edge_indicator(I) if term == "edge" else None
    v, *_ = oracle.step(I, phi, term=term, g=g, order=order, reinit=reinit, padding=padding)
    ref = independent_variant_step(I, phi, term, g=g, order=order, reinit=reinit,
                                   padding=padding)
    np.testing.assert_allclose(v, ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("padding", ["zero", "replicate"])
def test_table1_evolution_against_independent_formulation(padding):
    I = rng_image((1, 9, 10), 90)
    phi0 = rng_phi(9, 10, 91)
    phi = phi0.copy()
    for _ in range(5):
        v_ref = independent_variant_step(I, phi, "region", order="table1", padding=padding)
        phi = v_ref                   # Table I: the next iteration starts from v
    v, mask, st = oracle.evolve(I, phi0, iterations=5, order="table1", padding=padding)
    np.testing.assert_allclose(v, v_ref, rtol=1e-11, atol=1e-12)
    assert np.array_equal(mask.astype(bool), v_ref >= 0)


def test_table1_order_keeps_v_within_one_and_replicate_keeps_constants():
    I = rng_image((1, 20, 24), 92)
    phi0 = rng_phi(20, 24, 93)
    for padding in ("zero", "replicate"):
        v, _, _ = oracle.evolve(I, phi0, iterations=4, order="table1", padding=padding)
        assert np.abs(v).max() <= 1.0 + 1e-12
    # a constant LSF has no gradient, so u = phi: replicate padding keeps it,
    # zero padding pulls the border toward 0
    g = np.full((12, 14), 0.5)
    ones = np.ones((12, 14))
    v_rep, *_ = oracle.step(I[:, :12, :14], ones, term="edge", g=g, padding="replicate")
    v_zero, *_ = oracle.step(I[:, :12, :14], ones, term="edge", g=g)
    np.testing.assert_allclose(v_rep, 1.0, rtol=0, atol=1e-14)
    assert v_zero[0, 0] < 0.75 and abs(v_zero[6, 7] - 1.0) < 1e-14


def test_table1_tie_goes_to_plus():
    # constant image: R = 0 (degenerate), so u = phi; where phi = 0 the
    # re-initialisation before smoothing must give +1
    I = np.full((1, 7, 7), 0.4)
    phi = np.full((7, 7), -1.0)
    phi[2:5, 2:5] = 0.0
    v, *_ = oracle.step(I, phi, ts=1, order="table1")
    assert (v[2:5, 2:5] == 1.0).all() and (v[0] == -1.0).all()


def test_results_do_not_depend_on_the_thread_count():
    # the per-pixel maps and max|D| may run on several threads; every value,
    # sum and count must come out the same as on one thread (sizes above the
    # threshold at which the maps go parallel)
    I = rng_image((3, 260, 270), 94)
    phi0 = rng_phi(260, 270, 95)
    g = oracle.edge_indicator(I, 1.0, 9, 255.0)
    runs = []
    try:
        for n in (1, 4, 0):
            oracle.set_threads(n)
            v, mask, st = oracle.evolve(I, phi0, iterations=3)
            ve, _, ste = oracle.evolve(I, phi0, "edge", g=g, iterations=3,
                                       padding="replicate")
            runs.append((v, mask, st, ve, ste, oracle.edge_indicator(I, 1.0, 9, 255.0)))
    finally:
        oracle.set_threads(0)
    for other in runs[1:]:
        assert np.array_equal(runs[0][0], other[0]) and np.array_equal(runs[0][1], other[1])
        assert runs[0][2]["norm"] == other[2]["norm"]
        assert np.array_equal(runs[0][2]["c_plus"], other[2]["c_plus"])
        assert np.array_equal(runs[0][3], other[3]) and np.array_equal(runs[0][5], other[5])


# ---------------------------------------------------------------- re-initialisation schedule, flip count, early stop
def hand_evolve(I, phi0, iterations, period=1, frac=0.0, order="listing",
                sigma=1.0, ts=9, dt=15.0):
    """The whole region-term loop written out by hand on independent_step /
    independent_variant_step.

    Re-initialisation (Table I step 3; Sec. III-D, Step 3: "periodically")
    comes after every `period`-th iteration, i.e. after iterations
    period-1, 2*period-1, ... (0-based); period 1 = every iteration, 0 = never.
    The sign changes of an iteration compare v >= 0 with the LSF it started
    from, phi >= 0; Step 5 stops after the first iteration with fewer than
    frac * H * W of them.  Returns (v, list of per-iteration sign changes)."""
    N = phi0.size
    phi = phi0.copy()
    history = []
    for n in range(iterations):
        reinit = period == 1 or (period > 1 and n % period == period - 1)
        if order == "listing":
            v = independent_step(I, phi, "region", dt=dt, sigma=sigma, ts=ts)
        else:
            v = independent_variant_step(I, phi, "region", dt=dt, sigma=sigma, ts=ts,
                                         order="table1", reinit=reinit)
        changed = 0
        for y in range(phi.shape[0]):
            for x in range(phi.shape[1]):
                if (v[y, x] >= 0) != (phi[y, x] >= 0):
                    changed += 1
        history.append(changed)
        if order == "listing" and reinit:
            phi = np.where(v >= 0, 1.0, -1.0)
        else:
            phi = v
        if frac > 0 and changed < frac * N:
            break
    return v, history


@pytest.mark.parametrize("period", [2, 3])
@pytest.mark.parametrize("order", ["listing", "table1"])
def test_reinit_period_schedule_against_hand_loop(period, order):
    img, truth, _ = scenes.rect_scene(16, 20, 8, 6, noise=0.05)
    phi0 = scenes.circle_phi(16, 20, radius=5)
    its = 2 * period + 1          # ends one iteration after a re-initialisation
    v_ref, hist = hand_evolve(img.astype(np.float64), phi0, its, period=period,
                              order=order)
    v, mask, st = oracle.evolve(img, phi0, iterations=its, reinit_period=period,
                                order=order)
    np.testing.assert_allclose(v, v_ref, rtol=1e-11, atol=1e-12)
    assert st["iterations_run"] == its and st["last_flips"] == hist[-1]
    # the schedule matters: the same run re-initialising after iterations
    # 0, period, 2*period, ... (one iteration early) gives another v
    shifted = phi0.copy()
    for n in range(its):
        early = n % period == 0
        if order == "listing":
            w = independent_step(img.astype(np.float64), shifted, "region")
            shifted = np.where(w >= 0, 1.0, -1.0) if early else w
        else:
            w = independent_variant_step(img.astype(np.float64), shifted, "region",
                                         order="table1", reinit=early)
            shifted = w
    assert np.abs(w - v).max() > 1e-6


def test_sign_changes_counted_against_the_starting_lsf():
    img, truth, _ = scenes.rect_scene(32, 32, 14, 10, noise=0.05)
    phi0 = scenes.circle_phi(32, 32, radius=8)
    I = img.astype(np.float64)
    v_ref, hist = hand_evolve(I, phi0, 6)
    assert all(h > 0 for h in hist)          # non-zero counts throughout
    for its in (1, 3, 6):
        _, _, st = oracle.evolve(img, phi0, iterations=its)
        assert st["last_flips"] == hist[its - 1]
    # real-valued LSF between re-initialisations (period 3)
    _, hist3 = hand_evolve(I, phi0, 5, period=3)
    _, _, st = oracle.evolve(img, phi0, iterations=5, reinit_period=3)
    assert st["last_flips"] == hist3[-1]


def test_zero_lsf_value_is_not_a_sign_change():
    # TS = 1 and a constant image make v = phi exactly; a pixel with phi = 0
    # keeps v = 0, on the phi >= 0 side both times: no sign change.
    I = np.full((1, 6, 7), 0.3)
    phi0 = np.where(np.arange(7)[None, :] < 3, 1.0, -1.0) * np.ones((6, 7))
    phi0[1, 5] = 0.0
    phi0[4, 1] = 0.0
    _, _, st = oracle.evolve(I, phi0, ts=1, iterations=1)
    assert st["last_flips"] == 0


def test_early_stop_after_several_iterations():
    img, truth, _ = scenes.rect_scene(32, 32, 14, 10, noise=0.05)
    phi0 = scenes.circle_phi(32, 32, radius=8)
    I = img.astype(np.float64)
    N = 32 * 32                          # a power of two: k / N is exact
    _, hist = hand_evolve(I, phi0, 12)
    # an iteration k >= 1 whose count is below every earlier one
    ks = [k for k in range(1, len(hist)) if 0 < hist[k] < min(hist[:k])]
    assert ks, hist
    k = ks[0]
    # threshold between the counts: the loop stops right after iteration k
    frac = (hist[k] + 0.5) / N
    v_ref, h = hand_evolve(I, phi0, 12, frac=frac)
    v, mask, st = oracle.evolve(img, phi0, iterations=12, early_stop_frac=frac)
    assert len(h) == k + 1 and st["iterations_run"] == k + 1
    assert st["last_flips"] == hist[k]
    np.testing.assert_allclose(v, v_ref, rtol=1e-11, atol=1e-12)
    # a threshold equal to the count does not stop there (the rule is strict)
    frac = hist[k] / N
    v_ref, h = hand_evolve(I, phi0, 12, frac=frac)
    v, mask, st = oracle.evolve(img, phi0, iterations=12, early_stop_frac=frac)
    assert st["iterations_run"] == len(h) and len(h) > k + 1
    assert st["last_flips"] == h[-1]
    np.testing.assert_allclose(v, v_ref, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------- given statistics (row strips)
@pytest.mark.parametrize("B,term", [(1, "region"), (3, "region"), (1, "edge")])
def test_step_with_given_statistics(B, term):
    # with the image's own statistics the step is the ordinary step; on a
    # row strip with r + 1 halo rows and the whole image's statistics the
    # owned rows are those of the whole image's step (Eq. 18 and the
    # smoothing reach r + 1 rows)
    I = rng_image((B, 23, 17), 120 + B)
    phi = rng_phi(23, 17, 121)
    g = oracle.edge_indicator(I) if term == "edge" else None
    v, norm, cp, cm, z = oracle.step(I, phi, term=term, g=g, sigma=1.5, ts=7)
    v2 = oracle.step_given(I, phi, cp, cm, norm, z, term=term, g=g, sigma=1.5, ts=7)
    np.testing.assert_array_equal(v, v2)
    h = 4                                     # r + 1 for TS 7
    y0, y1 = 9, 15
    sl = slice(y0 - h, y1 + h)
    gs = g[sl] if g is not None else None
    vs = oracle.step_given(I[:, sl], phi[sl], cp, cm, norm, z, term=term, g=gs, sigma=1.5,
                           ts=7)
    np.testing.assert_array_equal(vs[h:h + (y1 - y0)], v[y0:y1])
    # a strip at the image's top edge has no halo above
    vt = oracle.step_given(I[:, :6 + h], phi[:6 + h], cp, cm, norm, z, term=term,
                           g=g[:6 + h] if g is not None else None, sigma=1.5, ts=7)
    np.testing.assert_array_equal(vt[:6], v[:6])
