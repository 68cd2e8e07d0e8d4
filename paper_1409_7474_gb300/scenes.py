"""Seeded synthetic scenes and initial level set functions.

These generators are the only code shared by the GPU path's tests/benchmark
and the FP64 oracle's checks.  They draw images and initial LSFs; they hold
none of the method's arithmetic.

The paper's experiments use Google Maps RGB images (Table II) that are not
available here.  The scenes below stand in for them with the structure the
paper extracts: bright roofs (concrete), dark road strips (asphalt), a
runway, on a flat background, with additive Gaussian noise (Sec. III-E.3 uses
additive white noise) and, for the multi-band scene, smooth illumination
ramps.  Every random choice comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rect_scene",
    "circle_phi",
    "box_phi",
    "multiband_scene",
    "large_scene",
    "tile_scene",
]


def circle_phi(H: int, W: int, cy: float | None = None, cx: float | None = None,
               radius: float = 64.0, inside: float = 1.0) -> np.ndarray:
    """Binary LSF of Eq. 13: ``inside`` within the circle, ``-inside`` outside.

    The default centre is the image centre ((H-1)/2, (W-1)/2).
    """
    cy = (H - 1) / 2.0 if cy is None else cy
    cx = (W - 1) / 2.0 if cx is None else cx
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = (xx - cx) ** 2 + (yy - cy) ** 2
    phi = np.where(d2 <= radius * radius, inside, -inside)
    return phi.astype(np.float32)


def box_phi(H: int, W: int, boxes, inside: float = -1.0) -> np.ndarray:
    """Binary LSF: ``inside`` within any box (y0, x0, y1, x1; half-open),
    ``-inside`` elsewhere.  The edge term needs phi < 0 inside a zero level
    curve that encloses the object (Sec. III-E.2), hence the default."""
    phi = np.full((H, W), -inside, np.float32)
    for (y0, x0, y1, x1) in boxes:
        phi[max(y0, 0):min(y1, H), max(x0, 0):min(x1, W)] = inside
    return phi


def rect_scene(H: int = 256, W: int = 256, rect_w: int = 100, rect_h: int = 60,
               background: float = 0.3, foreground: float = 0.7,
               noise: float = 0.05, seed_pos: int = 1, seed_noise: int = 2):
    """Two-level image: one axis-aligned rectangle on a flat background.

    The rectangle's top-left corner is drawn uniformly so that it lies fully
    inside the image (seed ``seed_pos``); N(0, noise^2) is added (seed
    ``seed_noise``).  Returns (image[1, H, W] float32, truth[H, W] bool,
    box (y0, x0, y1, x1)).
    """
    rng = np.random.default_rng(seed_pos)
    y0 = int(rng.integers(0, H - rect_h + 1))
    x0 = int(rng.integers(0, W - rect_w + 1))
    truth = np.zeros((H, W), bool)
    truth[y0:y0 + rect_h, x0:x0 + rect_w] = True
    img = np.where(truth, foreground, background).astype(np.float64)
    if noise > 0:
        img = img + np.random.default_rng(seed_noise).normal(0.0, noise, (H, W))
    return img.astype(np.float32)[None], truth, (y0, x0, y0 + rect_h, x0 + rect_w)


def _stamp_rotated_rect(cls, label, cy, cx, h, w, angle):
    H, W = cls.shape
    half = 0.5 * math.hypot(h, w) + 1
    ya, yb = max(int(cy - half), 0), min(int(cy + half) + 1, H)
    xa, xb = max(int(cx - half), 0), min(int(cx + half) + 1, W)
    if ya >= yb or xa >= xb:
        return
    yy, xx = np.mgrid[ya:yb, xa:xb]
    c, s = math.cos(angle), math.sin(angle)
    dy, dx = yy - cy, xx - cx
    u = c * dx + s * dy
    v = -s * dx + c * dy
    inside = (np.abs(u) <= w / 2.0) & (np.abs(v) <= h / 2.0)
    cls[ya:yb, xa:xb][inside] = label


def _stamp_segment(cls, label, p0, p1, width):
    H, W = cls.shape
    (y0, x0), (y1, x1) = p0, p1
    r = width / 2.0
    ya, yb = max(int(min(y0, y1) - r) - 1, 0), min(int(max(y0, y1) + r) + 2, H)
    xa, xb = max(int(min(x0, x1) - r) - 1, 0), min(int(max(x0, x1) + r) + 2, W)
    if ya >= yb or xa >= xb:
        return
    yy, xx = np.mgrid[ya:yb, xa:xb].astype(np.float64)
    vy, vx = y1 - y0, x1 - x0
    L2 = vy * vy + vx * vx
    if L2 == 0:
        t = np.zeros_like(yy)
    else:
        t = np.clip(((yy - y0) * vy + (xx - x0) * vx) / L2, 0.0, 1.0)
    d2 = (yy - (y0 + t * vy)) ** 2 + (xx - (x0 + t * vx)) ** 2
    cls[ya:yb, xa:xb][d2 <= r * r] = label


def multiband_scene(H: int = 2048, W: int = 2048, B: int = 4, seed: int = 7,
                    n_roofs: int = 40, noise: float = 0.03,
                    ramp: float = 0.1):
    """Four-band (B, G, R, NIR) uint16 scene.

    Classes: 0 background, 1 road, 2 roof, 3 runway.  6-12 road polylines
    8-20 px wide; ``n_roofs`` rectangles with sides 20-80 px at random
    orientations; one 60 x 1500 px runway.  Per-class band means are drawn
    from U(0.15, 0.85); N(0, noise^2) is added per band; a multiplicative
    illumination ramp 1 +/- ``ramp`` varies linearly in x and y.  Values are
    stored as uint16 (value * 65535, rounded, clipped).

    Returns a dict with ``image`` (B, H, W) uint16, ``classes`` (H, W) uint8,
    ``runway_box`` and ``roof_boxes`` (y0, x0, y1, x1).
    """
    rng = np.random.default_rng(seed)
    cls = np.zeros((H, W), np.uint8)
    # runway first so roads and roofs may cross it
    rw_len, rw_wid = min(1500, W - 40), 60
    ry = int(rng.integers(40, H - rw_wid - 40))
    rx = int(rng.integers(20, W - rw_len - 20 + 1))
    cls[ry:ry + rw_wid, rx:rx + rw_len] = 3
    runway_box = (ry, rx, ry + rw_wid, rx + rw_len)
    n_roads = int(rng.integers(6, 13))
    for _ in range(n_roads):
        width = float(rng.uniform(8, 20))
        n_pts = int(rng.integers(3, 7))
        pts = [(float(rng.uniform(0, H)), float(rng.uniform(0, W)))]
        for _ in range(n_pts - 1):
            ang = float(rng.uniform(0, 2 * math.pi))
            step = float(rng.uniform(150, 500))
            y = min(max(pts[-1][0] + step * math.sin(ang), 0), H - 1)
            x = min(max(pts[-1][1] + step * math.cos(ang), 0), W - 1)
            pts.append((y, x))
        for a, b in zip(pts[:-1], pts[1:]):
            _stamp_segment(cls, 1, a, b, width)
    roof_boxes = []
    for _ in range(n_roofs):
        h = float(rng.uniform(20, 80))
        w = float(rng.uniform(20, 80))
        cy = float(rng.uniform(50, H - 50))
        cx = float(rng.uniform(50, W - 50))
        ang = float(rng.uniform(0, math.pi))
        _stamp_rotated_rect(cls, 2, cy, cx, h, w, ang)
        half = 0.5 * math.hypot(h, w)
        roof_boxes.append((int(cy - half), int(cx - half), int(cy + half) + 1,
                           int(cx + half) + 1))
    means = rng.uniform(0.15, 0.85, size=(4, B))
    img = means[cls].transpose(2, 0, 1).astype(np.float64)  # (B, H, W)
    yy = np.linspace(-1.0, 1.0, H)[:, None]
    xx = np.linspace(-1.0, 1.0, W)[None, :]
    gy, gx = rng.uniform(-1, 1, size=2)
    norm = max(abs(gy) + abs(gx), 1e-9)
    illum = 1.0 + ramp * (gy * yy + gx * xx) / norm
    img = img * illum[None]
    img = img + rng.normal(0.0, noise, size=img.shape)
    img = np.clip(np.rint(img * 65535.0), 0, 65535).astype(np.uint16)
    return {"image": img, "classes": cls, "runway_box": runway_box,
            "roof_boxes": roof_boxes}


def large_scene(H: int = 8192, W: int = 8192, n_roofs: int = 2000,
                n_roads: int = 200, noise: float = 0.05, seed: int = 11,
                background: float = 0.3, roof: float = 0.7,
                road: float = 0.15):
    """Single-band scene: the two-level rectangle generator scaled up.

    ``n_roofs`` axis-aligned bright rectangles with sides 20-80 px and
    ``n_roads`` dark straight strips 8-20 px wide running across part of the
    image (horizontal or vertical), on a flat background, plus N(0, noise^2).
    Returns a dict with ``image`` (1, H, W) float32, ``truth`` (H, W) bool
    (roofs) and ``roof_boxes``.
    """
    rng = np.random.default_rng(seed)
    img = np.full((H, W), background, np.float32)
    for _ in range(n_roads):
        width = int(rng.integers(8, 21))
        length = int(rng.integers(H // 8, H // 2 + 1))
        if rng.random() < 0.5:
            y = int(rng.integers(0, H - width))
            x = int(rng.integers(0, max(W - length, 1)))
            img[y:y + width, x:x + length] = road
        else:
            x = int(rng.integers(0, W - width))
            y = int(rng.integers(0, max(H - length, 1)))
            img[y:y + length, x:x + width] = road
    truth = np.zeros((H, W), bool)
    roof_boxes = []
    for _ in range(n_roofs):
        h = int(rng.integers(20, 81))
        w = int(rng.integers(20, 81))
        y = int(rng.integers(0, H - h))
        x = int(rng.integers(0, W - w))
        img[y:y + h, x:x + w] = roof
        truth[y:y + h, x:x + w] = True
        roof_boxes.append((y, x, y + h, x + w))
    if noise > 0:
        nrng = np.random.default_rng(seed + 1)
        for y0 in range(0, H, 1024):
            y1 = min(y0 + 1024, H)
            img[y0:y1] += nrng.standard_normal((y1 - y0, W), np.float32) * np.float32(noise)
    return {"image": img[None], "truth": truth, "roof_boxes": roof_boxes}


def tile_scene(side_h: int, side_w: int, bands: int, seed: int,
               noise: float = 0.05):
    """One tile of the rectangle generator, for batched and served work.

    A bright rectangle whose sides are 20-60 % of the tile on a flat
    background; multi-band tiles repeat it with per-band levels drawn from
    U(0.15, 0.85).  Returns (image[bands, H, W] float32, box).
    """
    rng = np.random.default_rng(seed)
    rh = max(int(side_h * rng.uniform(0.2, 0.6)), 1)
    rw = max(int(side_w * rng.uniform(0.2, 0.6)), 1)
    y0 = int(rng.integers(0, side_h - rh + 1))
    x0 = int(rng.integers(0, side_w - rw + 1))
    truth = np.zeros((side_h, side_w), bool)
    truth[y0:y0 + rh, x0:x0 + rw] = True
    if bands == 1:
        levels = np.array([[0.3], [0.7]])
    else:
        levels = rng.uniform(0.15, 0.85, size=(2, bands))
    img = levels[truth.astype(np.int64)].transpose(2, 0, 1)
    img = img + rng.normal(0.0, noise, size=img.shape)
    return img.astype(np.float32), (y0, x0, y0 + rh, x0 + rw)


def batch_problems(n: int, seed: int, min_side: int = 128, max_side: int = 1024,
                   cap_range=(100, 600), early_stop_frac: float = 1e-4):
    """A work list of n independent images of uneven size (tile_scene).

    Sides are log-uniform in [min_side, max_side] (height and width drawn
    separately); half the images have one band and half four; half use the
    region term and half the edge term; each has an iteration cap drawn
    uniformly from cap_range (inclusive) and an early stop when fewer than
    early_stop_frac * H * W pixels change sign.  phi0 is +1 inside a centred
    circle of radius min(H, W) / 3 (region) or -1 inside a box 10 % of the
    tile outside the object (edge).  Returns a list of dicts with the keys
    image, phi0, term, iterations, early_stop_frac.
    """
    rng = np.random.default_rng(seed)
    lo, hi = np.log(min_side), np.log(max_side)
    out = []
    for i in range(n):
        H = int(round(np.exp(rng.uniform(lo, hi))))
        W = int(round(np.exp(rng.uniform(lo, hi))))
        bands = 1 if rng.random() < 0.5 else 4
        term = "region" if rng.random() < 0.5 else "edge"
        cap = int(rng.integers(cap_range[0], cap_range[1] + 1))
        img, (y0, x0, y1, x1) = tile_scene(H, W, bands, seed=int(rng.integers(1 << 31)))
        if term == "region":
            phi0 = circle_phi(H, W, radius=min(H, W) / 3.0)
        else:
            my, mx = max(int(0.1 * H), 2), max(int(0.1 * W), 2)
            phi0 = box_phi(H, W, [(max(y0 - my, 0), max(x0 - mx, 0),
                                   min(y1 + my, H), min(x1 + mx, W))])
        out.append({"image": img, "phi0": phi0, "term": term, "iterations": cap,
                    "early_stop_frac": early_stop_frac})
    return out
