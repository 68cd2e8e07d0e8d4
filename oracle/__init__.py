"""FP64 CPU oracle for the fast level set evolutions (arXiv 1409.7474).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never calls it and shares no code with it.

The arithmetic lives in ``lse_oracle.c`` (plain C, double precision); this
module only builds it with gcc and marshals numpy arrays.  The build enables
OpenMP when gcc has it: the per-pixel maps then run their rows on several
threads (``OMP_NUM_THREADS`` caps them), with results independent of the
thread count.
Each wrapper names the part of the paper it follows; the C file's header has
the full list and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lse_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_lse_oracle.so")
# A test may point the wrapper at another build of the same source (the
# mutation test compiles deliberately broken copies to show the pins fail).
_LIB_OVERRIDE = os.environ.get("LSE_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

TERM_REGION = 0
TERM_EDGE = 1
MAX_BANDS = 8


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("iterations_run", ctypes.c_int),
        ("last_flips", ctypes.c_longlong),
        ("area_plus", ctypes.c_longlong),
        ("c_plus", ctypes.c_double * MAX_BANDS),
        ("c_minus", ctypes.c_double * MAX_BANDS),
        ("norm", ctypes.c_double),
        ("degenerate", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile lse_oracle.c into a shared library next to it.

    ``-ffp-contract=off`` keeps gcc from fusing multiply-adds, so the x86 and
    Arm builds round identically.  ``-fopenmp`` is dropped when gcc cannot
    build with it.
    """
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                "-fPIC", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base + ["-fopenmp"], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if _LIB_OVERRIDE:
                lib = ctypes.CDLL(_LIB_OVERRIDE)
            else:
                build()
                lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i = ctypes.c_int
            d = ctypes.c_double
            lib.oracle_set_threads.argtypes = [i]
            lib.oracle_set_threads.restype = None
            lib.oracle_gaussian_taps.argtypes = [d, i, dp]
            lib.oracle_gaussian_taps.restype = None
            lib.oracle_gradient.argtypes = [dp, i, i, dp, dp]
            lib.oracle_gradient.restype = None
            lib.oracle_conv_same.argtypes = [dp, i, i, dp, i, dp]
            lib.oracle_conv_same.restype = None
            lib.oracle_conv_same_padded.argtypes = [dp, i, i, dp, i, i, dp]
            lib.oracle_conv_same_padded.restype = None
            lib.oracle_step_variant.argtypes = [dp, i, i, i, i, dp, dp, d, d, i, i, i, i,
                                                dp, dp, dp, dp]
            lib.oracle_step_variant.restype = i
            lib.oracle_evolve_variant.argtypes = [dp, i, i, i, i, dp, dp, d, d, i, i, i, d,
                                                  i, i, dp, ctypes.POINTER(ctypes.c_ubyte),
                                                  ctypes.POINTER(OracleStats)]
            lib.oracle_evolve_variant.restype = i
            lib.oracle_edge_indicator.argtypes = [dp, i, i, i, d, i, d, dp]
            lib.oracle_edge_indicator.restype = None
            lib.oracle_region_stats.argtypes = [dp, i, i, i, dp, dp, dp]
            lib.oracle_region_stats.restype = ctypes.c_longlong
            lib.oracle_update.argtypes = [dp, i, i, i, i, dp, dp, d, dp]
            lib.oracle_update.restype = i
            lib.oracle_region_force.argtypes = [dp, i, i, i, dp, dp, dp, dp, dp]
            lib.oracle_region_force.restype = i
            lib.oracle_step.argtypes = [dp, i, i, i, i, dp, dp, d, d, i, dp,
                                        dp, dp, dp]
            lib.oracle_step.restype = i
            lib.oracle_step_sampled.argtypes = [dp, i, i, i, i, dp, dp, d, d,
                                                i, i, ip, ip, dp, dp, dp, dp]
            lib.oracle_step_sampled.restype = i
            lib.oracle_step_given.argtypes = [dp, i, i, i, i, dp, dp, d, d, i, dp, dp, d, i,
                                              dp]
            lib.oracle_step_given.restype = None
            lib.oracle_evolve.argtypes = [dp, i, i, i, i, dp, dp, d, d, i, i,
                                          i, d, dp,
                                          ctypes.POINTER(ctypes.c_ubyte),
                                          ctypes.POINTER(OracleStats)]
            lib.oracle_evolve.restype = i
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))



def set_threads(n: int) -> None:
    """Threads the per-pixel maps may use (0: the OpenMP default).  Results do
    not depend on it; a caller that runs several oracle calls side by side
    sets 1."""
    _load().oracle_set_threads(int(n))

def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _image3(image) -> np.ndarray:
    img = _f64(image)
    if img.ndim == 2:
        img = img[None]
    if img.ndim != 3:
        raise ValueError("image must be H x W or B x H x W")
    return img


def gaussian_taps(sigma: float, ts: int) -> np.ndarray:
    """TS x TS normalised Gaussian G_sigma (Table I step 4)."""
    G = np.empty((ts, ts), np.float64)
    _load().oracle_gaussian_taps(float(sigma), int(ts), _ptr(G))
    return G


def gradient(f):
    """(f_x, f_y) with the listing's central / one-sided differences."""
    f = _f64(f)
    H, W = f.shape
    fx = np.empty_like(f)
    fy = np.empty_like(f)
    _load().oracle_gradient(_ptr(f), H, W, _ptr(fx), _ptr(fy))
    return fx, fy


ORDERS = {"listing": 0, "table1": 1}
PADDINGS = {"zero": 0, "replicate": 1}


def conv_same(f, G, padding: str = "zero"):
    """'same'-size 2-D convolution (Table I step 4), zero padding (the
    listing's) or replicate padding (the nearest image value)."""
    f = _f64(f)
    G = _f64(G)
    H, W = f.shape
    out = np.empty_like(f)
    if padding == "zero":
        _load().oracle_conv_same(_ptr(f), H, W, _ptr(G), G.shape[0], _ptr(out))
    else:
        _load().oracle_conv_same_padded(_ptr(f), H, W, _ptr(G), G.shape[0],
                                        PADDINGS[padding], _ptr(out))
    return out


def edge_indicator(image, sigma1: float = 1.0, ts1: int = 9,
                   edge_scale: float = 255.0) -> np.ndarray:
    """g(I) of Eq. 14 on the band mean scaled by edge_scale."""
    img = _image3(image)
    B, H, W = img.shape
    g = np.empty((H, W), np.float64)
    _load().oracle_edge_indicator(_ptr(img), H, W, B, float(sigma1), int(ts1),
                                  float(edge_scale), _ptr(g))
    return g


def region_stats(image, phi):
    """(c_plus[B], c_minus[B], |{phi >= 0}|) of Eq. 15."""
    img = _image3(image)
    B, H, W = img.shape
    phi = _f64(phi)
    cp = np.zeros(B)
    cm = np.zeros(B)
    n = _load().oracle_region_stats(_ptr(img), H, W, B, _ptr(phi), _ptr(cp),
                                    _ptr(cm))
    return cp, cm, int(n)


def region_force(image, phi):
    """(R, max|D|, c_plus, c_minus, zero_force) of Eq. 17."""
    img = _image3(image)
    B, H, W = img.shape
    phi = _f64(phi)
    R = np.empty((H, W))
    norm = np.zeros(1)
    cp = np.zeros(B)
    cm = np.zeros(B)
    z = _load().oracle_region_force(_ptr(img), H, W, B, _ptr(phi), _ptr(R),
                                    _ptr(norm), _ptr(cp), _ptr(cm))
    return R, float(norm[0]), cp, cm, bool(z)


def _term(term) -> int:
    if term in (TERM_REGION, "region"):
        return TERM_REGION
    if term in (TERM_EDGE, "edge"):
        return TERM_EDGE
    raise ValueError(f"unknown term {term!r}")


def update(image, phi, term="region", g=None, dt: float = 15.0):
    """u = phi + dt R |grad phi| (Eq. 18), before smoothing."""
    img = _image3(image)
    B, H, W = img.shape
    phi = _f64(phi)
    gg = _f64(g) if g is not None else None
    u = np.empty((H, W))
    z = _load().oracle_update(_ptr(img), H, W, B, _term(term), _ptr(gg),
                              _ptr(phi), float(dt), _ptr(u))
    return u, bool(z)


def step(image, phi, term="region", g=None, dt: float = 15.0,
         sigma: float = 1.0, ts: int = 9, order: str = "listing",
         reinit: bool = True, padding: str = "zero"):
    """One iteration v = G_sigma * (phi + dt R |grad phi|), not binarised.
    In the Table I order with ``reinit`` the update is binarised before the
    smoothing.  Returns (v, norm, c_plus, c_minus, zero_force).
    """
    img = _image3(image)
    B, H, W = img.shape
    phi = _f64(phi)
    gg = _f64(g) if g is not None else None
    v = np.empty((H, W))
    norm = np.zeros(1)
    cp = np.zeros(B)
    cm = np.zeros(B)
    if order == "listing" and padding == "zero":
        z = _load().oracle_step(_ptr(img), H, W, B, _term(term), _ptr(gg),
                                _ptr(phi), float(dt), float(sigma), int(ts),
                                _ptr(v), _ptr(norm), _ptr(cp), _ptr(cm))
    else:
        z = _load().oracle_step_variant(_ptr(img), H, W, B, _term(term), _ptr(gg),
                                        _ptr(phi), float(dt), float(sigma), int(ts),
                                        ORDERS[order], int(bool(reinit)), PADDINGS[padding],
                                        _ptr(v), _ptr(norm), _ptr(cp), _ptr(cm))
    return v, float(norm[0]), cp, cm, bool(z)


def step_given(image, phi, c_plus, c_minus, norm, zero_force=False, term="region", g=None,
               dt: float = 15.0, sigma: float = 1.0, ts: int = 9):
    """One iteration (Eq. 18, Table I step 4) with the region statistics given
    (c+ / c- per band, the normaliser M of Eq. 17) instead of taken from phi:
    a row strip of a larger image stepping with the whole image's
    statistics.  Not re-initialised."""
    img = _image3(image)
    B, H, W = img.shape
    phi = _f64(phi)
    gg = _f64(g) if g is not None else None
    cp = _f64(np.resize(np.asarray(c_plus, np.float64), B))
    cm = _f64(np.resize(np.asarray(c_minus, np.float64), B))
    v = np.empty((H, W))
    _load().oracle_step_given(_ptr(img), H, W, B, _term(term), _ptr(gg), _ptr(phi), float(dt),
                              float(sigma), int(ts), _ptr(cp), _ptr(cm), float(norm),
                              int(bool(zero_force)), _ptr(v))
    return v


def step_sampled(image, phi, ys, xs, term="region", g=None, dt: float = 15.0,
                 sigma: float = 1.0, ts: int = 9):
    """One iteration evaluated only at the pixels (ys[k], xs[k]).

    Returns (v_samples, norm, c_plus, c_minus, zero_force).
    """
    img = _image3(image)
    B, H, W = img.shape
    phi = _f64(phi)
    gg = _f64(g) if g is not None else None
    ys = np.ascontiguousarray(np.asarray(ys, dtype=np.int32))
    xs = np.ascontiguousarray(np.asarray(xs, dtype=np.int32))
    n = int(ys.size)
    v = np.empty(n)
    norm = np.zeros(1)
    cp = np.zeros(B)
    cm = np.zeros(B)
    ip = ctypes.POINTER(ctypes.c_int)
    z = _load().oracle_step_sampled(
        _ptr(img), H, W, B, _term(term), _ptr(gg), _ptr(phi), float(dt),
        float(sigma), int(ts), n, ys.ctypes.data_as(ip), xs.ctypes.data_as(ip),
        _ptr(v), _ptr(norm), _ptr(cp), _ptr(cm))
    return v, float(norm[0]), cp, cm, bool(z)


def evolve(image, phi0, term="region", g=None, dt: float = 15.0,
           sigma: float = 1.0, ts: int = 9, iterations: int = 200,
           reinit_period: int = 1, early_stop_frac: float = 0.0,
           order: str = "listing", padding: str = "zero"):
    """The whole evolution of Table I (in the listing's step order unless
    ``order`` = "table1").  Returns (v, mask, stats_dict)."""
    img = _image3(image)
    B, H, W = img.shape
    phi0 = _f64(phi0)
    gg = _f64(g) if g is not None else None
    v = np.empty((H, W))
    mask = np.empty((H, W), np.uint8)
    st = OracleStats()
    if order == "listing" and padding == "zero":
        rc = _load().oracle_evolve(
            _ptr(img), H, W, B, _term(term), _ptr(gg), _ptr(phi0), float(dt),
            float(sigma), int(ts), int(iterations), int(reinit_period),
            float(early_stop_frac), _ptr(v),
            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), ctypes.byref(st))
    else:
        rc = _load().oracle_evolve_variant(
            _ptr(img), H, W, B, _term(term), _ptr(gg), _ptr(phi0), float(dt),
            float(sigma), int(ts), int(iterations), int(reinit_period),
            float(early_stop_frac), ORDERS[order], PADDINGS[padding], _ptr(v),
            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle_evolve rejected its arguments")
    stats = {
        "iterations_run": st.iterations_run,
        "last_flips": st.last_flips,
        "area_plus": st.area_plus,
        "c_plus": np.array(st.c_plus[:B]),
        "c_minus": np.array(st.c_minus[:B]),
        "norm": st.norm,
        "degenerate": bool(st.degenerate),
    }
    return v, mask, stats
