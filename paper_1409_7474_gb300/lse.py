"""Thin ctypes binding of the C ABI in ``include/lse.h``.

Argument marshalling only: every step of the evolution runs in the CUDA
library ``liblse.so`` built in-tree by ``paper_1409_7474_gb300._build``.  The
binding accepts torch tensors (CUDA or CPU) and numpy arrays; CPU buffers are
passed to the library as host pointers and staged by it.  There is no CPU
fallback: if the library is missing this module raises on import.

Names follow the C ABI: ``create``/``Context``, ``precompute_edge``,
``evolve``, ``destroy``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

try:
    import torch
except ImportError:  # the binding itself only needs ctypes and numpy
    torch = None

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblse.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'` "
        "(the library has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

# ------------------------------------------------------------------ C types
LSE_OK = 0
LSE_ERR_INVALID_ARG = 1
LSE_ERR_OOM = 2
LSE_ERR_CUDA = 3
LSE_ERR_NONFINITE = 4
LSE_ERR_TIMEOUT = 5
LSE_WARN_DEGENERATE = 6
STATUS_NAMES = {0: "LSE_OK", 1: "LSE_ERR_INVALID_ARG", 2: "LSE_ERR_OOM",
                3: "LSE_ERR_CUDA", 4: "LSE_ERR_NONFINITE", 5: "LSE_ERR_TIMEOUT",
                6: "LSE_WARN_DEGENERATE"}

TERM_REGION = 0
TERM_EDGE = 1
F32, F16, BF16, U16 = 0, 1, 2, 3
STORAGE = {"f32": F32, "f16": F16, "bf16": BF16}
ORDERS = {"listing": 0, "table1": 1}        # lse_order
PADDINGS = {"zero": 0, "replicate": 1}      # lse_padding


class Params(ctypes.Structure):
    _fields_ = [("term", ctypes.c_int), ("dt", ctypes.c_float),
                ("sigma", ctypes.c_float), ("ts", ctypes.c_int),
                ("iterations", ctypes.c_int), ("reinit_period", ctypes.c_int),
                ("early_stop_frac", ctypes.c_float), ("storage", ctypes.c_int),
                ("order", ctypes.c_int), ("padding", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations_run", ctypes.c_int), ("last_flips", ctypes.c_longlong),
                ("area_plus", ctypes.c_longlong), ("c_plus", ctypes.c_double * 8),
                ("c_minus", ctypes.c_double * 8), ("norm", ctypes.c_double),
                ("elapsed_ms", ctypes.c_float), ("status", ctypes.c_int)]

    def to_dict(self, bands: int = 8) -> dict:
        return {"iterations_run": self.iterations_run,
                "last_flips": self.last_flips, "area_plus": self.area_plus,
                "c_plus": list(self.c_plus[:bands]),
                "c_minus": list(self.c_minus[:bands]), "norm": self.norm,
                "elapsed_ms": self.elapsed_ms,
                "status": STATUS_NAMES.get(self.status, str(self.status))}


class Problem(ctypes.Structure):
    """lse_problem: one image of lse_evolve_batch (device pointers)."""
    _fields_ = [("image", ctypes.c_void_p), ("dtype", ctypes.c_int),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("B", ctypes.c_int),
                ("g", ctypes.c_void_p), ("phi0", ctypes.c_void_p), ("params", Params),
                ("phi_out", ctypes.c_void_p), ("mask_out", ctypes.c_void_p)]


STRIP_SUMS_WORDS = 23                # an lse_strip_sums record in 64-bit words
STRIP_SUM_INT_WORDS = 19             # npix .. sum_a: integers the ranks add


class StripSums(ctypes.Structure):
    """lse_strip_sums: partial statistics of a strip's owned rows, or their
    totals over the ranks."""
    _fields_ = [("npix", ctypes.c_longlong), ("n_plus", ctypes.c_longlong),
                ("flips", ctypes.c_longlong), ("sum_w", ctypes.c_longlong * 8),
                ("sum_a", ctypes.c_longlong * 8), ("imin", ctypes.c_double),
                ("imax", ctypes.c_double), ("amax", ctypes.c_double),
                ("fix_k", ctypes.c_int), ("bands", ctypes.c_int)]


_vp = ctypes.c_void_p
_lib.lse_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t, ctypes.c_int]
_lib.lse_create.restype = ctypes.c_int
_lib.lse_destroy.argtypes = [_vp]
_lib.lse_destroy.restype = None
_lib.lse_last_error.argtypes = [_vp]
_lib.lse_last_error.restype = ctypes.c_char_p
_lib.lse_precompute_edge.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                     ctypes.c_float, _vp, _vp]
_lib.lse_precompute_edge.restype = ctypes.c_int
_lib.lse_evolve.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int, _vp, _vp, ctypes.POINTER(Params), _vp, _vp,
                            ctypes.POINTER(Stats), _vp]
_lib.lse_evolve.restype = ctypes.c_int
_lib.lse_get_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
_lib.lse_get_stats.restype = ctypes.c_int
_lib.lse_version.argtypes = []
_lib.lse_version.restype = ctypes.c_char_p
_lib.lse_kernel_launches.argtypes = [_vp]
_lib.lse_kernel_launches.restype = ctypes.c_ulonglong
_lib.lse_evolve_static.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                   ctypes.POINTER(Params), _vp, _vp, ctypes.POINTER(Stats),
                                   _vp]
_lib.lse_evolve_static.restype = ctypes.c_int
_lib.lse_evolve_batch.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                                  ctypes.POINTER(Stats), _vp]
_lib.lse_evolve_batch.restype = ctypes.c_int
_lib.lse_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                              ctypes.POINTER(ctypes.c_int), _vp]
_lib.lse_autotune.restype = ctypes.c_int
_lib.lse_server_create.argtypes = [_vp, ctypes.c_size_t, ctypes.POINTER(_vp)]
_lib.lse_server_create.restype = ctypes.c_int
_lib.lse_server_destroy.argtypes = [_vp]
_lib.lse_server_destroy.restype = None
_lib.lse_server_submit.argtypes = [_vp, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_longlong)]
_lib.lse_server_submit.restype = ctypes.c_int
_lib.lse_server_advance.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp]
_lib.lse_server_advance.restype = ctypes.c_int
_lib.lse_server_poll.argtypes = [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(Stats)]
_lib.lse_server_poll.restype = ctypes.c_int
_lib.lse_strip_scale.argtypes = [ctypes.c_double, ctypes.c_longlong]
_lib.lse_strip_scale.restype = ctypes.c_int
_lib.lse_strip_partials.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                    ctypes.c_int, _vp, _vp]
_lib.lse_strip_partials.restype = ctypes.c_int
_lib.lse_strip_dmax.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(StripSums), ctypes.c_float,
                                ctypes.POINTER(ctypes.c_double), _vp]
_lib.lse_strip_dmax.restype = ctypes.c_int
_lib.lse_strip_step.argtypes = [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(Params),
                                _vp, ctypes.c_double, _vp, _vp]
_lib.lse_strip_step.restype = ctypes.c_int
_lib.lse_strip_status.argtypes = [_vp, _vp]
_lib.lse_strip_status.restype = ctypes.c_int

SYMBOLS = ("lse_create", "lse_destroy", "lse_last_error", "lse_precompute_edge",
           "lse_evolve", "lse_get_stats", "lse_version", "lse_kernel_launches",
           "lse_evolve_static",
           "lse_evolve_batch", "lse_autotune", "lse_server_create", "lse_server_destroy",
           "lse_server_submit", "lse_server_advance", "lse_server_poll",
           "lse_strip_scale", "lse_strip_partials", "lse_strip_dmax", "lse_strip_step",
           "lse_strip_status")
STATIC_MAX_PIXELS = 262144


class LseError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def version() -> str:
    return _lib.lse_version().decode()


# ------------------------------------------------------------------ marshalling
def _is_torch(x) -> bool:
    return torch is not None and isinstance(x, torch.Tensor)


def _dtype_code(x) -> int:
    if _is_torch(x):
        m = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}
        if hasattr(torch, "uint16"):
            m[torch.uint16] = U16
        if x.dtype not in m:
            raise TypeError(f"unsupported image dtype {x.dtype}")
        return m[x.dtype]
    m = {np.dtype(np.float32): F32, np.dtype(np.float16): F16, np.dtype(np.uint16): U16}
    if x.dtype not in m:
        raise TypeError(f"unsupported image dtype {x.dtype}")
    return m[x.dtype]


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("arrays must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def _shape3(image):
    shp = tuple(image.shape)
    if len(shp) == 2:
        return 1, shp[0], shp[1]
    if len(shp) == 3:
        return shp
    raise ValueError("image must be H x W or B x H x W")


def _stream_ptr(stream, device: int):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    if torch is not None and torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    return ctypes.c_void_p(0)


def _empty_like_place(ref, shape, np_dtype, torch_dtype):
    if _is_torch(ref):
        return torch.empty(shape, dtype=torch_dtype, device=ref.device,
                           pin_memory=False)
    return np.empty(shape, dtype=np_dtype)


class Context:
    """An ``lse_ctx``: device scratch for images up to ``max_pixels`` pixels
    and ``max_bands`` bands on CUDA device ``device``."""

    def __init__(self, device: int = 0, max_pixels: int = 1 << 20,
                 max_bands: int = 4):
        h = ctypes.c_void_p()
        rc = _lib.lse_create(ctypes.byref(h), int(device), int(max_pixels), int(max_bands))
        if rc != LSE_OK:
            raise LseError(rc, _lib.lse_last_error(None).decode())
        self._h = h
        self.device = int(device)
        self.max_pixels = int(max_pixels)
        self.max_bands = int(max_bands)

    # -- lifetime
    def destroy(self):
        if getattr(self, "_h", None):
            _lib.lse_destroy(self._h)
            self._h = None

    close = destroy

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def _check(self, rc: int):
        if rc != LSE_OK:
            raise LseError(rc, _lib.lse_last_error(self._h).decode())

    # -- calls
    def precompute_edge(self, image, sigma1: float = 1.0, ts1: int = 9,
                        edge_scale: float = 255.0, out=None, stream=None):
        """g(I) of Eq. 14 (H x W float32), on the image's device or host."""
        B, H, W = _shape3(image)
        if out is None:
            out = _empty_like_place(image, (H, W), np.float32,
                                    torch.float32 if torch is not None else None)
        self._check(_lib.lse_precompute_edge(
            self._h, _ptr(image), _dtype_code(image), H, W, B, float(sigma1),
            int(ts1), float(edge_scale), _ptr(out), _stream_ptr(stream, self.device)))
        return out

    def evolve(self, image, phi0, term: str = "region", g=None, dt: float = 15.0,
               sigma: float = 1.0, ts: int = 9, iterations: int = 200,
               reinit_period: int = 1, early_stop_frac: float = 0.0,
               phi_out=None, mask_out=None, stream=None, sync: bool = True,
               storage: str = "f32", order: str = "listing", padding: str = "zero"):
        """Runs the evolution.  Returns (phi_out, mask_out, stats or None).

        With ``sync`` the call waits for the stream and returns the statistics
        dict; otherwise it returns at once and ``stats()`` reads them after the
        caller synchronises.  ``storage`` ("f32", "f16" or "bf16") is the type
        of the work planes in HBM (``lse_params.storage``); ``order``
        ("listing" or "table1") and ``padding`` ("zero" or "replicate") are
        ``lse_params.order`` and ``lse_params.padding``."""
        term_code = TERM_REGION if term in ("region", TERM_REGION) else TERM_EDGE
        ref = image if image is not None else phi0
        if image is not None:
            B, H, W = _shape3(image)
            dcode = _dtype_code(image)
        else:
            B, (H, W), dcode = 1, tuple(phi0.shape), F32
        if phi_out is None:
            phi_out = _empty_like_place(ref, (H, W), np.float32,
                                        torch.float32 if torch is not None else None)
        if mask_out is None:
            mask_out = _empty_like_place(ref, (H, W), np.uint8,
                                         torch.uint8 if torch is not None else None)
        p = Params(term_code, float(dt), float(sigma), int(ts), int(iterations),
                   int(reinit_period), float(early_stop_frac), STORAGE[storage],
                   ORDERS[order], PADDINGS[padding])
        st = Stats()
        rc = _lib.lse_evolve(self._h, _ptr(image) if term_code == TERM_REGION else None,
                             dcode, H, W, B,
                             _ptr(g) if term_code == TERM_EDGE else None, _ptr(phi0),
                             ctypes.byref(p), _ptr(phi_out), _ptr(mask_out),
                             ctypes.byref(st) if sync else None,
                             _stream_ptr(stream, self.device))
        self._check(rc)
        return phi_out, mask_out, (st.to_dict(B) if sync else None)

    def evolve_batch(self, items, use_graph: bool = True, stream=None):
        """lse_evolve_batch over `items`, a list of dicts with the keys of
        ``evolve`` (image or g, phi0, term, dt, sigma, ts, iterations,
        reinit_period, early_stop_frac, storage, and optionally phi_out /
        mask_out), all CUDA tensors.  Returns a list of (phi_out, mask_out,
        stats)."""
        n = len(items)
        probs = (Problem * n)()
        outs = []
        for i, it in enumerate(items):
            probs[i], phi_out, mask_out, B = _problem(it)
            outs.append((phi_out, mask_out, B))
        st = (Stats * n)()
        self._check(_lib.lse_evolve_batch(self._h, n, probs, 1 if use_graph else 0, st,
                                          _stream_ptr(stream, self.device)))
        return [(o[0], o[1], st[i].to_dict(o[2])) for i, o in enumerate(outs)]

    def autotune(self, items, iterations: int = 12, stream=None):
        """lse_autotune over `items` (dicts as in ``evolve_batch``): times both
        tile heights on them and keeps the faster per shape class in this
        context.  Returns each item's chosen tile height in rows (0 where the
        tile form does not apply)."""
        n = len(items)
        probs = (Problem * n)()
        for i, it in enumerate(items):
            probs[i] = _problem(it)[0]
        rows = (ctypes.c_int * n)()
        self._check(_lib.lse_autotune(self._h, n, probs, int(iterations), rows,
                                      _stream_ptr(stream, self.device)))
        return list(rows)

    # -- row strips (lse_strip_*)
    def strip_partials(self, image, phi, row0: int, row1: int, fix_k: int = 0,
                       phi_prev=None, bands: int = None, out=None, stream=None):
        """lse_strip_partials over rows [row0, row1) of a strip: image
        (B x Hs x W, or None for the edge term), phi / phi_prev (Hs x W
        float32, or None).  Returns a StripSums (synchronous), or, with
        ``out`` a CUDA int64 tensor of STRIP_SUMS_WORDS words, writes the
        record there without waiting and returns ``out``."""
        if image is not None:
            B, Hs, W = _shape3(image)
            dcode = _dtype_code(image)
        else:
            B = bands or 1
            Hs, W = tuple(phi.shape)
            dcode = F32
        dev_out = out is not None
        if dev_out:
            if out.numel() * out.element_size() < ctypes.sizeof(StripSums):
                raise ValueError("out is smaller than an lse_strip_sums record")
            ptr = _ptr(out)
        else:
            out = StripSums()
            ptr = ctypes.byref(out)
        self._check(_lib.lse_strip_partials(
            self._h, _ptr(image), dcode, Hs, W, B, int(row0), int(row1), _ptr(phi),
            _ptr(phi_prev), int(fix_k), ptr, _stream_ptr(stream, self.device)))
        return out

    def strip_status(self, stream=None) -> None:
        """lse_strip_status: raises LseError for a device-side condition that
        strip calls found since the last report."""
        self._check(_lib.lse_strip_status(self._h, _stream_ptr(stream, self.device)))

    def strip_dmax(self, image, row0: int, row1: int, totals: StripSums, dt: float = 15.0,
                   stream=None) -> float:
        """lse_strip_dmax: max |D| over rows [row0, row1) of the strip for the
        totals' statistics (vector images)."""
        B, Hs, W = _shape3(image)
        out = ctypes.c_double()
        self._check(_lib.lse_strip_dmax(
            self._h, _ptr(image), _dtype_code(image), Hs, W, B, int(row0), int(row1),
            ctypes.byref(totals), float(dt), ctypes.byref(out),
            _stream_ptr(stream, self.device)))
        return out.value

    def strip_step(self, image, phi, totals: StripSums = None, norm: float = 0.0,
                   term: str = "region", g=None, binarise_in: bool = False,
                   dt: float = 15.0, sigma: float = 1.0, ts: int = 9, v_out=None,
                   stream=None):
        """lse_strip_step: one iteration on a strip with the whole image's
        statistics.  Returns v_out (Hs x W float32, on phi's device)."""
        term_code = TERM_REGION if term in ("region", TERM_REGION) else TERM_EDGE
        Hs, W = tuple(phi.shape)
        if term_code == TERM_REGION:
            B, _, _ = _shape3(image)
            dcode = _dtype_code(image)
        else:
            B, dcode = 1, F32
        if v_out is None:
            v_out = _empty_like_place(phi, (Hs, W), np.float32,
                                      torch.float32 if torch is not None else None)
        p = Params(term_code, float(dt), float(sigma), int(ts), 1, 0, 0.0, F32, 0, 0)
        if totals is None:
            tptr = None
        elif isinstance(totals, StripSums):
            tptr = ctypes.byref(totals)
        else:
            tptr = _ptr(totals)            # a device record (CUDA tensor)
        self._check(_lib.lse_strip_step(
            self._h, _ptr(image) if term_code == TERM_REGION else None, dcode,
            _ptr(g) if term_code == TERM_EDGE else None, Hs, W, B, _ptr(phi),
            int(bool(binarise_in)), ctypes.byref(p), tptr, float(norm), _ptr(v_out),
            _stream_ptr(stream, self.device)))
        return v_out

    def kernel_launches(self) -> int:
        """lse_kernel_launches: kernels this context's evolve and
        precompute_edge calls have enqueued."""
        return int(_lib.lse_kernel_launches(self._h))

    def stats(self, bands: int = 8) -> dict:
        st = Stats()
        self._check(_lib.lse_get_stats(self._h, ctypes.byref(st)))
        return st.to_dict(bands)


def _problem(it: dict):
    """An lse_problem from a dict of CUDA tensors (see Context.evolve_batch);
    returns (problem, phi_out, mask_out, bands)."""
    term = it.get("term", "region")
    term_code = TERM_REGION if term in ("region", TERM_REGION) else TERM_EDGE
    phi0 = it["phi0"]
    H, W = (int(d) for d in phi0.shape)
    image = it.get("image") if term_code == TERM_REGION else None
    if image is not None:
        B, _, _ = _shape3(image)
        dcode = _dtype_code(image)
    else:
        B, dcode = 1, F32
    phi_out = it.get("phi_out")
    if phi_out is None:
        phi_out = torch.empty((H, W), dtype=torch.float32, device=phi0.device)
    mask_out = it.get("mask_out")
    if mask_out is None:
        mask_out = torch.empty((H, W), dtype=torch.uint8, device=phi0.device)
    p = Params(term_code, float(it.get("dt", 15.0)), float(it.get("sigma", 1.0)),
               int(it.get("ts", 9)), int(it.get("iterations", 200)),
               int(it.get("reinit_period", 1)), float(it.get("early_stop_frac", 0.0)),
               STORAGE[it.get("storage", "f32")])
    prob = Problem(_ptr(image), dcode, H, W, B,
                   _ptr(it.get("g")) if term_code == TERM_EDGE else None,
                   _ptr(phi0), p, _ptr(phi_out), _ptr(mask_out))
    return prob, phi_out, mask_out, B


class Server:
    """An lse_server on a Context: continuous batching of requests within a
    device-memory budget (bytes)."""

    QUEUED, RUNNING, DONE = 0, 1, 2

    def __init__(self, ctx: Context, budget_bytes: int):
        h = ctypes.c_void_p()
        ctx._check(_lib.lse_server_create(ctx._h, int(budget_bytes), ctypes.byref(h)))
        self._h = h
        self.ctx = ctx
        self._keep = {}      # the tensors of each request until it is done

    def submit(self, item: dict) -> int:
        """Queues a request (a dict as in Context.evolve_batch); returns its id."""
        prob, phi_out, mask_out, B = _problem(item)
        rid = ctypes.c_longlong()
        self.ctx._check(_lib.lse_server_submit(self._h, ctypes.byref(prob), ctypes.byref(rid)))
        self._keep[rid.value] = (item, phi_out, mask_out, B)
        return rid.value

    def advance(self, ticks: int, stream=None) -> int:
        """Admits, runs `ticks` iterations of every running request, retires
        the finished ones; returns the number still running."""
        running = ctypes.c_int()
        self.ctx._check(_lib.lse_server_advance(self._h, int(ticks), ctypes.byref(running),
                                                _stream_ptr(stream, self.ctx.device)))
        return running.value

    def poll(self, rid: int):
        """None while queued or running; (phi_out, mask_out, stats) once done."""
        state = ctypes.c_int()
        st = Stats()
        self.ctx._check(_lib.lse_server_poll(self._h, int(rid), ctypes.byref(state),
                                             ctypes.byref(st)))
        if state.value != self.DONE:
            return None
        item, phi_out, mask_out, B = self._keep.pop(rid)
        return phi_out, mask_out, st.to_dict(B)

    def destroy(self):
        if getattr(self, "_h", None):
            _lib.lse_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def create(device: int = 0, max_pixels: int = 1 << 20, max_bands: int = 4) -> Context:
    return Context(device, max_pixels, max_bands)


def destroy(ctx: Context) -> None:
    ctx.destroy()


def strip_scale(amax: float, npix: int) -> int:
    """lse_strip_scale: the fixed-point exponent of the strips' sums."""
    return int(_lib.lse_strip_scale(float(amax), int(npix)))


def raw_library():
    """The loaded ctypes CDLL (for tests that call the C ABI directly)."""
    return _lib
