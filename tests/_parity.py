"""Helpers shared by the parity tests (no method arithmetic)."""
import numpy as np
from scipy import ndimage


def contour_ring(mask: np.ndarray) -> np.ndarray:
    """Pixels with a 4-neighbour of the other mask value."""
    m = mask.astype(bool)
    cross = ndimage.generate_binary_structure(2, 1)
    return (ndimage.binary_dilation(m, cross) & ~m) | (m & ~ndimage.binary_erosion(m, cross, border_value=1))


def mask_report(gpu_mask: np.ndarray, ref_mask: np.ndarray) -> dict:
    """Disagreement of two masks and how far it lies from the reference's
    contour (Chebyshev distance; 'far' counts pixels more than 1 px away)."""
    g = gpu_mask.astype(bool)
    r = ref_mask.astype(bool)
    bad = g != r
    near = ndimage.binary_dilation(contour_ring(r), np.ones((3, 3), bool))
    return {"disagree": int(bad.sum()), "frac": float(bad.mean()),
            "far": int((bad & ~near).sum())}


def assert_mask_parity(gpu_mask, ref_mask, max_frac=5e-4):
    rep = mask_report(gpu_mask, ref_mask)
    assert rep["frac"] <= max_frac and rep["far"] == 0, rep
    return rep


class step_launches:
    """Within the block lse_evolve launches one kernel per step (LSE_PERSIST=0,
    read at every call).  Batches and the server advance their images one
    step per launch; vector images there take the band passes, and this is
    how a single call reproduces that path to compare bit for bit."""

    def __init__(self, on=True):
        self.on = on

    def __enter__(self):
        import os
        self._old = os.environ.get("LSE_PERSIST")
        if self.on:
            os.environ["LSE_PERSIST"] = "0"
        return self

    def __exit__(self, *exc):
        import os
        if self._old is None:
            os.environ.pop("LSE_PERSIST", None)
        else:
            os.environ["LSE_PERSIST"] = self._old
        return False


def is_vector_region(it):
    img = it.get("image")
    return it.get("term", "region") == "region" and img is not None and img.shape[0] > 1
