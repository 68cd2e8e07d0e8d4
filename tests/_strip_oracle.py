"""A strip's arithmetic done by the FP64 oracle: the checker's stand-in for
the library's LibraryCompute in the row-strip driver's tests.

Each method restates, for the owned rows of one strip, what the oracle's
whole-image step takes from the whole image: the region statistics of
Eq. 15 as plain sums (FP64), the normaliser of Eq. 17 as a maximum over the
owned pixels (one band: its closed form at the image's extremes, which is
where the oracle's maximum over pixels lies, D being affine in I), and the
step itself through ``oracle.step_given``.
"""
import numpy as np

import oracle
from paper_1409_7474_gb300 import strips

CONTRAST_TOL = 1e-6       # the oracle's degenerate-contrast rule


class OracleCompute:
    def __init__(self, part, image, g=None, term="region", dt=15.0, sigma=1.0, ts=9):
        self.part = part
        self.image = None if image is None else np.asarray(image, np.float64).reshape(
            (-1, part.rows, part.W))
        self.g = None if g is None else np.asarray(g, np.float64)
        self.term = term
        self.dt, self.sigma, self.ts = dt, sigma, ts
        self.calls = {"partials": 0, "dmax": 0, "step": 0}

    def _own(self, a):
        lo, hi = self.part.own
        return a[..., lo:hi, :]

    def range(self):
        I = self._own(self.image)
        return float(I[0].min()), float(I[0].max()), float(np.abs(I).max())

    def scale(self, amax, npix):
        return 0

    def partials(self, phi, phi_prev, fix_k):
        self.calls["partials"] += 1
        p = self._own(np.asarray(phi))
        plus = p >= 0.0
        flips = 0 if phi_prev is None else int(np.count_nonzero(
            plus != (self._own(np.asarray(phi_prev)) >= 0.0)))
        if self.term == "region":
            I = self._own(self.image)
            s = np.where(plus, 1.0, -1.0)
            sw = np.array([np.sum(s * I[b]) for b in range(I.shape[0])])
            sa = np.array([np.sum(I[b]) for b in range(I.shape[0])])
        else:
            sw = sa = np.zeros(1)
        return strips.Partials(int(np.count_nonzero(plus)), flips, sw, sa)

    def _coeffs(self, tot):
        cp, cm = strips.means(tot)
        zero = tot.n_plus == 0 or tot.n_plus == tot.npix
        contrast = np.max(np.abs(cp - cm))
        scale = np.max(np.abs(cp) + np.abs(cm))
        zero = zero or contrast <= CONTRAST_TOL * scale
        return cp, cm, bool(zero)

    def dmax(self, tot):
        self.calls["dmax"] += 1
        cp, cm, zero = self._coeffs(tot)
        if zero:
            return 0.0
        I = self._own(self.image)
        D = np.zeros(I.shape[1:])
        for b in range(I.shape[0]):
            D = D + (cp[b] - cm[b]) * (2.0 * I[b] - cp[b] - cm[b])
        return float(np.max(np.abs(D))) if D.size else 0.0

    def step(self, phi, binarise_in, tot, norm):
        self.calls["step"] += 1
        phi = np.asarray(phi, np.float64)
        if binarise_in:
            phi = np.where(phi >= 0.0, 1.0, -1.0)
        if self.term == "edge":
            zeros = np.zeros((1, self.part.rows, self.part.W))
            return oracle.step_given(zeros, phi, [0.0], [0.0], 0.0, False, term="edge",
                                     g=self.g, dt=self.dt, sigma=self.sigma, ts=self.ts)
        cp, cm, zero = self._coeffs(tot)
        B = self.image.shape[0]
        if not zero and B == 1:
            d = cp[0] - cm[0]
            norm = max(abs(d * (2.0 * tot.imax - cp[0] - cm[0])),
                       abs(d * (2.0 * tot.imin - cp[0] - cm[0])))
        if not norm > 0.0:
            zero = True
        return oracle.step_given(self.image, phi, cp, cm, norm, zero, term="region",
                                 dt=self.dt, sigma=self.sigma, ts=self.ts)
