"""FP64 periodic orthonormal Daubechies DWT and the wavelet Sobolev embedding
E_s / its adjoint E_s* (test infrastructure only).

Paper Sec. 4: the multiresolution basis {phi_lambda, psi_lambda} of Def. 4.1
(Eq. multid_wavelet), the diagonal level scaling of Prop. 4.2, the discrete
transform W of Sec. 4 (coefficient string [cA_m, cH_m, cV_m, cD_m, ..., cD_1])
and E_s* X = W^{-1}(D W X).

Readings taken here (the paper fixes no boundary mode and its level weights
disagree between the inline formula and the matrix D):
  * periodic boundary, orthonormal filters, so W^{-1} = W^T;
  * the level-i detail block (i = 1 finest, i = m coarsest) is scaled by
    2^{-s(m-i+o)} (o = level offset, default 0) in E_s* = S_s W and in
    E_s = W^T S_s, so E_s E_s* = W^T S_s^2 W carries 2^{-2s(m-i)} on level i
    as in the inline formula of Sec. 4; cA_m keeps weight 1.

One analysis level along an axis of length n (n even), filter length L:
    a_k = sum_j h_j x[(2k+j) mod n],   d_k = sum_j g_j x[(2k+j) mod n],
    g_j = (-1)^j h_{L-1-j},  k = 0 .. n/2-1.
2D: x (last array axis) first, then y.  Bands: H = (x low, y high),
V = (x high, y low), D = (x high, y high), stored in the paper's order
cH, cV, cD.  3D: seven bands in the binary order (z,y,x) = 001 .. 111, a 1
meaning high-pass on that axis.  Every band is stored row-major.
"""
from math import comb, sqrt

import numpy as np

FAMILIES = {1: "haar", 2: "db2", 4: "db4"}


def daubechies(nv: int) -> np.ndarray:
    """Orthonormal Daubechies low-pass filter with nv vanishing moments
    (2*nv taps, sum = sqrt(2)), extremal phase, built by spectral
    factorisation of |m0|^2 = cos^{2nv}(xi/2) P(sin^2(xi/2)) with
    P(y) = sum_{k<nv} C(nv-1+k, k) y^k (Daubechies' construction)."""
    if nv == 1:
        return np.array([1.0, 1.0]) / sqrt(2.0)
    p = np.array([comb(nv - 1 + k, k) for k in range(nv)], dtype=np.float64)  # ascending in y
    yroots = np.roots(p[::-1])
    zroots = []
    for yr in yroots:
        # y = (2 - z - 1/z)/4  <=>  z^2 - (2 - 4y) z + 1 = 0 ; keep the root outside the unit circle
        b = 2.0 - 4.0 * yr
        disc = np.sqrt(b * b - 4.0 + 0j)
        z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
        zroots.append(z1 if abs(z1) > 1.0 else z2)
    poly = np.array([1.0 + 0j])  # ascending coefficients in z
    for zr in zroots:
        poly = np.convolve(poly, np.array([-zr, 1.0]))
    for _ in range(nv):
        poly = np.convolve(poly, np.array([1.0, 1.0]))
    h = poly.real
    return h * (sqrt(2.0) / h.sum())


def highpass(h: np.ndarray) -> np.ndarray:
    L = len(h)
    return np.array([(-1) ** j * h[L - 1 - j] for j in range(L)])


def _analysis_axis(x, h, g, axis):
    n = x.shape[axis]
    k = np.arange(n // 2)
    a = 0.0
    d = 0.0
    for j in range(len(h)):
        xs = np.take(x, (2 * k + j) % n, axis=axis)
        a = a + h[j] * xs
        d = d + g[j] * xs
    return a, d


def _synthesis_axis(a, d, h, g, axis):
    n = 2 * a.shape[axis]
    shape = list(a.shape)
    shape[axis] = n
    x = np.zeros(shape)
    k = np.arange(n // 2)
    xm = np.moveaxis(x, axis, 0)
    am = np.moveaxis(a, axis, 0)
    dm = np.moveaxis(d, axis, 0)
    for j in range(len(h)):
        idx = (2 * k + j) % n  # distinct for fixed j
        xm[idx] += h[j] * am + g[j] * dm
    return x


def _band_codes(dim):
    return [2, 1, 3] if dim == 2 else list(range(1, 8))


def _analysis_level(x, h, g):
    """One level: returns (approximation, [detail bands in storage order])."""
    dim = x.ndim
    parts = {0: x}  # code -> array ; bit a set = high-pass along spatial axis a (0 = x)
    for a in range(dim):
        axis = dim - 1 - a
        new = {}
        for code, arr in parts.items():
            lo, hi = _analysis_axis(arr, h, g, axis)
            new[code] = lo
            new[code | (1 << a)] = hi
        parts = new
    return parts[0], [parts[c] for c in _band_codes(dim)]


def _synthesis_level(approx, details, h, g):
    dim = approx.ndim
    parts = {0: approx}
    for c, band in zip(_band_codes(dim), details):
        parts[c] = band
    for a in reversed(range(dim)):
        axis = dim - 1 - a
        new = {}
        for code in [c for c in parts if not (c >> a) & 1]:
            new[code] = _synthesis_axis(parts[code], parts[code | (1 << a)], h, g, axis)
        parts = new
    return parts[0]


class Wavelet:
    """Periodic orthonormal Daubechies transform of `levels` levels on grids of
    shape `shape` (every extent divisible by 2**levels)."""

    def __init__(self, shape, family: int, levels: int, level_offset: int = 0):
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        if family not in FAMILIES:
            raise ValueError("family must be 1 (haar), 2 (db2) or 4 (db4)")
        if levels < 0 or any(s % (1 << levels) for s in self.shape):
            raise ValueError("levels must be >= 0 and every extent divisible by 2**levels")
        self.levels = int(levels)
        self.level_offset = int(level_offset)
        self.h = daubechies(family)
        self.g = highpass(self.h)

    def level_weight(self, i: int, s: float) -> float:
        """Weight of the level-i detail block in E_s* (i = 1 finest)."""
        return 2.0 ** (-s * (self.levels - i + self.level_offset))

    def dwt(self, x):
        """W x as the flat coefficient string [cA_m, bands_m, ..., bands_1]."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        details = []
        a = x
        for _ in range(self.levels):
            a, bands = _analysis_level(a, self.h, self.g)
            details.append(bands)
        out = [a.ravel()]
        for bands in reversed(details):  # coarsest level first
            out.extend(b.ravel() for b in bands)
        return np.concatenate(out)

    def _split(self, u):
        u = np.asarray(u, dtype=np.float64).ravel()
        m = self.levels
        cshape = tuple(s >> m for s in self.shape)
        pos = int(np.prod(cshape))
        approx = u[:pos].reshape(cshape)
        details = {}
        nb = (1 << self.dim) - 1
        for i in range(m, 0, -1):
            bshape = tuple(s >> i for s in self.shape)
            sz = int(np.prod(bshape))
            details[i] = [u[pos + b * sz: pos + (b + 1) * sz].reshape(bshape) for b in range(nb)]
            pos += nb * sz
        assert pos == u.size
        return approx, details

    def idwt(self, u):
        """W^T u (= W^{-1} u) back to an array of `shape`."""
        approx, details = self._split(u)
        a = approx
        for i in range(self.levels, 0, -1):
            a = _synthesis_level(a, details[i], self.h, self.g)
        return a

    def scale(self, u, s: float):
        """S_s u: level-i details times 2^{-s(m-i+o)}, cA unchanged."""
        approx, details = self._split(u)
        out = [approx.ravel()]
        for i in range(self.levels, 0, -1):
            out.extend(self.level_weight(i, s) * b.ravel() for b in details[i])
        return np.concatenate(out)

    def EsT(self, x, s: float):
        """E_s* x = S_s W x (image -> coefficients)."""
        return self.scale(self.dwt(x), s)

    def Es(self, u, s: float):
        """E_s u = W^T S_s u (coefficients -> image)."""
        return self.idwt(self.scale(u, s))
