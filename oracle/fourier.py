"""Fourier form of the Sobolev embedding (test infrastructure only).

Paper Sec. 4 (implementation): the adjoint embedding acts in the Fourier
domain as multiplication by the Bessel potential (1 + 4 pi^2 |xi|^2)^{-s},
E_s* X = ifft(B . fft(X)) with B that potential sampled on the discrete
frequencies.  In the coefficient formulation used here (H = E_s* K* K E_s
+ alpha I, x = E_s u) the paper's operator is the covariance Gamma = E_s E_s*,
so the Fourier prior's E_s is the filter with the square root of the
potential, (1 + 4 pi^2 |xi|^2)^{-s/2}; it is real and symmetric, so E_s* = E_s.

Units: lengths are measured in units of `length_cells` grid cells, so DFT
index k on an axis of n cells is the frequency xi = k * length_cells / n
(cycles per unit).  numpy's FFT serves as the transform.
"""
import numpy as np


class FourierPrior:
    def __init__(self, shape, length_cells=1.0):
        self.shape = tuple(int(s) for s in shape)
        self.length_cells = float(length_cells)
        xi2 = 0.0
        for ax, n in enumerate(self.shape):
            xi = np.fft.fftfreq(n) * n * self.length_cells / n
            xi2 = xi2 + (xi ** 2).reshape([n if k == ax else 1 for k in range(len(self.shape))])
        self.potential = 1.0 + 4.0 * np.pi ** 2 * xi2  # (1 + 4 pi^2 |xi|^2)

    def Es(self, u, s):
        """E_s u = ifft((1 + 4 pi^2 |xi|^2)^{-s/2} fft(u)) (real)."""
        u = np.asarray(u, dtype=np.float64).reshape(self.shape)
        return np.fft.ifftn(self.potential ** (-s / 2.0) * np.fft.fftn(u)).real

    def EsT(self, x, s):
        """E_s* = E_s (the multiplier is real and even); returns a flat vector."""
        return self.Es(x, s).ravel()

    def Gamma(self, x, s):
        """The paper's E_s* of Sec. 4: ifft((1 + 4 pi^2 |xi|^2)^{-s} fft(x))."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        return np.fft.ifftn(self.potential ** (-s) * np.fft.fftn(x)).real
