"""Pins of the oracle's Fourier-form prior (paper Sec. 4: E_s* = ifft(B fft)
with the Bessel potential B = (1 + 4 pi^2 |xi|^2)^{-s}): at s = 3/2 in 2D the
covariance kernel is the Ornstein-Uhlenbeck function exp(-|x|)/(2 pi) (the
paper's worked case), s = 0 is the identity, Fourier modes are eigenvectors
with the potential's value, the operator is symmetric, E_a E_b = E_{a+b}, and
E_s E_s* is the paper's operator."""
import numpy as np
import pytest

from oracle import FourierPrior


def test_ornstein_uhlenbeck_kernel():
    n, lc = 256, 16.0
    fp = FourierPrior((n, n), lc)
    delta = np.zeros((n, n))
    delta[0, 0] = 1.0
    g = fp.Gamma(delta, 1.5) * lc ** 2  # kernel per unit area, lengths in units of lc cells
    j = np.arange(n)
    d = np.minimum(j, n - j) / lc
    r = np.sqrt(d[:, None] ** 2 + d[None, :] ** 2)
    ref = np.exp(-r) / (2 * np.pi)
    m = (r >= 0.5) & (r <= 4.0)
    assert np.max(np.abs(g[m] - ref[m]) / ref[m]) < 1e-3


def test_identity_modes_symmetry_semigroup():
    shape = (16, 32)
    fp = FourierPrior(shape, 2.0)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(shape)
    np.testing.assert_allclose(fp.Es(u, 0.0), u, atol=1e-13)
    # a Fourier mode is an eigenvector: eigenvalue (1 + 4 pi^2 |xi|^2)^{-s/2}
    ky, kx = 3, 5
    yy, xx = np.meshgrid(np.arange(16), np.arange(32), indexing="ij")
    mode = np.cos(2 * np.pi * (ky * yy / 16 + kx * xx / 32))
    xi2 = (ky * 2.0 / 16) ** 2 + (kx * 2.0 / 32) ** 2
    np.testing.assert_allclose(fp.Es(mode, 1.5), (1 + 4 * np.pi ** 2 * xi2) ** -0.75 * mode, atol=1e-12)
    # symmetric: <E u, v> = <u, E v>
    v = rng.standard_normal(shape)
    assert abs(np.sum(fp.Es(u, 1.0) * v) - np.sum(u * fp.Es(v, 1.0))) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(v)
    np.testing.assert_allclose(fp.Es(fp.Es(u, 0.7), 1.1), fp.Es(u, 1.8), atol=1e-12)
    np.testing.assert_allclose(fp.Es(fp.EsT(u, 1.2).reshape(shape), 1.2), fp.Gamma(u, 1.2), atol=1e-12)


@pytest.mark.parametrize("s", [0.5, 2.0])
def test_smoothing_decays_high_frequencies(s):
    fp = FourierPrior((64, 64), 4.0)
    noise = np.random.default_rng(1).standard_normal((64, 64))
    out = fp.Es(noise, s)
    spec_in = np.abs(np.fft.fft2(noise))
    spec_out = np.abs(np.fft.fft2(out))
    ratio = spec_out / spec_in
    np.testing.assert_allclose(ratio, fp.potential ** (-s / 2), rtol=1e-9)
    assert ratio[32, 32] < ratio[1, 1] < 1.0
