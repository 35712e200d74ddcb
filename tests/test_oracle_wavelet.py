"""Pins of the oracle's wavelet part (paper Sec. 4) against facts outside it:
published filter tables, the closed form of db2, orthonormality of the
multiresolution basis (Def. 4.1), hand values for Haar, and the exact
eigenstructure that Prop. 4.2's diagonal level scaling gives E_s E_s*."""
import os
from math import sqrt

import numpy as np
import pytest

from oracle import Wavelet, daubechies, highpass

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "daubechies_filters.txt")


def _golden_filters():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        out[int(parts[0])] = np.array([float(v) for v in parts[1:]])
    return out


@pytest.mark.parametrize("nv", [2, 4])
def test_filters_match_published_table(nv):
    ref = _golden_filters()[nv]
    np.testing.assert_allclose(daubechies(nv), ref, rtol=0, atol=1e-11)


def test_db2_closed_form():
    s3 = sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * sqrt(2.0))
    np.testing.assert_allclose(daubechies(2), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("nv", [1, 2, 4])
def test_filter_identities(nv):
    h = daubechies(nv)
    assert len(h) == 2 * nv
    assert abs(h.sum() - sqrt(2.0)) < 1e-14
    for k in range(nv):  # double-shift orthonormality
        assert abs(np.dot(h[: len(h) - 2 * k], h[2 * k:]) - (1.0 if k == 0 else 0.0)) < 1e-14
    g = highpass(h)
    j = np.arange(len(h), dtype=np.float64)
    for p in range(nv):  # nv vanishing moments of the wavelet
        assert abs(np.sum(g * j ** p)) < 1e-11 * (len(h) ** p)
    assert abs(np.dot(h, g)) < 1e-15


def test_haar_2x2_hand_values():
    w = Wavelet((2, 2), 1, 1)
    x = np.array([[1.0, 2.0], [3.0, 4.0]])  # row = y, column = x
    u = w.dwt(x)
    # cA = sum/2 ; cH = (row0 - row1)/2 ; cV = (col0 - col1)/2 ; cD = (1 - 2 - 3 + 4)/2
    np.testing.assert_allclose(u, [5.0, -2.0, -1.0, 0.0], atol=1e-15)


@pytest.mark.parametrize("shape,family,levels", [
    ((16, 16), 1, 4), ((16, 16), 2, 3), ((16, 16), 4, 4), ((32, 64), 4, 3), ((8, 8, 8), 4, 3), ((16, 8, 8), 2, 2)])
def test_perfect_reconstruction_and_energy(shape, family, levels):
    rng = np.random.default_rng(7)
    w = Wavelet(shape, family, levels)
    x = rng.standard_normal(shape)
    u = w.dwt(x)
    assert u.size == x.size
    assert np.linalg.norm(w.idwt(u) - x) / np.linalg.norm(x) < 1e-14
    assert abs(np.linalg.norm(u) - np.linalg.norm(x)) / np.linalg.norm(x) < 1e-14


def _dense(f, n):
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(np.asarray(f(e)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("shape,family,levels", [((16, 16), 4, 4), ((16, 16), 2, 2), ((8, 8, 8), 4, 3)])
def test_dense_transform_is_orthogonal(shape, family, levels):
    w = Wavelet(shape, family, levels)
    N = int(np.prod(shape))
    W = _dense(lambda e: w.dwt(e.reshape(shape)), N)
    np.testing.assert_allclose(W.T @ W, np.eye(N), atol=1e-13)
    Wi = _dense(lambda e: w.idwt(e).ravel(), N)
    np.testing.assert_allclose(Wi, W.T, atol=1e-14)


@pytest.mark.parametrize("shape,levels,s", [((16, 16), 1, 1.0), ((16, 16), 2, 1.5), ((16, 16), 3, 1.0),
                                            ((16, 16), 4, 2.0), ((8, 8, 8), 2, 1.0)])
def test_EsEsT_eigenstructure(shape, levels, s):
    """E_s E_s* = W^T S_s^2 W: eigenvalue 1 on cA_m (multiplicity (n/2^m)^d)
    and 2^{-2s(m-i)} on level-i details (multiplicity (2^d-1)(n/2^i)^d)."""
    w = Wavelet(shape, 4, levels)
    d = len(shape)
    N = int(np.prod(shape))
    G = _dense(lambda e: w.Es(w.EsT(e.reshape(shape), s), s).ravel(), N)
    np.testing.assert_allclose(G, G.T, atol=1e-13)
    ev = np.sort(np.linalg.eigvalsh(G))
    expect = [1.0] * (N >> (d * levels))
    for i in range(1, levels + 1):
        expect += [2.0 ** (-2 * s * (levels - i))] * ((2 ** d - 1) * (N >> (d * i)))
    np.testing.assert_allclose(ev, np.sort(expect), atol=1e-12)


def test_s_zero_is_identity():
    w = Wavelet((16, 16), 4, 3)
    x = np.random.default_rng(3).standard_normal((16, 16))
    np.testing.assert_allclose(w.Es(w.EsT(x, 0.0), 0.0), x, atol=1e-14)


def test_Es_is_adjoint_of_EsT():
    shape = (16, 32)
    w = Wavelet(shape, 4, 3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape)
    u = rng.standard_normal(x.size)
    lhs = np.dot(w.EsT(x, 1.3), u)
    rhs = np.sum(x * w.Es(u, 1.3))
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(u)


def test_wavelet_is_level_detail_eigenvector():
    """A single detail coefficient at level i is mapped by E_s E_s* to
    2^{-2s(m-i)} times itself (the inline weight of the paper's Sec. 4)."""
    shape, m, s = (32, 32), 4, 1.5
    w = Wavelet(shape, 4, m)
    sizes = [(32 >> m) ** 2] + sum([[(32 >> i) ** 2] * 3 for i in range(m, 0, -1)], [])
    starts = np.cumsum([0] + sizes)
    for band, lev in [(1, m), (4, m - 1), (len(sizes) - 1, 1)]:
        u = np.zeros(32 * 32)
        u[starts[band] + 1] = 1.0
        x = w.idwt(u)
        v = w.dwt(w.Es(w.EsT(x, s), s))
        np.testing.assert_allclose(v, 2.0 ** (-2 * s * (m - lev)) * u, atol=1e-13)
