"""Pins of the oracle's wave part (paper Sec. 2: the IVP of Eq. (wave_equation),
the measurement map K and its adjoint) against facts outside it: the exact
Chebyshev solution of a discrete Dirichlet sine mode, the 3D spherical-wave
closed form, Taylor accuracy of the composed stencil, exactness of bilinear
sampling on linear fields, conservation of the discrete energy below the CFL
limit, blow-up above it, the adjoint identity and the eliminated
pressure-only form of the same scheme."""
from math import cos, pi, sin, sqrt

import numpy as np
import pytest

from oracle import Wave

STAG = {2: [1.0], 4: [9 / 8, -1 / 24], 6: [75 / 64, -25 / 384, 3 / 640],
        8: [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168]}


def _dense(f, n):
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(np.asarray(f(e)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("shape", [(24, 20), (10, 12, 9)])
def test_dot_product_adjoint(order, shape):
    rng = np.random.default_rng(order)
    h = 1e-4
    c = 1400 + 200 * rng.random(shape)
    dt = 0.3 * h / c.max()
    d = len(shape)
    ns = 5
    sens = np.stack([rng.uniform(0, (s - 1) * h, ns) for s in shape[::-1]], axis=1)
    wv = Wave(shape, h, dt, 37, order, c, sens)
    x = rng.standard_normal(shape)
    y = rng.standard_normal((ns, 37))
    Kx, Ky = wv.forward(x), wv.adjoint(y)
    assert abs(np.sum(Kx * y) - np.sum(x * Ky)) <= 1e-13 * np.linalg.norm(Kx) * np.linalg.norm(y)
    assert d == len(shape)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_dense_adjoint_is_transpose(order):
    shape, nt = (8, 8), 20
    h = 1e-4
    rng = np.random.default_rng(10 + order)
    c = 1450 + 100 * rng.random(shape)
    dt = 0.3 * h / c.max()
    sens = np.array([[1.5e-4, 2.5e-4], [6.2e-4, 3.3e-4], [0.0, 7e-4]])
    wv = Wave(shape, h, dt, nt, order, c, sens)
    K = _dense(lambda e: wv.forward(e.reshape(shape)), 64)
    Ks = _dense(lambda e: wv.adjoint(e.reshape(3, nt)), 3 * nt)
    np.testing.assert_allclose(Ks, K.T, atol=1e-14 * np.abs(K).max())


@pytest.mark.parametrize("nt", [1, 2, 3])
def test_adjoint_short_time_axis(nt):
    shape = (9, 11)
    rng = np.random.default_rng(nt)
    wv = Wave(shape, 1e-4, 2e-8, nt, 4, 1500.0, np.array([[3e-4, 4e-4]]))
    K = _dense(lambda e: wv.forward(e.reshape(shape)), 99)
    Ks = _dense(lambda e: wv.adjoint(e.reshape(1, nt)), nt)
    np.testing.assert_allclose(Ks, K.T, atol=1e-15)
    if nt == 1:  # y_0 = S x: the bilinear weights themselves, summing to 1
        assert abs(K.sum() - 1.0) < 1e-14
    assert rng is not None


def test_chebyshev_sine_mode_order2():
    """Order 2, constant c, Dirichlet sine mode phi: the scheme gives exactly
    P^n = cos(n theta) phi with cos(theta) = 1 - kappa*lambda/2 and
    lambda = sum_axes 4 sin^2(pi k_a / (2 (n_a + 1)))."""
    ny, nx, ky, kx = 13, 17, 3, 5
    h, c = 1e-4, 1500.0
    dt = 0.5 * h / c
    kappa = (c * dt / h) ** 2
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.sin(pi * kx * (xx + 1) / (nx + 1)) * np.sin(pi * ky * (yy + 1) / (ny + 1))
    lam = 4 * sin(pi * kx / (2 * (nx + 1))) ** 2 + 4 * sin(pi * ky / (2 * (ny + 1))) ** 2
    theta = np.arccos(1 - kappa * lam / 2)
    wv = Wave((ny, nx), h, dt, 60, 2, c, np.zeros((0, 2)))
    hist = wv.history(phi)
    for n in range(60):
        np.testing.assert_allclose(hist[n], cos(n * theta) * phi, atol=1e-12)


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_composed_stencil_taylor_order(order):
    """LP^0 = 2 (P^1 - P^0)/kappa is the composed Laplacian; on a smooth
    interior Gaussian its error against the exact Laplacian falls like
    h^order under refinement."""
    errs = []
    for n in (40, 80):
        L = 1.0
        hh = L / n
        g = (np.arange(n) - (n - 1) / 2) * hh
        yy, xx = np.meshgrid(g, g, indexing="ij")
        sg = 0.08
        r2 = xx ** 2 + yy ** 2
        f = np.exp(-r2 / (2 * sg * sg))
        lap = f * (r2 / sg ** 4 - 2 / sg ** 2)
        dt = 0.1 * hh
        wv = Wave((n, n), hh, dt, 2, order, 1.0, np.zeros((0, 2)))
        hist = wv.history(f)
        kappa = (dt / hh) ** 2
        Lnum = 2 * (hist[1] - hist[0]) / kappa / hh ** 2
        errs.append(np.abs(Lnum - lap).max() / np.abs(lap).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > order - 0.6, (errs, rate)


def test_spherical_wave_closed_form_3d():
    """3D constant c, radial Gaussian p0 = f(r): the exact solution is
    p(r,t) = [(r-ct) f(r-ct) + (r+ct) f(r+ct)] / (2r).  Checked before the
    wave reaches the boundary; the error must be small and shrink under
    refinement at fixed CFL."""
    errs = []
    for n in (32, 64):
        Lbox = 1.0
        hh = Lbox / n
        c = 1.0
        dt = 0.3 * hh / c
        g = (np.arange(n) - (n - 1) / 2) * hh
        zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
        r = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
        sg = 0.06

        def f(rr):
            return np.exp(-rr ** 2 / (2 * sg * sg))

        T = 0.2
        nt = int(round(T / dt)) + 1
        t = (nt - 1) * dt
        wv = Wave((n, n, n), hh, dt, nt, 4, c, np.zeros((0, 3)))
        hist = wv.history(f(r))
        exact = ((r - c * t) * f(r - c * t) + (r + c * t) * f(r + c * t)) / (2 * np.maximum(r, 1e-12))
        exact[r < 1e-12] = 0.0
        mask = (r > 2 * hh) & (r < 0.4)
        errs.append(np.abs(hist[-1][mask] - exact[mask]).max() / np.abs(exact[mask]).max())
    assert errs[1] < 0.02, errs
    assert errs[1] < errs[0] / 2.5, errs


def test_bilinear_sampling_exact_on_linear_fields():
    shape = (12, 15)
    h = 2e-4
    rng = np.random.default_rng(5)
    sens = np.stack([rng.uniform(0, 14 * h, 20), rng.uniform(0, 11 * h, 20)], axis=1)
    sens[0] = [14 * h, 11 * h]  # the far corner
    sens[1] = [0.0, 0.0]
    yy, xx = np.meshgrid(np.arange(12) * h, np.arange(15) * h, indexing="ij")
    x0 = 0.3 + 2.0 * xx - 5.0 * yy
    wv = Wave(shape, h, 1e-8, 1, 8, 1500.0, sens)
    y = wv.forward(x0)[:, 0]
    np.testing.assert_allclose(y, 0.3 + 2.0 * sens[:, 0] - 5.0 * sens[:, 1], atol=1e-14)


def test_trilinear_sampling_exact_on_linear_fields():
    shape = (6, 7, 8)
    h = 1e-4
    rng = np.random.default_rng(6)
    sens = np.stack([rng.uniform(0, 7 * h, 9), rng.uniform(0, 6 * h, 9), rng.uniform(0, 5 * h, 9)], axis=1)
    zz, yy, xx = np.meshgrid(np.arange(6) * h, np.arange(7) * h, np.arange(8) * h, indexing="ij")
    wv = Wave(shape, h, 1e-8, 1, 4, 1500.0, sens)
    y = wv.forward(1.0 + xx + 2 * yy - 3 * zz)[:, 0]
    np.testing.assert_allclose(y, 1.0 + sens[:, 0] + 2 * sens[:, 1] - 3 * sens[:, 2], atol=1e-13)


def _composed_L(shape, order):
    """Dense L = -G^T G from the staggered difference G written as a matrix
    on the zero-extended grid (independent of the oracle's loops)."""
    c = STAG[order]
    M = len(c)
    d = len(shape)
    N = int(np.prod(shape))
    L = np.zeros((N, N))
    for a in range(d):
        axis = d - 1 - a
        na = shape[axis]
        G1 = np.zeros((na + 2 * M - 1, na))
        for f in range(na + 2 * M - 1):
            i = f - M
            for k in range(1, M + 1):
                if 0 <= i + k < na:
                    G1[f, i + k] += c[k - 1]
                if 0 <= i + 1 - k < na:
                    G1[f, i + 1 - k] -= c[k - 1]
        L1 = -(G1.T @ G1)
        mats = [np.eye(s) for s in shape]
        mats[axis] = L1
        K = mats[0]
        for mtx in mats[1:]:
            K = np.kron(K, mtx)
        L += K
    return L


@pytest.mark.parametrize("order", [2, 4, 8])
def test_pressure_only_form_matches(order):
    """Eliminating v gives P^{n+1} = 2P^n - P^{n-1} + kappa (L P^n) with
    P^1 = P^0 + kappa (L P^0)/2; the staggered oracle must agree."""
    shape = (9, 11)
    rng = np.random.default_rng(20 + order)
    c = 1450 + 100 * rng.random(shape)
    h = 1e-4
    dt = 0.3 * h / c.max()
    kap = ((c * dt / h) ** 2).ravel()
    L = _composed_L(shape, order)
    x = rng.standard_normal(shape).ravel()
    nt = 40
    P = [x, x + 0.5 * kap * (L @ x)]
    for _ in range(2, nt):
        P.append(2 * P[-1] - P[-2] + kap * (L @ P[-1]))
    hist = Wave(shape, h, dt, nt, order, c, np.zeros((0, 2))).history(x.reshape(shape))
    for n in range(nt):
        np.testing.assert_allclose(hist[n].ravel(), P[n], atol=1e-12 * np.abs(x).max())


def _cfl_limit(order, d):
    return 1.0 / (sqrt(d) * sum(abs(v) for v in STAG[order]))


@pytest.mark.parametrize("order", [2, 8])
def test_energy_conserved_below_cfl(order):
    shape = (20, 24)
    rng = np.random.default_rng(30 + order)
    c = 1400 + 200 * rng.random(shape)
    h = 1e-4
    dt = 0.95 * _cfl_limit(order, 2) * h / c.max()
    kap = ((c * dt / h) ** 2).ravel()
    L = _composed_L(shape, order)
    hist = Wave(shape, h, dt, 300, order, c, np.zeros((0, 2))).history(rng.standard_normal(shape))
    P = hist.reshape(300, -1)
    E = [np.sum((P[n + 1] - P[n]) ** 2 / kap) - P[n + 1] @ (L @ P[n]) for n in range(299)]
    E = np.array(E)
    assert E.min() > 0
    assert np.abs(E - E[0]).max() < 1e-11 * E[0]


def test_blowup_above_cfl():
    shape = (20, 20)
    h = 1e-4
    dt = 1.05 * _cfl_limit(4, 2) * h / 1500.0
    x = np.random.default_rng(1).standard_normal(shape)
    hist = Wave(shape, h, dt, 600, 4, 1500.0, np.zeros((0, 2))).history(x)
    assert np.abs(hist[-1]).max() > 1e3 * np.abs(x).max()


@pytest.mark.parametrize("shape,order", [((14, 17), 2), ((16, 12), 8), ((8, 9, 10), 4)])
def test_kappa_grad_matches_finite_differences(shape, order):
    """d<r, K x>/d kappa from the reverse sweep against central differences of
    the FP64 forward map under kappa -> kappa + eps delta (kappa = (c dt/h)^2)."""
    rng = np.random.default_rng(40 + order)
    h = 1e-4
    c = 1450 + 100 * rng.random(shape)
    dt = 0.3 * h / 1600.0
    nt = 45
    sens = np.stack([rng.uniform(0, (s - 1) * h, 6) for s in shape[::-1]], axis=1)
    x = rng.standard_normal(shape)
    r = rng.standard_normal((6, nt))
    g = Wave(shape, h, dt, nt, order, c, sens).kappa_grad(x, r)
    kap = (c * dt / h) ** 2
    for trial in range(3):
        delta = kap * 1e-3 * rng.standard_normal(shape)
        eps = 1e-3

        def J(k):
            cc = np.sqrt(k) * h / dt
            return float(np.sum(r * Wave(shape, h, dt, nt, order, cc, sens).forward(x)))

        fd = (J(kap + eps * delta) - J(kap - eps * delta)) / (2 * eps)
        assert abs(fd - float(np.sum(g * delta))) <= 1e-7 * np.linalg.norm(g) * np.linalg.norm(delta) + 1e-12 * abs(fd)
