"""Pins of the oracle's absorbing layer (this implementation's reading of the paper's
PML: damping sigma p in the pressure equation, trapezoidal in time; see
oracle/fdtd.c): sigma = 0 is the undamped program, a uniform sigma on a
Dirichlet sine mode follows the closed form of the damped three-level
recurrence, the discrete energy falls by exactly the dissipation term, the
adjoint is the transpose, the quadratic profile has its hand values, and the
layer absorbs an outgoing pulse."""
from math import pi, sin

import numpy as np
import pytest

from oracle import Wave, sponge_sigma, sponge_sigma_max

from test_oracle_fdtd import _cfl_limit, _composed_L, _dense


def test_profile_hand_values():
    s = sponge_sigma((7, 9), 3, 1.0)
    # x axis (9 cells): d = 0 1 2 3 4 3 2 1 0 -> 1, 4/9, 1/9, 0, 0, 0, 1/9, 4/9, 1
    row = np.array([1, 4 / 9, 1 / 9, 0, 0, 0, 1 / 9, 4 / 9, 1])
    np.testing.assert_allclose(s[3], row, atol=1e-15)  # middle row: y contributes 0 (d = 3)
    np.testing.assert_allclose(s[0], row + 1.0, atol=1e-15)  # face row: y contributes sigma_max
    assert s[3, 4] == 0.0 and s[0, 0] == 2.0
    assert sponge_sigma((5, 5), 0, 1.0).max() == 0.0
    np.testing.assert_allclose(sponge_sigma_max(1500.0, 10, 1e-4, 1e-3), 3 * 1500 * np.log(1e3) / (2 * 10 * 1e-4))


def test_zero_sigma_is_undamped():
    rng = np.random.default_rng(1)
    shape, h = (18, 22), 1e-4
    c = 1400 + 200 * rng.random(shape)
    dt = 0.3 * h / c.max()
    sens = np.stack([rng.uniform(0, (s - 1) * h, 5) for s in shape[::-1]], axis=1)
    a = Wave(shape, h, dt, 70, 6, c, sens)
    b = Wave(shape, h, dt, 70, 6, c, sens, sigma=np.zeros(shape))
    x, y = rng.standard_normal(shape), rng.standard_normal((5, 70))
    np.testing.assert_array_equal(a.forward(x), b.forward(x))
    np.testing.assert_array_equal(a.adjoint(y), b.adjoint(y))


def test_uniform_damping_sine_mode_closed_form():
    """Order 2, constant c and sigma, Dirichlet sine mode phi (L phi = -lam phi):
    the damped three-level recurrence P^{n+1} = (1+a) P^n - a P^{n-1} - b kappa lam P^n
    with P^0 = phi, P^1 = (a - b kappa lam / 2) phi has the closed form
    P^n = (A r1^n + B r2^n) phi, r1, r2 the roots of r^2 - (1 + a - b kappa lam) r + a."""
    ny, nx, ky, kx = 13, 17, 3, 5
    h, c = 1e-4, 1500.0
    dt = 0.5 * h / c
    kappa = (c * dt / h) ** 2
    sigma = 0.08 / dt  # sigma dt / 2 = 0.04
    q = sigma * dt / 2
    a, b = (1 - q) / (1 + q), 1 / (1 + q)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.sin(pi * kx * (xx + 1) / (nx + 1)) * np.sin(pi * ky * (yy + 1) / (ny + 1))
    lam = 4 * sin(pi * kx / (2 * (nx + 1))) ** 2 + 4 * sin(pi * ky / (2 * (ny + 1))) ** 2
    tr = 1 + a - b * kappa * lam
    disc = np.sqrt(complex(tr * tr - 4 * a))
    r1, r2 = (tr + disc) / 2, (tr - disc) / 2
    p1 = a - b * kappa * lam / 2
    B = (p1 - r1) / (r2 - r1)
    A = 1 - B
    hist = Wave((ny, nx), h, dt, 80, 2, c, np.zeros((0, 2)), sigma=np.full((ny, nx), sigma)).history(phi)
    for n in range(80):
        amp = (A * r1 ** n + B * r2 ** n).real
        np.testing.assert_allclose(hist[n], amp * phi, atol=1e-12)
    assert abs(r1) < 1 and abs(r2) < 1  # the mode decays


@pytest.mark.parametrize("order", [2, 8])
def test_energy_falls_by_the_dissipation_term(order):
    """E^{n+1/2} = sum (P^{n+1}-P^n)^2/kappa - P^{n+1}.L P^n obeys
    E^{n+1/2} - E^{n-1/2} = -sum (sigma dt/2) / kappa (P^{n+1} - P^{n-1})^2
    for the damped scheme (varying c and sigma)."""
    shape = (20, 24)
    rng = np.random.default_rng(30 + order)
    c = 1400 + 200 * rng.random(shape)
    h = 1e-4
    dt = 0.9 * _cfl_limit(order, 2) * h / c.max()
    kap = ((c * dt / h) ** 2).ravel()
    sig = sponge_sigma(shape, 5, 0.3 / dt)
    q = (sig * dt / 2).ravel()
    L = _composed_L(shape, order)
    hist = Wave(shape, h, dt, 200, order, c, np.zeros((0, 2)), sigma=sig).history(rng.standard_normal(shape))
    P = hist.reshape(200, -1)
    E = np.array([np.sum((P[n + 1] - P[n]) ** 2 / kap) - P[n + 1] @ (L @ P[n]) for n in range(199)])
    diss = np.array([np.sum(q / kap * (P[n + 1] - P[n - 1]) ** 2) for n in range(1, 199)])
    np.testing.assert_allclose(E[1:] - E[:-1], -diss, atol=1e-10 * E[0])
    assert E[-1] < 0.5 * E[0]


@pytest.mark.parametrize("shape,order", [((16, 21), 4), ((12, 10), 8), ((9, 10, 11), 2)])
def test_dot_product_damped(shape, order):
    rng = np.random.default_rng(7 + order)
    h = 1e-4
    c = 1450 + 100 * rng.random(shape)
    dt = 0.3 * h / c.max()
    sens = np.stack([rng.uniform(0, (s - 1) * h, 7) for s in shape[::-1]], axis=1)
    wv = Wave(shape, h, dt, 60, order, c, sens, sigma=sponge_sigma(shape, 4, 0.5 / dt))
    x, y = rng.standard_normal(shape), rng.standard_normal((7, 60))
    lhs, rhs = float(np.sum(wv.forward(x) * y)), float(np.sum(x * wv.adjoint(y)))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10


def test_dense_adjoint_is_transpose_damped():
    shape, h, nt = (8, 8), 1e-4, 20
    rng = np.random.default_rng(3)
    dt = 0.3 * h / 1500
    sens = np.stack([rng.uniform(0, 7 * h, 3) for _ in range(2)], axis=1)
    wv = Wave(shape, h, dt, nt, 4, 1500.0, sens, sigma=sponge_sigma(shape, 3, 0.6 / dt))
    K = _dense(lambda v: wv.forward(v.reshape(shape)).ravel(), 64)
    Kt = _dense(lambda v: wv.adjoint(v.reshape(3, nt)).ravel(), 3 * nt)
    np.testing.assert_allclose(K, Kt.T, atol=1e-14 * np.abs(K).max())


def test_layer_absorbs_an_outgoing_pulse():
    """A centred Gaussian pulse on 96^2 (order 8, c = 1500, CFL 0.3), run for
    the time it takes to cross the grid four times: with a 10-cell layer
    (nominal reflection 1e-3) under 1 % of the initial energy is left, while
    the reflecting box keeps its energy."""
    n, h, c = 96, 1e-4, 1500.0
    dt = 0.3 * h / c
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x0 = np.exp(-((xx - n / 2) ** 2 + (yy - n / 2) ** 2) / (2 * 3.0 ** 2))
    nt = int(4 * n / 0.3)
    sig = sponge_sigma((n, n), 10, sponge_sigma_max(c, 10, h))

    def energy(p1, p0):  # potential proxy + kinetic proxy (kappa = 0.09)
        return float(np.sum(p1 ** 2) + np.sum((p1 - p0) ** 2) / 0.09)

    for name, s in (("box", None), ("layer", sig)):
        hist = Wave((n, n), h, dt, nt, 8, c, np.zeros((0, 2)), sigma=s).history(x0)
        e0, e1 = energy(hist[1], hist[0]), energy(hist[-1], hist[-2])
        if name == "box":
            assert e1 > 0.3 * e0
        else:
            assert e1 < 1e-2 * e0
