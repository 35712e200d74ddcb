"""Pins of the oracle's GMRES (the paper's solver on the image-space system
A x = f, A = E_s E_s* K* K + alpha I) and Landweber iteration, on problems
small enough for dense matrices: the GMRES iterate is the least-squares
minimiser over the Krylov space built by brute force, its residual log is the
true residual, it reaches the direct solution at full dimension and there
coincides with CG's image (the same minimiser); Landweber matches its
polynomial closed form and decreases J."""
import numpy as np
import pytest

import oracle
from oracle import krylov


def tiny(seed=0, shape=(8, 8), nt=24, ns=5, levels=1, family=2):
    rng = np.random.default_rng(seed)
    h = 1e-4
    dt = 0.3 * h / 1500.0
    sens = np.stack([rng.uniform(0, (s - 1) * h, ns) for s in shape[::-1]], axis=1)
    wave = oracle.Wave(shape, h, dt, nt, 4, 1500.0, sens)
    wav = oracle.Wavelet(shape, family, levels)
    y = rng.standard_normal((ns, nt))
    return wave, wav, y, rng


def dense(op, n):
    return np.stack([op(np.eye(n)[i]) for i in range(n)], axis=1)


def test_gmres_iterate_is_krylov_least_squares():
    wave, wav, y, _ = tiny(1)
    alpha, s = 0.05, 1.0
    A = krylov.image_op(wave, wav, s, alpha)
    f = wav.Es(wav.EsT(wave.adjoint(y), s), s).ravel()
    for k in (1, 2, 3, 5):
        x, res, _ = krylov.gmres(wave, wav, y, alpha, s, k)
        # brute force: minimise ||f - A x|| over span{f, A f, ..., A^{k-1} f}
        Kr = [f]
        for _ in range(k - 1):
            Kr.append(A(Kr[-1]))
        Kr = np.stack(Kr, axis=1)
        AK = np.stack([A(Kr[:, i]) for i in range(k)], axis=1)
        c = np.linalg.lstsq(AK, f, rcond=None)[0]
        np.testing.assert_allclose(x.ravel(), Kr @ c, rtol=1e-7, atol=1e-10 * np.abs(Kr @ c).max())
        np.testing.assert_allclose(res[-1], np.linalg.norm(f - A(x.ravel())), rtol=1e-8)


def test_gmres_residuals_and_full_dimension():
    wave, wav, y, _ = tiny(2)
    alpha, s = 0.02, 1.5
    n = wave.N
    x, res, J = krylov.gmres(wave, wav, y, alpha, s, n)
    assert np.all(np.diff(res) <= 1e-12 * res[0])
    Ad = dense(krylov.image_op(wave, wav, s, alpha), n)
    f = wav.Es(wav.EsT(wave.adjoint(y), s), s).ravel()
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(Ad, f), rtol=1e-8, atol=1e-12)
    # the paper's system and the coefficient system have the same minimiser
    _, x_cg, _ = oracle.cg(wave, wav, y, alpha, s, 3 * n)
    np.testing.assert_allclose(x, x_cg, rtol=1e-7, atol=1e-10 * np.abs(x).max())
    assert J[-1] <= J[0]


def test_landweber_closed_form_and_descent():
    wave, wav, y, _ = tiny(3)
    alpha, s = 0.1, 1.0
    n = wave.N
    Hd = dense(oracle.normal_op(wave, wav, s, alpha), n)
    b = oracle.rhs(wave, wav, y, s)
    lam = float(np.linalg.eigvalsh(0.5 * (Hd + Hd.T)).max())
    omega = 1.0 / lam
    k = 7
    u, x, J = krylov.landweber(wave, wav, y, alpha, s, k, omega)
    M = np.eye(n) - omega * Hd
    ref = sum(np.linalg.matrix_power(M, i) @ (omega * b) for i in range(k))
    np.testing.assert_allclose(u, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    assert np.all(np.diff(J) <= 0)
    # J at the exact minimiser bounds every iterate from below
    u_star = np.linalg.solve(Hd, b)
    assert krylov.objective(wave, wav, y, alpha, s, u_star) <= J.min() + 1e-12 * J[0]


def test_coefficients_invert_Es():
    wave, wav, _, rng = tiny(4, shape=(16, 16), levels=3)
    u = rng.standard_normal(wave.N)
    for s in (0.0, 1.0, 2.0):
        np.testing.assert_allclose(krylov.coefficients(wav, wav.Es(u, s), s), u, rtol=1e-12, atol=1e-12)
