"""Pins of the oracle's CG solve of paper Eq. (linear_minimization) in
coefficient form: agreement with a dense direct solve, monotone error in the
energy norm, the 1 + 2k wave-evaluation count of Sec. 5, the equivalence with
the paper's non-symmetric system, and convergence of a noise-free
reconstruction."""
import numpy as np
import pytest

import synth
from oracle import Wave, Wavelet, cg, cg_converged, normal_op, rhs


def _small(n=16, nt=40, order=4, family=4, levels=2, ns=12, seed=3):
    rng = np.random.default_rng(seed)
    h = 1e-4
    c = 1450 + 100 * rng.random((n, n))
    dt = 0.3 * h / c.max()
    wave = Wave((n, n), h, dt, nt, order, c, synth.circle(n, h, ns))
    wav = Wavelet((n, n), family, levels)
    return wave, wav, rng


def _dense(f, n):
    return np.stack([f(np.eye(n)[i]) for i in range(n)], axis=1)


def test_cg_matches_dense_solve():
    wave, wav, rng = _small()
    s, alpha = 1.0, 0.05
    N = 256
    y = rng.standard_normal((wave.ns, wave.nt))
    Hd = _dense(normal_op(wave, wav, s, alpha), N)
    np.testing.assert_allclose(Hd, Hd.T, atol=1e-12 * np.abs(Hd).max())
    assert np.linalg.eigvalsh(Hd).min() >= alpha * (1 - 1e-10)
    b = rhs(wave, wav, y, s)
    u_ref = np.linalg.solve(Hd, b)
    u, x, log = cg(wave, wav, y, alpha, s, 120)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-9
    np.testing.assert_allclose(x, wav.Es(u_ref, s), atol=1e-9 * np.abs(x).max())
    # energy-norm error decreases monotonically along the CG iterates
    errs = []
    for k in range(1, 30):
        uk, _, _ = cg(wave, wav, y, alpha, s, k)
        e = uk - u_ref
        errs.append(e @ Hd @ e)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


def test_equivalent_to_paper_system():
    """x = E_s u solves (Gamma K*K + alpha I) x = Gamma K* y with
    Gamma = E_s E_s*, the paper's operator with its covariance."""
    wave, wav, rng = _small(seed=4)
    s, alpha = 1.5, 0.02
    y = rng.standard_normal((wave.ns, wave.nt))
    u, x, _ = cg(wave, wav, y, alpha, s, 200)

    def gamma(v):
        return wav.Es(wav.EsT(v, s), s)

    lhs = gamma(wave.adjoint(wave.forward(x))) + alpha * x
    rhs_ = gamma(wave.adjoint(y))
    assert np.linalg.norm(lhs - rhs_) / np.linalg.norm(rhs_) < 1e-9


@pytest.mark.parametrize("k", [0, 1, 5, 15])
def test_wave_evaluation_count(k):
    """k CG iterations cost 1 + 2k wave evaluations (15 iterations -> 31)."""
    wave, wav, rng = _small(n=12, nt=10, levels=1, family=2)
    y = rng.standard_normal((wave.ns, wave.nt))
    wave.evaluations = 0
    cg(wave, wav, y, 0.1, 1.0, k)
    assert wave.evaluations == 1 + 2 * k


def test_noise_free_reconstruction_converges():
    n = 32
    w = synth.workload("small", n=n, nt=160, order=4, family=2, levels=2, ns=64)
    wave = Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors)
    wav = Wavelet(w.shape, w.family, w.levels)
    y = wave.forward(w.x_true)
    errs = []
    for k in (5, 20, 60):
        _, x, _ = cg(wave, wav, y, 1e-8, 1.0, k)
        errs.append(np.linalg.norm(x - w.x_true) / np.linalg.norm(w.x_true))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05, errs


def test_cg_converged_is_the_dense_minimiser():
    """The converged solve (residual tolerance) reaches the dense direct
    solution of the normal equations, and reports a true residual below the
    tolerance; a plain fixed-count CG with fewer iterations does not."""
    wave, wav, rng = _small(seed=6)
    s, alpha = 2.0, 1e-3
    y = rng.standard_normal((wave.ns, wave.nt))
    Hd = _dense(normal_op(wave, wav, s, alpha), 256)
    u_ref = np.linalg.solve(Hd, rhs(wave, wav, y, s))
    u, x, k, rel_res = cg_converged(wave, wav, y, alpha, s, rtol=1e-11)
    assert rel_res <= 1e-10
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-8
    u5, _, _ = cg(wave, wav, y, alpha, s, 5)
    assert np.linalg.norm(u5 - u_ref) / np.linalg.norm(u_ref) > 1e-4
    assert k > 5


def test_cg_snapshots_are_the_fixed_count_iterates():
    """An iterate recorded on the way equals a separate run stopped there."""
    wave, wav, rng = _small(seed=7)
    y = rng.standard_normal((wave.ns, wave.nt))
    _, x12, _, snaps = cg(wave, wav, y, 0.02, 1.0, 12, snapshots=(5, 9))
    assert sorted(snaps) == [5, 9]
    for k in (5, 9):
        _, xk, _ = cg(wave, wav, y, 0.02, 1.0, k)
        np.testing.assert_array_equal(snaps[k], xk)
    _, x12b, _ = cg(wave, wav, y, 0.02, 1.0, 12)
    np.testing.assert_array_equal(x12, x12b)

