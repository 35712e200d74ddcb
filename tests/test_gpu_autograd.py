"""Differentiation through torch.autograd: the backward of every wrapper is the
library's adjoint kernel.  Checked by the dot-product identity, by central
finite differences of the FP64 oracle's objective (eps = 1e-3) along random
directions, and by the oracle's FP64 gradient.

Objective (paper Eq. reg_functional with the coefficient form of
Eq. linear_minimization): J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu


def _oracle_J_parts(wave, wav, u, y, s):
    """(K E_s u - y) in FP64."""
    return wave.forward(wav.Es(u, s)) - y


def _check(w, ndir, seed, tol_grad=1e-5, tol_fd=1e-5):
    torch = need_gpu()
    from paper_2507_02401_gb300 import autograd as ag
    plan, wave, wav = make_pair(w)
    rng = np.random.default_rng(seed)
    s, alpha = w.s[0], 1e-3
    y = synth.add_noise(wave.forward(w.x_true), w.noise, rng)
    u0 = wav.EsT(w.x_true, s) * 0.7 + 0.05 * rng.standard_normal(w.N)

    # GPU gradient through autograd
    ut = torch.tensor(u0, dtype=torch.float32, device="cuda", requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    J = ag.reconstruction_loss(plan, ut, yt, alpha, s)
    J.backward()
    g = ut.grad.double().cpu().numpy()

    # FP64 oracle gradient: E_s* K* (K E_s u - y) + alpha u
    res = _oracle_J_parts(wave, wav, u0, y, s)
    g_ref = wav.EsT(wave.adjoint(res), s) + alpha * u0
    assert rel(g, g_ref) <= tol_grad
    # the objective's value (library, FP64 reductions) against the oracle's
    J_ref = 0.5 * float(np.sum(res * res)) + 0.5 * alpha * float(u0 @ u0)
    assert abs(float(J) - J_ref) <= 1e-5 * J_ref

    # central differences of the FP64 objective; K is linear, so
    # K E_s (u +- eps d) = K E_s u +- eps K E_s d exactly (up to FP64 rounding)
    eps = 1e-3

    def J64(rr, uu):
        return 0.5 * float(np.sum(rr * rr)) + 0.5 * alpha * float(uu @ uu)

    worst = 0.0
    for _ in range(ndir):
        d = rng.standard_normal(w.N)
        Kd = wave.forward(wav.Es(d, s))
        fd = (J64(res + eps * Kd, u0 + eps * d) - J64(res - eps * Kd, u0 - eps * d)) / (2 * eps)
        worst = max(worst, abs(fd - float(g @ d)) / (np.linalg.norm(g_ref) * np.linalg.norm(d)))
    assert worst <= tol_fd, worst
    return plan


def test_autograd_small_many_directions():
    """256 x 256, constant c, order 8, 600 steps, 180-degree arc, db4 4 levels,
    s = 1.5: 64 random directions."""
    w = synth.workload("arc", n=256, nt=600, ns=96, levels=4)
    _check(w, 64, seed=1)


def test_autograd_full_arc_1024():
    """The differentiation workload at full size: 1024 x 1024, constant c,
    order 8, 3000 steps, 256 sensors on a 180-degree arc, db4 6 levels,
    s = 1.5 (16 directions; each costs the oracle one 3000-step solve)."""
    _check(synth.workload("arc"), 16, seed=2)


def test_dot_product_through_autograd():
    """<K x, y> = <x, grad_x <K x, y>> with the gradient from backward."""
    torch = need_gpu()
    from paper_2507_02401_gb300 import autograd as ag
    w = synth.workload("vessels", n=128, nt=400, levels=3)
    plan, _, _ = make_pair(w)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(w.shape, device="cuda", generator=g, requires_grad=True)
    y = torch.randn((w.ns, w.nt), device="cuda", generator=g)
    Kx = ag.K(plan, x)
    (Kx.double() * y.double()).sum().backward()
    lhs = float((Kx.double() * y.double()).sum())
    rhs = float((x.double() * x.grad.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(Kx.double().norm() * y.double().norm())
    # and the transposed wrapper's backward is K
    yy = torch.randn((w.ns, w.nt), device="cuda", generator=g, requires_grad=True)
    xx = torch.randn(w.shape, device="cuda", generator=g)
    Kty = ag.Kt(plan, yy)
    (Kty.double() * xx.double()).sum().backward()
    assert rel(yy.grad.cpu().numpy(), plan.forward(xx).cpu().numpy()) <= 1e-7
