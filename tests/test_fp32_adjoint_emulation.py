"""Why the 2D adjoint kernels keep a compensated state: an FP32 emulation of
their arithmetic, in numpy, against the FP64 oracle (CPU only).

The adjoint recurrence of the increment-form leapfrog (paper Sec. 2, the
transpose of K) is run in Z = kappa Q:

    G^m = G^{m+1} + S^T r_m + L Z^{m+1},   Z^m = Z^{m+1} + kappa G^m,
    x   = S^T r_0 + G^1 + 1/2 L Z^1,

once plainly in FP32 (pair-form stencil (a + b) - 2c, as a textbook kernel
would) and once as the kernels do it (Z as a TwoSum pair, Z through the
difference form (a - c) + (b - c), Z_lo through its own stencil).  With data
simulated from a phantom the state Z integrates the data over time and grows
far beyond the result, and the plain recurrence loses an order of magnitude
of accuracy; this is the reason the per-step, batched and persistent 2D
kernels carry Z_lo.  The emulation is a model of the kernels' operation
order, not the CUDA path (the GPU tests check that)."""
import numpy as np
import pytest

import oracle
import synth

F = np.float32


def staggered_order8_weights():
    """Composed Laplacian weights w_1..w_7 of the order-8 staggered first derivative (Fornberg's
    coefficients 1225/1024, -245/3072, 49/5120, -5/7168): w = -(g * g) on the non-negative offsets."""
    c = [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168]
    g = np.array([-v for v in c[::-1]] + c)
    return (-np.correlate(g, g, "full"))[len(g) - 1:]


def laplacian_f32(P, w, diff):
    """sum over both axes and offsets m of w_m [(a - c) + (b - c)] (diff) or w_m [(a + b) - 2c],
    each tap rounded to FP32 and accumulated with one rounding, zero outside the grid."""
    R = len(w) - 1
    n0, n1 = P.shape
    Pp = np.zeros((n0 + 2 * R, n1 + 2 * R), F)
    Pp[R:-R, R:-R] = P
    c2 = (P + P).astype(F)
    acc = np.zeros(P.shape, F)
    for ax in (0, 1):
        for m in range(1, R + 1):
            if ax == 0:
                a, b = Pp[R + m:n0 + R + m, R:-R], Pp[R - m:n0 + R - m, R:-R]
            else:
                a, b = Pp[R:-R, R + m:n1 + R + m], Pp[R:-R, R - m:n1 + R - m]
            t = ((a - P).astype(F) + (b - P).astype(F)) if diff else ((a + b).astype(F) - c2)
            acc = (np.float64(F(w[m])) * t.astype(np.float64) + acc.astype(np.float64)).astype(F)
    return acc


def two_sum(a, b):
    s = (a + b).astype(F)
    bp = (s - a).astype(F)
    return s, ((a - (s - bp)) + (b - bp)).astype(F)


def adjoint_f32(y, kappa, sensors, h, w, compensated):
    n0, n1 = kappa.shape
    pos = sensors / h
    ix = np.minimum(np.floor(pos[:, 0]).astype(int), n1 - 2)
    iy = np.minimum(np.floor(pos[:, 1]).astype(int), n0 - 2)
    fx, fy = pos[:, 0] - ix, pos[:, 1] - iy
    corners = [((1 - fx) * (1 - fy), iy, ix), (fx * (1 - fy), iy, ix + 1), ((1 - fx) * fy, iy + 1, ix),
               (fx * fy, iy + 1, ix + 1)]

    def inject(t):
        acc = np.zeros(kappa.shape, F)
        for wk, cy, cx in corners:
            np.add.at(acc, (cy, cx), (wk.astype(F) * y[:, t].astype(F)).astype(F))
        return acc

    kh = kappa.astype(F)
    Z = np.zeros(kappa.shape, F)
    Zl = np.zeros(kappa.shape, F)
    G = np.zeros(kappa.shape, F)

    def lap():
        if compensated:
            return (laplacian_f32(Z, w, True) + laplacian_f32(Zl, w, False)).astype(F)
        return laplacian_f32(Z, w, False)

    for m in range(y.shape[1] - 1, 0, -1):
        G = (G + (inject(m) + lap()).astype(F)).astype(F)
        u = (kh * G).astype(F)
        if compensated:
            Z, e = two_sum(Z, u)
            Zl = (Zl + e).astype(F)
        else:
            Z = (Z + u).astype(F)
    return ((inject(0) + G).astype(F) + (F(0.5) * lap()).astype(F)).astype(F)


@pytest.fixture(scope="module")
def case():
    w = synth.workload("vessels", n=96, nt=500, levels=3)
    wave = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors)
    y = synth.add_noise(wave.forward(w.x_true), w.noise, np.random.default_rng(77))
    kappa = (w.c_array() * w.dt / w.h) ** 2
    return w, y, kappa, wave.adjoint(y)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_weights_are_zero_sum():
    w = staggered_order8_weights()
    assert abs(w[0] + 2 * w[1:].sum()) < 1e-14  # the composed 1D stencil annihilates constants


def test_compensated_state_is_an_order_of_magnitude_closer(case):
    w, y, kappa, x_ref = case
    wts = staggered_order8_weights()
    e_plain = rel(adjoint_f32(y, kappa, w.sensors, w.h, wts, False), x_ref)
    e_comp = rel(adjoint_f32(y, kappa, w.sensors, w.h, wts, True), x_ref)
    assert e_comp < 1e-6          # 2.8e-7 at this size
    assert e_plain > 5 * e_comp   # 3.7e-6 at this size; 1.9e-5 at 512^2 / 1500 steps
