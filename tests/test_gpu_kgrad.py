"""Medium gradient d<r, K x>/d kappa on the GPU (checkpointed adjoint) against
the FP64 oracle's reverse sweep of the staggered program, against central
differences of the FP64 forward map at full size, and for invariance under
the checkpoint interval."""
import numpy as np
import pytest

import synth
from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("shape,nt,order,varc", [((48, 72), 200, 8, True), ((64, 64), 300, 2, False),
                                                 ((20, 24, 18), 80, 4, False), ((16, 20, 24), 60, 8, True)])
def test_grad_kappa_matches_oracle(shape, nt, order, varc):
    need_gpu()
    w = custom(shape, nt, order, varc, 9, seed=len(shape) * 10 + order)
    plan, wave, _ = make_pair(w)
    rng = np.random.default_rng(3)
    r = rng.standard_normal((w.ns, w.nt))
    g_ref = wave.kappa_grad(w.x_true, r)
    g = plan.grad_kappa(w.x_true, r).cpu().numpy()
    assert rel(g, g_ref) <= TOL


def test_grad_kappa_independent_of_checkpoint_interval():
    need_gpu()
    w = custom((64, 96), 150, 8, True, 12, seed=4)
    plan, _, _ = make_pair(w)
    r = np.random.default_rng(4).standard_normal((w.ns, w.nt))
    gs = [plan.grad_kappa(w.x_true, r, segment=s).cpu().numpy() for s in (1, 0, 7, w.nt - 1)]
    for g in gs[1:]:
        assert np.array_equal(g, gs[0])


def test_grad_kappa_full_arc_1024_finite_differences():
    """1024 x 1024, c = 1500, order 8, 3000 steps, 256 sensors on a 180-degree
    arc, sqrt(nt) = 55-step checkpoints: <g, delta> against central differences
    of the FP64 oracle's <r, K(kappa) x> along two random directions."""
    need_gpu()
    import oracle
    w = synth.workload("arc")
    plan, wave, _ = make_pair(w)
    rng = np.random.default_rng(11)
    r = wave.forward(w.x_true) - synth.add_noise(wave.forward(w.x_true), 0.05, rng)
    g = plan.grad_kappa(w.x_true, r).cpu().numpy().astype(np.float64)
    kap = (w.c_array() * w.dt / w.h) ** 2
    eps = 1e-3

    def J(k):
        cc = np.sqrt(k) * w.h / w.dt
        return float(np.sum(r * oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, cc, w.sensors).forward(w.x_true)))

    for _ in range(2):
        # a smooth perturbation of the medium (a random speed map rescaled to +-1e-3 of kappa)
        sm = synth.speed_map(w.shape, rng, sigma=40.0, lo=-1.0, hi=1.0)
        delta = kap * 1e-3 * sm
        fd = (J(kap + eps * delta) - J(kap - eps * delta)) / (2 * eps)
        assert abs(fd - float(np.sum(g * delta))) <= 1e-4 * abs(fd)
