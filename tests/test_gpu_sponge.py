"""Absorbing layer on the GPU (pat_plan_set_sponge) against the FP64 oracle's
damped program: K and K* (relative L2 <= 1e-5) through the persistent engine
and the per-step engine (TMA kernel for orders 2 and 8 with a constant
medium, order 4 varying medium whose adjoint runs the compensated kernel, the
plain kernel for nx not divisible by 4), short time axes, the default
damping rate, a CG solve (<= 1e-4), the GPU dot-product identity, and the
calls that refuse a layer."""
import numpy as np
import pytest

import oracle
from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5

CASES = [
    # shape, nt, order, varc, ns, width
    ((96, 128), 300, 8, False, 24, 10),
    ((72, 136), 250, 2, False, 17, 8),
    ((80, 96), 200, 4, True, 12, 10),
    ((66, 70), 180, 6, False, 9, 6),   # nx % 4 != 0: plain per-step kernel
]


def damped_pair(w, width, sigma_max):
    plan, _, wav = make_pair(w)
    plan.set_sponge(width, sigma_max)
    sigma = oracle.sponge_sigma(w.shape, width, sigma_max)
    wave = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors, sigma=sigma)
    return plan, wave, wav


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"-o{c[2]}" + ("v" if c[3] else ""))
@pytest.mark.parametrize("path", [1, 2], ids=["persistent", "step"])
def test_sponge_forward_adjoint_parity(case, path):
    need_gpu()
    shape, nt, order, varc, ns, width = case
    w = custom(shape, nt, order, varc, ns, seed=sum(shape) + order)
    smax = oracle.sponge_sigma_max(float(np.max(w.c_array())), width, w.h)
    plan, wave, _ = damped_pair(w, width, smax)
    plan.path = path
    y = plan.forward(w.x_true).cpu().numpy()
    y_ref = wave.forward(w.x_true)
    assert rel(y, y_ref) <= TOL_OP
    # the layer changes the data (it is not a no-op)
    undamped = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors).forward(w.x_true)
    assert rel(y_ref, undamped) > 1e-3
    r = np.random.default_rng(7).standard_normal((w.ns, w.nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP
    assert plan.check() == 0


@pytest.mark.parametrize("nt", [1, 2, 3, 5])
@pytest.mark.parametrize("path", [1, 2], ids=["persistent", "step"])
def test_sponge_short_time_axis(nt, path):
    need_gpu()
    w = custom((72, 136), nt, 8, False, 6, seed=nt)
    plan, wave, _ = damped_pair(w, 8, 0.4 / w.dt)
    plan.path = path
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    r = np.random.default_rng(nt).standard_normal((w.ns, nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP


def test_sponge_default_rate_and_removal():
    need_gpu()
    w = custom((64, 96), 150, 8, False, 10, seed=3)
    smax = oracle.sponge_sigma_max(1500.0, 10, w.h)
    a, _, _ = damped_pair(w, 10, smax)
    b, _, _ = make_pair(w)
    b.set_sponge(10)  # default rate
    ya, yb = a.forward(w.x_true).cpu().numpy(), b.forward(w.x_true).cpu().numpy()
    assert rel(yb, ya) <= 1e-6
    b.set_sponge(0)  # removed: the reflecting box again
    _, wave, _ = make_pair(w)
    for path in (1, 2):
        b.path = path
        assert rel(b.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP


def test_sponge_dot_product_and_solve():
    need_gpu()
    w = custom((96, 96), 250, 8, True, 20, seed=11, family=4, levels=3)
    plan, wave, wav = damped_pair(w, 10, 0.3 / w.dt)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(w.shape)
    y = rng.standard_normal((w.ns, w.nt))
    Kx = plan.forward(x).double().cpu().numpy()
    Ky = plan.adjoint(y).double().cpu().numpy()
    assert abs(float(np.sum(Kx * y)) - float(np.sum(x * Ky))) <= 1e-5 * np.linalg.norm(Kx) * np.linalg.norm(y)
    data = wave.forward(w.x_true)
    alpha = 1e-3 * float(np.sum(wave.adjoint(data) ** 2)) / float(np.sum(data ** 2))  # on the scale of ||K||^2
    _, xg, _ = plan.solve(data, alpha, 1.0, 10)
    _, xr, _ = oracle.cg(wave, wav, data, alpha, 1.0, 10)
    assert rel(xg.cpu().numpy(), xr) <= 1e-4


def test_sponge_refusals():
    torch = need_gpu()
    from paper_2507_02401_gb300 import _lib
    w3 = custom((16, 20, 24), 30, 4, False, 4, seed=1)
    p3, _, _ = make_pair(w3)
    with pytest.raises(_lib.PatError):
        p3.set_sponge(4)  # 3D
    w = custom((64, 64), 60, 8, False, 5, seed=2)
    p, _, _ = make_pair(w)
    with pytest.raises(_lib.PatError):
        p.set_sponge(40)  # wider than half the grid
    with pytest.raises(_lib.PatError):
        p.set_sponge(-1)
    p.set_sponge(8)
    r = np.zeros((w.ns, w.nt))
    with pytest.raises(_lib.PatError):
        p.grad_kappa(w.x_true, r)
    q, _, _ = make_pair(custom((64, 64), 60, 8, False, 5, seed=3))
    with pytest.raises(_lib.PatError):
        _lib.pat_batch_create([p.handle, q.handle])
    torch.cuda.synchronize()
