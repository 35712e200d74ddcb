"""GMRES (the paper's solver, on the image-space system with Gamma = E_s E_s*)
and the Landweber iteration on the GPU against the FP64 oracle: final image,
residual and objective logs (relative L2 <= 1e-4, the reconstruction bound),
host-array arguments, and GMRES reaching CG's minimiser."""
import numpy as np
import pytest

import oracle
from oracle import krylov
from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_X = 1e-4


def problem(shape=(64, 64), nt=200, order=8, varc=True, ns=24, seed=5, levels=3):
    w = custom(shape, nt, order, varc, ns, seed=seed, family=4, levels=levels)
    plan, wave, wav = make_pair(w)
    y = synth_data(w, wave, seed)
    # alpha on the scale of ||K||^2 (Rayleigh quotient of K K* on the data)
    alpha = 1e-2 * float(np.sum(wave.adjoint(y) ** 2)) / float(np.sum(y ** 2))
    return w, plan, wave, wav, y, alpha


def synth_data(w, wave, seed):
    import synth
    return synth.add_noise(wave.forward(w.x_true), 0.01, np.random.default_rng(seed))


@pytest.mark.parametrize("s", [1.0, 2.0])
def test_gmres_matches_oracle(s):
    need_gpu()
    w, plan, wave, wav, y, alpha = problem()
    iters = 12
    x, res, J = plan.solve_gmres(y, alpha, s, iters, want_log=True)
    x_ref, res_ref, J_ref = krylov.gmres(wave, wav, y, alpha, s, iters)
    assert rel(x.cpu().numpy(), x_ref) <= TOL_X
    assert rel(res, res_ref) <= TOL_X
    assert rel(J, J_ref) <= TOL_X
    assert np.all(np.diff(res) <= 1e-6 * res[0])


def test_landweber_matches_oracle():
    need_gpu()
    w, plan, wave, wav, y, alpha = problem(shape=(48, 72), order=4, varc=False, seed=7)
    s = 1.5
    # omega below 1 / lambda_max from a few oracle power iterations
    H = oracle.normal_op(wave, wav, s, alpha)
    v = np.random.default_rng(0).standard_normal(wave.N)
    for _ in range(20):
        v = H(v)
        lam = float(np.linalg.norm(v))
        v /= lam
    omega = 0.9 / lam
    iters = 15
    u, x, J = plan.solve_landweber(y, alpha, s, iters, omega, want_log=True)
    u_ref, x_ref, J_ref = krylov.landweber(wave, wav, y, alpha, s, iters, omega)
    assert rel(u.cpu().numpy(), u_ref) <= TOL_X
    assert rel(x.cpu().numpy(), x_ref) <= TOL_X
    assert rel(J, J_ref) <= TOL_X
    assert np.all(np.diff(J) <= 1e-6 * J[0])


def test_gmres_host_arrays_and_cg_minimiser():
    need_gpu()
    from paper_2507_02401_gb300 import _lib
    w, plan, wave, wav, y, alpha = problem(shape=(32, 32), nt=120, order=2, varc=False, seed=9, levels=2)
    s = 1.0
    x_host = np.zeros(w.shape, dtype=np.float32)
    res = np.zeros(41)
    _lib.pat_solve_gmres(plan.handle, np.ascontiguousarray(y, dtype=np.float32), alpha, s, 40, x_host, res, None,
                         None)
    x_dev, _, _ = plan.solve_gmres(y, alpha, s, 40)
    assert rel(x_host, x_dev.cpu().numpy()) <= 1e-6
    # 40 GMRES iterations and 60 CG iterations reach the same minimiser
    _, x_cg, _ = plan.solve(y, alpha, s, 60)
    assert rel(x_host, x_cg.cpu().numpy()) <= 1e-3
    assert res[-1] <= 1e-3 * res[0]
