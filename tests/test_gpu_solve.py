"""GPU CG solve (FP32 vectors, FP64 device scalars) against the oracle's FP64
CG at the same iteration count.  Bound on the final reconstruction: relative
L2 error <= 1e-4."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_X = 1e-4


def lambda_max(wave, wav, s, iters=15, seed=0):
    """Power iteration on E_s* K* K E_s (oracle, FP64)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(wave.N)
    v /= np.linalg.norm(v)
    lam = 0.0
    H = oracle.normal_op(wave, wav, s, 0.0)
    for _ in range(iters):
        hv = H(v)
        lam = float(np.linalg.norm(hv))
        v = hv / lam
    return lam


def data(w, wave, seed=7):
    return synth.add_noise(wave.forward(w.x_true), w.noise, np.random.default_rng(seed))


@pytest.mark.parametrize("family", [1, 2])
def test_small_circle_solve(family):
    """64 x 64, c = 1500, order 2, 250 steps, 32 sensors on a circle, 1% noise,
    Haar / db2 with 3 levels, s = 1, alpha = 1e-2 (relative), 50 iterations."""
    need_gpu()
    w = synth.workload("small", family=family)
    plan, wave, wav = make_pair(w)
    y = data(w, wave)
    s = w.s[0]
    alpha = w.alpha[0] * lambda_max(wave, wav, s)
    u_ref, x_ref, log_ref = oracle.cg(wave, wav, y, alpha, s, w.iters)
    u, x, log = plan.solve(y, alpha, s, w.iters, want_log=True)
    assert plan.check() == 0
    assert rel(x.cpu().numpy(), x_ref) <= TOL_X
    assert rel(u.cpu().numpy(), u_ref) <= TOL_X
    lg = log.cpu().numpy()
    np.testing.assert_allclose(lg[:10], log_ref[:10], rtol=1e-4)


def test_varc_order8_solve_and_warm_start():
    need_gpu()
    w = synth.workload("vessels", n=128, nt=400, levels=4, iters=30)
    plan, wave, wav = make_pair(w)
    y = data(w, wave)
    s = 2.0
    alpha = 1e-2 * lambda_max(wave, wav, s)
    u_ref, x_ref, _ = oracle.cg(wave, wav, y, alpha, s, 20)
    u, x, _ = plan.solve(y, alpha, s, 20)
    assert rel(x.cpu().numpy(), x_ref) <= TOL_X
    # warm start from u20 for 10 more iterations
    u2_ref, x2_ref, _ = oracle.cg(wave, wav, y, alpha, s, 10, u0=u_ref)
    u2, x2, _ = plan.solve(y, alpha, s, 10, u0=u)
    assert rel(x2.cpu().numpy(), x2_ref) <= TOL_X
    assert plan.check() == 0


def test_breakdown_is_reported_not_raised():
    """y = 0 gives b = 0, r = p = 0 and p.q = 0 at the first iteration: the
    solver stops, keeps u = 0 and reports PAT_ERR_BREAKDOWN."""
    need_gpu()
    from paper_2507_02401_gb300 import _lib
    w = synth.workload("small", n=32, nt=60, levels=2)
    plan, _, _ = make_pair(w)
    u, x, _ = plan.solve(np.zeros((w.ns, w.nt)), 1e-3, 1.0, 3)
    assert plan.check() == _lib.PAT_ERR_BREAKDOWN
    assert float(u.abs().max()) == 0.0
    assert plan.check() == 0  # cleared after being reported


def test_timeout_is_reported_not_hung():
    """A zero wait bound makes the persistent engine give up at its first
    unsatisfied inter-tile wait; the call returns, the plan reports
    PAT_ERR_TIMEOUT and the next call (with the normal bound) is correct."""
    torch = need_gpu()
    from paper_2507_02401_gb300 import _lib
    w = synth.workload("vessels", n=256, nt=400, levels=3)
    plan, wave, _ = make_pair(w, path=1)
    _lib.pat_plan_set_timeout(plan.handle, 0)
    for _ in range(5):
        plan.forward(w.x_true)
    st = plan.check()
    assert st in (0, _lib.PAT_ERR_TIMEOUT)
    _lib.pat_plan_set_timeout(plan.handle, 2_000_000_000)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= 1e-5
    assert plan.check() == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("varc", [True, False])
def test_solve_multi_matches_single_solves(varc):
    """pat_solve_multi: three right-hand sides (a pair in two-field launches
    of the persistent engine, then one alone) give bit for bit the images of
    three pat_solve calls, and each is within the solve bound of the oracle's
    CG with the same data, alpha and s."""
    torch = need_gpu()
    w = synth.workload("vessels", n=128, nt=400, levels=4, iters=12) if varc else synth.workload("small", n=96,
                                                                                                   nt=200, order=8)
    plan, wave, wav = make_pair(w)
    assert plan.path == 1
    rng = np.random.default_rng(31)
    ys = [synth.add_noise(wave.forward(w.x_true), w.noise, rng) for _ in range(3)]
    alphas, ss = [3e-3, 1e-2, 2e-2], [1.0, 2.0, 1.5]
    iters = 8
    xs = plan.solve_multi(ys, alphas, ss, iters)
    assert plan.check() == 0
    for y, a, s, x in zip(ys, alphas, ss, xs):
        _, x1, _ = plan.solve(y, a, s, iters)
        assert torch.equal(x, x1)
        _, x_ref, _ = oracle.cg(wave, wav, y, a, s, iters)
        assert rel(x.cpu().numpy(), x_ref) <= TOL_X

