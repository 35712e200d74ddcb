"""Parity at the full workload sizes, in the engine configuration the
benchmark times (persistent engine for the 512 x 512 varying-medium case,
TMA plane-pipeline engine for the 256^3 volume).

  * 512 x 512, smooth random c in [1400, 1600], order 8, 1500 steps, 512
    sensors on a circle: K and K* against the oracle, then the full
    100-iteration solve (paper Sec. 5: a fixed iteration count) at the
    workload's worst conditioning (s = 2, alpha = 1e-3 relative) and at
    s = 1, alpha = 1e-2; alpha_abs = alpha_rel * lambda_max with lambda_max
    from the oracle, the same absolute number on both sides (accuracy bound
    per conditioning band, reading A14: see the test).
  * 1024 x 1024, constant c, order 8, 3000 steps, 256 sensors on a 180-degree
    arc: K, and K* of noisy data simulated from the phantom and of random data.
  * 256^3, constant c, order 4, 4096 sensors on a sphere, the full 800 steps:
    K of the phantom and K* of noisy data simulated from it.
  * 96^3 volume of the same recipe (order 4, 300 steps, 3D db4 with 3 levels):
    the 30-iteration CG solve against the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_OP, TOL_X = 1e-5, 1e-4


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


@pytest.fixture(scope="module")
def vessels():
    need_gpu()
    w = synth.workload("vessels")
    plan, wave, wav = make_pair(w)
    y_clean = wave.forward(w.x_true)
    y = synth.add_noise(y_clean, w.noise, np.random.default_rng(77))
    yield w, plan, wave, wav, y_clean, y
    plan.close()


def test_vessels_512_operators(vessels):
    w, plan, wave, wav, y_clean, y = vessels
    assert plan.path == 1  # persistent engine, as benchmarked
    assert rel(plan.forward(w.x_true).cpu().numpy(), y_clean) <= TOL_OP
    assert rel(plan.adjoint(y).cpu().numpy(), wave.adjoint(y)) <= TOL_OP


# Beyond this many CG steps past the fixed count, the oracle's iterate stands in for the minimiser:
# at s = 2, alpha_rel = 1e-3 the FP64 iterates after 100 / 150 / 200 steps are 1.4e-3 / 4.9e-5 / 2.1e-6
# from the converged solution.
EXTRA_ITERS = 50


@pytest.mark.parametrize("s,alpha_rel", [(2.0, 1e-3), (1.0, 1e-2)])
def test_vessels_512_solve_100_iterations(vessels, s, alpha_rel):
    """The workload's full 100 CG iterations against the oracle's, per
    reading A14 of the accuracy bound:
      * alpha_rel >= 1e-2: the final image within 1e-4 of the oracle's at the
        same iteration count;
      * alpha_rel < 1e-2 (s = 2): CG is far from converged after 100 steps
        and its iterate is sensitive to any rounding (FP64 oracle runs: FP32
        rounding of the CG vectors alone, exact operator, moves the
        100-step iterate by 2.9e-4; a random 1e-6 operator perturbation by
        2.8e-4; the GPU by the same).  There the GPU's 100-step image must be
        as accurate as the oracle's against the oracle's iterate 50 steps
        further on (within 10 % of the oracle's own distance), and within the
        band bound 1e-3 of the oracle's 100-step image.
    The FP64 CG scalars of the first 20 iterations are compared as well."""
    w, plan, wave, wav, _, y = vessels
    assert w.iters == 100
    alpha = alpha_rel * lambda_max(wave, wav, s)
    ill = alpha_rel < 1e-2
    _, x_far, log_ref, snaps = oracle.cg(wave, wav, y, alpha, s, w.iters + (EXTRA_ITERS if ill else 0),
                                         snapshots=(w.iters,))
    x_ref = snaps[w.iters]
    _, x, log = plan.solve(y, alpha, s, w.iters, want_log=True)
    assert plan.check() == 0
    xg = x.cpu().numpy()
    err = rel(xg, x_ref)
    print(f"512^2 s={s} alpha_rel={alpha_rel}: final image rel. error {err:.3e}")
    np.testing.assert_allclose(log.cpu().numpy()[:20], log_ref[:20], rtol=1e-3)
    if not ill:
        assert err <= TOL_X
        return
    e_gpu, e_ora = rel(xg, x_far), rel(x_ref, x_far)
    print(f"  against the oracle's {w.iters + EXTRA_ITERS}-step iterate: GPU {e_gpu:.4e}, oracle {e_ora:.4e}")
    assert abs(e_gpu - e_ora) <= 0.1 * e_ora
    assert err <= 1e-3


def test_arc_1024_operators():
    need_gpu()
    w = synth.workload("arc")
    plan, wave, _ = make_pair(w)
    y_ref = wave.forward(w.x_true)
    assert rel(plan.forward(w.x_true).cpu().numpy(), y_ref) <= TOL_OP
    y = synth.add_noise(y_ref, w.noise, np.random.default_rng(78))  # data simulated from the phantom
    assert rel(plan.adjoint(y).cpu().numpy(), wave.adjoint(y)) <= TOL_OP
    r = np.random.default_rng(2).standard_normal((w.ns, w.nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP
    plan.close()


def test_tree_256_cubed_800_steps():
    """The volume's full time axis: K of the phantom and K* of noisy data
    simulated from it (the adjoint's hardest case: the adjoint state carries
    the data's large time integral)."""
    need_gpu()
    w = synth.workload("tree3d")
    assert w.nt == 800 and w.shape == (256, 256, 256)
    plan, wave, wav = make_pair(w)
    y_clean = wave.forward(w.x_true)
    e_k = rel(plan.forward(w.x_true).cpu().numpy(), y_clean)
    y = synth.add_noise(y_clean, w.noise, np.random.default_rng(79))
    e_kt = rel(plan.adjoint(y).cpu().numpy(), wave.adjoint(y))
    print(f"256^3 / 800 steps: K {e_k:.3e}  K* (noisy phantom data) {e_kt:.3e}")
    assert e_k <= TOL_OP
    assert e_kt <= TOL_OP
    x = w.x_true
    assert rel(plan.EsT(x, 1.0).cpu().numpy(), wav.EsT(x, 1.0)) <= TOL_OP
    # the synthesis E_s at the full size too (E_s* above: z-marching levels 1-2, plane-parallel 3-4)
    u = np.random.default_rng(80).standard_normal(x.size)
    assert rel(plan.Es(u, 1.0).cpu().numpy(), wav.Es(u, 1.0)) <= TOL_OP
    plan.close()


def test_tree3d_solve_30_iterations():
    """3D CG solve (30 iterations, s = 1, alpha = 1e-2 relative) on a 96^3
    volume of the 3D workload's recipe, against the oracle's FP64 CG."""
    need_gpu()
    w = synth.workload("tree3d", n=96, nt=300, ns=1024, levels=3)
    plan, wave, wav = make_pair(w)
    y = synth.add_noise(wave.forward(w.x_true), w.noise, np.random.default_rng(80))
    s = w.s[0]
    alpha = w.alpha[0] * lambda_max(wave, wav, s, iters=10)
    _, x_ref, log_ref = oracle.cg(wave, wav, y, alpha, s, w.iters)
    _, x, log = plan.solve(y, alpha, s, w.iters, want_log=True)
    assert plan.check() == 0
    err = rel(x.cpu().numpy(), x_ref)
    print(f"96^3 3D solve, 30 iterations: final image rel. error {err:.3e}")
    assert err <= TOL_X
    np.testing.assert_allclose(log.cpu().numpy()[:10], log_ref[:10], rtol=1e-3)
    plan.close()
