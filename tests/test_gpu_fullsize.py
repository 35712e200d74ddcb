"""Parity at the full workload sizes, in the engine configuration the
benchmark times (persistent engine for the 512 x 512 varying-medium case).

  * 512 x 512, smooth random c in [1400, 1600], order 8, 1500 steps, 512
    sensors on a circle: K and K* against the oracle, then a 10-iteration
    solve (the full 100 iterations would cost the oracle ~200 wave solves).
  * 1024 x 1024, constant c, order 8, 3000 steps, 256 sensors on a 180-degree
    arc: K, and K* of noisy data simulated from the phantom and of random data.
  * 256^3, constant c, order 4, 4096 sensors on a sphere: K and K* over the
    first 60 steps (the per-step launch configuration is the one the 800-step
    run uses).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu


def test_vessels_512_operators_and_solve():
    need_gpu()
    w = synth.workload("vessels")
    plan, wave, wav = make_pair(w)
    assert plan.path == 1  # persistent engine, as benchmarked
    y_clean_ref = wave.forward(w.x_true)
    assert rel(plan.forward(w.x_true).cpu().numpy(), y_clean_ref) <= 1e-5
    y = synth.add_noise(y_clean_ref, w.noise, np.random.default_rng(77))
    assert rel(plan.adjoint(y).cpu().numpy(), wave.adjoint(y)) <= 1e-5
    alpha = 1.0e-3  # absolute; identical for both sides
    s = 1.0
    _, x_ref, _ = oracle.cg(wave, wav, y, alpha, s, 10)
    _, x, _ = plan.solve(y, alpha, s, 10)
    assert plan.check() == 0
    assert rel(x.cpu().numpy(), x_ref) <= 1e-4


def test_arc_1024_operators():
    need_gpu()
    w = synth.workload("arc")
    plan, wave, _ = make_pair(w)
    y_ref = wave.forward(w.x_true)
    assert rel(plan.forward(w.x_true).cpu().numpy(), y_ref) <= 1e-5
    y = synth.add_noise(y_ref, w.noise, np.random.default_rng(78))  # data simulated from the phantom
    assert rel(plan.adjoint(y).cpu().numpy(), wave.adjoint(y)) <= 1e-5
    r = np.random.default_rng(2).standard_normal((w.ns, w.nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= 1e-5


def test_tree_256_cubed_operators():
    need_gpu()
    w = synth.workload("tree3d", nt=60)
    plan, wave, wav = make_pair(w)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= 1e-5
    r = np.random.default_rng(3).standard_normal((w.ns, w.nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= 1e-5
    x = w.x_true
    assert rel(plan.EsT(x, 1.0).cpu().numpy(), wav.EsT(x, 1.0)) <= 1e-5
