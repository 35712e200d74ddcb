"""Limited-view workload end to end on the GPU at a size the oracle finishes
in seconds (64 x 64, 80 sensors on one side or two adjacent sides, absorbing
layer, data simulated by the oracle on the twice-finer grid): GMRES (the
paper's solver) and CG against the oracle's (relative L2 <= 1e-4), and the
reconstruction approaching the phantom."""
import numpy as np
import pytest

import oracle
from oracle import krylov
import synth
from gpu_helpers import need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sides", [1, 2])
def test_limited_view_gmres_and_cg(sides):
    need_gpu()
    from paper_2507_02401_gb300 import Plan
    w = synth.workload("limited", n=64, sides=sides, levels=3)
    ex = w.extra
    smax = oracle.sponge_sigma_max(1500.0, ex["layer"], w.h)
    fine = oracle.Wave((128, 128), ex["h_fine"], ex["dt_fine"], ex["nt_fine"], w.order, 1500.0, w.sensors,
                       sigma=oracle.sponge_sigma((128, 128), 2 * ex["layer"], smax))
    y = synth.add_noise(fine.forward(ex["x_fine"])[:, ::2], w.noise, np.random.default_rng(3))
    wave = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, 1500.0, w.sensors,
                       sigma=oracle.sponge_sigma(w.shape, ex["layer"], smax))
    wav = oracle.Wavelet(w.shape, w.family, w.levels)
    plan = Plan(w.shape, w.h, w.dt, w.nt, w.order, 1500.0, w.sensors, w.family, w.levels)
    plan.set_sponge(ex["layer"], smax)
    alpha = 1e-2 * float(np.sum(wave.adjoint(y) ** 2)) / float(np.sum(y ** 2))
    s = 1.0
    x, res, J = plan.solve_gmres(y, alpha, s, 10, want_log=True)
    x_ref, res_ref, J_ref = krylov.gmres(wave, wav, y, alpha, s, 10)
    assert rel(x.cpu().numpy(), x_ref) <= 1e-4
    assert rel(J, J_ref) <= 1e-4
    _, xc, _ = plan.solve(y, alpha, s, 10)
    _, xc_ref, _ = oracle.cg(wave, wav, y, alpha, s, 10)
    assert rel(xc.cpu().numpy(), xc_ref) <= 1e-4
    err = np.linalg.norm(x.cpu().numpy() - w.x_true) / np.linalg.norm(w.x_true)
    assert err < 0.9
