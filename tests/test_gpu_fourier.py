"""Fourier-form prior on the GPU (pat_plan_set_prior kind 1, hand-written
radix-2 FFTs) against the oracle's numpy-FFT filter: E_s / E_s* (relative L2
<= 1e-5) over shapes, s and length units; the Ornstein-Uhlenbeck kernel of
the paper's worked case; a CG reconstruction with this prior (<= 1e-4); and
the shapes it refuses."""
import numpy as np
import pytest

import oracle
from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu


def fourier_plan(shape, lc, nt=30, order=4, seed=0):
    w = custom(shape, nt, order, False, 4, seed=seed, family=2, levels=0)
    plan, wave, _ = make_pair(w)
    plan.set_prior(1, lc)
    return w, plan, wave, oracle.FourierPrior(shape, lc)


@pytest.mark.parametrize("shape,lc", [((64, 128), 1.0), ((256, 256), 8.0), ((512, 64), 3.5), ((16, 16), 2.0)])
@pytest.mark.parametrize("s", [0.0, 1.0, 1.5, 2.5])
def test_fourier_Es_parity(shape, lc, s):
    need_gpu()
    w, plan, _, fp = fourier_plan(shape, lc)
    u = np.random.default_rng(1).standard_normal(shape)
    assert rel(plan.Es(u.ravel(), s).cpu().numpy(), fp.Es(u, s)) <= 1e-5
    assert rel(plan.EsT(u, s).cpu().numpy(), fp.EsT(u, s)) <= 1e-5


def test_fourier_ornstein_uhlenbeck_kernel_on_gpu():
    need_gpu()
    n, lc = 256, 16.0
    w, plan, _, _ = fourier_plan((n, n), lc)
    delta = np.zeros((n, n), dtype=np.float32)
    delta[0, 0] = 1.0
    g = plan.Es(plan.EsT(delta, 1.5), 1.5).cpu().numpy().astype(np.float64) * lc ** 2
    j = np.arange(n)
    d = np.minimum(j, n - j) / lc
    r = np.sqrt(d[:, None] ** 2 + d[None, :] ** 2)
    ref = np.exp(-r) / (2 * np.pi)
    m = (r >= 0.5) & (r <= 3.0)
    assert np.max(np.abs(g[m] - ref[m]) / ref[m]) < 2e-3


def test_fourier_prior_cg_solve():
    need_gpu()
    import synth
    w = custom((64, 64), 200, 8, True, 24, seed=3, family=2, levels=0)
    plan, wave, _ = make_pair(w)
    plan.set_prior(1, 4.0)
    fp = oracle.FourierPrior(w.shape, 4.0)
    y = synth.add_noise(wave.forward(w.x_true), 0.01, np.random.default_rng(2))
    alpha = 1e-2 * float(np.sum(wave.adjoint(y) ** 2)) / float(np.sum(y ** 2))
    _, x, _ = plan.solve(y, alpha, 1.5, 12)
    _, x_ref, _ = oracle.cg(wave, fp, y, alpha, 1.5, 12)
    assert rel(x.cpu().numpy(), x_ref) <= 1e-4


def test_fourier_prior_refusals():
    need_gpu()
    from paper_2507_02401_gb300 import _lib
    w = custom((48, 64), 20, 2, False, 3, seed=4, family=2, levels=0)
    p, _, _ = make_pair(w)
    with pytest.raises(_lib.PatError):
        p.set_prior(1, 1.0)  # 48 is not a power of two
    w3 = custom((16, 16, 16), 20, 2, False, 3, seed=5, family=2, levels=0)
    p3, _, _ = make_pair(w3)
    with pytest.raises(_lib.PatError):
        p3.set_prior(1, 1.0)  # 3D
    w2 = custom((64, 64), 20, 2, False, 3, seed=6, family=2, levels=0)
    p2, _, _ = make_pair(w2)
    with pytest.raises(_lib.PatError):
        p2.set_prior(1, 0.0)
    p2.set_prior(1, 2.0)
    p2.set_prior(0)  # back to the wavelet form (levels 0: identity)
    u = np.random.default_rng(0).standard_normal(w2.N).astype(np.float32)
    assert np.array_equal(p2.Es(u, 1.0).cpu().numpy().ravel(), u)
