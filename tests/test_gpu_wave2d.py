"""2D per-step engine through the TMA tile-pipeline kernel.

Parity with the FP64 oracle (relative L2 <= 1e-5 per operator) on grids that
span several 64 x 64 tiles with ragged edges, every stencil order, constant
and varying media, short time axes, a field address the kernel cannot take
(the forward falls back per step, the adjoint stages its output), agreement
with the plain per-step kernel, the medium gradient, and the full-size
512 x 512 order-8 forward map and adjoint (varying and constant medium; the
adjoint with noisy data simulated from the phantom, the case that needs the
compensated adjoint state, and with random data)."""
import numpy as np
import pytest

import synth
from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5

CASES = [
    # shape (ny, nx), nt, order, varc, ns
    ((70, 132), 150, 8, False, 20),   # 3 x 2 tiles, ragged in x and y
    ((200, 196), 120, 2, False, 31),
    ((130, 68), 100, 4, True, 12),
    ((64, 256), 90, 6, True, 9),
    ((16, 8), 40, 8, False, 3),       # narrower than one tile
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"-o{c[2]}" + ("v" if c[3] else ""))
def test_tma2d_forward_adjoint_parity(case):
    need_gpu()
    shape, nt, order, varc, ns = case
    w = custom(shape, nt, order, varc, ns, seed=sum(shape) + order)
    plan, wave, _ = make_pair(w, path=2)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    r = np.random.default_rng(7).standard_normal((w.ns, w.nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP
    assert plan.check() == 0


@pytest.mark.parametrize("nt", [1, 2, 3, 4])
@pytest.mark.parametrize("varc", [False, True])
def test_tma2d_short_time_axis(nt, varc):
    need_gpu()
    w = custom((72, 136), nt, 8, varc, 6, seed=nt)
    plan, wave, _ = make_pair(w, path=2)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    r = np.random.default_rng(nt).standard_normal((w.ns, nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP


@pytest.mark.parametrize("varc", [False, True])
def test_tma2d_matches_plain_kernel(monkeypatch, varc):
    need_gpu()
    w = custom((192, 256), 300, 8, varc, 40, seed=5)
    a, _, _ = make_pair(w, path=2)
    monkeypatch.setenv("PAT_STEP2D", "plain")
    b, _, _ = make_pair(w, path=2)
    monkeypatch.delenv("PAT_STEP2D")
    assert rel(a.forward(w.x_true).cpu().numpy(), b.forward(w.x_true).cpu().numpy()) <= 2e-6
    r = np.random.default_rng(1).standard_normal((w.ns, w.nt))
    # both adjoints are compensated (the TMA kernel in Z = kappa Q, the plain kernel in Q)
    assert rel(a.adjoint(r).cpu().numpy(), b.adjoint(r).cpu().numpy()) <= 2e-6


def test_tma2d_unaligned_field_falls_back():
    torch = need_gpu()
    w = custom((96, 128), 80, 4, False, 8, seed=3)
    plan, wave, _ = make_pair(w, path=2)
    buf = torch.zeros(w.x_true.size + 1, device="cuda", dtype=torch.float32)
    x = buf[1:].view(w.shape)  # 4-byte offset: not a 16-byte aligned field
    x.copy_(torch.as_tensor(w.x_true, dtype=torch.float32))
    assert x.data_ptr() % 16 != 0
    assert rel(plan.forward(x).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    r = np.random.default_rng(3).standard_normal((w.ns, w.nt))
    out = buf[1:].view(w.shape)
    plan.adjoint(r, out=out)
    assert rel(out.cpu().numpy(), wave.adjoint(r)) <= TOL_OP


@pytest.mark.parametrize("varc", [False, True])
def test_tma2d_grad_kappa(varc):
    need_gpu()
    w = custom((72, 136), 120, 8, varc, 9, seed=8)
    plan, wave, _ = make_pair(w, path=2)
    r = np.random.default_rng(2).standard_normal((w.ns, w.nt))
    assert rel(plan.grad_kappa(w.x_true, r).cpu().numpy(), wave.kappa_grad(w.x_true, r)) <= 1e-5


def test_tma2d_vessels_512_forward_full_size():
    """512 x 512, order 8, varying c, 1500 steps, 512 sensors through the
    per-step engine (the default engine there is the persistent one)."""
    need_gpu()
    w = synth.workload("vessels")
    plan, wave, _ = make_pair(w, path=2)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP


@pytest.mark.parametrize("medium", ["varying", "constant"])
def test_tma2d_vessels_512_adjoint_full_size(medium):
    """The adjoint through the TMA kernel (Z = kappa Q as a compensated pair) at the full
    512 x 512, order 8, 1500-step workload: noisy data simulated from the phantom (an
    uncompensated FP32 adjoint reaches ~2e-5 there, in FP32 emulation) and random data."""
    need_gpu()
    w = synth.workload("vessels")
    if medium == "constant":
        w.c = 1500.0
    plan, wave, _ = make_pair(w, path=2)
    y = synth.add_noise(wave.forward(w.x_true), w.noise, np.random.default_rng(77))
    assert rel(plan.adjoint(y).cpu().numpy(), wave.adjoint(y)) <= TOL_OP
    r = np.random.default_rng(2).standard_normal((w.ns, w.nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP
