"""3D constant-medium wave steps through the TMA plane-pipeline kernel.

Parity with the FP64 oracle (relative L2 <= 1e-5 per operator) on volumes
that span several 64 x 16 column tiles and z chunks with ragged edges in all
three directions, every stencil order, the short time axes, a field address
the kernel cannot take (it falls back per step), agreement with the plain
per-step kernel, and the medium gradient."""
import numpy as np
import pytest

from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5

CASES = [
    # shape (nz, ny, nx), nt, order, ns
    ((40, 37, 132), 60, 4, 20),   # 3 x 3 tiles, ragged x/y, ragged z chunk
    ((24, 20, 68), 40, 8, 9),
    ((18, 33, 64), 50, 2, 7),
    ((35, 16, 8), 30, 6, 5),      # narrower than one tile
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"-o{c[2]}")
def test_tma_forward_adjoint_parity(case):
    need_gpu()
    shape, nt, order, ns = case
    w = custom(shape, nt, order, False, ns, seed=sum(shape) + order)
    plan, wave, _ = make_pair(w)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    r = np.random.default_rng(7).standard_normal((w.ns, w.nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP
    assert plan.check() == 0


@pytest.mark.parametrize("nt", [1, 2, 3, 4])
def test_tma_short_time_axis(nt):
    need_gpu()
    w = custom((20, 24, 36), nt, 8, False, 6, seed=nt)
    plan, wave, _ = make_pair(w)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    r = np.random.default_rng(nt).standard_normal((w.ns, nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP


def test_tma_matches_plain_kernel(monkeypatch):
    need_gpu()
    w = custom((48, 40, 96), 120, 4, False, 30, seed=5)
    a, _, _ = make_pair(w)
    monkeypatch.setenv("PAT_STEP3D", "plain")
    b, _, _ = make_pair(w)
    monkeypatch.delenv("PAT_STEP3D")
    assert rel(a.forward(w.x_true).cpu().numpy(), b.forward(w.x_true).cpu().numpy()) <= 2e-6
    r = np.random.default_rng(1).standard_normal((w.ns, w.nt))
    assert rel(a.adjoint(r).cpu().numpy(), b.adjoint(r).cpu().numpy()) <= 2e-6


def test_unaligned_field_falls_back():
    torch = need_gpu()
    w = custom((20, 18, 40), 40, 4, False, 8, seed=3)
    plan, wave, _ = make_pair(w)
    buf = torch.zeros(w.x_true.size + 1, device="cuda", dtype=torch.float32)
    x = buf[1:].view(w.shape)  # 4-byte offset: not a 16-byte aligned field
    x.copy_(torch.as_tensor(w.x_true, dtype=torch.float32))
    assert x.data_ptr() % 16 != 0
    assert rel(plan.forward(x).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP


def test_tma_grad_kappa():
    need_gpu()
    w = custom((20, 24, 36), 60, 4, False, 9, seed=8)
    plan, wave, _ = make_pair(w)
    r = np.random.default_rng(2).standard_normal((w.ns, w.nt))
    assert rel(plan.grad_kappa(w.x_true, r).cpu().numpy(), wave.kappa_grad(w.x_true, r)) <= 1e-5
