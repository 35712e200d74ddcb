"""GPU parity of the C-ABI operators against the FP64 oracle.

Tolerance: relative L2 error <= 1e-5 per operator application (K, K*, E_s,
E_s*), the bound the reconstruction path is held to; FP32 fields against an
FP64 oracle.  Sizes span several 64 x 32 tiles and ragged tile edges."""
import numpy as np
import pytest

from gpu_helpers import custom, make_pair, need_gpu, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5

WAVE_CASES = [
    # shape, nt, order, varc, ns
    ((64, 64), 250, 2, False, 32),
    ((90, 70), 120, 8, True, 17),     # ragged in both tile directions
    ((33, 130), 60, 4, True, 9),
    ((128, 96), 200, 6, False, 40),
    ((20, 18, 22), 60, 4, False, 12),  # 3D
    ((17, 24, 35), 40, 8, True, 7),
    ((16, 16, 16), 30, 2, True, 5),
]


@pytest.mark.parametrize("case", WAVE_CASES, ids=lambda c: "x".join(map(str, c[0])) + f"-o{c[2]}")
@pytest.mark.parametrize("path", [1, 2], ids=["persistent", "step"])
def test_forward_adjoint_parity(case, path):
    torch = need_gpu()
    shape, nt, order, varc, ns = case
    if path == 1 and len(shape) == 3:
        pytest.skip("persistent engine is 2D only")
    w = custom(shape, nt, order, varc, ns, seed=hash(case) % 1000)
    plan, wave, _ = make_pair(w, path=path)
    rng = np.random.default_rng(5)
    y_ref = wave.forward(w.x_true)
    y = plan.forward(w.x_true).cpu().numpy()
    assert rel(y, y_ref) <= TOL_OP
    r = rng.standard_normal((w.ns, w.nt))
    x_ref = wave.adjoint(r)
    x = plan.adjoint(r).cpu().numpy()
    assert rel(x, x_ref) <= TOL_OP
    assert plan.check() == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("nt", [1, 2, 3, 5])
@pytest.mark.parametrize("path", [1, 2], ids=["persistent", "step"])
def test_short_time_axis(nt, path):
    need_gpu()
    w = custom((40, 72), nt, 8, True, 6, seed=nt)
    plan, wave, _ = make_pair(w, path=path)
    assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
    r = np.random.default_rng(nt).standard_normal((w.ns, nt))
    assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP


@pytest.mark.parametrize("path", [1, 2], ids=["persistent", "step"])
def test_gpu_dot_product(path):
    need_gpu()
    w = custom((96, 128), 300, 8, True, 24, seed=11)
    plan, _, _ = make_pair(w, path=path)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(w.shape)
    y = rng.standard_normal((w.ns, w.nt))
    Kx = plan.forward(x).double().cpu().numpy()
    Ky = plan.adjoint(y).double().cpu().numpy()
    lhs, rhs = float(np.sum(Kx * y)), float(np.sum(x * Ky))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Kx) * np.linalg.norm(y)


def test_engines_agree():
    need_gpu()
    w = custom((128, 128), 400, 8, True, 50, seed=21)
    a, _, _ = make_pair(w, path=1)
    b, _, _ = make_pair(w, path=2)
    ya, yb = a.forward(w.x_true).cpu().numpy(), b.forward(w.x_true).cpu().numpy()
    assert rel(ya, yb) <= 2e-6


def test_sensors_on_cells_and_edges():
    need_gpu()
    shape = (64, 64)
    w = custom(shape, 80, 4, False, 4, seed=2)
    h = w.h
    w.sensors = np.array([[0.0, 0.0], [63 * h, 63 * h], [10 * h, 20 * h], [63 * h, 0.0], [31.5 * h, 7.25 * h]])
    for path in (1, 2):
        plan, wave, _ = make_pair(w, path=path)
        assert rel(plan.forward(w.x_true).cpu().numpy(), wave.forward(w.x_true)) <= TOL_OP
        r = np.random.default_rng(1).standard_normal((5, 80))
        assert rel(plan.adjoint(r).cpu().numpy(), wave.adjoint(r)) <= TOL_OP


# Shapes are (ny, nx) / (nz, ny, nx).  Levels of width nx % 8 == 0 take the HBM-rate kernels (2D fused
# level, 3D fused level with z-marching); narrower levels the generic ones: the cases mix both, with
# ragged CTA blocks (coefficient widths not multiples of the 64 x 16 / 32 x 8 blocks), several CTAs per
# axis and per z chunk, coarse levels shorter than the filter halo (periodic wrap repeated), and 3D
# levels with many columns and few planes (a CTA's share of the work spans several columns).  3D levels
# whose (column, output plane) items fit in one wave take the plane-parallel kernel, larger ones the
# z-marching kernel (the last three cases, the last with ragged column blocks).
WAVELET_CASES = [((64, 64), 1, 3), ((64, 64), 2, 3), ((128, 64), 4, 5), ((16, 16), 4, 4), ((32, 32, 32), 4, 3),
                 ((16, 8, 8), 2, 2), ((512, 512), 4, 5), ((72, 1032), 4, 3), ((264, 136), 2, 3), ((16, 64), 4, 3),
                 ((8, 256), 4, 3), ((24, 40, 48), 4, 2), ((32, 24, 136), 4, 2), ((64, 64, 64), 4, 4),
                 ((16, 16, 72), 1, 3), ((8, 512, 1024), 4, 2), ((32, 256, 1024), 4, 2), ((16, 328, 1032), 4, 2)]


@pytest.mark.parametrize("shape,family,levels", WAVELET_CASES)
@pytest.mark.parametrize("s", [0.0, 1.0, 1.5])
def test_Es_EsT_parity(shape, family, levels, s):
    need_gpu()
    w = custom(shape, 2, 2, False, 1, seed=4, family=family, levels=levels)
    plan, _, wav = make_pair(w, level_offset=1 if s == 1.5 else 0)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(shape)
    assert rel(plan.EsT(x, s).cpu().numpy(), wav.EsT(x, s)) <= TOL_OP
    u = rng.standard_normal(x.size)
    assert rel(plan.Es(u, s).cpu().numpy(), wav.Es(u, s)) <= TOL_OP


def test_host_pointer_path_matches_device():
    torch = need_gpu()
    from paper_2507_02401_gb300 import _lib
    w = custom((64, 96), 100, 8, True, 10, seed=9, family=4, levels=2)
    plan, _, _ = make_pair(w)
    x = w.x_true.astype(np.float32)
    y_dev = plan.forward(x).cpu().numpy()
    y_host = np.zeros((w.ns, w.nt), np.float32)
    _lib.pat_forward(plan.handle, x, y_host, None)
    np.testing.assert_array_equal(y_host, y_dev)
    u_host = np.zeros(x.size, np.float32)
    _lib.pat_EsT(plan.handle, 1.0, x, u_host, None)
    np.testing.assert_array_equal(u_host, plan.EsT(x, 1.0).cpu().numpy())
    torch.cuda.synchronize()


def test_deterministic():
    need_gpu()
    w = custom((96, 96), 150, 8, True, 20, seed=13, family=4, levels=2)
    plan, _, _ = make_pair(w)
    y = plan.forward(w.x_true).cpu().numpy()
    u1, x1, _ = plan.solve(y, 1e-3, 1.0, 5)
    u2, x2, _ = plan.solve(y, 1e-3, 1.0, 5)
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    assert np.array_equal(plan.forward(w.x_true).cpu().numpy(), y)


def test_validation_errors():
    need_gpu()
    from paper_2507_02401_gb300 import Plan, PatError, _lib
    h = 1e-4
    sens = np.array([[1e-3, 1e-3]])
    with pytest.raises(PatError) as e:
        Plan((64, 64), h, 0.8 * h / 1500, 10, 2, 1500.0, sens, 2, 2)  # CFL 0.8 > 0.707
    assert e.value.status == _lib.PAT_ERR_CFL
    with pytest.raises(PatError) as e:
        Plan((64, 64), h, 0.3 * h / 1500, 10, 2, 1500.0, np.array([[7e-3, 1e-3]]), 2, 2)
    assert e.value.status == _lib.PAT_ERR_INVALID
    with pytest.raises(PatError) as e:
        Plan((60, 64), h, 0.3 * h / 1500, 10, 2, 1500.0, sens, 2, 3)  # 60 % 8 != 0
    assert e.value.status == _lib.PAT_ERR_INVALID
    with pytest.raises(PatError) as e:
        Plan((64, 64), h, 0.3 * h / 1500, 10, 3, 1500.0, sens, 2, 2)
    assert e.value.status == _lib.PAT_ERR_INVALID
    c = np.full((64, 64), 1500.0)
    c[3, 4] = np.nan
    with pytest.raises(PatError) as e:
        Plan((64, 64), h, 0.3 * h / 1500, 10, 2, c, sens, 2, 2)
    assert e.value.status == _lib.PAT_ERR_INVALID
