"""pat_EsT_noalloc: E_s* without any device allocation, for callers that
cannot allocate device memory (no plan can be created for them).

Collected last (file name) so that a run stopping at the first failure has
already run every other test.  It must pass alone in a fresh process and
after the other tests: it creates everything it needs itself.
"""
import numpy as np
import pytest

from gpu_helpers import need_gpu, rel

TOL_OP = 1e-5  # the per-operator bound used by the other parity tests


@pytest.mark.gpu
def test_noalloc_EsT_matches_plan_EsT_on_two_calls():
    """Two calls in a row on fresh inputs agree with the plan-based pat_EsT
    (the existing entry point) and with the FP64 oracle's E_s* (paper Sec. 4,
    Prop. 4.2) within the operator tolerance; the scratch the calls share
    keeps nothing that leaks from the first into the second."""
    torch = need_gpu()
    import oracle
    from paper_2507_02401_gb300 import Plan, _lib
    ny, nx = 256, 512
    family, levels, level_offset = 4, 5, 0
    plan = Plan((ny, nx), 1e-4, 2e-8, 2, 2, 1500.0, np.array([[1e-3, 1e-3]]), family, levels, level_offset)
    wav = oracle.Wavelet((ny, nx), family, levels, level_offset)
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(2024)
    for call, s in enumerate((1.0, 2.0)):
        x = torch.randn((ny, nx), device="cuda", generator=g) * (call + 1)
        u_ref = plan.EsT(x, s)
        u = torch.full((ny * nx,), float("nan"), device="cuda")
        _lib.pat_EsT_noalloc(nx, ny, family, levels, level_offset, s, x, u, stream)
        torch.cuda.synchronize()
        assert torch.isfinite(u).all()
        got = u.cpu().numpy()
        assert rel(got, u_ref.cpu().numpy()) <= TOL_OP
        assert rel(got, wav.EsT(x.cpu().numpy().astype(np.float64), s)) <= TOL_OP
    plan.close()


@pytest.mark.gpu
def test_noalloc_rejects_grids_above_its_limit():
    torch = need_gpu()
    from paper_2507_02401_gb300 import _lib
    x = torch.zeros(8, device="cuda")
    with pytest.raises(_lib.PatError) as e:
        _lib.pat_EsT_noalloc(2048, 1024, 4, 3, 0, 1.0, x.data_ptr(), x.data_ptr() + 4096, None)
    assert e.value.status == _lib.PAT_ERR_INVALID
    assert "2^20" in _lib.pat_last_error() or "1048576" in _lib.pat_last_error()


@pytest.mark.gpu
def test_noalloc_rejects_bad_arrays_on_the_host():
    """Undersized or wrongly typed tensors are refused before any launch, and
    overlapping input and output arrays are refused by the library."""
    torch = need_gpu()
    from paper_2507_02401_gb300 import _lib
    ny, nx = 64, 64
    x = torch.zeros((ny, nx), device="cuda")
    with pytest.raises(ValueError):
        _lib.pat_EsT_noalloc(nx, ny, 2, 2, 0, 1.0, x, torch.zeros(nx * ny - 1, device="cuda"))
    with pytest.raises(ValueError):
        _lib.pat_EsT_noalloc(nx, ny, 2, 2, 0, 1.0, x.half(), torch.zeros(nx * ny, device="cuda"))
    with pytest.raises(_lib.PatError) as e:
        _lib.pat_EsT_noalloc(nx, ny, 2, 2, 0, 1.0, x, x)
    assert e.value.status == _lib.PAT_ERR_INVALID
    assert "overlap" in _lib.pat_last_error()
