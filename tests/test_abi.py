"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/pat.h declares; the Python binding mirrors those names;
plan validation (host logic) rejects bad problems before touching the GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pat.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pat_[a-zA-Z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_02401_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2507_02401_gb300 import build
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_binding_mirrors_header():
    from paper_2507_02401_gb300 import _lib
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(_lib, n)), n


def test_last_error_without_gpu(lib):
    from paper_2507_02401_gb300 import _lib
    assert isinstance(_lib.pat_last_error(), str)


def _plan_args(dt_cfl=0.3, sensors=None, n=(64, 64), order=2, levels=2, c=None, nt=10, family=2):
    from paper_2507_02401_gb300 import _lib
    grid = _lib.pat_grid()
    grid.dim = 2
    grid.n[0], grid.n[1], grid.n[2] = n[1], n[0], 1
    grid.h = 1e-4
    wav = _lib.pat_wavelet()
    wav.family, wav.levels, wav.level_offset = family, levels, 0
    sens = np.array([[1e-3, 2e-3]]) if sensors is None else sensors
    return grid, c, 1500.0, sens, len(sens), dt_cfl * 1e-4 / 1500.0, nt, order, wav


@pytest.mark.parametrize("kw,status", [
    (dict(dt_cfl=0.75, order=2), 2),            # CFL above 1/sqrt(2)
    (dict(dt_cfl=0.56, order=8), 2),            # above 1/(sqrt 2 * 1.2863) = 0.5497
    (dict(sensors=np.array([[7e-3, 1e-3]])), 1),  # outside the grid
    (dict(sensors=np.array([[-1e-9, 1e-3]])), 1),
    (dict(order=5), 1),
    (dict(levels=7), 1),                         # 64 % 128 != 0
    (dict(family=3), 1),
    (dict(nt=0), 1),
    (dict(c=np.full((64, 64), np.nan)), 1),
])
def test_validation_rejects_before_gpu_work(lib, kw, status):
    from paper_2507_02401_gb300 import _lib
    with pytest.raises(_lib.PatError) as e:
        _lib.pat_plan_create(*_plan_args(**kw))
    assert e.value.status == status
    assert len(_lib.pat_last_error()) > 0


def test_cfl_limit_boundary(lib):
    """The stated limits: 1/sqrt(2) (2D order 2), 1/(sqrt(3)*(9/8+1/24)) (3D
    order 4) -- a plan just above is rejected with PAT_ERR_CFL."""
    from paper_2507_02401_gb300 import _lib
    with pytest.raises(_lib.PatError) as e:
        _lib.pat_plan_create(*_plan_args(dt_cfl=0.7072, order=2))
    assert e.value.status == _lib.PAT_ERR_CFL
