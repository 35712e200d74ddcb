"""Shared helpers of the GPU parity tests: build matching CUDA plans and
oracle objects from one seeded workload description."""
import numpy as np
import pytest

import synth


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    return torch


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_pair(w, path=None, level_offset=0):
    """(cuda Plan, oracle Wave, oracle Wavelet) for a synth.Workload."""
    import oracle
    from paper_2507_02401_gb300 import Plan
    c = w.c if np.ndim(w.c) == 0 else w.c_array()
    plan = Plan(w.shape, w.h, w.dt, w.nt, w.order, c, w.sensors, w.family, w.levels, level_offset)
    if path is not None:
        plan.path = path
    wave = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, w.c_array(), w.sensors)
    wav = oracle.Wavelet(w.shape, w.family, w.levels, level_offset)
    return plan, wave, wav


def custom(shape, nt, order, varc, ns, seed, family=2, levels=0, layout="random"):
    """Small seeded workload of arbitrary (possibly ragged) shape."""
    rng = np.random.default_rng(seed)
    h = 1e-4
    c = synth.speed_map(shape, rng, sigma=3.0) if varc else 1500.0
    cmax = float(np.max(c))
    dt = 0.3 * h / cmax
    d = len(shape)
    if layout == "random":
        sens = np.stack([rng.uniform(0, (s - 1) * h, ns) for s in shape[::-1]], axis=1)
    else:
        sens = synth.circle(min(shape), h, ns) if d == 2 else synth.fibonacci_sphere(min(shape), h, ns)
    x = synth.blobs(shape, 3, rng, sigma=(1.5, 3.0))
    return synth.Workload("custom", tuple(shape), h, c, dt, nt, order, sens, family, levels, [1.0], [1e-2], 10,
                          0.01, x, seed)
