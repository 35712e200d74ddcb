"""Seeded workload descriptions.

Each workload fixes grid, medium, time axis, stencil order, sensors, wavelet,
smoothness s, relative regularisation alpha, CG iterations, noise level and
the true initial pressure.  Time step: CFL 0.3, dt = 0.3 h / c_max; the grid
spacing is h = 0.1 mm.  Seeds: workload index + 1000 unless given.
"""
from dataclasses import dataclass, field
from math import ceil, sqrt

import numpy as np

from . import phantoms, sensors

H = 1.0e-4
CFL = 0.3


@dataclass
class Workload:
    name: str
    shape: tuple
    h: float
    c: object  # float (constant) or array of `shape`
    dt: float
    nt: int
    order: int
    sensors: np.ndarray
    family: int
    levels: int
    s: list
    alpha: list  # relative: alpha_abs = alpha * lambda_max(E_s* K* K E_s)
    iters: int
    noise: float
    x_true: np.ndarray
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def dim(self):
        return len(self.shape)

    @property
    def N(self):
        return int(np.prod(self.shape))

    @property
    def ns(self):
        return int(self.sensors.shape[0])

    @property
    def c_max(self):
        return float(np.max(self.c))

    def c_array(self):
        return np.ascontiguousarray(np.broadcast_to(np.asarray(self.c, dtype=np.float64), self.shape))


def add_noise(y, level, rng):
    """y + level * max|y| * xi, xi standard normal (noise relative to the
    maximum signal amplitude, as in the paper's data simulation)."""
    y = np.asarray(y, dtype=np.float64)
    return y + level * np.max(np.abs(y)) * rng.standard_normal(y.shape)


def _dt(h, cmax):
    return CFL * h / cmax


def small_2d(n=64, nt=250, order=2, family=2, levels=3, ns=32, seed=1000, varc=False, iters=50):
    """2D n x n grid, constant c = 1500 m/s (or a smooth random map), sensors on
    a full circle, 3 Gaussian blobs, 1% noise, s = 1, alpha = 1e-2."""
    rng = np.random.default_rng(seed)
    c = phantoms.speed_map((n, n), rng, sigma=max(n / 32.0, 1.0)) if varc else 1500.0
    x = phantoms.blobs((n, n), 3, rng)
    cmax = float(np.max(c))
    return Workload("2d-%d-o%d" % (n, order), (n, n), H, c, _dt(H, cmax), nt, order, sensors.circle(n, H, ns),
                    family, levels, [1.0], [1e-2], iters, 0.01, x, seed)


def vessels_2d(n=512, nt=1500, order=8, ns=512, levels=5, seed=1001, iters=100):
    """2D grid with a smooth random speed map in [1400, 1600] m/s (white noise
    Gaussian-filtered with sigma = n/32 px), sensors on a full circle, p0 = 4
    blobs + 6 Bezier vessels of width 1-3 px, 2% noise, db4,
    s in {1, 2} x alpha in {1e-3, 1e-2}."""
    rng = np.random.default_rng(seed)
    c = phantoms.speed_map((n, n), rng, sigma=n / 32.0)
    x = phantoms.blobs((n, n), 4, rng) + phantoms.vessels2d((n, n), 6, rng)
    return Workload("2d-%d-o%d-varc" % (n, order), (n, n), H, c, _dt(H, float(c.max())), nt, order,
                    sensors.circle(n, H, ns), 4, levels, [1.0, 2.0], [1e-3, 1e-2], iters, 0.02, x, seed)


def arc_2d(n=1024, nt=3000, order=8, ns=256, levels=6, seed=1002, iters=100):
    """Limited view: constant c, sensors on a 180-degree arc, db4, s = 1.5."""
    rng = np.random.default_rng(seed)
    x = phantoms.blobs((n, n), 4, rng) + phantoms.vessels2d((n, n), 6, rng)
    return Workload("2d-%d-o%d-arc" % (n, order), (n, n), H, 1500.0, _dt(H, 1500.0), nt, order,
                    sensors.arc(n, H, ns), 4, levels, [1.5], [1e-2], iters, 0.01, x, seed)


def limited_view(n=512, sides=1, ns=80, order=8, levels=5, seed=1005, iters=15, layer=10, refine=2):
    """The paper's experiment in synthetic form: n x n, c = 1500 m/s, an
    absorbing layer of `layer` cells, `ns` point sensors on one side (sides=1:
    a row `layer`+1 cells inside the top face) or split over two adjacent sides
    (sides=2: the top row and the left column), p0 = 4 blobs + 6 Bezier
    vessels, 2% noise, db4, s in {0, 0.5, 1, 1.5, 2}, 15 iterations, alpha
    1e-2 (relative).  Against the inverse crime the data are to be simulated
    on a grid `refine` times finer (spacing h/refine, time step dt/refine,
    the same sensor positions) and sampled at every `refine`-th time step;
    the fine-grid phantom is extra["x_fine"] and x_true is its refine x refine
    block mean.  nt covers the grid diagonal at CFL 0.3."""
    rng = np.random.default_rng(seed)
    nf = n * refine
    xf = phantoms.blobs((nf, nf), 4, rng, sigma=(2.0 * refine, 6.0 * refine)) + phantoms.vessels2d(
        (nf, nf), 6, rng, width=tuple(w * refine for w in (1, 2, 3)))
    x = xf.reshape(n, refine, n, refine).mean(axis=(1, 3))
    d = (layer + 1) * H
    lo, hi = (layer + 4) * H, (n - layer - 5) * H
    if sides == 1:
        pos = np.stack([np.linspace(lo, hi, ns), np.full(ns, d)], axis=1)
    else:
        a = ns // 2
        top = np.stack([np.linspace(lo, hi, a), np.full(a, d)], axis=1)
        left = np.stack([np.full(ns - a, d), np.linspace(lo, hi, ns - a)], axis=1)
        pos = np.concatenate([top, left])
    nt = int(ceil(sqrt(2.0) * n / CFL))
    w = Workload("2d-%d-o%d-limited%d" % (n, order, sides), (n, n), H, 1500.0, _dt(H, 1500.0), nt, order, pos, 4,
                 levels, [0.0, 0.5, 1.0, 1.5, 2.0], [1e-2], iters, 0.02, x, seed)
    w.extra.update(x_fine=xf, refine=refine, layer=layer, h_fine=H / refine, dt_fine=_dt(H, 1500.0) / refine,
                   nt_fine=refine * (nt - 1) + 1)
    return w


def tree_3d(n=256, nt=800, order=4, ns=4096, levels=4, seed=1004, iters=30):
    """3D grid, constant c, sensors on a Fibonacci sphere, p0 = vessel tree +
    5 blobs, 1% noise, 3D db4, s = 1, alpha = 1e-2."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    x = phantoms.vessel_tree3d(shape, rng, r_max=max(1.0, 4.0 * n / 256.0)) + phantoms.blobs(
        shape, 5, rng, sigma=(max(1.0, 2.0 * n / 256.0), max(1.5, 6.0 * n / 256.0)))
    return Workload("3d-%d-o%d" % (n, order), shape, H, 1500.0, _dt(H, 1500.0), nt, order,
                    sensors.fibonacci_sphere(n, H, ns), 4, levels, [1.0], [1e-2], iters, 0.01, x, seed)


def batched_workloads(count=64, seed=1003, sizes=(128, 192, 256, 384, 512), iters=50, levels=4, order=8):
    """Independent 2D reconstructions of uneven size: n from `sizes`, constant
    c, nt = ceil(sqrt(2) n / 0.3) (the grid diagonal at CFL 0.3), Ns in
    [64, 512] on a full circle or a 180-degree arc, alpha log-uniform in
    [1e-4, 1e-1], s in {1, 1.5, 2}, db4."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        ns = int(rng.integers(64, 513))
        lay = sensors.circle(n, H, ns) if rng.random() < 0.5 else sensors.arc(n, H, ns)
        nt = int(ceil(sqrt(2.0) * n / CFL))
        alpha = float(10.0 ** rng.uniform(-4.0, -1.0))
        s = float(rng.choice([1.0, 1.5, 2.0]))
        x = phantoms.blobs((n, n), 3, rng) + phantoms.vessels2d((n, n), 3, rng)
        out.append(Workload("batch-%d-%d" % (i, n), (n, n), H, 1500.0, _dt(H, 1500.0), nt, order, lay, 4,
                            levels, [s], [alpha], iters, 0.01, x, seed))
    return out


WORKLOADS = {
    "small": small_2d,
    "vessels": vessels_2d,
    "arc": arc_2d,
    "tree3d": tree_3d,
    "limited": limited_view,
}


def workload(name, **kw):
    return WORKLOADS[name](**kw)
