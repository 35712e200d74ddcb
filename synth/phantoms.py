"""Seeded initial-pressure phantoms and speed-of-sound maps.

All coordinates are in pixels/voxels of the array (x = last axis).
"""
import numpy as np
from scipy.ndimage import gaussian_filter


def _grid(shape):
    return np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")


def blobs(shape, count, rng, amp=(0.5, 1.0), sigma=(2.0, 6.0), radius_frac=0.3):
    """Sum of `count` isotropic Gaussian blobs, amplitude U[amp], width U[sigma]
    pixels, centres uniform in the disk/ball of radius radius_frac*n around the
    grid centre."""
    shape = tuple(shape)
    d = len(shape)
    n = min(shape)
    centre = np.array([(s - 1) / 2.0 for s in shape])
    coords = _grid(shape)
    out = np.zeros(shape)
    for _ in range(count):
        while True:  # rejection sample a point of the unit ball
            v = rng.uniform(-1.0, 1.0, d)
            if v @ v <= 1.0:
                break
        c = centre + radius_frac * n * v
        a = rng.uniform(*amp)
        sg = rng.uniform(*sigma)
        r2 = sum((coords[k] - c[k]) ** 2 for k in range(d))
        out += a * np.exp(-r2 / (2.0 * sg * sg))
    return out


def _tube(out, p0, p1, radius, amp):
    """Max-composite a straight tube of given radius (pixels) between p0 and p1
    (array-order coordinates); linear 1-pixel soft edge."""
    shape = out.shape
    d = len(shape)
    lo = np.maximum(np.floor(np.minimum(p0, p1) - radius - 2).astype(int), 0)
    hi = np.minimum(np.ceil(np.maximum(p0, p1) + radius + 2).astype(int) + 1, np.array(shape))
    if np.any(hi <= lo):
        return
    sl = tuple(slice(lo[k], hi[k]) for k in range(d))
    coords = np.meshgrid(*[np.arange(lo[k], hi[k], dtype=np.float64) for k in range(d)], indexing="ij")
    seg = p1 - p0
    L2 = float(seg @ seg)
    t = sum((coords[k] - p0[k]) * seg[k] for k in range(d)) / max(L2, 1e-12)
    t = np.clip(t, 0.0, 1.0)
    dist2 = sum((coords[k] - (p0[k] + t * seg[k])) ** 2 for k in range(d))
    val = amp * np.clip(radius + 0.5 - np.sqrt(dist2), 0.0, 1.0)
    out[sl] = np.maximum(out[sl], val)


def vessels2d(shape, count, rng, width=(1, 2, 3), amp=(0.5, 1.0), radius_frac=0.3, segments=48):
    """`count` thin vessel-like curves: cubic Bezier splines with four control
    points in the central disk, width drawn from `width` pixels."""
    shape = tuple(shape)
    n = min(shape)
    centre = np.array([(s - 1) / 2.0 for s in shape])
    out = np.zeros(shape)
    t = np.linspace(0.0, 1.0, segments + 1)
    B = np.stack([(1 - t) ** 3, 3 * t * (1 - t) ** 2, 3 * t ** 2 * (1 - t), t ** 3], axis=1)
    for _ in range(count):
        ctrl = []
        for _k in range(4):
            while True:
                v = rng.uniform(-1.0, 1.0, 2)
                if v @ v <= 1.0:
                    break
            ctrl.append(centre + radius_frac * n * v)
        pts = B @ np.array(ctrl)
        w = float(rng.choice(np.asarray(width)))
        a = rng.uniform(*amp)
        for k in range(segments):
            _tube(out, pts[k], pts[k + 1], w / 2.0, a)
    return out


def vessel_tree3d(shape, rng, depth=4, r_max=4.0, r_min=1.0, amp=(0.5, 1.0), radius_frac=0.3):
    """Binary-branching vessel tree: a trunk through the central region, each
    segment splitting in two at its end, radius tapering from r_max to r_min
    voxels over `depth` generations."""
    shape = tuple(shape)
    n = min(shape)
    centre = np.array([(s - 1) / 2.0 for s in shape])
    out = np.zeros(shape)
    a = rng.uniform(*amp)
    start = centre + np.array([0.0, 0.0, -radius_frac * n])
    direction = np.array([0.0, 0.0, 1.0]) + 0.2 * rng.standard_normal(3)
    stack = [(start, direction / np.linalg.norm(direction), 0)]
    seg_len = radius_frac * n * 0.7
    while stack:
        p, dvec, gen = stack.pop()
        r = r_max + (r_min - r_max) * gen / max(depth - 1, 1)
        q = p + seg_len * (0.75 ** gen) * dvec
        q = np.clip(q, centre - radius_frac * n, centre + radius_frac * n)
        _tube(out, p, q, r, a)
        if gen + 1 < depth:
            for _ in range(2):
                nd = dvec + 0.8 * rng.standard_normal(3)
                stack.append((q, nd / np.linalg.norm(nd), gen + 1))
    return out


def speed_map(shape, rng, sigma=16.0, lo=1400.0, hi=1600.0):
    """Smooth random speed of sound: white noise, Gaussian-filtered with
    standard deviation `sigma` pixels, affinely rescaled to [lo, hi] m/s."""
    noise = rng.standard_normal(tuple(shape))
    sm = gaussian_filter(noise, sigma, mode="wrap")
    sm = (sm - sm.min()) / (sm.max() - sm.min())
    return lo + (hi - lo) * sm
