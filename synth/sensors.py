"""Point-sensor layouts, returned as (Ns, d) coordinates (x, y[, z]) in metres
with cell i at coordinate i*h and the grid centre at (n-1)*h/2."""
import numpy as np


def circle(n, h, count, radius_frac=0.45):
    """`count` sensors evenly on a full circle of radius radius_frac*n*h."""
    c = (n - 1) * h / 2.0
    r = radius_frac * n * h
    th = 2.0 * np.pi * np.arange(count) / count
    return np.stack([c + r * np.cos(th), c + r * np.sin(th)], axis=1)


def arc(n, h, count, radius_frac=0.45, theta0=0.0, theta1=np.pi):
    """`count` sensors on the arc theta in [theta0, theta1], endpoints included."""
    c = (n - 1) * h / 2.0
    r = radius_frac * n * h
    th = theta0 + (theta1 - theta0) * np.arange(count) / max(count - 1, 1)
    return np.stack([c + r * np.cos(th), c + r * np.sin(th)], axis=1)


def fibonacci_sphere(n, h, count, radius_frac=0.45):
    """`count` near-uniform sensors on a sphere (golden-angle spiral)."""
    c = (n - 1) * h / 2.0
    r = radius_frac * n * h
    k = np.arange(count) + 0.5
    z = 1.0 - 2.0 * k / count
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - np.sqrt(5.0)) * np.arange(count)
    return np.stack([c + r * rho * np.cos(phi), c + r * rho * np.sin(phi), c + r * z], axis=1)


def line(n, h, count, side="bottom", margin=2):
    """`count` equidistant sensors along one side of a square grid, `margin`
    cells inside the edge (sides: bottom, top, left, right)."""
    lo, hi = margin * h, (n - 1 - margin) * h
    t = lo + (hi - lo) * np.arange(count) / max(count - 1, 1)
    e0, e1 = lo, hi
    if side == "bottom":
        return np.stack([t, np.full(count, e0)], axis=1)
    if side == "top":
        return np.stack([t, np.full(count, e1)], axis=1)
    if side == "left":
        return np.stack([np.full(count, e0), t], axis=1)
    if side == "right":
        return np.stack([np.full(count, e1), t], axis=1)
    raise ValueError(side)
