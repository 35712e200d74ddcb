"""ctypes front end of the FP64 C oracle for K and K* (test infrastructure only).

Paper Sec. 2.2: K maps the initial pressure p0 (N cells) to the sensor traces
y in R^{Ns x Nt}; here the wave IVP of Eq. (wave_equation) is discretised as
the literal staggered pressure/velocity leapfrog described in fdtd.c, and K*
is the reverse sweep of that program (its exact transpose).
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        sig = [ctypes.c_int, ip, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
               dp, dp, dp]
        for name in ("oracle_forward", "oracle_adjoint"):
            f = getattr(_lib, name)
            f.argtypes = sig
            f.restype = ctypes.c_int
        sig_d = sig[:9] + [dp, dp, dp]  # ... sensors, sigma, in, out
        for name in ("oracle_forward_damped", "oracle_adjoint_damped"):
            f = getattr(_lib, name)
            f.argtypes = sig_d
            f.restype = ctypes.c_int
        _lib.oracle_forward_history_damped.argtypes = [ctypes.c_int, ip, ctypes.c_double, ctypes.c_double,
                                                       ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        _lib.oracle_forward_history_damped.restype = ctypes.c_int
        _lib.oracle_forward_history.argtypes = [ctypes.c_int, ip, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int, dp, dp, dp]
        _lib.oracle_forward_history.restype = ctypes.c_int
        _lib.oracle_kappa_grad.argtypes = sig + [dp]
        _lib.oracle_kappa_grad.restype = ctypes.c_int
        _lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib.oracle_max_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Wave:
    """Geometry + medium of one problem.

    shape: grid shape in array order, (ny, nx) or (nz, ny, nx), x fastest.
    h: spacing [m]; dt: time step [s]; nt: number of samples (P^0 .. P^{nt-1});
    order: 2, 4, 6 or 8; c: scalar or array of shape `shape` [m/s];
    sensors: (Ns, dim) coordinates (x, y[, z]) in metres, cell i at i*h.
    """

    def __init__(self, shape, h, dt, nt, order, c, sensors, sigma=None):
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        self.h, self.dt, self.nt, self.order = float(h), float(dt), int(nt), int(order)
        c = np.asarray(c, dtype=np.float64)
        self.c = np.ascontiguousarray(np.broadcast_to(c, self.shape), dtype=np.float64)
        self.sensors = np.ascontiguousarray(np.asarray(sensors, dtype=np.float64).reshape(-1, self.dim))
        self.ns = self.sensors.shape[0]
        self.n3 = np.array(list(self.shape[::-1]) + [1] * (3 - self.dim), dtype=np.int32)
        self.N = int(np.prod(self.shape))
        self.evaluations = 0  # wave-equation solves performed (forward or adjoint)
        # damping rate of the absorbing layer [1/s] per cell, or None (see fdtd.c and sponge_sigma)
        self.sigma = None if sigma is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(sigma, dtype=np.float64), self.shape))

    def _args(self):
        return (self.dim, self.n3.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.h, self.dt, self.nt,
                self.order, _dp(self.c), self.ns, _dp(self.sensors))

    def forward(self, x):
        """y = K x, shape (Ns, nt)."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(self.shape))
        y = np.zeros((self.ns, self.nt), dtype=np.float64)
        if self.sigma is None:
            rc = _load().oracle_forward(*self._args(), _dp(x), _dp(y))
        else:
            rc = _load().oracle_forward_damped(*self._args(), _dp(self.sigma), _dp(x), _dp(y))
        if rc != 0:
            raise ValueError(f"oracle_forward failed ({rc})")
        self.evaluations += 1
        return y

    def adjoint(self, y):
        """x = K* y, shape `shape`."""
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(self.ns, self.nt))
        x = np.zeros(self.shape, dtype=np.float64)
        if self.sigma is None:
            rc = _load().oracle_adjoint(*self._args(), _dp(y), _dp(x))
        else:
            rc = _load().oracle_adjoint_damped(*self._args(), _dp(self.sigma), _dp(y), _dp(x))
        if rc != 0:
            raise ValueError(f"oracle_adjoint failed ({rc})")
        self.evaluations += 1
        return x

    def kappa_grad(self, x, r):
        """g = d<r, K x>/d kappa per cell, kappa = (c dt / h)^2 (shape `shape`); undamped program."""
        if self.sigma is not None:
            raise ValueError("kappa_grad is defined for the undamped program")
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(self.shape))
        r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(self.ns, self.nt))
        g = np.zeros(self.shape, dtype=np.float64)
        rc = _load().oracle_kappa_grad(*self._args(), _dp(x), _dp(r), _dp(g))
        if rc != 0:
            raise ValueError(f"oracle_kappa_grad failed ({rc})")
        return g

    def history(self, x):
        """All pressure fields P^0..P^{nt-1}, shape (nt,) + shape."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(self.shape))
        hist = np.zeros((self.nt,) + self.shape, dtype=np.float64)
        lib = _load()
        n3 = self.n3.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if self.sigma is None:
            rc = lib.oracle_forward_history(self.dim, n3, self.h, self.dt, self.nt, self.order, _dp(self.c), _dp(x),
                                            _dp(hist))
        else:
            rc = lib.oracle_forward_history_damped(self.dim, n3, self.h, self.dt, self.nt, self.order, _dp(self.c),
                                                   _dp(self.sigma), _dp(x), _dp(hist))
        if rc != 0:
            raise ValueError(f"oracle_forward_history failed ({rc})")
        return hist


def sponge_sigma(shape, width, sigma_max):
    """Damping rate of the absorbing layer (this implementation's reading of the paper's
    PML): within `width` cells of each grid face, sigma grows quadratically
    from 0 (at `width` cells from the face) to sigma_max (on the face); the
    contributions of the axes add up, so corners are damped twice.  For a
    cell at index i of an axis with n cells, d = min(i, n - 1 - i) and the
    axis contributes sigma_max * ((width - d) / width)^2 when d < width."""
    shape = tuple(int(s) for s in shape)
    sigma = np.zeros(shape, dtype=np.float64)
    if width <= 0:
        return sigma
    for ax, n in enumerate(shape):
        i = np.arange(n)
        d = np.minimum(i, n - 1 - i).astype(np.float64)
        prof = np.where(d < width, sigma_max * ((width - d) / width) ** 2, 0.0)
        sigma += prof.reshape([n if k == ax else 1 for k in range(len(shape))])
    return sigma


def sponge_sigma_max(c_max, width, h, reflection=1e-3):
    """sigma_max of the quadratic profile for a nominal reflection coefficient:
    3 c_max ln(1/R) / (2 width h) (the usual rule for a quadratic absorbing
    profile)."""
    return 3.0 * c_max * np.log(1.0 / reflection) / (2.0 * width * h)
