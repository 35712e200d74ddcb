"""Plan: owning Python handle of a pat_plan (argument marshalling only)."""
import numpy as np
import torch

from . import _lib


class Plan:
    """One reconstruction problem on the GPU.

    shape    grid shape in array order, (ny, nx) or (nz, ny, nx), x fastest
    h, dt    spacing [m] and time step [s];  nt samples (P^0 .. P^{nt-1})
    order    staggered order 2/4/6/8;  c: scalar [m/s] or array of `shape`
    sensors  (Ns, d) coordinates (x, y[, z]) [m]
    family, levels, level_offset: periodic Daubechies wavelet of E_s
    """

    def __init__(self, shape, h, dt, nt, order, c, sensors, family=4, levels=3, level_offset=0, stream=None):
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        grid = _lib.pat_grid()
        grid.dim = self.dim
        n = list(self.shape[::-1]) + [1] * (3 - self.dim)
        for i in range(3):
            grid.n[i] = n[i]
        grid.h = float(h)
        wav = _lib.pat_wavelet()
        wav.family, wav.levels, wav.level_offset = int(family), int(levels), int(level_offset)
        c_arr = None
        c0 = 0.0
        if np.ndim(c) == 0:
            c0 = float(c)
        else:
            c_arr = np.ascontiguousarray(np.broadcast_to(np.asarray(c, dtype=np.float64), self.shape))
        sens = np.ascontiguousarray(np.asarray(sensors, dtype=np.float64).reshape(-1, self.dim))
        self.ns = sens.shape[0]
        self.nt = int(nt)
        self.N = int(np.prod(self.shape))
        self.handle = _lib.pat_plan_create(grid, c_arr, c0, sens, self.ns, float(dt), self.nt, int(order), wav, stream)

    def close(self):
        if getattr(self, "handle", None):
            _lib.pat_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- helpers
    def _stream(self, stream):
        if stream is not None:
            return stream
        if torch.cuda.is_available():
            return torch.cuda.current_stream()
        return None

    @staticmethod
    def _f32(t, device="cuda"):
        if isinstance(t, torch.Tensor):
            return t.to(device=device, dtype=torch.float32).contiguous()
        return torch.as_tensor(np.ascontiguousarray(t, dtype=np.float32), device=device)

    @property
    def path(self):
        return _lib.pat_plan_get_path(self.handle)

    @path.setter
    def path(self, p):
        _lib.pat_plan_set_path(self.handle, p)

    def set_prior(self, kind, length_cells=1.0, stream=None):
        """kind 0: wavelet form of E_s (default); 1: Fourier form with lengths in
        units of `length_cells` cells (2D, power-of-two extents)."""
        _lib.pat_plan_set_prior(self.handle, kind, length_cells, self._stream(stream))

    def set_sponge(self, width, sigma_max=0.0, stream=None):
        """Absorbing layer of `width` cells (0 removes it); sigma_max 0 selects
        the nominal-reflection-1e-3 default.  2D plans only."""
        _lib.pat_plan_set_sponge(self.handle, width, sigma_max, self._stream(stream))

    def check(self, stream=None):
        return _lib.pat_plan_check(self.handle, self._stream(stream))

    # -------------------------------------------------------------- operators
    def forward(self, x, out=None, stream=None):
        """y = K x on the device; returns a (Ns, nt) float32 tensor."""
        x = self._f32(x)
        y = out if out is not None else torch.empty((self.ns, self.nt), device="cuda", dtype=torch.float32)
        _lib.pat_forward(self.handle, x, y, self._stream(stream))
        return y

    def adjoint(self, y, out=None, stream=None):
        """x = K* y; returns a float32 tensor of `shape`."""
        y = self._f32(y)
        x = out if out is not None else torch.empty(self.shape, device="cuda", dtype=torch.float32)
        _lib.pat_adjoint(self.handle, y, x, self._stream(stream))
        return x

    def Es(self, u, s, out=None, stream=None):
        u = self._f32(u)
        x = out if out is not None else torch.empty(self.shape, device="cuda", dtype=torch.float32)
        _lib.pat_Es(self.handle, s, u, x, self._stream(stream))
        return x

    def EsT(self, x, s, out=None, stream=None):
        x = self._f32(x)
        u = out if out is not None else torch.empty(self.N, device="cuda", dtype=torch.float32)
        _lib.pat_EsT(self.handle, s, x, u, self._stream(stream))
        return u

    def grad_kappa(self, x, r, segment=0, stream=None):
        """d<r, K x>/d kappa per cell (float32 tensor of `shape`)."""
        x = self._f32(x)
        r = self._f32(r)
        g = torch.empty(self.shape, device="cuda", dtype=torch.float32)
        _lib.pat_grad_kappa(self.handle, x, r, g, segment, self._stream(stream))
        return g

    def solve(self, y, alpha, s, iters, u0=None, want_log=False, stream=None):
        """CG solve; returns (u, x, log) as device tensors (log: (iters, 3) float64 or None)."""
        y = self._f32(y)
        u = torch.empty(self.N, device="cuda", dtype=torch.float32)
        x = torch.empty(self.shape, device="cuda", dtype=torch.float32)
        log = torch.zeros((max(iters, 1), 3), device="cuda", dtype=torch.float64) if want_log else None
        u0t = self._f32(u0) if u0 is not None else None
        _lib.pat_solve(self.handle, y, alpha, s, iters, u0t, u, x, log, self._stream(stream))
        return u, x, (log[:iters] if want_log else None)


    def solve_multi(self, ys, alphas, ss, iters, stream=None):
        """CG for several right-hand sides of this plan (two per wave launch on
        the persistent engine); returns the images."""
        ys = [self._f32(y) for y in ys]
        xs = [torch.empty(self.shape, device="cuda", dtype=torch.float32) for _ in ys]
        _lib.pat_solve_multi(self.handle, ys, alphas, ss, iters, xs, self._stream(stream))
        return xs

    def solve_gmres(self, y, alpha, s, iters, want_log=False, stream=None):
        """GMRES on the paper's image-space system; returns (x, res, J) with
        res and J numpy arrays of iters+1 values (None unless want_log)."""
        y = self._f32(y)
        x = torch.empty(self.shape, device="cuda", dtype=torch.float32)
        res = np.zeros(iters + 1) if want_log else None
        J = np.zeros(iters + 1) if want_log else None
        _lib.pat_solve_gmres(self.handle, y, alpha, s, iters, x, res, J, self._stream(stream))
        return x, res, J

    def solve_landweber(self, y, alpha, s, iters, omega, want_log=False, stream=None):
        """Landweber iteration; returns (u, x, J) (J: numpy, iters+1 values, or None)."""
        y = self._f32(y)
        u = torch.empty(self.N, device="cuda", dtype=torch.float32)
        x = torch.empty(self.shape, device="cuda", dtype=torch.float32)
        J = np.zeros(iters + 1) if want_log else None
        _lib.pat_solve_landweber(self.handle, y, alpha, s, iters, omega, u, x, J, self._stream(stream))
        return u, x, J


class Batch:
    """Many 2D plans (one stencil order) advanced together by the batched engine
    (all instances' tiles in one table; tile height and launch form -- one
    launch per time step, or one cooperative launch per K / K* -- chosen by
    the library's autotuner when the batch is created).  The plans must
    outlive the batch and are not used concurrently with it."""

    def __init__(self, plans, stream=None):
        self.plans = list(plans)
        self.handle = _lib.pat_batch_create([p.handle for p in self.plans], stream)

    def close(self):
        if getattr(self, "handle", None):
            _lib.pat_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream):
        return stream if stream is not None else torch.cuda.current_stream()

    @property
    def info(self):
        d = _lib.pat_batch_info(self.handle)
        runall, ms = _lib.pat_batch_launch(self.handle, -1)
        d.update(launch="one per application" if runall else "one per step", launch_tune_ms=ms)
        return d

    def set_launch(self, mode):
        """0: autotuner's choice, 1: one launch per time step, 2: one cooperative launch per K / K*."""
        _lib.pat_batch_launch(self.handle, mode)

    def forward(self, xs, outs=None, stream=None):
        """[K_i x_i] for every instance; returns a list of (Ns_i, nt_i) tensors."""
        xs = [Plan._f32(x) for x in xs]
        ys = outs or [torch.empty((p.ns, p.nt), device="cuda", dtype=torch.float32) for p in self.plans]
        _lib.pat_batch_forward(self.handle, xs, ys, self._stream(stream))
        return ys

    def adjoint(self, ys, outs=None, stream=None):
        ys = [Plan._f32(y) for y in ys]
        xs = outs or [torch.empty(p.shape, device="cuda", dtype=torch.float32) for p in self.plans]
        _lib.pat_batch_adjoint(self.handle, ys, xs, self._stream(stream))
        return xs

    def solve(self, ys, alphas, ss, iters, outs=None, stream=None):
        """CG for every instance; returns (images, status, per-instance statuses)."""
        ys = [Plan._f32(y) for y in ys]
        xs = outs or [torch.empty(p.shape, device="cuda", dtype=torch.float32) for p in self.plans]
        rc, per = _lib.pat_batch_solve(self.handle, ys, alphas, ss, iters, xs, self._stream(stream))
        return xs, rc, per
