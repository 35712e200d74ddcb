"""ctypes binding of libpat.so: the C ABI of include/pat.h, same names,
argument marshalling only.  Every operator runs in the CUDA library; there is
no fallback: if the library cannot be loaded, loading raises.

Array arguments accept torch tensors (float32/float64, contiguous, on the
device or the host), numpy arrays (host) or raw integer addresses; streams
accept a torch.cuda.Stream, an integer cudaStream_t or None (legacy default
stream).
"""
import ctypes
import os

import numpy as np

from . import build as _build

c_int, c_double, c_void_p, c_longlong = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong

PAT_OK, PAT_ERR_INVALID, PAT_ERR_CFL, PAT_ERR_CUDA, PAT_ERR_OOM, PAT_ERR_TIMEOUT, PAT_ERR_BREAKDOWN = range(7)
STATUS_NAMES = {0: "PAT_OK", 1: "PAT_ERR_INVALID", 2: "PAT_ERR_CFL", 3: "PAT_ERR_CUDA", 4: "PAT_ERR_OOM",
                5: "PAT_ERR_TIMEOUT", 6: "PAT_ERR_BREAKDOWN"}
PAT_PATH_AUTO, PAT_PATH_PERSISTENT, PAT_PATH_STEP = 0, 1, 2


class pat_grid(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int * 3), ("h", c_double)]


class pat_wavelet(ctypes.Structure):
    _fields_ = [("family", c_int), ("levels", c_int), ("level_offset", c_int)]


# (name, restype, argtypes) of every symbol declared in include/pat.h
SIGNATURES = [
    ("pat_plan_create", c_int, [ctypes.POINTER(pat_grid), c_void_p, c_double, c_void_p, c_int, c_double, c_int,
                                c_int, ctypes.POINTER(pat_wavelet), c_void_p, ctypes.POINTER(c_void_p)]),
    ("pat_plan_destroy", None, [c_void_p]),
    ("pat_plan_info", c_int, [c_void_p, ctypes.POINTER(c_longlong), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    ("pat_forward", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("pat_adjoint", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("pat_Es", c_int, [c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    ("pat_EsT", c_int, [c_void_p, c_double, c_void_p, c_void_p, c_void_p]),
    ("pat_solve", c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                          c_void_p]),
    ("pat_solve_gmres", c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_void_p, c_void_p, c_void_p,
                                c_void_p]),
    ("pat_solve_landweber", c_int, [c_void_p, c_void_p, c_double, c_double, c_int, c_double, c_void_p, c_void_p,
                                    c_void_p, c_void_p]),
    ("pat_solve_multi", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    ("pat_objective", c_int, [c_void_p, c_void_p, c_double, c_double, c_void_p, ctypes.POINTER(c_double),
                              c_void_p, c_void_p]),
    ("pat_solve_batched", c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                  c_void_p]),
    ("pat_batch_create", c_int, [c_void_p, c_int, c_void_p, ctypes.POINTER(c_void_p)]),
    ("pat_batch_destroy", None, [c_void_p]),
    ("pat_batch_forward", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("pat_batch_adjoint", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("pat_batch_solve", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("pat_batch_info", c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_longlong),
                               ctypes.POINTER(c_double)]),
    ("pat_batch_launch", c_int, [c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    ("pat_grad_kappa", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    ("pat_plan_check", c_int, [c_void_p, c_void_p]),
    ("pat_plan_set_path", c_int, [c_void_p, c_int]),
    ("pat_plan_get_path", c_int, [c_void_p, ctypes.POINTER(c_int)]),
    ("pat_plan_set_timeout", c_int, [c_void_p, c_longlong]),
    ("pat_plan_set_sponge", c_int, [c_void_p, c_int, c_double, c_void_p]),
    ("pat_plan_set_prior", c_int, [c_void_p, c_int, c_double, c_void_p]),
    ("pat_plan_profile", c_int, [c_void_p, c_int]),
    ("pat_plan_profile_read", c_int, [c_void_p, ctypes.POINTER(c_longlong), ctypes.POINTER(c_int),
                                      ctypes.POINTER(c_double), ctypes.POINTER(c_longlong)]),
    ("pat_EsT_noalloc", c_int, [c_int, c_int, c_int, c_int, c_int, c_double, c_void_p, c_void_p, c_void_p]),
    ("pat_last_error", ctypes.c_char_p, []),
]

_lib = None


class PatError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib_path():
    return _build.LIB_PATH


def load(build_if_missing=True):
    """Load libpat.so (building it first if absent and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libpat.so not built at {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != PAT_OK:
        raise PatError(status, load().pat_last_error().decode())
    return status


def ptr(a):
    """Address of an array argument (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def stream_handle(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


# ------------------------------------------------------------ raw C ABI calls
def pat_plan_create(grid, c, c0, sensors, ns, dt, nt, order, wavelet, stream=None):
    out = c_void_p()
    _check(load().pat_plan_create(ctypes.byref(grid), ptr(c), float(c0), ptr(sensors), int(ns), float(dt), int(nt),
                                  int(order), ctypes.byref(wavelet), stream_handle(stream), ctypes.byref(out)))
    return out.value


def pat_plan_destroy(plan):
    load().pat_plan_destroy(plan)


def pat_plan_info(plan):
    n, ns, nt = c_longlong(), c_int(), c_int()
    _check(load().pat_plan_info(plan, ctypes.byref(n), ctypes.byref(ns), ctypes.byref(nt)))
    return n.value, ns.value, nt.value


def pat_forward(plan, x, y, stream=None):
    return _check(load().pat_forward(plan, ptr(x), ptr(y), stream_handle(stream)))


def pat_adjoint(plan, y, x, stream=None):
    return _check(load().pat_adjoint(plan, ptr(y), ptr(x), stream_handle(stream)))


def pat_Es(plan, s, u, x, stream=None):
    return _check(load().pat_Es(plan, float(s), ptr(u), ptr(x), stream_handle(stream)))


def pat_EsT(plan, s, x, u, stream=None):
    return _check(load().pat_EsT(plan, float(s), ptr(x), ptr(u), stream_handle(stream)))


def pat_solve(plan, y, alpha, s, iters, u0, u, x, log=None, stream=None):
    return _check(load().pat_solve(plan, ptr(y), float(alpha), float(s), int(iters), ptr(u0), ptr(u), ptr(x),
                                   ptr(log), stream_handle(stream)))


def pat_solve_gmres(plan, y, alpha, s, iters, x, res=None, J=None, stream=None):
    """res, J: None or float64 numpy arrays of iters+1 values (host)."""
    return _check(load().pat_solve_gmres(plan, ptr(y), float(alpha), float(s), int(iters), ptr(x), ptr(res), ptr(J),
                                         stream_handle(stream)))


def pat_solve_landweber(plan, y, alpha, s, iters, omega, u=None, x=None, J=None, stream=None):
    return _check(load().pat_solve_landweber(plan, ptr(y), float(alpha), float(s), int(iters), float(omega), ptr(u),
                                             ptr(x), ptr(J), stream_handle(stream)))


def pat_solve_batched(plans, ys, alphas, ss, iters, xs, stream=None):
    B = len(plans)
    P = (c_void_p * B)(*plans)
    Y = (c_void_p * B)(*[ptr(y) for y in ys])
    A = (c_double * B)(*[float(a) for a in alphas])
    S = (c_double * B)(*[float(s) for s in ss])
    X = (c_void_p * B)(*[ptr(x) for x in xs])
    st = (c_int * B)()
    rc = load().pat_solve_batched(P, B, Y, A, S, int(iters), X, st, stream_handle(stream))
    return rc, [int(v) for v in st]


def _ptrs(arrs):
    return (c_void_p * len(arrs))(*[ptr(a) for a in arrs])


def pat_batch_create(plans, stream=None):
    B = len(plans)
    out = c_void_p()
    _check(load().pat_batch_create((c_void_p * B)(*plans), B, stream_handle(stream), ctypes.byref(out)))
    return out.value


def pat_batch_destroy(batch):
    load().pat_batch_destroy(batch)


def pat_batch_forward(batch, xs, ys, stream=None):
    return _check(load().pat_batch_forward(batch, _ptrs(xs), _ptrs(ys), stream_handle(stream)))


def pat_batch_adjoint(batch, ys, xs, stream=None):
    return _check(load().pat_batch_adjoint(batch, _ptrs(ys), _ptrs(xs), stream_handle(stream)))


def pat_batch_solve(batch, ys, alphas, ss, iters, xs, stream=None):
    """Returns (status, per-instance statuses); no exception for device-side statuses."""
    B = len(ys)
    A = (c_double * B)(*[float(a) for a in alphas])
    S = (c_double * B)(*[float(s) for s in ss])
    st = (c_int * B)()
    rc = load().pat_batch_solve(batch, _ptrs(ys), A, S, int(iters), _ptrs(xs), st, stream_handle(stream))
    if rc in (PAT_ERR_INVALID, PAT_ERR_CUDA, PAT_ERR_OOM):
        _check(rc)
    return rc, [int(v) for v in st]


def pat_batch_info(batch):
    rows, ctas, nodes, tune = c_int(), c_int(), c_longlong(), (c_double * 2)()
    _check(load().pat_batch_info(batch, ctypes.byref(rows), ctypes.byref(ctas), ctypes.byref(nodes), tune))
    return {"tile_rows": rows.value, "ctas": ctas.value, "graph_nodes": nodes.value, "tune_ms": [tune[0], tune[1]]}


def pat_grad_kappa(plan, x, r, g, segment=0, stream=None):
    return _check(load().pat_grad_kappa(plan, ptr(x), ptr(r), ptr(g), int(segment), stream_handle(stream)))


def pat_plan_check(plan, stream=None):
    """Synchronise and return the plan's device status (no exception)."""
    return int(load().pat_plan_check(plan, stream_handle(stream)))


def pat_plan_set_path(plan, path):
    return _check(load().pat_plan_set_path(plan, int(path)))


def pat_plan_get_path(plan):
    v = c_int()
    _check(load().pat_plan_get_path(plan, ctypes.byref(v)))
    return v.value


def pat_plan_set_sponge(plan, width, sigma_max=0.0, stream=None):
    return _check(load().pat_plan_set_sponge(plan, int(width), float(sigma_max), stream_handle(stream)))


def pat_plan_set_prior(plan, kind, length_cells=1.0, stream=None):
    return _check(load().pat_plan_set_prior(plan, int(kind), float(length_cells), stream_handle(stream)))


def pat_plan_set_timeout(plan, timeout_ns):
    return _check(load().pat_plan_set_timeout(plan, int(timeout_ns)))


def pat_plan_profile(plan, enable):
    return _check(load().pat_plan_profile(plan, int(enable)))


def pat_plan_profile_read(plan):
    """(kernels launched, wave applications, their device ms, point-updates)."""
    k, calls, ms, pts = c_longlong(), c_int(), c_double(), c_longlong()
    _check(load().pat_plan_profile_read(plan, ctypes.byref(k), ctypes.byref(calls), ctypes.byref(ms),
                                        ctypes.byref(pts)))
    return k.value, calls.value, ms.value, pts.value


def pat_EsT_noalloc(nx, ny, family, levels, level_offset, s, x, u, stream=None):
    """E_s* of a 2D image without any device allocation (device arrays only).

    The C side cannot see array lengths, so tensors are checked here: float32,
    on a CUDA device, at least nx*ny elements."""
    for name, t in (("x", x), ("u", u)):
        if hasattr(t, "data_ptr"):
            import torch
            if t.dtype != torch.float32 or not t.is_cuda or t.numel() < int(nx) * int(ny):
                raise ValueError(f"pat_EsT_noalloc: {name} must be a float32 CUDA tensor of at least nx*ny = "
                                 f"{int(nx) * int(ny)} elements (got {t.dtype}, {t.device}, {t.numel()})")
    return _check(load().pat_EsT_noalloc(int(nx), int(ny), int(family), int(levels), int(level_offset), float(s),
                                         ptr(x), ptr(u), stream_handle(stream)))


def pat_solve_multi(plan, ys, alphas, ss, iters, xs, stream=None):
    """Several CG solves of one plan, two per wave launch on the persistent
    engine (device arrays only); returns the status."""
    n = len(ys)
    if not (len(xs) == len(alphas) == len(ss) == n):
        raise ValueError("ys, alphas, ss and xs must have the same length")
    yp = (c_void_p * n)(*[ptr(y) for y in ys])
    xp = (c_void_p * n)(*[ptr(x) for x in xs])
    ap = (c_double * n)(*[float(a) for a in alphas])
    sp = (c_double * n)(*[float(v) for v in ss])
    return _check(load().pat_solve_multi(plan, n, yp, ap, sp, int(iters), xp, stream_handle(stream)))


def pat_objective(plan, y, alpha, s, u, grad=None, stream=None):
    """J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2 (returned); the gradient
    is written to `grad` when given."""
    J = c_double()
    _check(load().pat_objective(plan, ptr(y), float(alpha), float(s), ptr(u), ctypes.byref(J), ptr(grad),
                                stream_handle(stream)))
    return J.value


def pat_batch_launch(batch, mode=-1):
    """Set (mode 0 auto, 1 per step, 2 one launch per application) or query the
    batched launch form; returns (runall, [ms per-step, ms one-launch])."""
    ra = c_int()
    ms = (c_double * 2)()
    _check(load().pat_batch_launch(batch, int(mode), ctypes.byref(ra), ms))
    return ra.value, [ms[0], ms[1]]


def pat_last_error():
    return load().pat_last_error().decode()
