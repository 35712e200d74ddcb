"""FP64 conjugate-gradient solve of the regularised PAT problem (test
infrastructure only).

Paper Eq. (linear_minimization): (E_s* K* K + alpha I) x = E_s* K* p.  The
same minimiser is reached on the symmetric positive definite system in wavelet
coefficients

    (E_s* K* K E_s + alpha I) u = E_s* K* y,   x = E_s u,

because multiplying it by E_s gives (E_s E_s* K* K + alpha I)(E_s u) =
E_s E_s* K* y, the paper's system with its covariance E_s E_s*, and E_s is
invertible.  Plain CG from u0 (default 0) for a fixed number of iterations;
each iteration costs one K and one K*, plus one K* for the right-hand side
(the 1 + 2k count of Sec. 5).  alpha is absolute.
"""
import numpy as np


class Breakdown(RuntimeError):
    pass


def normal_op(wave, wav, s, alpha):
    """p -> E_s* K* K E_s p + alpha p."""
    def H(p):
        return wav.EsT(wave.adjoint(wave.forward(wav.Es(p, s))), s).ravel() + alpha * p
    return H


def rhs(wave, wav, y, s):
    """b = E_s* K* y."""
    return wav.EsT(wave.adjoint(y), s).ravel()


def cg(wave, wav, y, alpha, s, iters, u0=None, snapshots=None):
    """Returns (u, x, log) with log[k] = (rr_k, pq_k, a_k) per iteration.
    With `snapshots` (iteration counts), returns (u, x, log, {k: x_k}) with
    the image E_s u_k after k iterations of this same run."""
    H = normal_op(wave, wav, s, alpha)
    b = rhs(wave, wav, y, s)
    if u0 is None:
        u = np.zeros_like(b)
        r = b.copy()
    else:
        u = np.asarray(u0, dtype=np.float64).ravel().copy()
        r = b - H(u)
    p = r.copy()
    rr = float(r @ r)
    log = []
    snaps = {}
    for _ in range(iters):
        q = H(p)
        pq = float(p @ q)
        if not np.isfinite(pq) or pq <= 0.0:
            raise Breakdown(f"p.q = {pq}")
        a = rr / pq
        u += a * p
        r -= a * q
        rr_new = float(r @ r)
        log.append((rr, pq, a))
        p = r + (rr_new / rr) * p
        rr = rr_new
        if snapshots is not None and len(log) in snapshots:
            snaps[len(log)] = wav.Es(u, s)
    if snapshots is not None:
        return u, wav.Es(u, s), np.array(log), snaps
    return u, wav.Es(u, s), np.array(log)


def cg_converged(wave, wav, y, alpha, s, rtol=1e-10, max_iters=3000):
    """The minimiser itself (reading A14's "converged solution"): the same CG,
    run until ||b - H u|| <= rtol ||b|| with the residual recomputed from u
    (not the recurrence) at the end.  Returns (u, x, iterations, rel_res)."""
    H = normal_op(wave, wav, s, alpha)
    b = rhs(wave, wav, y, s)
    nb = float(np.linalg.norm(b))
    u = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    k = 0
    while k < max_iters and np.sqrt(rr) > rtol * nb:
        q = H(p)
        pq = float(p @ q)
        if not np.isfinite(pq) or pq <= 0.0:
            raise Breakdown(f"p.q = {pq}")
        a = rr / pq
        u += a * p
        r -= a * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        k += 1
    rel_res = float(np.linalg.norm(b - H(u)) / nb)
    return u, wav.Es(u, s), k, rel_res

