"""FP64 Landweber iteration and GMRES for the regularised PAT problem (test
infrastructure only).

GMRES is the paper's solver (Sec. 4 and 5: GMRES on the non-symmetric image-
space system of Eq. linear_minimization with the covariance Gamma = E_s E_s*
in place of the paper's "E_s*"):

    A x = f,   A = Gamma K* K + alpha I,   f = Gamma K* y.

Arnoldi with modified Gram-Schmidt builds an orthonormal basis V_k of the
Krylov space K_k(A, r_0) and the (k+1) x k Hessenberg matrix H_k with
A V_k = V_{k+1} H_k; the iterate x_k = x_0 + V_k z minimises ||f - A x|| over
x_0 + K_k, i.e. z solves the small least-squares problem
min ||beta e_1 - H_k z|| (numpy's least-squares routine serves as that step).

Landweber is gradient descent on J(u) = 1/2 ||K E_s u - y||^2 + alpha/2
||u||^2 in wavelet coefficients: u_{k+1} = u_k - omega (H u_k - b) with
H = E_s* K* K E_s + alpha I, b = E_s* K* y (converges for 0 < omega <
2 / lambda_max(H)).

Both record J along the iterates (the J-per-iterate curves); for an image x,
u = E_s^{-1} x = S_s^{-1} W x.
"""
import numpy as np

from .solve import normal_op, rhs


def objective(wave, wav, y, alpha, s, u):
    """J(u) = 1/2 ||K E_s u - y||^2 + alpha/2 ||u||^2."""
    r = wave.forward(wav.Es(u, s)) - y
    return 0.5 * float(np.sum(r * r)) + 0.5 * alpha * float(u @ u)


def coefficients(wav, x, s):
    """u = E_s^{-1} x = S_s^{-1} W x (W orthonormal, S_s diagonal)."""
    return wav.scale(wav.dwt(x), -s)


def landweber(wave, wav, y, alpha, s, iters, omega, u0=None):
    """Returns (u, x, J) with J[k] = J(u_k) for k = 0 .. iters."""
    H = normal_op(wave, wav, s, alpha)
    b = rhs(wave, wav, y, s)
    u = np.zeros_like(b) if u0 is None else np.asarray(u0, dtype=np.float64).ravel().copy()
    J = [objective(wave, wav, y, alpha, s, u)]
    for _ in range(iters):
        u = u - omega * (H(u) - b)
        J.append(objective(wave, wav, y, alpha, s, u))
    return u, wav.Es(u, s), np.array(J)


def image_op(wave, wav, s, alpha):
    """x -> Gamma K* K x + alpha x with Gamma = E_s E_s*."""
    def A(x):
        x = x.reshape(wave.shape)
        g = wave.adjoint(wave.forward(x))
        return wav.Es(wav.EsT(g, s), s).ravel() + alpha * x.ravel()
    return A


def gmres(wave, wav, y, alpha, s, iters, x0=None):
    """Returns (x, res, J): res[k] = ||f - A x_k|| and J[k] = J(E_s^{-1} x_k)
    for k = 0 .. iters (x_0 = 0 unless given)."""
    A = image_op(wave, wav, s, alpha)
    f = wav.Es(wav.EsT(wave.adjoint(y), s), s).ravel()
    x0 = np.zeros(wave.N) if x0 is None else np.asarray(x0, dtype=np.float64).ravel()
    r0 = f - A(x0)
    beta = float(np.linalg.norm(r0))
    V = [r0 / beta] if beta > 0 else []
    Hh = np.zeros((iters + 1, iters))
    res = [beta]
    J = [objective(wave, wav, y, alpha, s, coefficients(wav, x0.reshape(wave.shape), s))]
    x = x0.copy()
    for j in range(iters):
        if beta == 0.0:
            res.append(0.0)
            J.append(J[-1])
            continue
        w = A(V[j])
        for i in range(j + 1):  # modified Gram-Schmidt
            Hh[i, j] = float(V[i] @ w)
            w = w - Hh[i, j] * V[i]
        Hh[j + 1, j] = float(np.linalg.norm(w))
        e1 = np.zeros(j + 2)
        e1[0] = beta
        z = np.linalg.lstsq(Hh[:j + 2, :j + 1], e1, rcond=None)[0]
        x = x0 + np.stack(V, axis=1) @ z
        res.append(float(np.linalg.norm(e1 - Hh[:j + 2, :j + 1] @ z)))
        J.append(objective(wave, wav, y, alpha, s, coefficients(wav, x.reshape(wave.shape), s)))
        if Hh[j + 1, j] == 0.0:  # lucky breakdown: x is exact
            V.append(np.zeros_like(w))
        else:
            V.append(w / Hh[j + 1, j])
    return x.reshape(wave.shape), np.array(res), np.array(J)
