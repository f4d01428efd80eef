"""R-preconditioned Krylov least-squares solvers in FP64 (Sec. 3.2.3, Alg. 5).

Test infrastructure only.

CGLS with R as right preconditioner is CG on the normal equations of A R^{-1}.
Alg. 5 as printed has two slips, read here as follows:
  * the step length is alpha = gamma / delta (the printed ``gamma/gamma1`` uses a
    value not yet defined in the first iteration; delta is computed on the line
    before and otherwise unused, and the cited cgls.m uses gamma/delta);
  * the solution update uses the unpreconditioned direction, x += alpha R^{-1} p
    (the printed ``x + alpha*p`` adds a preconditioned-space vector to x).
The printed initialisation s = A^T r, p = s also lacks the preconditioner; the
preconditioned form s = R^{-T} A^T r is used (it is what the loop body computes).

LSQR (Paige and Saunders 1982, named by the paper as the more stable
equivalent, Sec. 5) is applied to the same operator A R^{-1}.

Stop test (the paper omits it): eta_est = ||R^{-T} A^T r|| / (||A||_F ||x||) <= tol.
For an exact R this quantity equals ||A (x - x*)|| / (||A||_F ||x||), an upper
bound on the Karlson-Walden estimate of the least-squares backward error.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_triangular


def _rinv(R, v):
    return solve_triangular(R, v, lower=False)


def _rinvT(R, v):
    return solve_triangular(R, v, lower=False, trans="T")


def cgls(A, b, R, tol: float = 1e-12, maxit: int = 200, x0=None):
    """Preconditioned CGLS (Alg. 5, corrected). Returns (x, iterations, eta history)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    anorm = np.linalg.norm(A)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    s = _rinvT(R, A.T @ r)
    p = s.copy()
    gamma = float(s @ s)
    hist = []
    it = 0
    for it in range(1, maxit + 1):
        t = _rinv(R, p)
        q = A @ t
        delta = float(q @ q)
        if delta == 0.0:
            it -= 1
            break
        alpha = gamma / delta
        x += alpha * t
        r -= alpha * q
        s = _rinvT(R, A.T @ r)
        gamma1 = gamma
        gamma = float(s @ s)
        xn = np.linalg.norm(x)
        eta = math.sqrt(gamma) / (anorm * xn) if xn > 0 else math.inf
        hist.append(eta)
        if eta <= tol:
            break
        beta = gamma / gamma1
        p = s + beta * p
    return x, it, hist


def lsqr(A, b, R, tol: float = 1e-12, maxit: int = 200):
    """LSQR on the right-preconditioned operator B = A R^{-1}; x = R^{-1} y.

    Golub-Kahan bidiagonalisation: beta u = b, alpha v = B^T u, then each step
    beta u = B v - alpha u, alpha v = B^T u - beta v, a plane rotation of the
    bidiagonal, and the updates y += (phi/rho) w, w = v - (theta/rho) w. The
    iterate is kept in x-space with d = R^{-1} w.
    Returns (x, iterations, eta history)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = A.shape
    anorm = np.linalg.norm(A)
    x = np.zeros(n)
    beta = np.linalg.norm(b)
    u = b / beta
    v = _rinvT(R, A.T @ u)
    alpha = np.linalg.norm(v)
    v = v / alpha
    d = _rinv(R, v)
    phibar, rhobar = beta, alpha
    hist = []
    it = 0
    for it in range(1, maxit + 1):
        u = A @ _rinv(R, v) - alpha * u
        beta = np.linalg.norm(u)
        if beta > 0:
            u /= beta
        v_new = _rinvT(R, A.T @ u) - beta * v
        alpha = np.linalg.norm(v_new)
        if alpha > 0:
            v_new /= alpha
        rho = math.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x += (phi / rho) * d
        d = _rinv(R, v_new) - (theta / rho) * d
        v = v_new
        xn = np.linalg.norm(x)
        # ||B^T r_k|| = phibar * alpha * |c| (Paige and Saunders, Sec. 5)
        eta = (phibar * alpha * abs(c)) / (anorm * xn) if xn > 0 else math.inf
        hist.append(eta)
        if eta <= tol:
            break
    return x, it, hist
