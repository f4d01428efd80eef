"""Accuracy measures for QR factors and least-squares solutions, in FP64.

Test infrastructure only.

QR (Sec. 3.2.1): backward error ||A - QR|| / ||A|| and orthogonality
||I - Q^T Q||, in the 2-norm (power iteration) and the Frobenius norm; the
experiments also quote ||I - Q^T Q|| / N (Fig. qr_accu).

Least squares (Sec. 3.2.2 uses the raw A^T (A x - b)); normalised forms:
  eta_ls     = ||A^T r|| / (||A||_F ||r||)                      (LSQR-style)
  eta_cons   = ||r|| / (||A||_F ||x|| + ||b||)                 (compatible systems)
  eta_kw     = ||(A^T A + xi^2 I)^{-1/2} A^T r|| / (||A||_F ||x||), xi = ||r|| / ||x||
               the Karlson-Walden estimate of the smallest ||dA||_F / ||A||_F that
               makes x an exact least-squares solution of (A + dA, b)
  eta_opt    = exact smallest such ||dA||_F / ||A||_F (Walden, Karlson and Sun 1995):
               min(xi, sigma_min([A, xi (I - r r^T / ||r||^2)])) / ||A||_F (tiny cases only)
Residuals and A^T r use the compensated dot product (oracle.direct).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_triangular

from . import direct


def norm2_est(apply, applyT, n: int, iters: int = 30, seed: int = 0) -> float:
    """Largest singular value of an operator by power iteration on op^T op."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    s = 0.0
    for _ in range(iters):
        w = applyT(apply(v))
        nw = np.linalg.norm(w)
        if nw == 0:
            return 0.0
        s = math.sqrt(nw)
        v = w / nw
    return s


def qr_factorization_error(A, Q, R, norm: str = "fro") -> float:
    A = np.asarray(A, dtype=np.float64)
    E = A - np.asarray(Q, dtype=np.float64) @ np.asarray(R, dtype=np.float64)
    if norm == "fro":
        return float(np.linalg.norm(E) / np.linalg.norm(A))
    n = A.shape[1]
    e2 = norm2_est(lambda v: E @ v, lambda w: E.T @ w, n)
    a2 = norm2_est(lambda v: A @ v, lambda w: A.T @ w, n)
    return e2 / a2


def orthogonality(Q, norm: str = "fro") -> float:
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[1]
    G = np.eye(n) - Q.T @ Q
    if norm == "fro":
        return float(np.linalg.norm(G))
    if norm == "perN":
        return float(np.linalg.norm(G, 2)) / n
    return float(np.linalg.norm(G, 2))


def eta_ls(A32, b, x) -> float:
    r = direct.residual(A32, x, b)
    u = direct.atr(A32, r)
    an = np.linalg.norm(np.asarray(A32, dtype=np.float64))
    return float(np.linalg.norm(u) / (an * np.linalg.norm(r)))


def eta_consistent(A32, b, x) -> float:
    r = direct.residual(A32, x, b)
    an = np.linalg.norm(np.asarray(A32, dtype=np.float64))
    return float(np.linalg.norm(r) / (an * np.linalg.norm(x) + np.linalg.norm(b)))


def eta_kw(A32, b, x) -> float:
    """Karlson-Walden estimate, via the R factor of [A; xi I]: (A^T A + xi^2 I) = Rt^T Rt,
    so ||(A^T A + xi^2 I)^{-1/2} z|| = ||Rt^{-T} z||."""
    A = np.asarray(A32, dtype=np.float64)
    m, n = A.shape
    r = direct.residual(A32, x, b)
    u = direct.atr(A32, r)
    xn = float(np.linalg.norm(x))
    xi = float(np.linalg.norm(r)) / xn
    _, Rt = direct.householder_qr(np.vstack([A, xi * np.eye(n)]))
    z = solve_triangular(Rt, u, lower=False, trans="T")
    return float(np.linalg.norm(z) / (xn * np.linalg.norm(A)))


def eta_kw_eigh(A32, b, x) -> float:
    """Same estimate through an eigendecomposition of A^T A + xi^2 I (second, independent route)."""
    A = np.asarray(A32, dtype=np.float64)
    n = A.shape[1]
    r = direct.residual(A32, x, b)
    u = direct.atr(A32, r)
    xn = float(np.linalg.norm(x))
    xi = float(np.linalg.norm(r)) / xn
    w, V = np.linalg.eigh(A.T @ A + xi * xi * np.eye(n))
    z = V @ ((V.T @ u) / np.sqrt(w))
    return float(np.linalg.norm(z) / (xn * np.linalg.norm(A)))


def eta_optimal(A32, b, x) -> float:
    """Exact optimal backward error (perturbing A only), for tiny problems."""
    A = np.asarray(A32, dtype=np.float64)
    m, n = A.shape
    r = direct.residual(A32, x, b)
    xn = float(np.linalg.norm(x))
    rn = float(np.linalg.norm(r))
    xi = rn / xn
    if rn == 0.0:
        return 0.0
    P = np.eye(m) - np.outer(r, r) / (rn * rn)
    smin = np.linalg.svd(np.hstack([A, xi * P]), compute_uv=False)[-1]
    return float(min(xi, smin) / np.linalg.norm(A))


def forward_error(x, x_ref) -> float:
    return float(np.linalg.norm(np.asarray(x) - np.asarray(x_ref)) / np.linalg.norm(x_ref))
