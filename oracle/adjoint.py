"""Gradient of the least-squares solution map, in FP64 (test infrastructure only).

The paper has no adjoint; this is the textbook sensitivity of
x*(A, b) = (A^T A)^{-1} A^T b. For a loss L(x*) with g = dL/dx:
  z      = (A^T A)^{-1} g
  dL/db  = A z
  dL/dA  = r z^T - (A z) x^T,   r = b - A x
(differentiate A^T (b - A x) = 0: A^T A dx = dA^T r + A^T db - A^T dA x).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import direct


def lls_grad(A, b, x, g):
    """(dL/dA, dL/db) for given x = x*(A, b) and g = dL/dx, using the oracle's R."""
    A = np.asarray(A, dtype=np.float64)
    _, R = direct.householder_qr(A)
    z = solve_triangular(R, solve_triangular(R, g, lower=False, trans="T"), lower=False)
    r = np.asarray(b, dtype=np.float64) - A @ x
    Az = A @ z
    return np.outer(r, z) - np.outer(Az, x), Az
