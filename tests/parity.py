"""Parity predicates shared by the GPU tests (test infrastructure; no arithmetic of the method).

R factors are compared entry by entry, each entry's difference measured against the norm of
its column of the oracle's R. A normwise bound over the whole of R can hide a localized
mistake (one wrong tile of a wide R moves the Frobenius norm by little); this measure sees
any single entry that is off by more than the bound times its column's size.
"""
import numpy as np


def r_entry_err(R, Ro):
    """max over i, j of |R_ij - Ro_ij| / ||Ro[:, j]||_2 (columns of Ro that are zero count
    their entries' absolute differences)."""
    R = np.asarray(R, dtype=np.float64)
    Ro = np.asarray(Ro, dtype=np.float64)
    cn = np.linalg.norm(Ro, axis=0)
    cn = np.where(cn > 0.0, cn, 1.0)
    return float((np.abs(R - Ro) / cn[None, :]).max())


def kw_bound(A, R, tol=1e-12):
    """The Karlson-Walden backward error the stop test guarantees. The solver stops on
    eta_est = ||R^-T A^T r|| / (||A||_F ||x||) <= tol, and eta_kw <= ||(A^T A)^-1/2 R^T|| eta_est
    = eta_est / sigma_min(A R^-1); with a coarse R (FP8 products) sigma_min drops below one."""
    A = np.asarray(A, dtype=np.float64)
    Rinv = np.linalg.inv(np.asarray(R, dtype=np.float64))
    smin = np.linalg.svd(A @ Rinv, compute_uv=False)[-1]
    return tol / smin * (1 + 1e-6)
