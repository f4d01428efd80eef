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
