"""FP64 Householder QR and direct least-squares solve (Sec. 2.2, Alg. 1, Eq. qr_lls).

Test infrastructure only: thin ctypes wrappers over householder.c.
x* = R^{-1} (Q^T b) for the stored FP32 A and FP64 b, promoted to FP64.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        dp, fp, i = C.POINTER(C.c_double), C.POINTER(C.c_float), C.c_int
        _lib.oracle_householder_qr.argtypes = [i, i, dp, i, dp]
        _lib.oracle_apply_qt.argtypes = [i, i, dp, i, dp, dp]
        _lib.oracle_form_q.argtypes = [i, i, dp, i, dp, dp, i]
        _lib.oracle_back_substitute.argtypes = [i, dp, i, dp, dp]
        _lib.oracle_lls.argtypes = [i, i, dp, i, dp, dp]
        _lib.oracle_residual_f32.argtypes = [i, i, fp, i, dp, dp, dp]
        _lib.oracle_atr_f32.argtypes = [i, i, fp, i, dp, dp]
        for f in ("oracle_householder_qr", "oracle_back_substitute", "oracle_lls"):
            getattr(_lib, f).restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def householder_qr(A) -> tuple[np.ndarray, np.ndarray]:
    """Reduced QR of A (m x n, m >= n) in FP64: Q (m x n), R (n x n).

    Normalised so that diag(R) >= 0, which makes (Q, R) unique for full column
    rank (the form every Gram-Schmidt variant produces).
    """
    W = np.asfortranarray(np.array(A, dtype=np.float64, copy=True))
    m, n = W.shape
    tau = np.zeros(n)
    rc = lib().oracle_householder_qr(m, n, _dp(W), m, _dp(tau))
    if rc != 0:
        raise ValueError("bad shape for QR")
    R = np.triu(W[:n, :n]).copy()
    Q = np.zeros((m, n), order="F")
    lib().oracle_form_q(m, n, _dp(W), m, _dp(tau), _dp(Q), m)
    d = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * d, R * d[:, None]


def lls(A, b) -> np.ndarray:
    """x* = argmin ||A x - b||_2 by Alg. 1 (Householder QR, Q^T b, back substitution)."""
    W = np.asfortranarray(np.array(A, dtype=np.float64))
    m, n = W.shape
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n)
    rc = lib().oracle_lls(m, n, _dp(W), m, _dp(bb), _dp(x))
    if rc == -2:
        raise np.linalg.LinAlgError("singular R")
    if rc != 0:
        raise ValueError("bad shape for least squares")
    return x


def residual(A32, x, b) -> np.ndarray:
    """r = b - A x for FP32 A, evaluated as if in twice FP64 precision (Dot2)."""
    A = np.asfortranarray(A32, dtype=np.float32)
    m, n = A.shape
    xx = np.ascontiguousarray(x, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    r = np.zeros(m)
    lib().oracle_residual_f32(m, n, _fp(A), m, _dp(xx), _dp(bb), _dp(r))
    return r


def atr(A32, r) -> np.ndarray:
    """A^T r for FP32 A with the compensated dot product."""
    A = np.asfortranarray(A32, dtype=np.float32)
    m, n = A.shape
    rr = np.ascontiguousarray(r, dtype=np.float64)
    u = np.zeros(n)
    lib().oracle_atr_f32(m, n, _fp(A), m, _dp(rr), _dp(u))
    return u
