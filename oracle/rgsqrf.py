"""Recursive Gram-Schmidt QR (RGSQRF) with a communication-avoiding panel, in FP64.

Test infrastructure only. Follows the paper's method step by step:

* Alg. 2 (Sec. 3.1.2, Eq. recqr): split the columns in two, factor the left
  half, R12 = Q1^T A2, A2 <- A2 - Q1 R12, factor the right half. The two
  products are the low-precision GEMMs: their inputs are rounded to the GEMM
  precision (``lowprec``), the products accumulate exactly here (FP64 stands in
  for the FP32 accumulator).
* The recursion stops at panels of at most ``panel_width`` columns (the paper:
  32-column panels, Sec. 3.1.3). Split point w1 = panel_width * ceil(w / (2 panel_width)).
* Panel = CAQR/TSQR (Eq. caqr, steps 1-5): split rows into blocks, factor each
  block independently, stack the R factors, factor the stack (recursively),
  multiply each block's Q by its slice of the stack's Q.
* Leaf factorization: CGS2 (classical Gram-Schmidt with one full
  reorthogonalization) or MGS (Alg. 4).

Every Gram-Schmidt variant yields R with a positive diagonal, so for full
column rank the exact-arithmetic factors are the unique QR factors.
"""
from __future__ import annotations

import math

import numpy as np

from .lowprec import round_to, scaled_round


def cgs2(A: np.ndarray):
    """CGS2 of an m x b block (m >= b): per column k,
    h = Q_<k^T a_k, a_k -= Q_<k h, repeated once, R_<k,k = h + h', R_kk = ||a_k||, q_k = a_k / R_kk.
    A column that is exactly zero after projection gives q_k = 0 and R_kk = 0."""
    A = np.asarray(A, dtype=np.float64)
    m, b = A.shape
    Q = np.zeros((m, b))
    R = np.zeros((b, b))
    for k in range(b):
        a = A[:, k].copy()
        h1 = Q[:, :k].T @ a
        a -= Q[:, :k] @ h1
        h2 = Q[:, :k].T @ a
        a -= Q[:, :k] @ h2
        R[:k, k] = h1 + h2
        nrm = math.sqrt(float(a @ a))
        R[k, k] = nrm
        Q[:, k] = a / nrm if nrm > 0.0 else 0.0
    return Q, R


def mgs(A: np.ndarray):
    """Modified Gram-Schmidt, Alg. 4: normalise column k, then remove its
    component from every later column."""
    Q = np.array(A, dtype=np.float64, copy=True)
    m, b = Q.shape
    R = np.zeros((b, b))
    for k in range(b):
        nrm = math.sqrt(float(Q[:, k] @ Q[:, k]))
        R[k, k] = nrm
        Q[:, k] = Q[:, k] / nrm if nrm > 0.0 else 0.0
        R[k, k + 1:] = Q[:, k] @ Q[:, k + 1:]
        Q[:, k + 1:] -= np.outer(Q[:, k], R[k, k + 1:])
    return Q, R


LEAVES = {"cgs2": cgs2, "mgs": mgs}


def row_blocks(m: int, leaf_rows: int):
    """Balanced contiguous row blocks: ceil(m / leaf_rows) blocks whose sizes differ by at most one."""
    nb = max(1, -(-m // leaf_rows))
    base, extra = divmod(m, nb)
    starts, s = [], 0
    for i in range(nb):
        sz = base + (1 if i < extra else 0)
        starts.append((s, s + sz))
        s += sz
    return starts


def tsqr(A: np.ndarray, leaf_rows: int = 256, leaf: str = "cgs2"):
    """CAQR panel of Eq. caqr.

    1. A = [A_1; ...; A_p], A_i = Q_1i R_i (independent leaf factorizations)
    2. stack S = [R_1; ...; R_p]
    3. S = Q_2 R (the same procedure applied to S, until one block remains)
    4. Q_i = Q_1i Q_2i, Q_2i the i-th b-row slice of Q_2
    5. A = Q R
    """
    A = np.asarray(A, dtype=np.float64)
    m, b = A.shape
    f = LEAVES[leaf]
    if m <= leaf_rows:
        return f(A)
    blocks = row_blocks(m, leaf_rows)
    if any(e - s < b for s, e in blocks):
        return f(A)
    factors = [f(A[s:e]) for s, e in blocks]                 # step 1
    S = np.vstack([R for _, R in factors])                   # step 2
    Q2, R = tsqr(S, leaf_rows, leaf)                         # step 3
    Q = np.vstack([Qi @ Q2[i * b:(i + 1) * b]                 # step 4
                   for i, (Qi, _) in enumerate(factors)])
    return Q, R                                              # step 5


def split_point(w: int, panel_width: int) -> int:
    """Left width of a recursion node of width w: a multiple of the panel width near w/2."""
    return panel_width * (-(-w // (2 * panel_width)))


def rgsqrf(A: np.ndarray, panel_width: int = 32, prec: str = "fp16",
           leaf_rows: int = 256, leaf: str = "cgs2"):
    """Alg. 2 with the GEMM inputs rounded to ``prec`` ('fp16', 'bf16', 'fp32', 'fp64').

    R12 = (round(Q1)^T round(A2 * 2^e)) * 2^-e           (projection, A2 columns scaled)
    A2  = A2 - (round(Q1) round(R12 * 2^f)) * 2^-f        (update, R12 columns scaled)
    Q1 is not scaled for FP16/BF16 (|q| <= 1). For 'fp8' (E4M3, whose normal range starts at
    2^-6, above the ~m^-1/2 entries of Q) Q1's columns are scaled too, Q1l = round(Q1 2^s):
    R12 = 2^-s (Q1l^T A2l) 2^-e, and the update uses Q1 R12 = Q1l (2^-s R12), so R12's rows
    are divided by 2^s before its own column scaling. Returns (Q, R) in FP64.
    """
    W = np.array(A, dtype=np.float64, copy=True)
    m, n = W.shape
    R = np.zeros((n, n))

    def rec(c0: int, w: int):
        if w <= panel_width:
            Qp, Rp = tsqr(W[:, c0:c0 + w], leaf_rows, leaf)
            W[:, c0:c0 + w] = Qp
            R[c0:c0 + w, c0:c0 + w] = Rp
            return
        w1 = split_point(w, panel_width)
        rec(c0, w1)
        if prec == "fp8":
            Q1l, s = scaled_round(W[:, c0:c0 + w1], prec)
        else:
            Q1l, s = round_to(prec, W[:, c0:c0 + w1]), np.zeros(w1, dtype=np.int64)
        A2l, e = scaled_round(W[:, c0 + w1:c0 + w], prec)
        R12 = np.ldexp(np.ldexp(Q1l.T @ A2l, -e[None, :]), -s[:, None])
        R[c0:c0 + w1, c0 + w1:c0 + w] = R12
        R12l, f = scaled_round(np.ldexp(R12, -s[:, None]), prec)
        W[:, c0 + w1:c0 + w] -= np.ldexp(Q1l @ R12l, -f[None, :])
        rec(c0 + w1, w - w1)

    rec(0, n)
    return W, R


def rgsqrf_reorth(A: np.ndarray, panel_width: int = 32, prec: str = "fp16", leaf_rows: int = 256,
                  leaf: str = "cgs2"):
    """Re-orthogonalized RGSQRF: A = Q1 R1, then Q1 = Q2 R2 by the same recursion, returning
    (Q2, R2 R1). The second pass restores the orthogonality the recursion loses with growing
    condition number (the paper's remedy for ill-conditioned inputs, Sec. 4.2.1)."""
    Q1, R1 = rgsqrf(A, panel_width, prec, leaf_rows, leaf)
    Q2, R2 = rgsqrf(Q1, panel_width, prec, leaf_rows, leaf)
    return Q2, R2 @ R1
