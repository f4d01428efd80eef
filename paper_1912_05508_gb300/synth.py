"""Seeded synthetic inputs shaped like the paper's least-squares workloads.

This module builds test and benchmark matrices only; it contains none of the
factorization or solver arithmetic, and both the CPU oracle tests and the
GPU path draw their inputs from it.

Matrix families follow the paper's experiment section (Sec. 4.2): i.i.d.
uniform (0,1) and (-1,1), standard normal, and A = U diag(sigma) V^T with a
prescribed condition number and a geometric, arithmetic or clustered singular
value distribution (the paper used MAGMA's generator, which is not available;
these are rebuilt from the definitions).

Conventions: every matrix is returned column-major-ready as a numpy array of
shape (m, n); callers that need Fortran order use ``np.asfortranarray``.
A is rounded to FP32 (the problem is defined for the stored FP32 A); b and
x_true are FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SPECTRA = ("geometric", "arithmetic", "cluster")


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def haar_orthonormal(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """m x n matrix with Haar-distributed orthonormal columns (FP64).

    Q factor of an m x n standard normal matrix with its columns multiplied by
    sign(diag R), which makes the distribution Haar (Mezzadri 2007).
    """
    g = rng.standard_normal((m, n))
    q, r = np.linalg.qr(g, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def spectrum(kind: str, n: int, kappa: float) -> np.ndarray:
    """Singular values sigma_1 >= ... >= sigma_n with sigma_1 / sigma_n = kappa.

    geometric : log sigma_i evenly spaced from 0 to -log kappa (matrix type 3 of Sec. 4.2)
    arithmetic: sigma_i evenly spaced from 1 to 1/kappa (type 4)
    cluster   : all ones except the smallest, which is 1/kappa (type 5)
    """
    if n == 1:
        return np.ones(1)
    i = np.arange(n, dtype=np.float64)
    if kind == "geometric":
        return kappa ** (-i / (n - 1))
    if kind == "arithmetic":
        return 1.0 - i * (1.0 - 1.0 / kappa) / (n - 1)
    if kind == "cluster":
        s = np.ones(n)
        s[-1] = 1.0 / kappa
        return s
    raise ValueError(f"unknown spectrum {kind!r}")


@dataclass
class LLSProblem:
    A: np.ndarray        # (m, n) float32
    b: np.ndarray        # (m,) float64
    x_true: np.ndarray   # (n,) float64, exact LS solution of the FP64 problem before A is rounded
    sigma: np.ndarray    # singular values used to build A
    kind: str
    kappa: float
    seed: int


def svd_lls(m: int, n: int, kind: str = "geometric", kappa: float = 1e3,
            seed: int = 1, noise: float = 1e-6) -> LLSProblem:
    """A = U diag(sigma) V^T (Haar U, V), x_true ~ N(0, I), b = A x_true + e.

    e is orthogonal to range(A) with ||e|| = noise * ||A x_true||, so x_true is
    the exact least-squares solution of the FP64 problem. A is then rounded to
    FP32; after that rounding x_true is no longer exact (perturbation of order
    kappa * u32), and exact solutions must come from solving the rounded problem.
    """
    rng = rng_for(seed)
    U = haar_orthonormal(rng, m, n)
    V = haar_orthonormal(rng, n, n)
    sig = spectrum(kind, n, kappa)
    A64 = (U * sig) @ V.T
    x = rng.standard_normal(n)
    Ax = A64 @ x
    b = Ax.copy()
    if noise > 0.0 and m > n:
        g = rng.standard_normal(m)
        w = g - U @ (U.T @ g)
        w -= U @ (U.T @ w)          # second pass keeps w orthogonal to range(U) to ~1e-16
        b = Ax + noise * np.linalg.norm(Ax) * w / np.linalg.norm(w)
    return LLSProblem(A=A64.astype(np.float32), b=b, x_true=x, sigma=sig,
                      kind=kind, kappa=kappa, seed=seed)


def random_dense(m: int, n: int, kind: str = "normal", seed: int = 0) -> np.ndarray:
    """i.i.d. matrices of Sec. 4.2 types 1 and 2: 'uniform01', 'uniform11', 'normal'."""
    rng = rng_for(seed)
    if kind == "uniform01":
        A = rng.random((m, n))
    elif kind == "uniform11":
        A = 2.0 * rng.random((m, n)) - 1.0
    elif kind == "normal":
        A = rng.standard_normal((m, n))
    else:
        raise ValueError(kind)
    return A.astype(np.float32)


def scaled_gaussian(m: int, n: int, seed: int = 11, lo: float = -2.0, hi: float = 2.0,
                    dtype=np.float32) -> np.ndarray:
    """N(0,1) entries with column j rescaled to norm 10**U(lo, hi).

    Stresses per-column range handling of the low-precision products.
    Generated column block by column block to bound host memory.
    """
    rng = rng_for(seed)
    expo = rng.uniform(lo, hi, size=n)
    A = np.empty((m, n), dtype=dtype, order="F")
    blk = max(1, min(n, (1 << 26) // max(m, 1)))
    for j0 in range(0, n, blk):
        j1 = min(n, j0 + blk)
        g = rng.standard_normal((m, j1 - j0))
        g *= (10.0 ** expo[j0:j1]) / np.linalg.norm(g, axis=0)
        A[:, j0:j1] = g
    return A


def batched_shapes(count: int = 4096, seed: int = 13, m_range=(256, 4096),
                   n_range=(16, 512), ratio: int = 4, kappa_exp=(1.0, 5.0)):
    """Rejection-sampled uneven shapes: n ~ U{n_range}, m ~ U{m_range}, kept if m >= ratio*n.

    Returns (ms, ns, kappas) as int32, int32, float64 arrays.
    """
    rng = rng_for(seed)
    ms, ns = [], []
    while len(ms) < count:
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        if m >= ratio * n:
            ms.append(m)
            ns.append(n)
    kap = 10.0 ** rng.uniform(kappa_exp[0], kappa_exp[1], size=count)
    return np.array(ms, np.int32), np.array(ns, np.int32), kap


def upper_triangular_test(n: int, seed: int = 0, diag_lo: float = 0.5) -> np.ndarray:
    """Well-conditioned upper-triangular matrix with positive diagonal (FP64)."""
    rng = rng_for(seed)
    T = np.triu(rng.standard_normal((n, n))) / math.sqrt(n)
    T[np.diag_indices(n)] = diag_lo + rng.random(n)
    return T


def svd_lls_torch(m: int, n: int, kind: str = "geometric", kappa: float = 1e3, seed: int = 2,
                  noise: float = 1e-6, device="cuda"):
    """Device-side version of ``svd_lls`` for large problems (FP64 generation with torch).

    Returns (A, b, x_true): A an (m, n) column-major FP32 device tensor (strides (1, m)),
    b and x_true FP64 device vectors. The Haar factors come from torch.linalg.qr of
    Gaussian matrices; this is input construction only.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f64 = torch.float64

    def haar(rows, cols):
        G = torch.randn(rows, cols, generator=g, dtype=f64, device=device)
        Q, R = torch.linalg.qr(G)
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1.0
        return Q * d

    U = haar(m, n)
    V = haar(n, n)
    sig = torch.from_numpy(spectrum(kind, n, kappa)).to(device=device, dtype=f64)
    A64 = (U * sig) @ V.T
    del V
    x = torch.randn(n, generator=g, dtype=f64, device=device)
    Ax = A64 @ x
    b = Ax.clone()
    if noise > 0.0 and m > n:
        w = torch.randn(m, generator=g, dtype=f64, device=device)
        w = w - U @ (U.T @ w)
        w = w - U @ (U.T @ w)
        b = Ax + noise * torch.linalg.norm(Ax) * w / torch.linalg.norm(w)
    del U
    A = torch.empty((n, m), dtype=torch.float32, device=device).t()
    A.copy_(A64)
    del A64
    torch.cuda.empty_cache()
    return A, b, x


def scaled_gaussian_torch(m: int, n: int, seed: int = 11, lo: float = -2.0, hi: float = 2.0, device="cuda"):
    """Device-side ``scaled_gaussian``: N(0, 1) entries with column j scaled to norm 10**U(lo, hi),
    as an (m, n) column-major FP32 tensor, generated 1024 columns at a time."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    A = torch.empty((n, m), dtype=torch.float32, device=device).t()
    expo = torch.empty(n, dtype=torch.float64, device=device).uniform_(lo, hi, generator=g)
    for j0 in range(0, n, 1024):
        j1 = min(n, j0 + 1024)
        blk = torch.randn((j1 - j0, m), generator=g, dtype=torch.float32, device=device)
        scale = (10.0 ** expo[j0:j1]) / torch.linalg.norm(blk.double(), dim=1)
        A[:, j0:j1] = (blk.double() * scale[:, None]).float().t()
    return A


def batched_problems_torch(count: int = 4096, seed: int = 13, m_range=(256, 4096), n_range=(16, 512),
                           kappa_exp=(1.0, 5.0), device="cuda"):
    """The uneven batch on the device: shapes from ``batched_shapes``, problem i an SVD problem
    (``svd_lls_torch``, geometric spectrum with its kappa, seed seed * 10007 + i).
    Returns (As, bs, kappas)."""
    ms, ns, kap = batched_shapes(count, seed=seed, m_range=m_range, n_range=n_range, kappa_exp=kappa_exp)
    As, bs = [], []
    for i, (m, n, k) in enumerate(zip(ms, ns, kap)):
        A, b, _ = svd_lls_torch(int(m), int(n), "geometric", float(k), seed=seed * 10007 + i, device=device)
        As.append(A)
        bs.append(b)
    return As, bs, kap
