"""Pins for the oracle's FP64 Householder QR least squares (Alg. 1, Eq. qr_lls).

Every check is against something other than the oracle itself: exact rational
arithmetic, exact constructions (tests/golden), closed forms, invariants and
LAPACK via scipy.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

from golden_io import as_float, load
from oracle import direct
from paper_1912_05508_gb300 import synth


def exact_lls(Aint, bint):
    """Exact rational x* = (A^T A)^{-1} A^T b by Gaussian elimination (normal equations, Eq. ne)."""
    m, n = len(Aint), len(Aint[0])
    G = [[sum(Fraction(Aint[k][i]) * Aint[k][j] for k in range(m)) for j in range(n)] for i in range(n)]
    h = [sum(Fraction(Aint[k][i]) * bint[k] for k in range(m)) for i in range(n)]
    M = [G[i][:] + [h[i]] for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)], G


@pytest.mark.parametrize("seed,m,n", [(0, 3, 2), (1, 4, 3), (2, 5, 3), (3, 6, 4)])
def test_bruteforce_rational_tiny(seed, m, n):
    rng = np.random.default_rng(seed)
    while True:
        Aint = rng.integers(-4, 5, size=(m, n)).tolist()
        if np.linalg.matrix_rank(np.array(Aint, float)) == n:
            break
    bint = rng.integers(-5, 6, size=m).tolist()
    x_ex, G = exact_lls(Aint, bint)
    x = direct.lls(np.array(Aint, float), np.array(bint, float))
    np.testing.assert_allclose(x, [float(v) for v in x_ex], rtol=1e-12, atol=1e-12)
    Q, R = direct.householder_qr(np.array(Aint, float))
    # R^T R = A^T A exactly in rationals, so to rounding in FP64
    np.testing.assert_allclose(R.T @ R, np.array([[float(v) for v in row] for row in G]),
                               rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("name", ["lls_exact_6x3.txt", "lls_exact_9x4.txt", "lls_exact_5x1.txt"])
def test_golden_exact_construction(name):
    g = load(name)
    A, R, Q = as_float(g["A"]), as_float(g["R"]), as_float(g["Q"])
    x, b = as_float(g["x"]), as_float(g["b"])
    Qo, Ro = direct.householder_qr(A)
    np.testing.assert_allclose(Ro, R, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Qo, Q, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(direct.lls(A, b), x, rtol=1e-12, atol=1e-12)


def test_invariants_random():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((120, 37))
    b = rng.standard_normal(120)
    Q, R = direct.householder_qr(A)
    assert np.linalg.norm(A - Q @ R) <= 1e-14 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(37)) <= 1e-14
    assert np.allclose(np.tril(R, -1), 0.0) and (np.diag(R) > 0).all()
    x = direct.lls(A, b)
    # normal equations A^T (b - A x) = 0
    assert np.linalg.norm(A.T @ (b - A @ x)) <= 1e-13 * np.linalg.norm(A) ** 2 * np.linalg.norm(x)


def test_single_column_closed_form():
    rng = np.random.default_rng(5)
    a = rng.standard_normal(17)
    b = rng.standard_normal(17)
    Q, R = direct.householder_qr(a[:, None])
    assert abs(R[0, 0] - np.linalg.norm(a)) <= 1e-15 * np.linalg.norm(a)
    np.testing.assert_allclose(Q[:, 0], a / np.linalg.norm(a), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(direct.lls(a[:, None], b)[0], a @ b / (a @ a), rtol=1e-14)


def test_orthonormal_columns():
    rng = np.random.default_rng(6)
    U = synth.haar_orthonormal(rng, 40, 9)
    b = rng.standard_normal(40)
    Q, R = direct.householder_qr(U)
    np.testing.assert_allclose(R, np.eye(9), atol=1e-14)
    np.testing.assert_allclose(direct.lls(U, b), U.T @ b, atol=1e-14)


def test_upper_triangular_padded():
    R0 = synth.upper_triangular_test(6, seed=1)
    A = np.vstack([R0, np.zeros((5, 6))])
    b = np.arange(11, dtype=float)
    Q, R = direct.householder_qr(A)
    np.testing.assert_allclose(R, R0, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(direct.lls(A, b), scipy.linalg.solve_triangular(R0, b[:6]), rtol=1e-13)


def test_constructed_problem_recovers_x_true():
    # FP64 construction, no FP32 rounding: x_true is exact up to kappa * u64
    rng = synth.rng_for(3)
    U = synth.haar_orthonormal(rng, 300, 20)
    V = synth.haar_orthonormal(rng, 20, 20)
    s = synth.spectrum("geometric", 20, 1e4)
    A = (U * s) @ V.T
    x = rng.standard_normal(20)
    g = rng.standard_normal(300)
    e = g - U @ (U.T @ g)
    b = A @ x + 1e-2 * e
    xo = direct.lls(A, b)
    assert np.linalg.norm(xo - x) / np.linalg.norm(x) <= 1e4 * 1e-14


def test_library_pin_scipy():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((200, 50))
    b = rng.standard_normal(200)
    xs = scipy.linalg.lstsq(A, b)[0]
    np.testing.assert_allclose(direct.lls(A, b), xs, rtol=1e-11, atol=1e-12)
    _, Rs = scipy.linalg.qr(A, mode="economic")
    Rs = Rs * np.sign(np.diag(Rs))[:, None]
    np.testing.assert_allclose(direct.householder_qr(A)[1], Rs, rtol=1e-11, atol=1e-12)


def test_compensated_residual_beats_fp64_cancellation():
    # b = A x exactly representable pieces; the compensated residual is exact where FP64 is not
    rng = np.random.default_rng(9)
    A = rng.standard_normal((64, 8)).astype(np.float32)
    x = rng.standard_normal(8)
    exact = [sum(Fraction(float(A[i, j])) * Fraction(float(x[j])) for j in range(8)) for i in range(64)]
    b = np.array([float(v) for v in exact])
    r = direct.residual(A, x, b)
    r_ex = np.array([float(Fraction(float(b[i])) - exact[i]) for i in range(64)])
    np.testing.assert_allclose(r, r_ex, rtol=1e-10, atol=1e-30)
    u = direct.atr(A, r)
    u_ex = [sum(Fraction(float(A[i, j])) * Fraction(float(r[i])) for i in range(64)) for j in range(8)]
    np.testing.assert_allclose(u, [float(v) for v in u_ex], rtol=1e-15, atol=1e-300)


def test_bad_arguments():
    with pytest.raises(ValueError):
        direct.householder_qr(np.zeros((3, 5)))
    with pytest.raises(np.linalg.LinAlgError):
        direct.lls(np.zeros((5, 2)), np.ones(5))
