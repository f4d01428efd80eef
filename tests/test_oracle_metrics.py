"""Pins for the oracle's accuracy measures (oracle/metrics.py; Sec. 3.2.1 and 3.2.2).

Each measure is checked against a closed form it must reproduce on a constructed input, or
against an independent library route (SVD-based 2-norms), never against its own formula.
"""
import numpy as np
import pytest

from oracle import direct, metrics


def _orthonormal(rng, m, n):
    Q, _ = np.linalg.qr(rng.standard_normal((m, n)))
    return Q


@pytest.mark.parametrize("seed,m,n", [(0, 40, 7), (1, 90, 12), (2, 12, 12)])
def test_norm2_est_random_against_svd(seed, m, n):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    est = metrics.norm2_est(lambda v: A @ v, lambda w: A.T @ w, n, iters=200)
    assert est == pytest.approx(np.linalg.svd(A, compute_uv=False)[0], rel=1e-8)


def test_norm2_est_rank_one_closed_form():
    # ||u v^T||_2 = ||u|| ||v||, and one power step already lands on v
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(30), rng.standard_normal(9)
    A = np.outer(u, v)
    est = metrics.norm2_est(lambda z: A @ z, lambda w: A.T @ w, 9)
    assert est == pytest.approx(np.linalg.norm(u) * np.linalg.norm(v), rel=1e-13)


def test_norm2_est_diagonal_and_zero():
    d = np.array([0.5, -3.0, 2.0, 1e-3])
    D = np.diag(d)
    est = metrics.norm2_est(lambda z: D @ z, lambda w: D.T @ w, 4, iters=200)
    assert est == pytest.approx(3.0, rel=1e-10)
    Z = np.zeros((5, 3))
    assert metrics.norm2_est(lambda z: Z @ z, lambda w: Z.T @ w, 3) == 0.0


def test_qr_factorization_error_planted_entry_closed_form():
    # A = Q R exactly (to rounding); R' = R + delta e_i e_j^T gives A - Q R' = -delta q_i e_j^T,
    # whose 2-norm and F-norm are both |delta| (q_i is a unit vector)
    rng = np.random.default_rng(4)
    A = rng.standard_normal((60, 8))
    Q, R = direct.householder_qr(A)
    delta = 3e-4
    Rp = R.copy()
    Rp[2, 5] += delta
    a2 = np.linalg.svd(A, compute_uv=False)[0]
    got2 = metrics.qr_factorization_error(A, Q, Rp, norm="2")
    # ||E||_2 is exact (rank one); ||A||_2 by 30 power steps is a lower bound within 1 %
    # for this spectrum, so the ratio is at least the true one and at most 1 % above it
    assert delta / a2 * (1 - 1e-12) <= got2 <= 1.01 * delta / a2
    gotf = metrics.qr_factorization_error(A, Q, Rp, norm="fro")
    assert gotf == pytest.approx(delta / np.linalg.norm(A), rel=1e-6)
    assert metrics.qr_factorization_error(A, Q, R, norm="2") <= 1e-14


@pytest.mark.parametrize("norm", ["2", "perN", "fro"])
def test_orthogonality_scaled_columns_closed_form(norm):
    # Q = U diag(d) with orthonormal U: Q^T Q = diag(d^2), so I - Q^T Q = diag(1 - d^2)
    rng = np.random.default_rng(5)
    n = 6
    U = _orthonormal(rng, 50, n)
    d = np.array([1.0, 1.0 + 1e-3, 1.0 - 2e-3, 1.0, 1.0 + 5e-4, 1.0])
    Q = U * d
    g = np.abs(1.0 - d * d)
    want = {"2": g.max(), "perN": g.max() / n, "fro": np.sqrt((g * g).sum())}[norm]
    assert metrics.orthogonality(Q, norm=norm) == pytest.approx(want, rel=1e-9)


def test_orthogonality_perN_off_diagonal():
    # two unit columns at angle theta: I - Q^T Q = [[0, -c], [-c, 0]], 2-norm |c| = |cos theta|
    th = 1.2
    Q = np.array([[1.0, np.cos(th)], [0.0, np.sin(th)], [0.0, 0.0]])
    assert metrics.orthogonality(Q, norm="perN") == pytest.approx(abs(np.cos(th)) / 2, rel=1e-13)


def test_eta_consistent_closed_form():
    # A = [I; 0], b = [x; c]: r = b - A x = [0; c] exactly, ||A||_F = sqrt(n)
    n, m = 4, 9
    A = np.zeros((m, n), dtype=np.float32)
    A[:n, :n] = np.eye(n)
    x = np.array([1.0, -2.0, 0.5, 3.0])
    c = np.array([0.25, -1.0, 0.0, 2.0, 0.5])
    b = np.concatenate([x, c])
    want = np.linalg.norm(c) / (np.sqrt(n) * np.linalg.norm(x) + np.linalg.norm(b))
    assert metrics.eta_consistent(A, b, x) == pytest.approx(want, rel=1e-14)
    # a compatible system solved exactly has zero backward error
    assert metrics.eta_consistent(A, np.concatenate([x, np.zeros(m - n)]), x) == 0.0


def test_eta_consistent_bounds_the_optimal_backward_error_when_compatible():
    # for a nearly compatible system the consistent-case measure and the exact optimal
    # least-squares backward error (Walden-Karlson-Sun) agree to within a factor of a few
    rng = np.random.default_rng(6)
    A = rng.standard_normal((30, 5)).astype(np.float32)
    x = rng.standard_normal(5)
    b = A.astype(np.float64) @ x
    xp = x + 1e-9 * rng.standard_normal(5)
    ec = metrics.eta_consistent(A, b, xp)
    eo = metrics.eta_optimal(A, b, xp)
    assert 0.0 < eo <= 10 * ec and ec <= 10 * eo
