"""Pins for the oracle's R-preconditioned CGLS (Alg. 5, corrected) and LSQR,
the backward-error measures and the least-squares adjoint."""
import math

import numpy as np
import pytest
import scipy.optimize
import scipy.sparse.linalg
import torch

from oracle import adjoint, direct, krylov, metrics, rgsqrf
from paper_1912_05508_gb300 import synth


@pytest.fixture(scope="module")
def cfg_small():
    return synth.svd_lls(512, 48, "geometric", 1e3, seed=21)


@pytest.mark.parametrize("solver", [krylov.cgls, krylov.lsqr])
def test_exact_R_converges_in_one_or_two_steps(cfg_small, solver):
    # With the exact QR, kappa(A R^{-1}) = 1 and the iteration converges at once (Sec. 3.2.3).
    p = cfg_small
    xs = direct.lls(p.A, p.b)
    _, R = direct.householder_qr(p.A)
    x, it, _ = solver(p.A, p.b, R, tol=1e-13, maxit=20)
    assert it <= 2
    assert metrics.forward_error(x, xs) < p.kappa * 1e-13   # kappa * tol


def test_identity_preconditioner_is_plain_cgls_and_matches_scipy_lsqr():
    A = synth.random_dense(300, 20, "normal", seed=22).astype(np.float64)
    b = np.random.default_rng(22).standard_normal(300)
    xs = direct.lls(A, b)
    x, it, _ = krylov.cgls(A, b, np.eye(20), tol=1e-14, maxit=200)
    ref = scipy.sparse.linalg.lsqr(A, b, atol=1e-15, btol=1e-15, iter_lim=200)
    assert metrics.forward_error(x, xs) < 1e-12
    assert metrics.forward_error(ref[0], xs) < 1e-12
    # CG on the normal equations of a 20-column operator: at most ~n steps (+ a few for rounding)
    assert it <= 30 and abs(it - ref[2]) <= 6


@pytest.mark.parametrize("solver", [krylov.cgls, krylov.lsqr])
def test_lowprec_R_reaches_fp64_backward_error(cfg_small, solver):
    p = cfg_small
    xs = direct.lls(p.A, p.b)
    _, R = rgsqrf.rgsqrf(p.A, 16, "fp16", leaf_rows=128)
    x, it, hist = solver(p.A, p.b, R, tol=1e-13, maxit=200)
    assert hist[-1] <= 1e-13 and it < 60
    assert metrics.eta_kw(p.A, p.b, x) < 1e-12
    assert metrics.forward_error(x, xs) < 1e3 * 1e-12 * 10


def test_convergence_bound(cfg_small):
    # e_k <= 2 e_0 ((k-1)/(k+1))^k in the A^T A energy norm, k = kappa(A R^{-1}) (Sec. 3.2.3;
    # the printed bound omits the factor 2 and the norm).
    p = cfg_small
    A = p.A.astype(np.float64)
    xs = direct.lls(p.A, p.b)
    _, R = rgsqrf.rgsqrf(p.A, 16, "bf16", leaf_rows=128)
    sv = np.linalg.svd(A @ np.linalg.inv(R), compute_uv=False)
    kap = sv[0] / sv[-1]
    rho = (kap - 1) / (kap + 1)
    e0 = np.linalg.norm(A @ xs)
    for k in (2, 5, 10):
        x, _, _ = krylov.cgls(p.A, p.b, R, tol=0.0, maxit=k)
        assert np.linalg.norm(A @ (x - xs)) <= 2 * e0 * rho ** k * 1.01 + 1e-13 * e0


def test_stop_quantity_is_energy_norm_error(cfg_small):
    # with the exact R, ||R^{-T} A^T r|| = ||A (x - x*)||
    p = cfg_small
    A = p.A.astype(np.float64)
    xs = direct.lls(p.A, p.b)
    _, R = direct.householder_qr(p.A)
    x = xs + 1e-4 * np.random.default_rng(0).standard_normal(48)
    s = np.linalg.solve(R.T, A.T @ (p.b - A @ x))
    assert abs(np.linalg.norm(s) - np.linalg.norm(A @ (x - xs))) < 1e-9 * np.linalg.norm(s)


# ---- backward errors -----------------------------------------------------------------

def brute_force_backward_error(A, b, x, seed):
    """min ||dA||_F s.t. (A + dA)^T (b - (A + dA) x) = 0, by SLSQP from several starts."""
    m, n = A.shape
    rng = np.random.default_rng(seed)

    def cons(d):
        M = A + d.reshape(m, n)
        return M.T @ (b - M @ x)

    best = math.inf
    for _ in range(8):
        res = scipy.optimize.minimize(lambda d: d @ d, rng.standard_normal(m * n) * 1e-3,
                                      jac=lambda d: 2 * d,
                                      constraints=[{"type": "eq", "fun": cons}], method="SLSQP",
                                      options={"ftol": 1e-16, "maxiter": 500})
        if res.success and np.linalg.norm(cons(res.x)) < 1e-10:
            best = min(best, math.sqrt(res.fun))
    return best / np.linalg.norm(A)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_error_formulas_against_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    A32 = rng.standard_normal((5, 3)).astype(np.float32)
    b = rng.standard_normal(5)
    x = direct.lls(A32, b) + 1e-3 * rng.standard_normal(3)
    opt = metrics.eta_optimal(A32, b, x)
    bf = brute_force_backward_error(A32.astype(np.float64), b, x, seed)
    kw = metrics.eta_kw(A32, b, x)
    assert abs(opt - bf) <= 1e-5 * bf
    assert abs(kw - metrics.eta_kw_eigh(A32, b, x)) <= 1e-10 * kw
    assert 0.5 * opt <= kw <= 1.0001 * opt * math.sqrt(2)


def test_backward_error_of_exact_solution_and_the_ls_floor():
    p = synth.svd_lls(1024, 128, "geometric", 1e3, seed=1)
    xs = direct.lls(p.A, p.b)
    # The exact solution, stored in FP64, has backward error ~u64 ...
    assert metrics.eta_kw(p.A, p.b, xs) < 1e-15
    # ... while the LSQR-style ratio ||A^T r|| / (||A|| ||r||) cannot go below ~u64 ||b|| / ||r||
    assert metrics.eta_ls(p.A, p.b, xs) > 1e-12
    # and both are upper-bounded relations: kw <= ls (Stewart's first bound)
    x = xs * (1 + 1e-9)
    assert metrics.eta_kw(p.A, p.b, x) <= metrics.eta_ls(p.A, p.b, x) * 1.0001


# ---- adjoint -------------------------------------------------------------------------

def test_adjoint_against_central_differences():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((8, 4))
    b = rng.standard_normal(8)

    def loss(A_, b_):
        x = direct.lls(A_, b_)
        return float(x @ x)

    x = direct.lls(A, b)
    gA, gb = adjoint.lls_grad(A, b, x, 2 * x)
    h = 1e-6
    fdA = np.zeros_like(A)
    for i in range(8):
        for j in range(4):
            E = np.zeros_like(A)
            E[i, j] = h
            fdA[i, j] = (loss(A + E, b) - loss(A - E, b)) / (2 * h)
    fdb = np.array([(loss(A, b + h * np.eye(8)[i]) - loss(A, b - h * np.eye(8)[i])) / (2 * h)
                    for i in range(8)])
    np.testing.assert_allclose(gA, fdA, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(gb, fdb, rtol=1e-6, atol=1e-8)


def test_adjoint_against_torch_autograd_lstsq():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 6))
    b = rng.standard_normal(30)
    At = torch.tensor(A, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    xt = torch.linalg.lstsq(At, bt[:, None], driver="gelsd").solution[:, 0]
    (xt * xt).sum().backward()
    x = direct.lls(A, b)
    gA, gb = adjoint.lls_grad(A, b, x, 2 * x)
    np.testing.assert_allclose(gA, At.grad.numpy(), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(gb, bt.grad.numpy(), rtol=1e-9, atol=1e-11)
