"""Sensitivity of the oracle's pins: each test plants one plausible mistake in a copy of an
oracle step, on the CPU (a dropped term, a wrong sign, a wrong index, a transposed scale, a
typo of the printed listing), and checks that the predicate of the pin guarding that step
rejects the mutant while the unmodified oracle passes it.

The predicates are those of tests/test_oracle_rgsqrf.py, tests/test_oracle_krylov.py and
tests/test_oracle_direct.py; one more pin is added here: the recursion keeps a columnwise
backward error at the low-precision level for columns whose norms span twelve decades
(power-of-two column scaling, Sec. 3.1.2 range discussion).
"""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint, direct, krylov, metrics, rgsqrf
from oracle.lowprec import round_fp16, round_to, scaled_round
from paper_1912_05508_gb300 import synth

U16 = 2.0 ** -11


def ill_conditioned(m, n, kappa, seed):
    rng = synth.rng_for(seed)
    U = synth.haar_orthonormal(rng, m, n)
    V = synth.haar_orthonormal(rng, n, n)
    return (U * synth.spectrum("geometric", n, kappa)) @ V.T


# ---- Gram-Schmidt leaf: the second projection dropped -------------------------------------

def cgs1(A):
    """CGS2 with its reorthogonalization dropped (classical Gram-Schmidt)."""
    A = np.asarray(A, dtype=np.float64)
    m, b = A.shape
    Q, R = np.zeros((m, b)), np.zeros((b, b))
    for k in range(b):
        a = A[:, k].copy()
        h = Q[:, :k].T @ a
        a -= Q[:, :k] @ h
        R[:k, k] = h
        R[k, k] = math.sqrt(float(a @ a))
        Q[:, k] = a / R[k, k]
    return Q, R


def test_dropped_reorthogonalization_fails_the_orthogonality_pin():
    A = ill_conditioned(400, 24, 1e10, seed=4)
    pin = lambda Q: metrics.orthogonality(Q, "2") < 1e-14       # test_cgs2_keeps_orthogonality...
    assert pin(rgsqrf.cgs2(A)[0])
    assert not pin(cgs1(A)[0])


# ---- CAQR panel: the wrong slice of the stack's Q (step 4 of Eq. caqr) -------------------

def tsqr_wrong_slice(A, leaf_rows):
    m, b = A.shape
    blocks = rgsqrf.row_blocks(m, leaf_rows)
    factors = [rgsqrf.cgs2(A[s:e]) for s, e in blocks]
    Q2, R = rgsqrf.tsqr(np.vstack([R for _, R in factors]), leaf_rows)
    p = len(blocks)
    Q = np.vstack([Qi @ Q2[((i + 1) % p) * b:((i + 1) % p + 1) * b] for i, (Qi, _) in enumerate(factors)])
    return Q, R


def test_wrong_stack_slice_fails_the_tsqr_pin():
    A = ill_conditioned(4000, 32, 1e3, seed=4000)
    Qh, _ = direct.householder_qr(A)
    pin = lambda Q: np.allclose(Q, Qh, atol=1e-11) and metrics.orthogonality(Q, "2") < 1e-13
    assert pin(rgsqrf.tsqr(A, 256)[0])
    assert not pin(tsqr_wrong_slice(A, 256)[0])


# ---- the recursion (Alg. 2): sign of the update, the scale exponents ---------------------

def rgsqrf_mutant(A, panel_width, prec, mutation):
    """The oracle's recursion (FP16/BF16/FP64 products) with one mistake planted."""
    W = np.array(A, dtype=np.float64, copy=True)
    m, n = W.shape
    R = np.zeros((n, n))

    def rec(c0, w):
        if w <= panel_width:
            Qp, Rp = rgsqrf.tsqr(W[:, c0:c0 + w], 256)
            W[:, c0:c0 + w] = Qp
            R[c0:c0 + w, c0:c0 + w] = Rp
            return
        w1 = rgsqrf.split_point(w, panel_width)
        rec(c0, w1)
        Q1l = round_to(prec, W[:, c0:c0 + w1])
        A2l, e = scaled_round(W[:, c0 + w1:c0 + w], prec)
        if mutation == "exponent_of_another_column":
            e_un = np.roll(e, 1)
        else:
            e_un = e
        R12 = np.ldexp(Q1l.T @ A2l, -e_un[None, :])
        R[c0:c0 + w1, c0 + w1:c0 + w] = R12
        R12l, f = scaled_round(R12, prec)
        upd = Q1l @ R12l
        if mutation != "unscale_of_the_update_dropped":
            upd = np.ldexp(upd, -f[None, :])
        if mutation == "update_sign":
            W[:, c0 + w1:c0 + w] += upd
        else:
            W[:, c0 + w1:c0 + w] -= upd
        rec(c0 + w1, w - w1)

    rec(0, n)
    return W, R


def test_update_sign_fails_the_exact_products_pin():
    A = ill_conditioned(700, 100, 1e4, seed=100)
    _, Rh = direct.householder_qr(A)
    pin = lambda R: np.linalg.norm(R - Rh) <= 1e-11 * np.linalg.norm(Rh)   # test_rgsqrf_exact_products...
    assert pin(rgsqrf.rgsqrf(A, 32, "fp64", leaf_rows=256)[1])
    assert pin(rgsqrf_mutant(A, 32, "fp64", "none")[1])                    # the copy itself is faithful
    assert not pin(rgsqrf_mutant(A, 32, "fp64", "update_sign")[1])


def test_dropped_unscale_fails_the_low_precision_pin():
    A = ill_conditioned(1024, 96, 1e3, seed=7)
    pin = lambda Q, R: metrics.qr_factorization_error(A, Q, R) < 4 * U16   # test_rgsqrf_low_precision...
    assert pin(*rgsqrf.rgsqrf(A, 32, "fp16", leaf_rows=256))
    assert not pin(*rgsqrf_mutant(A, 32, "fp16", "unscale_of_the_update_dropped"))


def columnwise_backward_error(A, Q, R):
    E = np.asarray(A, dtype=np.float64) - Q @ R
    return float((np.linalg.norm(E, axis=0) / np.linalg.norm(A, axis=0)).max())


def test_recursion_keeps_columnwise_error_over_twelve_decades_of_column_norms():
    # The added pin: with per-column power-of-two scaling, every column of A - QR is small
    # relative to its own column, even for column norms from 1e-6 to 1e6 (FP16's normal range
    # alone spans about 2^-14 .. 2^16). A column scaled by another column's exponent loses
    # its low-precision copy and fails it.
    A = synth.scaled_gaussian(1500, 64, seed=12, lo=-6.0, hi=6.0).astype(np.float64)
    Q, R = rgsqrf.rgsqrf(A, 16, "fp16", leaf_rows=256)
    assert columnwise_backward_error(A, Q, R) <= 16 * U16
    Qm, Rm = rgsqrf_mutant(A, 16, "fp16", "exponent_of_another_column")
    assert columnwise_backward_error(A, Qm, Rm) > 16 * U16


# ---- rounding: truncation instead of round-to-nearest-even --------------------------------

def test_truncating_cast_fails_the_rounding_pin():
    x = np.random.default_rng(5).standard_normal(20000) * np.exp2(np.random.default_rng(6).integers(-12, 12, 20000))
    ref = torch.from_numpy(x).to(torch.float16).double().numpy()
    trunc = x.astype(np.float16)
    away = np.abs(trunc.astype(np.float64)) > np.abs(x)
    trunc[away] = np.nextafter(trunc[away], np.float16(0))
    assert np.array_equal(round_fp16(x), ref)                           # test_round_fp16_matches_torch_cast
    assert not np.array_equal(trunc.astype(np.float64), ref)


# ---- preconditioned CGLS (Alg. 5): the printed step length, x updated with p -------------

def cgls_mutant(A, b, R, mutation, tol=1e-13, maxit=20):
    with np.errstate(over="ignore", invalid="ignore"):    # a mutant may diverge
        return _cgls_mutant(A, b, R, mutation, tol, maxit)


def _cgls_mutant(A, b, R, mutation, tol, maxit):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    anorm = np.linalg.norm(A)
    x = np.zeros(n)
    r = b.astype(np.float64).copy()
    s = krylov._rinvT(R, A.T @ r)
    p = s.copy()
    gamma = gamma_prev = float(s @ s)
    it = 0
    for it in range(1, maxit + 1):
        if not (np.isfinite(p).all() and math.isfinite(gamma)):
            break                                          # a diverging mutant stops here
        t = krylov._rinv(R, p)
        q = A @ t
        delta = float(q @ q)
        alpha = gamma / gamma_prev if mutation == "printed_step_length" else gamma / delta
        x += alpha * (p if mutation == "x_updated_with_p" else t)
        r -= alpha * q
        if not np.isfinite(r).all():
            break
        s = krylov._rinvT(R, A.T @ r)
        gamma_prev, gamma = gamma, float(s @ s)
        xn = np.linalg.norm(x)
        if xn > 0 and math.sqrt(gamma) / (anorm * xn) <= tol:
            break
        beta = gamma_prev / gamma if mutation == "inverted_beta" else gamma / gamma_prev
        p = s + beta * p
    return x, it


@pytest.fixture(scope="module")
def cfg_small():
    return synth.svd_lls(512, 48, "geometric", 1e3, seed=21)


def test_x_updated_with_p_fails_the_exact_R_pin(cfg_small):
    # test_exact_R_converges_in_one_or_two_steps: with the exact R, <= 2 iterations and a
    # forward error below kappa * tol
    p = cfg_small
    xs = direct.lls(p.A, p.b)
    _, R = direct.householder_qr(p.A)
    pin = lambda x, it: it <= 2 and metrics.forward_error(x, xs) < p.kappa * 1e-13
    assert pin(*cgls_mutant(p.A, p.b, R, "none"))
    assert pin(*krylov.cgls(p.A, p.b, R, tol=1e-13, maxit=20)[:2])
    assert not pin(*cgls_mutant(p.A, p.b, R, "x_updated_with_p"))


def test_printed_step_length_fails_the_low_precision_R_pin(cfg_small):
    # With the exact R, A R^-1 is orthonormal, delta = gamma and the printed step length
    # gamma / gamma_prev is 1, the right value, on the first step: the exact-R pin cannot see
    # this slip. With the FP16-product R of the recursion it can
    # (test_lowprec_R_reaches_fp64_backward_error: eta_kw < 1e-12 within 60 iterations).
    p = cfg_small
    xs = direct.lls(p.A, p.b)
    _, R = rgsqrf.rgsqrf(p.A, 16, "fp16", leaf_rows=128)
    def pin(x, it):
        with np.errstate(over="ignore"):
            if not (it < 60 and np.isfinite(x).all() and np.linalg.norm(x) < 1e100):
                return False
        return metrics.eta_kw(p.A, p.b, x) < 1e-12 and metrics.forward_error(x, xs) < 1e3 * 1e-12 * 10

    assert pin(*cgls_mutant(p.A, p.b, R, "none", maxit=200))
    assert not pin(*cgls_mutant(p.A, p.b, R, "printed_step_length", maxit=200))


def test_inverted_beta_fails_the_plain_cgls_pin():
    # test_identity_preconditioner_is_plain_cgls...: R = I converges within ~n steps
    A = synth.random_dense(300, 20, "normal", seed=22).astype(np.float64)
    b = np.random.default_rng(22).standard_normal(300)
    xs = direct.lls(A, b)
    pin = lambda x, it: it <= 30 and metrics.forward_error(x, xs) < 1e-12
    assert pin(*cgls_mutant(A, b, np.eye(20), "none", tol=1e-14, maxit=200))
    assert not pin(*cgls_mutant(A, b, np.eye(20), "inverted_beta", tol=1e-14, maxit=200))


# ---- the adjoint: the sign of the second rank-1 term ---------------------------------------

def test_adjoint_sign_mistake_fails_the_central_difference_pin():
    rng = np.random.default_rng(31)
    A = rng.standard_normal((8, 4))
    b = rng.standard_normal(8)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    g = 2 * x                                              # L = sum of squares of x
    gA, gb = adjoint.lls_grad(A, b, x, g)
    z = np.linalg.solve(A.T @ A, g)
    r = b - A @ x
    gA_mut = np.outer(r, z) + np.outer(A @ z, x)            # sign of the second term flipped
    L = lambda AA: float(np.sum(np.linalg.lstsq(AA, b, rcond=None)[0] ** 2))
    h = 1e-6 * np.linalg.norm(A)
    fd = np.zeros_like(A)
    for i in range(A.shape[0]):
        for j in range(A.shape[1]):
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h
            Am[i, j] -= h
            fd[i, j] = (L(Ap) - L(Am)) / (2 * h)
    pin = lambda G: np.linalg.norm(G - fd) <= 1e-6 * np.linalg.norm(fd)
    assert pin(gA)
    assert not pin(gA_mut)
