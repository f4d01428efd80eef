"""Pins for the oracle's recursive Gram-Schmidt QR (Alg. 2), CAQR panel (Eq. caqr),
CGS2 / MGS leaves (Alg. 4) and the low-precision rounding operations."""
import numpy as np
import pytest
import torch

from oracle import direct, metrics, rgsqrf
from oracle.lowprec import column_scale_exponents, round_bf16, round_fp8_e4m3, round_fp16, scaled_round
from paper_1912_05508_gb300 import synth


def ill_conditioned(m, n, kappa, seed):
    rng = synth.rng_for(seed)
    U = synth.haar_orthonormal(rng, m, n)
    V = synth.haar_orthonormal(rng, n, n)
    return (U * synth.spectrum("geometric", n, kappa)) @ V.T


# ---- rounding operations -------------------------------------------------------------

def test_round_fp16_matches_torch_cast():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-9, 5, 20000),
                        [65504.0, 65520.0, 6.0e-8, 2.0 ** -25, -0.0]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float64).numpy()
    got = round_fp16(x.astype(np.float64))
    assert np.array_equal(np.isinf(ref), np.isinf(got))
    fin = np.isfinite(ref)
    assert np.array_equal(ref[fin], got[fin])


def test_round_bf16_matches_torch_cast():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)).astype(np.float32)
    # exact ties: 1 + 2^-8 (odd neighbour below? no: 1.0 is even) and 1 + 3*2^-8
    x = np.concatenate([x, np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)], np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(round_bf16(x.astype(np.float64)), ref)
    assert round_bf16(np.array([1 + 2 ** -8]))[0] == 1.0           # tie to even (down)
    assert round_bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6  # tie to even (up)


def test_round_fp8_e4m3_matches_torch_cast():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(20000) * 10.0 ** rng.uniform(-4, 2.5, 20000)
    x = x[np.abs(x) < 440.0]
    x = np.concatenate([x, [448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -6, 0.0]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(round_fp8_e4m3(x32.astype(np.float64)), ref)
    # ties to even: 1 + 2^-4 lies halfway between 1 and 1 + 2^-3
    assert round_fp8_e4m3(np.array([1 + 2 ** -4]))[0] == 1.0
    assert round_fp8_e4m3(np.array([1 + 3 * 2 ** -4]))[0] == 1 + 2 ** -2
    # saturation (the GPU conversion's satfinite mode) instead of NaN
    assert np.array_equal(round_fp8_e4m3(np.array([500.0, -1e9])), np.array([448.0, -448.0]))


def test_column_scale_fp8_range():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((64, 30)) * 10.0 ** rng.uniform(-10, 10, 30)
    e = column_scale_exponents(X, "fp8")
    mx = np.abs(np.ldexp(X, e[None, :])).max(axis=0)
    assert ((mx >= 2.0 ** 7) & (mx < 2.0 ** 8)).all()
    Xl, _ = scaled_round(X, "fp8")
    np.testing.assert_allclose(np.ldexp(Xl, -e[None, :]), X, rtol=2.0 ** -4, atol=0)


def test_column_scale_is_exact_power_of_two_in_range():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((50, 40)) * 10.0 ** rng.uniform(-12, 12, 40)
    X[:, 3] = 0.0
    e = column_scale_exponents(X, "fp16")
    mx = np.abs(np.ldexp(X, e[None, :])).max(axis=0)
    nz = mx > 0
    assert ((mx[nz] >= 2.0 ** 14) & (mx[nz] < 2.0 ** 15)).all()
    assert e[3] == 0
    # scaling changes no significand bit: unscaling the rounded value is exact
    Xl, e2 = scaled_round(X, "fp16")
    assert np.array_equal(e, e2)
    back = np.ldexp(Xl, -e[None, :])
    np.testing.assert_allclose(back, X, rtol=2.0 ** -11, atol=0)
    assert np.array_equal(column_scale_exponents(X, "bf16"), np.zeros(40, dtype=np.int64))


# ---- Gram-Schmidt leaves -------------------------------------------------------------

@pytest.mark.parametrize("leaf", ["cgs2", "mgs"])
def test_leaf_matches_householder_well_conditioned(leaf):
    A = synth.random_dense(300, 16, "normal", seed=3).astype(np.float64)
    Q, R = rgsqrf.LEAVES[leaf](A)
    Qh, Rh = direct.householder_qr(A)
    np.testing.assert_allclose(R, Rh, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Q, Qh, rtol=1e-11, atol=1e-12)


def test_cgs2_keeps_orthogonality_where_mgs_loses_it():
    # MGS orthogonality loss grows like kappa * u (Bjorck 1967, cited in Sec. 3.2.1);
    # CGS2 keeps it at O(u) while kappa * u < 1. CGS without the second pass would lose ~kappa^2 u.
    A = ill_conditioned(400, 24, 1e10, seed=4)
    Qc, Rc = rgsqrf.cgs2(A)
    Qm, Rm = rgsqrf.mgs(A)
    assert metrics.orthogonality(Qc, "2") < 1e-14
    assert metrics.orthogonality(Qm, "2") > 1e-9
    assert metrics.qr_factorization_error(A, Qc, Rc) < 1e-15 * 24
    assert metrics.qr_factorization_error(A, Qm, Rm) < 1e-15 * 24


def test_cgs2_zero_column():
    A = np.zeros((10, 3))
    A[:, 0] = 1.0
    A[:, 2] = np.arange(10.0)
    Q, R = rgsqrf.cgs2(A)
    assert R[1, 1] == 0.0 and np.all(Q[:, 1] == 0.0)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)


# ---- CAQR panel ----------------------------------------------------------------------

def test_row_blocks_balanced_and_cover():
    for m in (1, 255, 256, 257, 1000, 4097):
        b = rgsqrf.row_blocks(m, 256)
        assert b[0][0] == 0 and b[-1][1] == m
        assert all(b[i][1] == b[i + 1][0] for i in range(len(b) - 1))
        sizes = [e - s for s, e in b]
        assert max(sizes) - min(sizes) <= 1 and max(sizes) <= 256


@pytest.mark.parametrize("m,b,leaf_rows", [(4000, 32, 256), (1000, 7, 64), (300, 32, 64)])
def test_tsqr_equals_unique_qr(m, b, leaf_rows):
    A = ill_conditioned(m, b, 1e3, seed=m)
    Q, R = rgsqrf.tsqr(A, leaf_rows)
    Qh, Rh = direct.householder_qr(A)
    np.testing.assert_allclose(R, Rh, rtol=0, atol=1e-13 * np.abs(Rh).max() * 1e3)
    assert metrics.orthogonality(Q, "2") < 1e-13
    np.testing.assert_allclose(Q, Qh, atol=1e-11)


# ---- recursion (Alg. 2) --------------------------------------------------------------

def test_split_point():
    assert rgsqrf.split_point(128, 32) == 64
    assert rgsqrf.split_point(96, 32) == 64
    assert rgsqrf.split_point(33, 32) == 32
    assert rgsqrf.split_point(4096, 32) == 2048


@pytest.mark.parametrize("n,pw", [(128, 32), (100, 32), (45, 16)])
def test_rgsqrf_exact_products_is_the_qr(n, pw):
    A = ill_conditioned(700, n, 1e4, seed=n)
    Q, R = rgsqrf.rgsqrf(A, pw, "fp64", leaf_rows=128)
    Qh, Rh = direct.householder_qr(A)
    assert np.linalg.norm(R - Rh) <= 1e-11 * np.linalg.norm(Rh)
    assert metrics.qr_factorization_error(A, Q, R) < 1e-14
    assert np.allclose(np.tril(R, -1), 0.0) and (np.diag(R) > 0).all()


@pytest.mark.parametrize("prec,u", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8), ("fp8", 2.0 ** -4)])
def test_rgsqrf_low_precision_error_scales_with_unit_roundoff(prec, u):
    # Backward error stays at the GEMM precision independent of kappa, orthogonality
    # loss grows with kappa (Sec. 3.2.1, Fig. qr_accu discussion).
    e_prev = None
    for kappa in (1e1, 1e3):
        A = ill_conditioned(1024, 96, kappa, seed=7)
        Q, R = rgsqrf.rgsqrf(A, 32, prec, leaf_rows=256)
        fe = metrics.qr_factorization_error(A, Q, R)
        orth = metrics.orthogonality(Q, "2")
        assert u / 64 < fe < 4 * u
        assert orth < 4 * u * kappa * 96 ** 0.5
        if e_prev is not None:
            assert orth > e_prev           # loses orthogonality as kappa grows
        e_prev = orth


def test_reorth_exact_products_is_the_qr():
    A = ill_conditioned(600, 80, 1e6, seed=21)
    Q, R = rgsqrf.rgsqrf_reorth(A, 16, "fp64", leaf_rows=128)
    Qh, Rh = direct.householder_qr(A)
    assert np.linalg.norm(R - Rh) <= 1e-9 * np.linalg.norm(Rh)
    assert metrics.orthogonality(Q) < 1e-14


def test_reorth_restores_orthogonality_of_low_precision_factors():
    A = ill_conditioned(1024, 96, 1e3, seed=22)
    Q1, R1 = rgsqrf.rgsqrf(A, 32, "fp16", leaf_rows=256)
    Q2, R2 = rgsqrf.rgsqrf_reorth(A, 32, "fp16", leaf_rows=256)
    o1, o2 = metrics.orthogonality(Q1, "2"), metrics.orthogonality(Q2, "2")
    assert o2 < o1 / 20
    assert o2 < 8 * 2.0 ** -11 * 96 ** 0.5
    assert metrics.qr_factorization_error(A, Q2, R2) < 8 * 2.0 ** -11
