"""GPU parity of qr_factor (Alg. 2 + Eq. caqr) against the CPU oracle, through the C ABI.

Tolerances
----------
* FP32 products: the factorization is a recursive Gram-Schmidt QR in FP32, so R matches
  the unique (positive-diagonal) FP64 R to c * kappa * u32 normwise, ||A - QR|| / ||A|| <=
  c * u32 and ||I - Q^T Q|| <= c * kappa * u32 (Sec. 3.2.1), with c ~ sqrt(n).
* FP16 / BF16 / FP8 products: the oracle runs the same recursion with the same rounding
  points in FP64. Rounding decisions can differ where the GPU's FP32 operand and the
  oracle's FP64 operand straddle a rounding boundary, so R agrees to c * u_low normwise
  (u16 = 2^-11, ubf16 = 2^-8, u8 = 2^-4 for E4M3); backward error <= 4 u_low;
  orthogonality <= c * kappa * u_low.
"""
import numpy as np
import pytest
import torch

from oracle import direct, metrics, rgsqrf
from paper_1912_05508_gb300 import lls, synth
from parity import r_entry_err

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
ULOW = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8, "fp8": 2.0 ** -4}


def svd_matrix(m, n, kappa, seed, kind="geometric"):
    return synth.svd_lls(m, n, kind, kappa, seed=seed, noise=0.0).A


def gpu_qr(A32, prec, pw=32):
    Q, R = lls.qr(lls.colmajor(A32), prec=prec, panel_width=pw)
    torch.cuda.synchronize()
    return Q.cpu().numpy().astype(np.float64), R.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,n", [(1000, 100), (4000, 32), (5000, 7), (300, 300), (257, 64)])
def test_fp32_products_match_householder(m, n):
    kappa = 1e3
    A = svd_matrix(m, n, kappa, seed=m + n)
    Q, R = gpu_qr(A, "fp32")
    Qh, Rh = direct.householder_qr(A)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert (np.diag(R) > 0).all()
    assert np.linalg.norm(R - Rh) / np.linalg.norm(Rh) <= 20 * kappa * U32 * n ** 0.5
    assert metrics.qr_factorization_error(A, Q, R) <= 10 * U32 * n ** 0.5
    # the recursion orthogonalises each right half once, so orthogonality decays like
    # kappa * u (Sec. 3.2.1), not like CGS2's O(u)
    assert metrics.orthogonality(Q, "2") <= 10 * kappa * U32 * n ** 0.5


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp8"])
@pytest.mark.parametrize("m,n,pw", [(1000, 100, 32), (2048, 256, 32), (777, 96, 16),
                                    # narrow nodes as single cooperative launches over many CTAs
                                    (20000, 96, 16), (9000, 72, 8), (12000, 256, 32)])
def test_lowprec_matches_oracle_recursion(prec, m, n, pw):
    if prec == "fp8" and pw % 16:
        pytest.skip("FP8 products take panel widths that are multiples of 16")
    kappa = 1e3
    A = svd_matrix(m, n, kappa, seed=3 * m + n)
    Q, R = gpu_qr(A, prec, pw)
    Qo, Ro = rgsqrf.rgsqrf(A, pw, prec, leaf_rows=256)
    u = ULOW[prec]
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 8 * u
    assert r_entry_err(R, Ro) <= 4 * u
    fe = metrics.qr_factorization_error(A, Q, R)
    assert fe <= 4 * u
    assert metrics.orthogonality(Q, "2") <= 4 * u * kappa * n ** 0.5
    # the oracle's own figures are of the same size (the products really are rounded)
    assert fe >= metrics.qr_factorization_error(A, Qo, Ro) / 16


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("m,n", [(40000, 64), (3000, 24), (600, 17), (20000, 48)])
def test_two_panel_blocks_match_oracle(prec, m, n):
    # The lowest recursion nodes (w1 = 16, w2 <= 16 at panel width 16) run as one launch:
    # left panel, the node's two products, right panel. m = 40000 takes four rows per thread
    # over 40 CTAs, m = 600 one CTA; n = 24 and 17 give ragged right halves, n = 48 a block
    # under a fused 32-wide node.
    kappa = 1e3
    A = svd_matrix(m, n, kappa, seed=m + 7 * n)
    Q, R = gpu_qr(A, prec, 16)
    Qo, Ro = rgsqrf.rgsqrf(A, 16, prec, leaf_rows=256)
    u = ULOW[prec]
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 8 * u
    assert r_entry_err(R, Ro) <= 4 * u
    fe = metrics.qr_factorization_error(A, Q, R)
    assert fe <= 4 * u
    assert metrics.orthogonality(Q, "2") <= 4 * u * kappa * n ** 0.5
    assert fe >= metrics.qr_factorization_error(A, Qo, Ro) / 16


def test_two_panel_block_is_one_launch():
    # At panel width 16 a 32-column factorization is one block: it takes as many launches as
    # a single 16-column panel.
    A = lls.colmajor(svd_matrix(5000, 32, 1e2, seed=5))

    def launches(n):
        An = A[:, :n]                                  # column-major view, ld 5000
        lls.qr(An, prec="fp16", panel_width=16)      # a first call may record its graph
        torch.cuda.synchronize()
        c0 = lls.lls_kernel_launch_count()
        lls.qr(An, prec="fp16", panel_width=16)
        torch.cuda.synchronize()
        return lls.lls_kernel_launch_count() - c0

    assert launches(32) == launches(16)


def test_column_scaling_handles_wide_column_range():
    # Column norms 10^U(-2, 2): without per-column scaling FP16 would lose the small columns.
    A = synth.scaled_gaussian(2000, 64, seed=11)
    Q, R = gpu_qr(A, "fp16")
    Qo, Ro = rgsqrf.rgsqrf(A, 32, "fp16")
    assert metrics.qr_factorization_error(A, Q, R) <= 4 * ULOW["fp16"]
    # columnwise relative error of A - QR stays at the FP16 level even for tiny columns
    E = A.astype(np.float64) - Q @ R
    colrel = np.linalg.norm(E, axis=0) / np.linalg.norm(A.astype(np.float64), axis=0)
    assert colrel.max() <= 16 * ULOW["fp16"]
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 8 * ULOW["fp16"]
    assert r_entry_err(R, Ro) <= 4 * ULOW["fp16"]


@pytest.mark.parametrize("pw", [16, 32])
def test_column_scaling_in_every_node_width(pw):
    # n = 256 puts nodes of w1 = 16/32/64 (one cooperative launch each) and w1 = 128 (the
    # tensor-core path) into one factorization. With column norms over twelve decades (beyond
    # FP16's range, subnormals included) a column scaled by another column's exponent loses
    # its low-precision copy; the R12 entries of that column, and the orthogonality of the
    # next Q, are then off by several u16 (the oracle with that mistake planted gives 5.5 and
    # 6 u16; the oracle itself 0.1 and 0.24 u16).
    A = synth.scaled_gaussian(9000, 256, seed=12, lo=-6.0, hi=6.0)
    Q, R = gpu_qr(A, "fp16", pw)
    Qo, Ro = rgsqrf.rgsqrf(A, pw, "fp16", leaf_rows=256)
    colrel = np.linalg.norm(R - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert colrel.max() <= 2 * ULOW["fp16"]
    assert r_entry_err(R, Ro) <= 2 * ULOW["fp16"]
    assert metrics.orthogonality(Q, "2") <= 2 * ULOW["fp16"]


def test_rank_deficient_column_gives_zero_diagonal():
    A = svd_matrix(600, 40, 10.0, seed=5)
    A[:, 17] = 0.0
    _, R = gpu_qr(A, "fp32")
    assert abs(R[17, 17]) <= 1e-6 * np.abs(np.diag(R)).max()


def test_q_optional_and_repeatable():
    A = svd_matrix(1500, 96, 1e2, seed=9)
    Ad = lls.colmajor(A)
    _, R1 = lls.qr(Ad, prec="fp16", want_q=False)
    _, R2 = lls.qr(Ad, prec="fp16", want_q=False)
    torch.cuda.synchronize()
    assert torch.equal(R1, R2)     # fixed reduction order: bitwise repeatable


@pytest.mark.parametrize("prec,u", [("fp32", U32), ("fp16", 2.0 ** -11)])
def test_reorth_restores_orthogonality(prec, u):
    # with the recursion's single projection per node, orthogonality decays with kappa; the
    # second pass brings it back to the product precision (oracle: oracle.rgsqrf.rgsqrf_reorth)
    kappa = 1e5 if prec == "fp32" else 1e3
    A = svd_matrix(2000, 128, kappa, seed=44)
    Q1, R1 = lls.qr(lls.colmajor(A), prec=prec, panel_width=16)
    Q2, R2 = lls.qr(lls.colmajor(A), prec=prec, panel_width=16, reorth=1)
    torch.cuda.synchronize()
    Q1, Q2 = Q1.cpu().numpy().astype(np.float64), Q2.cpu().numpy().astype(np.float64)
    R2 = R2.cpu().numpy().astype(np.float64)
    o1, o2 = metrics.orthogonality(Q1, "2"), metrics.orthogonality(Q2, "2")
    assert o2 < o1 / 10
    assert o2 <= 16 * u * 128 ** 0.5
    assert metrics.qr_factorization_error(A, Q2, R2) <= 16 * u * 128 ** 0.5
    assert np.allclose(np.tril(R2, -1), 0.0)


# ---- the paper's MGS leaf (Alg. 4) as the panel factorization (opts.panel_leaf = 1) ----

def graded(m, n, seed, kappa):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = kappa ** (-np.arange(n) / max(n - 1, 1))
    return ((U * s) @ V.T).astype(np.float32)


@pytest.mark.parametrize("m,b,kappa", [(3000, 16, 1e2), (32768, 16, 1e4), (65536, 13, 1e3), (4100, 8, 1e5)])
def test_mgs_panel_matches_oracle_mgs_tsqr(m, b, kappa):
    # one panel (n = panel width): CAQR with MGS leaves. MGS loses orthogonality like
    # kappa * u (CGS2 does not), so Q is bounded by c kappa u32; R is the unique
    # positive-diagonal factor, equal to the oracle's to c kappa u32 normwise.
    A = graded(m, b, m + b, kappa)
    Q, R = lls.qr(lls.colmajor(A), prec="fp32", panel_width=b, panel_leaf="mgs")
    torch.cuda.synchronize()
    Q, R = Q.cpu().numpy().astype(np.float64), R.cpu().numpy().astype(np.float64)
    A64 = A.astype(np.float64)
    Qo, Ro = rgsqrf.tsqr(A64, leaf_rows=1024, leaf="mgs")
    assert np.allclose(np.tril(R, -1), 0.0) and (np.diag(R) > 0).all()
    assert metrics.qr_factorization_error(A64, Q, R) <= 8 * b * U32
    assert metrics.orthogonality(Q, "2") <= 16 * b * kappa * U32
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 4 * np.sqrt(b) * kappa * U32 + 4 * b * U32
    assert r_entry_err(R, Ro) <= 4 * np.sqrt(b) * kappa * U32 + 4 * b * U32


def test_cgs2_panel_keeps_orthogonality_where_mgs_loses_it():
    A = graded(32768, 16, 5, 1e6)
    Qc, _ = lls.qr(lls.colmajor(A), prec="fp32", panel_width=16)
    Qm, _ = lls.qr(lls.colmajor(A), prec="fp32", panel_width=16, panel_leaf="mgs")
    torch.cuda.synchronize()
    oc = metrics.orthogonality(Qc.cpu().numpy().astype(np.float64), "2")
    om = metrics.orthogonality(Qm.cpu().numpy().astype(np.float64), "2")
    assert oc <= 64 * U32
    assert om > 100 * oc        # MGS: ~kappa u32


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_mgs_leaves_in_the_recursion_match_oracle(prec):
    A = svd_matrix(6000, 128, 1e3, seed=31)
    Q, R = lls.qr(lls.colmajor(A), prec=prec, panel_width=16, panel_leaf="mgs")
    torch.cuda.synchronize()
    Q, R = Q.cpu().numpy().astype(np.float64), R.cpu().numpy().astype(np.float64)
    Qo, Ro = rgsqrf.rgsqrf(A, 16, prec, leaf_rows=256, leaf="mgs")
    u = ULOW[prec]
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 8 * u
    assert r_entry_err(R, Ro) <= 4 * u
    assert metrics.qr_factorization_error(A, Q, R) <= 4 * u


def test_mgs_leaves_solve_to_fp64_target():
    p = synth.svd_lls(4096, 96, "geometric", 1e3, seed=33)
    x, info = lls.solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda(), panel_width=16, panel_leaf="mgs")
    assert info["status"] == 0, info
    xs = direct.lls(p.A, p.b)
    assert metrics.eta_kw(p.A, p.b, x.cpu().numpy()) <= 1e-12
    assert metrics.forward_error(x.cpu().numpy(), xs) <= 10 * p.kappa * 1e-12


def test_mgs_leaves_unsupported_where_built_for_cgs2_only():
    # a panel taller than one tree level (m > 65536 at width 16) and the batched solver
    A = torch.zeros((16, 70000), device="cuda").t()
    with pytest.raises(lls.LLSError) as e:
        lls.qr(A, prec="fp32", panel_width=16, panel_leaf="mgs")
    assert e.value.status == -6
    o = lls.make_options(panel_leaf="mgs", target="fp32")
    nb = lls.lls_solve_batched_workspace_size(1, [256], [16], o)
    ws = lls.workspace(max(nb, 1 << 20))
    Ab = torch.randn((16, 256), device="cuda").t()
    bb = torch.randn(256, dtype=torch.float64, device="cuda")
    xb = torch.empty(16, dtype=torch.float64, device="cuda")
    infos = (lls.lls_info * 1)()
    st = lls.lls_solve_batched(1, [256], [16], [Ab.data_ptr()], [256], [bb.data_ptr()], [xb.data_ptr()], None,
                               None, ws.data_ptr(), ws.numel(), o, infos, torch.cuda.current_stream().cuda_stream)
    assert st == -6
