"""GPU parity of the CAQR panel (Eq. caqr with CGS2 leaves) through lls_panel_qr.

Reference: the oracle's FP64 TSQR with CGS2 leaves (oracle.rgsqrf.tsqr), itself pinned against
Householder QR, brute force and the invariants in tests/test_oracle_rgsqrf.py.

Tolerances. The GPU panel runs CGS2 in FP32. CGS2 is backward stable and, for
kappa * u32 < 1, orthogonal to working precision: ||A - QR||_F / ||A||_F <= c u32 and
||I - Q^T Q||_F <= c u32 with c a small multiple of b. R is the unique positive-diagonal
factor, so it agrees with the oracle's to c * kappa * u32 normwise (c = 4 sqrt(b) here). The copy of Q in the
product precision must equal Q rounded to nearest even exactly.
"""
import numpy as np
import pytest
import torch

from oracle import metrics, rgsqrf
from paper_1912_05508_gb300 import lls
from parity import r_entry_err

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
TDT = {"fp16": torch.float16, "bf16": torch.bfloat16}


def panel(A32, prec="fp16"):
    m, b = A32.shape
    W = lls.colmajor(A32)
    Wh = torch.zeros((b, m), dtype=TDT.get(prec, torch.float16), device="cuda").t()
    R = torch.full((b, b), np.nan, dtype=torch.float32, device="cuda").t()
    ws = lls.workspace(lls.lls_panel_qr_workspace_size(m, b)).zero_()
    st = lls.lls_panel_qr(m, b, lls.PREC[prec], W.data_ptr(), m, Wh.data_ptr(), m, R.data_ptr(), b,
                          ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, lls.lls_status_string(st)
    torch.cuda.synchronize()
    return W, Wh, R


def graded(m, b, seed, kappa):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, b)))
    V, _ = np.linalg.qr(rng.standard_normal((b, b)))
    s = kappa ** (-np.arange(b) / max(b - 1, 1))
    return ((U * s) @ V.T).astype(np.float32)


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("m,b,kappa", [(1, 1, 1.0), (16, 16, 10.0), (1000, 7, 1e2), (1024, 16, 1e3),
                                       (1025, 32, 1e3), (4099, 13, 1e4), (32771, 16, 1e3),
                                       (70000, 32, 1e5),
                                       # one-level tree: 512-row leaves, stack of exactly 1024 rows
                                       (32768, 16, 1e3), (512, 16, 1e2), (513, 9, 1e2),
                                       # one-level tree with 1024-row leaves; deeper tree beyond
                                       (65536, 16, 1e4), (65537, 8, 1e2), (150000, 16, 1e3)])
def test_panel_matches_oracle_tsqr(prec, m, b, kappa):
    A = graded(m, b, m + b, kappa)
    W, Wh, R = panel(A, prec)
    Q = W.cpu().numpy().astype(np.float64)
    Rg = R.cpu().numpy().astype(np.float64)
    A64 = A.astype(np.float64)
    assert np.array_equal(np.tril(Rg, -1), np.zeros_like(Rg))
    assert (np.diag(Rg) > 0).all()
    assert metrics.qr_factorization_error(A64, Q, Rg) <= 8 * b * U32
    assert metrics.orthogonality(Q) <= 8 * b * U32
    Qo, Ro = rgsqrf.tsqr(A64, leaf_rows=1024)
    assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= 4 * np.sqrt(b) * kappa * U32 + 4 * b * U32
    assert r_entry_err(Rg, Ro) <= 4 * np.sqrt(b) * kappa * U32 + 4 * b * U32
    if prec != "fp32":
        assert torch.equal(Wh, W.to(TDT[prec]))


def test_panel_zero_column_gives_zero_q():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3000, 8)).astype(np.float32)
    A[:, 5] = 0.0
    W, _, R = panel(A, "fp16")
    Rg = R.cpu().numpy()
    assert Rg[5, 5] == 0.0
    assert np.all(W.cpu().numpy()[:, 5] == 0.0)
    Qo, Ro = rgsqrf.tsqr(A.astype(np.float64), leaf_rows=1024)
    assert Ro[5, 5] == 0.0


def test_panel_rejects_bad_arguments():
    ws = lls.workspace(1 << 20)
    z = torch.zeros(64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lls.lls_panel_qr(10, 33, 0, z.data_ptr(), 10, z.data_ptr(), 10, z.data_ptr(), 33, ws.data_ptr(),
                            ws.numel(), s) == -1
    assert lls.lls_panel_qr(4, 8, 0, z.data_ptr(), 4, z.data_ptr(), 4, z.data_ptr(), 8, ws.data_ptr(),
                            ws.numel(), s) == -1
    assert lls.lls_panel_qr(64, 8, 0, z.data_ptr(), 64, None, 64, z.data_ptr(), 8, ws.data_ptr(),
                            ws.numel(), s) == -1
    assert lls.lls_panel_qr(64, 8, 0, z.data_ptr(), 64, z.data_ptr(), 64, z.data_ptr(), 8, ws.data_ptr(),
                            16, s) == -4


# ---- the lowest recursion node in one launch (lls_panel_block_qr) ----------------------

ULOW = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


def block(A32, w1, prec):
    m, w = A32.shape
    W = lls.colmajor(A32)
    Wh = torch.zeros((w, m), dtype=TDT[prec], device="cuda").t()
    R = torch.full((w, w), np.nan, dtype=torch.float32, device="cuda").t()
    ws = lls.workspace(lls.lls_panel_block_qr_workspace_size(m, w1, w - w1)).zero_()
    st = lls.lls_panel_block_qr(m, w1, w - w1, lls.PREC[prec], W.data_ptr(), m, Wh.data_ptr(), m, R.data_ptr(),
                                w, ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, lls.lls_status_string(st)
    torch.cuda.synchronize()
    return W, Wh, R


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("m,w1,w2", [(40000, 16, 16), (32768, 16, 16), (65536, 16, 11), (5000, 16, 1),
                                     (700, 16, 5), (300, 12, 12), (1537, 9, 9)])
def test_block_matches_oracle_recursion(prec, m, w1, w2):
    # panel, node (low-precision products with column scaling), panel: the oracle's recursion
    # at panel width w1 takes the same steps in FP64 with the same rounding points
    kappa = 1e3
    A = graded(m, w1 + w2, 5 * m + w2, kappa)
    W, Wh, R = block(A, w1, prec)
    Q = W.cpu().numpy().astype(np.float64)
    Rg = R.cpu().numpy().astype(np.float64)
    Qo, Ro = rgsqrf.rgsqrf(A, w1, prec, leaf_rows=256)
    u = ULOW[prec]
    assert np.array_equal(np.tril(Rg, -1), np.zeros_like(Rg))
    assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= 8 * u
    assert r_entry_err(Rg, Ro) <= 4 * u
    assert metrics.qr_factorization_error(A, Q, Rg) <= 4 * u
    assert metrics.orthogonality(Q, "2") <= 4 * u * kappa * (w1 + w2) ** 0.5
    # the product-precision copy is Q rounded to nearest even
    assert torch.equal(Wh, W.to(TDT[prec]))


def test_block_reuses_its_workspace():
    # back-to-back calls on one zero-filled workspace give identical results (the barrier
    # words and column maxima are left ready for the next call)
    A = graded(20000, 32, 3, 1e2)
    m = A.shape[0]
    ws = lls.workspace(lls.lls_panel_block_qr_workspace_size(m, 16, 16)).zero_()
    outs = []
    for _ in range(3):
        W = lls.colmajor(A)
        Wh = torch.zeros((32, m), dtype=torch.float16, device="cuda").t()
        R = torch.zeros((32, 32), dtype=torch.float32, device="cuda").t()
        st = lls.lls_panel_block_qr(m, 16, 16, lls.PREC["fp16"], W.data_ptr(), m, Wh.data_ptr(), m, R.data_ptr(),
                                    32, ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
        assert st == 0
        outs.append((W, R))
    torch.cuda.synchronize()
    for W, R in outs[1:]:
        assert torch.equal(W, outs[0][0]) and torch.equal(R, outs[0][1])


def test_block_rejects_unsupported_shapes():
    ws = lls.workspace(lls.lls_panel_block_qr_workspace_size(70000, 16, 16)).zero_()
    z = torch.zeros(70000 * 32, device="cuda")
    h = torch.zeros(70000 * 32, dtype=torch.float16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    args = (z.data_ptr(), 70000, h.data_ptr(), 70000, z.data_ptr(), 32, ws.data_ptr(), ws.numel(), s)
    f16 = lls.PREC["fp16"]
    # beyond the one-level panel; left half not wider than 8; right half wider than the left
    assert lls.lls_panel_block_qr(70000, 16, 16, f16, *args) == -6
    assert lls.lls_panel_block_qr(4000, 8, 8, f16, *args) == -6
    assert lls.lls_panel_block_qr(4000, 12, 13, f16, *args) == -6
    # FP32 products, R too small, m below the width
    assert lls.lls_panel_block_qr(4000, 16, 16, lls.PREC["fp32"], *args) == -1
    assert lls.lls_panel_block_qr(4000, 16, 16, f16, z.data_ptr(), 70000, h.data_ptr(), 70000, z.data_ptr(), 31,
                                  ws.data_ptr(), ws.numel(), s) == -1
    assert lls.lls_panel_block_qr(20, 16, 16, f16, *args) == -1
