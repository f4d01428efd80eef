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
