"""GPU parity of the two tensor-core products of a recursion step (Alg. 2: projection and update),
through the kernel-level C entry points, against an FP64 product of the SAME rounded inputs.

Bound: with FP32 accumulation over K terms, |fl(sum) - sum| <= K * u32 * sum |a_k b_k|
(products of FP16/BF16 values are exact in FP32). The tests assert that bound elementwise
and a much tighter normwise statistic (random rounding errors grow like sqrt(K)).
"""
import numpy as np
import pytest
import torch

from paper_1912_05508_gb300 import lls

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
TDT = {"fp16": torch.float16, "bf16": torch.bfloat16}
PREC = {"fp16": 0, "bf16": 1}


def lowp_colmajor(X, prec, ld=None):
    """Device column-major low-precision copy (ld >= rows, multiple of 8) and its FP64 values."""
    m, n = X.shape
    ld = ld or (m + 7) // 8 * 8
    buf = torch.zeros((n, ld), dtype=TDT[prec], device="cuda")
    t = torch.from_numpy(np.ascontiguousarray(X.T)).to(TDT[prec])
    buf[:, :m] = t.cuda()
    vals = t.to(torch.float64).numpy().T
    return buf, ld, vals


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("m,w1,w2", [(1000, 32, 32), (4096, 128, 128), (2049, 96, 200),
                                     (300, 512, 300), (8192, 256, 520), (32768, 64, 64),
                                     # persistent kernel: ragged M and N tiles; several units per CTA
                                     (3000, 200, 136), (4096, 2048, 2048)])
def test_projection(prec, m, w1, w2):
    rng = np.random.default_rng(m + w1 + w2)
    Q = rng.standard_normal((m, w1)) / np.sqrt(m)
    e = rng.integers(-3, 4, size=w2).astype(np.int32)
    A = rng.standard_normal((m, w2)) * 2.0 ** 10
    Qd, ldh, Qv = lowp_colmajor(Q, prec)
    Ad, ldh2, Av = lowp_colmajor(A, prec, ldh)
    ed = torch.from_numpy(e).cuda()
    R12 = torch.zeros((w2, w1), dtype=torch.float32, device="cuda")
    ldrl = (w1 + 7) // 8 * 8
    R12l = torch.zeros((w2, ldrl), dtype=TDT[prec], device="cuda")
    f = torch.zeros(w2, dtype=torch.int32, device="cuda")
    nb = lls.lls_lowp_projection_workspace_size(m, w1, w2)
    ws = lls.workspace(nb)
    st = lls.lls_lowp_projection(m, w1, w2, PREC[prec], Qd.data_ptr(), Ad.data_ptr(), ldh, ed.data_ptr(),
                                 R12.data_ptr(), w1, R12l.data_ptr(), ldrl, f.data_ptr(), ws.data_ptr(),
                                 ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    got = R12.cpu().numpy().T.astype(np.float64)
    ref = np.ldexp(Qv.T @ Av, -e[None, :].astype(np.int64))
    mag = np.ldexp(np.abs(Qv).T @ np.abs(Av), -e[None, :].astype(np.int64))
    err = np.abs(got - ref)
    assert (err <= m * U32 * mag + 1e-30).all(), float((err / (mag + 1e-300)).max())
    assert np.linalg.norm(err) <= 16 * np.sqrt(m) * U32 * np.linalg.norm(mag)
    # the scaled low-precision copy: exponent in range and correctly rounded from R12
    fh = f.cpu().numpy()
    mx = np.abs(got).max(axis=0)
    if prec == "fp16":
        scaled = np.ldexp(mx, fh.astype(np.int64))
        nz = mx > 0
        assert ((scaled[nz] >= 2.0 ** 14) & (scaled[nz] < 2.0 ** 15)).all()
    else:
        assert (fh == 0).all()
    lowv = R12l.cpu().to(torch.float64).numpy()[:, :w1].T
    expect = torch.from_numpy(np.ldexp(got, fh[None, :].astype(np.int64)).astype(np.float32)).to(TDT[prec]).to(torch.float64).numpy()
    assert np.array_equal(lowv, expect)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("m,w1,w2", [(1000, 32, 32), (4096, 128, 128), (2049, 96, 200),
                                     (300, 64, 300), (8192, 256, 520), (777, 512, 64),
                                     # persistent kernel: ragged rows and a ragged K tile; several
                                     # tiles per CTA, so both accumulators and the A2 chunk ring wrap
                                     (2052, 96, 200), (4096, 512, 1024)])
def test_update(prec, m, w1, w2):
    rng = np.random.default_rng(7 * m + w1 + w2)
    Q = rng.standard_normal((m, w1)) / np.sqrt(m)
    Rl = rng.standard_normal((w1, w2)) * 2.0 ** 12
    fexp = rng.integers(-2, 6, size=w2).astype(np.int32)
    A2 = rng.standard_normal((m, w2)).astype(np.float32)
    Qd, ldh, Qv = lowp_colmajor(Q, prec)
    Rd, ldrl, Rv = lowp_colmajor(Rl, prec)
    A2d = lls.colmajor(A2)
    fd = torch.from_numpy(fexp).cuda()
    ws = lls.workspace(256)
    st = lls.lls_lowp_update(m, w1, w2, PREC[prec], Qd.data_ptr(), ldh, Rd.data_ptr(), ldrl, fd.data_ptr(),
                             A2d.data_ptr(), m, ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    got = A2d.cpu().numpy().astype(np.float64)
    prod = np.ldexp(Qv @ Rv, -fexp[None, :].astype(np.int64))
    mag = np.ldexp(np.abs(Qv) @ np.abs(Rv), -fexp[None, :].astype(np.int64))
    ref = A2.astype(np.float64) - prod
    err = np.abs(got - ref)
    assert (err <= (w1 + 2) * U32 * (mag + np.abs(ref)) + 1e-30).all(), float((err / (mag + 1e-300)).max())
