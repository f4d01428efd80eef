"""lls_lowp_projection_noalloc, the projection entry point that takes its scratch from a fixed
array inside the library instead of a caller workspace.

Its outputs must agree with lls_lowp_projection on the same inputs. Both run the same
kernels with the same split of the K loop and the same fixed order of summation, so R12, the
derived integer exponents f and the rounded low-precision copy R12l must agree bit for bit
(R12 is also held to the FP32 accumulation bound m * u32 * |Q1|^T |A2| against the exact
product, as in the product tests). Two calls in a
row with different inputs check that nothing left in the shared array by one call leaks into
the next. This file is collected last so that it also runs after every other test in one
process; it passes alone in a fresh process too, where its first call does the per-device
set-up.
"""
import numpy as np
import pytest
import torch

from paper_1912_05508_gb300 import lls

U32 = 2.0 ** -24
TDT = {"fp16": torch.float16, "bf16": torch.bfloat16}
PREC = {"fp16": 0, "bf16": 1}
LLS_ERR_TOO_LARGE = -7


def lowp_colmajor(X, prec, ld):
    m, n = X.shape
    buf = torch.zeros((n, ld), dtype=TDT[prec], device="cuda")
    t = torch.from_numpy(np.ascontiguousarray(X.T)).to(TDT[prec])
    buf[:, :m] = t.cuda()
    return buf, t.to(torch.float64).numpy().T


def outputs(w1, w2, prec):
    ldrl = (w1 + 7) // 8 * 8
    return (torch.full((w2, w1), np.nan, dtype=torch.float32, device="cuda"),
            torch.zeros((w2, ldrl), dtype=TDT[prec], device="cuda"),
            torch.full((w2,), -999, dtype=torch.int32, device="cuda"), ldrl)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,m,w1,w2", [("fp16", 4096, 128, 128), ("bf16", 2049, 96, 200)])
def test_noalloc_matches_workspace_projection_twice(prec, m, w1, w2):
    stream = torch.cuda.current_stream().cuda_stream
    ldh = (m + 7) // 8 * 8
    assert lls.lls_lowp_projection_workspace_size(m, w1, w2) <= 4 << 20
    for call in range(2):
        rng = np.random.default_rng(1000 * call + m + w1 + w2)
        Q = rng.standard_normal((m, w1)) / np.sqrt(m)
        A = rng.standard_normal((m, w2)) * 2.0 ** (10 - 4 * call)
        e = rng.integers(-3, 4, size=w2).astype(np.int32)
        Qd, Qv = lowp_colmajor(Q, prec, ldh)
        Ad, Av = lowp_colmajor(A, prec, ldh)
        ed = torch.from_numpy(e).cuda()

        R12a, R12la, fa, ldrl = outputs(w1, w2, prec)
        ws = lls.workspace(lls.lls_lowp_projection_workspace_size(m, w1, w2))
        st = lls.lls_lowp_projection(m, w1, w2, PREC[prec], Qd.data_ptr(), Ad.data_ptr(), ldh, ed.data_ptr(),
                                     R12a.data_ptr(), w1, R12la.data_ptr(), ldrl, fa.data_ptr(),
                                     ws.data_ptr(), ws.numel(), stream)
        assert st == 0

        R12b, R12lb, fb, _ = outputs(w1, w2, prec)
        st = lls.lls_lowp_projection_noalloc(m, w1, w2, PREC[prec], Qd.data_ptr(), Ad.data_ptr(), ldh,
                                             ed.data_ptr(), R12b.data_ptr(), w1, R12lb.data_ptr(), ldrl,
                                             fb.data_ptr(), stream)
        assert st == 0, lls.lls_status_string(st)
        torch.cuda.synchronize()

        b = R12b.cpu().numpy().T.astype(np.float64)
        mag = np.ldexp(np.abs(Qv).T @ np.abs(Av), -e[None, :].astype(np.int64))
        exact = np.ldexp(Qv.T @ Av, -e[None, :].astype(np.int64))
        assert np.isfinite(b).all()
        assert torch.equal(R12a, R12b), f"call {call}"
        assert (np.abs(b - exact) <= m * U32 * mag + 1e-30).all(), f"call {call}"
        assert torch.equal(fa, fb), f"call {call}"
        assert torch.equal(R12la[:, :w1], R12lb[:, :w1]), f"call {call}"


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    m, w = 32768, 256
    assert lls.lls_lowp_projection_workspace_size(m, w, w) > 4 << 20
    dummy = torch.zeros(8, dtype=torch.float16, device="cuda").data_ptr()
    st = lls.lls_lowp_projection_noalloc(m, w, w, 0, dummy, dummy, m, dummy, dummy, w, dummy, w, dummy,
                                         torch.cuda.current_stream().cuda_stream)
    assert st == LLS_ERR_TOO_LARGE
    assert "fixed scratch" in lls.lls_status_string(st)
