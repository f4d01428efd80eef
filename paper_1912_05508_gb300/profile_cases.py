"""Small, self-contained cases of the library's kernels for profiling (ncu) and timing.

    python -m paper_1912_05508_gb300.profile_cases <case>

Cases (each a few GB at most on the device, inputs larger than L2):
    products   the projection and the update of a top recursion node, 16384 x 2048 x 2048
               (FP16), two calls each through the kernel-level entry points;
    krylov     a solve of 16384 x 4096 (geometric spectrum, kappa = 1e3) capped at 6
               Krylov iterations;
    block      the lowest recursion node (two 16-column panels and the node between them)
               on 32768 rows, three calls;
    small      the 1024 x 128 LSQR solve to the FP32 target, three calls.
The krylov case keeps its generated input in the temporary folder, so a second run of the
same command (under a profiler, where torch's linear-algebra plugin may not load) reuses it.
"""
from __future__ import annotations

import os
import sys
import tempfile


def products():
    import torch
    from . import lls
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream().cuda_stream
    m, w1, w2 = 16384, 2048, 2048
    g = torch.Generator(device=dev).manual_seed(7)
    Q1l = (torch.randn((w1, m), device=dev, generator=g) / m ** 0.5).half().t()
    A2l = torch.randn((w2, m), device=dev, generator=g).half().t()
    A2 = torch.randn((w2, m), device=dev, generator=g).t()
    e = torch.zeros(w2, dtype=torch.int32, device=dev)
    R12 = torch.empty((w2, w1), device=dev)
    R12l = torch.zeros((w2, w1), dtype=torch.float16, device=dev)
    f = torch.zeros(w2, dtype=torch.int32, device=dev)
    ws = lls.workspace(lls.lls_lowp_projection_workspace_size(m, w1, w2), dev)
    for _ in range(2):
        assert lls.lls_lowp_projection(m, w1, w2, 0, Q1l.data_ptr(), A2l.data_ptr(), m, e.data_ptr(), R12.data_ptr(),
                                       w1, R12l.data_ptr(), w1, f.data_ptr(), ws.data_ptr(), ws.numel(), s) == 0
        R12l.zero_()
        f.zero_()
        assert lls.lls_lowp_update(m, w1, w2, 0, Q1l.data_ptr(), m, R12l.data_ptr(), w1, f.data_ptr(), A2.data_ptr(),
                                   m, ws.data_ptr(), ws.numel(), s) == 0
    torch.cuda.synchronize()


def krylov():
    import torch
    from . import lls, synth
    dev = torch.device("cuda", 0)
    path = os.path.join(tempfile.gettempdir(), "lls_profile_krylov_16384x4096.pt")
    if os.path.exists(path):
        d = torch.load(path)
        A = torch.empty((4096, 16384), dtype=torch.float32, device=dev).t()
        A.copy_(d["A"])
        b = d["b"].to(dev)
    else:
        A, b, _ = synth.svd_lls_torch(16384, 4096, "geometric", 1e3, seed=3, device=dev)
        torch.save({"A": A.cpu(), "b": b.cpu()}, path)
    lls.solve(A, b, panel_width=16, max_iter=6, tol=1e-300, check=False)
    torch.cuda.synchronize()


def block():
    import torch
    from . import lls
    dev = torch.device("cuda", 0)
    m, w = 32768, 32
    g = torch.Generator(device=dev).manual_seed(9)
    s = torch.cuda.current_stream().cuda_stream
    ws = lls.workspace(lls.lls_panel_block_qr_workspace_size(m, 16, 16), dev).zero_()
    for _ in range(3):
        W = torch.randn((w, m), device=dev, generator=g).t()
        Wh = torch.empty((w, m), dtype=torch.float16, device=dev).t()
        R = torch.empty((w, w), device=dev)
        assert lls.lls_panel_block_qr(m, 16, 16, 0, W.data_ptr(), m, Wh.data_ptr(), m, R.data_ptr(), w,
                                      ws.data_ptr(), ws.numel(), s) == 0
    torch.cuda.synchronize()


def small():
    import torch
    from . import lls, synth
    p = synth.svd_lls(1024, 128, "geometric", 1e3, seed=1)
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    for _ in range(3):
        lls.solve(A, b, target="fp32", krylov="lsqr")
    torch.cuda.synchronize()


CASES = {"products": products, "krylov": krylov, "block": block, "small": small}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        print(__doc__)
        sys.exit(2)
    CASES[sys.argv[1]]()
    print("ok", sys.argv[1])
