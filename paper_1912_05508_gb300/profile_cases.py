"""Small, self-contained cases of the library's kernels for profiling (ncu) and timing.

    python -m paper_1912_05508_gb300.profile_cases <case>

Cases (each a few GB at most on the device, inputs larger than L2):
    products   the projection and the update of a top recursion node, 16384 x 2048 x 2048
               (FP16), two calls each through the kernel-level entry points;
    krylov     a solve of 16384 x 4096 (geometric spectrum, kappa = 1e3) capped at 6
               Krylov iterations;
    block      the lowest recursion node (two 16-column panels and the node between them)
               on 32768 rows, three calls;
    small      the 1024 x 128 LSQR solve to the FP32 target, three calls;
    solve      the benchmark's solve, 32768 x 4096 (geometric spectrum, kappa = 1e3, seed 2,
               FP16 products, CGLS to the FP64 target), with the implementation choices the
               autotuner picks for it on a GB300 (panel width 16, blocks and narrow nodes as
               single launches, the persistent update with the one-tile-per-CTA projection;
               recorded here, not measured, so a profiler cannot change them), two solves:
               the launch list of the second is the steady-state one (512 MiB of A).
The krylov and solve cases keep their generated inputs in the temporary folder, so a second run
of the same command (under a profiler, where torch's linear-algebra plugin may not load) reuses
them.
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


def _problem(m, n, seed, dev):
    """The geometric-spectrum problem (kappa = 1e3) of the given seed, generated on the device
    once and kept in the temporary folder: a second run of the same command (under a profiler,
    where torch's linear-algebra plugin may not load) reuses it."""
    import torch
    from . import synth
    path = os.path.join(tempfile.gettempdir(), f"lls_profile_{m}x{n}_seed{seed}.pt")
    if os.path.exists(path):
        d = torch.load(path)
        A = torch.empty((n, m), dtype=torch.float32, device=dev).t()
        A.copy_(d["A"])
        return A, d["b"].to(dev)
    A, b, _ = synth.svd_lls_torch(m, n, "geometric", 1e3, seed=seed, device=dev)
    torch.save({"A": A.cpu(), "b": b.cpu()}, path)
    return A, b


def krylov():
    import torch
    from . import lls
    dev = torch.device("cuda", 0)
    A, b = _problem(16384, 4096, 3, dev)
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


def solve():
    import torch
    from . import lls
    dev = torch.device("cuda", 0)
    A, b = _problem(32768, 4096, 2, dev)
    t = lls.lls_tuning()
    t.panel_width, t.node_mode, t.gemm_kernel, t.batched_ctas_per_sm, t.krylov_ctas = 16, 0, 2, 0, 0
    assert lls.lls_tuning_set(0, 32768, 4096, lls.make_options(prec="fp16", target="fp64"), t) == 0
    for _ in range(2):
        x, info = lls.solve(A, b, prec="fp16", target="fp64")
        torch.cuda.synchronize()
    print("iters", info["iters"], "eta", info["eta"])


CASES = {"products": products, "krylov": krylov, "block": block, "small": small, "solve": solve}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        print(__doc__)
        sys.exit(2)
    CASES[sys.argv[1]]()
    print("ok", sys.argv[1])
