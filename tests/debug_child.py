"""Child process of tests/test_gpu_debug.py (not a test module).

    python tests/debug_child.py run <out.npz>      a fixed set of seeded calls; results saved
    python tests/debug_child.py inject <out.json>  the planted faults, each armed then disarmed

LLS_DEBUG in the environment selects the library build (0: release, 1: debug).
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1912_05508_gb300 import lls, synth  # noqa: E402


def run(out):
    dev = torch.device("cuda", 0)
    res = {}
    # a solve whose QR takes the block kernels, the fused nodes and the persistent products
    A, b, _ = synth.svd_lls_torch(8192, 512, "geometric", 1e3, seed=11, device=dev)
    x, info, R = lls.solve(A, b, prec="fp16", panel_width=16, want_r=True)
    res["solve_x"] = x.cpu().numpy()
    res["solve_R"] = R.cpu().numpy()
    res["solve_iters"] = np.array([info["iters"], info["status_code"]])
    # a ragged BF16 QR with a direct-start LSQR solve
    A2, b2, _ = synth.svd_lls_torch(3001, 97, "arithmetic", 1e2, seed=12, device=dev)
    Q, R2 = lls.qr(A2, prec="bf16", panel_width=16)
    res["qr_Q"] = Q.cpu().numpy()
    res["qr_R"] = R2.cpu().numpy()
    x2, info2 = lls.solve(A2, b2, prec="bf16", krylov="lsqr", x0="direct", panel_width=16)
    res["lsqr_x"] = x2.cpu().numpy()
    # a small uneven batch and its adjoint
    g = torch.Generator(device="cpu").manual_seed(13)
    shapes = [(300, 40), (1024, 128), (777, 5), (2048, 64)]
    As = [lls.colmajor(torch.randn(m, n, generator=g, dtype=torch.float64).float()) for m, n in shapes]
    bs = [torch.randn(m, generator=g, dtype=torch.float64).cuda() for m, _ in shapes]
    xs, infos, Rs = lls.solve_batched(As, bs, prec="fp16", target="fp64", want_r=True)
    gxs = [torch.ones_like(xv) for xv in xs]
    gAs, gbs = lls.backward(As, bs, xs, Rs, gxs, prec="fp16")
    for i in range(len(shapes)):
        res[f"batch_x{i}"] = xs[i].cpu().numpy()
        res[f"batch_gA{i}"] = gAs[i].cpu().numpy()
        res[f"batch_gb{i}"] = gbs[i].cpu().numpy()
    # the kernel-level panel and block entry points at a one-level shape of 64 leaves
    st = torch.cuda.current_stream().cuda_stream
    for (m, b) in [(32768, 16), (5000, 13), (9000, 8)]:
        W = lls.colmajor(torch.randn(m, b, generator=g, dtype=torch.float64).float())
        Wh = torch.zeros((b, m), dtype=torch.float16, device="cuda").t()
        R = torch.zeros((b, b), dtype=torch.float32, device="cuda").t()
        ws = lls.workspace(lls.lls_panel_qr_workspace_size(m, b)).zero_()
        for _ in range(2):   # the second call reuses the workspace as left by the first
            W2 = W.clone()
            assert lls.lls_panel_qr(m, b, lls.PREC["fp16"], W2.data_ptr(), m, Wh.data_ptr(), m, R.data_ptr(), b,
                                    ws.data_ptr(), ws.numel(), st) == 0
        res[f"panel_Q_{m}_{b}"] = W2.cpu().numpy()
        res[f"panel_R_{m}_{b}"] = R.cpu().numpy()
    m = 32768
    W = lls.colmajor(torch.randn(m, 32, generator=g, dtype=torch.float64).float())
    Wh = torch.zeros((32, m), dtype=torch.float16, device="cuda").t()
    R = torch.zeros((32, 32), dtype=torch.float32, device="cuda").t()
    ws = lls.workspace(lls.lls_panel_block_qr_workspace_size(m, 16, 16)).zero_()
    assert lls.lls_panel_block_qr(m, 16, 16, lls.PREC["fp16"], W.data_ptr(), m, Wh.data_ptr(), m, R.data_ptr(), 32,
                                  ws.data_ptr(), ws.numel(), st) == 0
    res["block_Q"] = W.cpu().numpy()
    res["block_R"] = R.cpu().numpy()
    torch.cuda.synchronize()
    np.savez(out, **res)


def inject(out):
    m, b = 2048, 16
    g = torch.Generator(device="cpu").manual_seed(14)
    A = torch.randn(m, b, generator=g, dtype=torch.float64).float()
    st = torch.cuda.current_stream().cuda_stream
    ws = lls.workspace(lls.lls_panel_qr_workspace_size(m, b)).zero_()
    res = {"debug_build": lls.load().lls_debug_build()}

    def panel():
        W = lls.colmajor(A)
        Wh = torch.zeros((b, m), dtype=torch.float16, device="cuda").t()
        R = torch.zeros((b, b), dtype=torch.float32, device="cuda").t()
        s = lls.lls_panel_qr(m, b, lls.PREC["fp16"], W.data_ptr(), m, Wh.data_ptr(), m, R.data_ptr(), b,
                             ws.data_ptr(), ws.numel(), st)
        torch.cuda.synchronize()
        return s, W.cpu()

    res["arm"] = lls.load().lls_debug_inject(1)
    res["armed_status"], W = panel()
    res["q_untouched"] = bool(torch.equal(W, A))
    res["disarm"] = lls.load().lls_debug_inject(0)
    res["disarmed_status"], W = panel()
    res["q_written"] = not bool(torch.equal(W, A))

    # mode 2: the panel's grid barrier waits for one CTA more than the grid holds
    A2 = lls.colmajor(torch.randn(4096, 64, generator=g, dtype=torch.float64).float())
    b2 = torch.randn(4096, generator=g, dtype=torch.float64).cuda()
    res["arm2"] = lls.load().lls_debug_inject(2)
    _, R = lls.qr(A2, prec="fp16", panel_width=16, want_q=False)
    torch.cuda.synchronize()
    res["armed_qr_diag_nan"] = bool(torch.isnan(torch.diagonal(R)).all())
    _, info = lls.solve(A2, b2, prec="fp16", panel_width=16, check=False)
    res["armed_solve_status"] = info["status_code"]
    res["disarm2"] = lls.load().lls_debug_inject(0)
    _, R = lls.qr(A2, prec="fp16", panel_width=16, want_q=False)
    torch.cuda.synchronize()
    res["disarmed_qr_diag_finite"] = bool(torch.isfinite(torch.diagonal(R)).all())
    _, info = lls.solve(A2, b2, prec="fp16", panel_width=16, check=False)
    res["disarmed_solve_status"] = info["status_code"]
    res["bad_mode"] = lls.load().lls_debug_inject(3)
    with open(out, "w") as fh:
        json.dump(res, fh)


if __name__ == "__main__":
    {"run": run, "inject": inject}[sys.argv[1]](sys.argv[2])
