"""GPU checks of lls_solve_host: the solve on page-locked host operands, with A uploaded in
column chunks on a side stream while the factorization runs.

The device work is the same sequence of kernels as lls_solve on device copies of A and b, so
x must agree with lls_solve bit for bit when both take the 16-byte-aligned product paths (m a
multiple of 4); the oracle (FP64 Householder) pins the accuracy.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import direct, metrics
from paper_1912_05508_gb300 import lls, synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def host_solve(A64, b64, lda=None, prec="fp16", target="fp64", reps=1):
    m, n = A64.shape
    lda = lda or m
    Ah = torch.zeros((n, lda), dtype=torch.float32, pin_memory=True)
    Ah[:, :m] = torch.from_numpy(np.ascontiguousarray(A64.T.astype(np.float32)))
    bh = torch.from_numpy(np.asarray(b64, dtype=np.float64)).pin_memory()
    xh = torch.full((n,), np.nan, dtype=torch.float64, pin_memory=True)
    o = lls.make_options(prec=prec, target=target)
    ws = lls.workspace(lls.lls_solve_host_workspace_size(m, n, o))
    info = lls.lls_info()
    s = torch.cuda.current_stream().cuda_stream
    xs = []
    for _ in range(reps):
        st = lls.lls_solve_host(m, n, Ah.data_ptr(), lda, bh.data_ptr(), xh.data_ptr(), ws.data_ptr(), ws.numel(),
                                o, info, s)
        assert st == 0, (st, lls.lls_status_string(st))
        xs.append(xh.numpy().copy())
    return xs, info


@pytest.mark.parametrize("m,n", [(1500, 96), (5000, 700), (3000, 40), (2048, 256)])
def test_host_solve_equals_device_solve(m, n):
    p = synth.svd_lls(m, n, "geometric", 1e3, seed=m + n)
    xs, info = host_solve(p.A, p.b)
    xd, infod = lls.solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda())
    assert info.iters == infod["iters"]
    assert np.array_equal(xs[0], xd.cpu().numpy())
    assert metrics.eta_kw(p.A, p.b, xs[0]) <= 1e-12
    assert metrics.forward_error(xs[0], direct.lls(p.A, p.b)) <= 10 * p.kappa * 1e-12


def test_host_solve_padded_lda_and_repeats():
    # lda > m on the host; repeated calls replay one graph and give the same x
    p = synth.svd_lls(2500, 200, "arithmetic", 1e2, seed=5)
    xs, info = host_solve(p.A, p.b, lda=2600, reps=3)
    assert info.status == 0
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[0], xs[2])
    assert metrics.eta_kw(p.A, p.b, xs[0]) <= 1e-12


def test_host_solve_fp32_target_bf16():
    p = synth.svd_lls(4000, 300, "geometric", 1e3, seed=9)
    xs, info = host_solve(p.A, p.b, prec="bf16", target="fp32")
    assert info.status == 0
    assert metrics.forward_error(xs[0], direct.lls(p.A, p.b)) <= 1e-5


def test_host_solve_rejects_memory_that_is_not_page_locked():
    m, n = 300, 20
    o = lls.make_options()
    ws = lls.workspace(lls.lls_solve_host_workspace_size(m, n, o))
    s = torch.cuda.current_stream().cuda_stream
    A = np.ones((n, m), dtype=np.float32)                # pageable host memory
    b = np.ones(m)
    x = np.zeros(n)
    Ad = torch.ones((n, m), device="cuda")               # device memory
    bp = torch.ones(m, dtype=torch.float64, pin_memory=True)
    xp = torch.zeros(n, dtype=torch.float64, pin_memory=True)
    assert lls.lls_solve_host(m, n, A.ctypes.data, m, b.ctypes.data, x.ctypes.data, ws.data_ptr(), ws.numel(),
                              o, None, s) == -1
    assert lls.lls_solve_host(m, n, Ad.data_ptr(), m, bp.data_ptr(), xp.data_ptr(), ws.data_ptr(), ws.numel(),
                              o, None, s) == -1
    Ap = torch.ones((n, m), dtype=torch.float32, pin_memory=True)
    assert lls.lls_solve_host(m, n, Ap.data_ptr(), m, bp.data_ptr(), xp.data_ptr(), ws.data_ptr(), 1024,
                              o, None, s) == -4


def test_host_solve_without_graphs():
    # LLS_NO_GRAPH (read once per process) enqueues directly: the chunk events then order the
    # side stream's uploads and the factorization at run time
    code = (
        "import sys, numpy as np, torch; sys.path.insert(0, %r); sys.path.insert(0, %r);"
        "from paper_1912_05508_gb300 import lls, synth; from test_gpu_host import host_solve;"
        "p = synth.svd_lls(3000, 330, 'geometric', 1e3, seed=21);"
        "xs, info = host_solve(p.A, p.b);"
        "xd, _ = lls.solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda());"
        "print(int(info.status), bool(np.array_equal(xs[0], xd.cpu().numpy())))"
    ) % (ROOT, os.path.join(ROOT, "tests"))
    env = dict(os.environ, LLS_NO_GRAPH="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().splitlines()[-1] == "0 True"
