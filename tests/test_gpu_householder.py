"""GPU parity of the plain Householder least-squares solver (Alg. 1) against the CPU oracle.

Tolerances: Householder QR is backward stable, so the computed x solves a problem perturbed
by c * u relative in the working precision; the forward error is then bounded by
c * kappa * u (+ kappa^2 u tan(theta), negligible for these small residuals). The tests use
c = 20 sqrt(n): FP64, u = 2^-53; FP32, u = 2^-24.
"""
import numpy as np
import pytest
import torch

from oracle import direct, metrics
from paper_1912_05508_gb300 import lls, synth

pytestmark = pytest.mark.gpu

U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m,n,kappa", [(1024, 128, 1e3), (3000, 45, 1e2), (96, 96, 10.0), (40, 1, 1.0),
                                       (5001, 300, 1e4), (20000, 70, 1e3)])
def test_householder_matches_oracle(prec, m, n, kappa):
    p = synth.svd_lls(m, n, "geometric", kappa, seed=m + n, noise=1e-6 if m > n else 0.0)
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    x = lls.householder_solve(A, b, prec=prec).cpu().numpy()
    torch.cuda.synchronize()
    xs = direct.lls(p.A, p.b)
    assert metrics.forward_error(x, xs) <= 20 * np.sqrt(n) * kappa * U[prec]


def test_householder_fp64_reaches_fp64_backward_error():
    p = synth.svd_lls(2048, 200, "cluster", 1e3, seed=3)
    x = lls.householder_solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda(), prec="fp64").cpu().numpy()
    assert metrics.eta_kw(p.A, p.b, x) <= 1e-14


def test_householder_rejects_bad_arguments():
    ws = lls.workspace(1 << 16)
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lls.lls_householder_solve(4, 8, 4, z.data_ptr(), 4, z.data_ptr(), z.data_ptr(), ws.data_ptr(),
                                     ws.numel(), s) == -1
    assert lls.lls_householder_solve(8, 4, 0, z.data_ptr(), 8, z.data_ptr(), z.data_ptr(), ws.data_ptr(),
                                     ws.numel(), s) == -1
    assert lls.lls_householder_solve(8, 4, 4, z.data_ptr(), 8, z.data_ptr(), z.data_ptr(), ws.data_ptr(),
                                     16, s) == -4
