"""GPU parity of lls_solve (RGSQRF-preconditioned CGLS, Alg. 5) against the CPU oracle.

Tolerances
----------
* FP64 target: the Karlson-Walden backward error of the returned x, evaluated by the
  oracle (compensated residual, FP64 QR of [A; xi I]), must be <= 1e-12 and the forward
  error against the oracle's x* <= 10 * kappa * 1e-12 (first-order perturbation bound).
* FP32 target: ||x - x*|| / ||x*|| <= 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import direct, metrics
from paper_1912_05508_gb300 import lls, synth

pytestmark = pytest.mark.gpu


def run(p, **kw):
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    x, info = lls.solve(A, b, **kw)
    return x.cpu().numpy(), info


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_fp64_target_config_small(prec):
    p = synth.svd_lls(1024, 128, "geometric", 1e3, seed=1)
    x, info = run(p, prec=prec, target="fp64")
    xs = direct.lls(p.A, p.b)
    assert info["status"] == 0, info
    assert metrics.eta_kw(p.A, p.b, x) <= 1e-12
    assert metrics.forward_error(x, xs) <= 10 * p.kappa * 1e-12
    assert info["eta"] <= 1e-12


@pytest.mark.parametrize("kind", ["geometric", "arithmetic", "cluster"])
def test_fp32_target(kind):
    p = synth.svd_lls(1024, 128, kind, 1e3, seed=2)
    x, info = run(p, prec="fp16", target="fp32")
    xs = direct.lls(p.A, p.b)
    assert info["status"] == 0, info
    assert metrics.forward_error(x, xs) <= 1e-5


@pytest.mark.parametrize("m,n", [(3000, 200), (700, 45), (96, 96), (40, 1)])
def test_ragged_and_degenerate_shapes(m, n):
    p = synth.svd_lls(m, n, "arithmetic", 1e2, seed=m + n, noise=1e-3 if m > n else 0.0)
    x, info = run(p, prec="fp16", target="fp64")
    xs = direct.lls(p.A, p.b)
    assert info["status"] == 0, info
    assert metrics.forward_error(x, xs) <= 10 * p.kappa * 1e-12


def test_singular_is_reported():
    p = synth.svd_lls(500, 30, "geometric", 10.0, seed=4)
    A = p.A.copy()
    A[:, 3] = 0.0
    Ad = lls.colmajor(A)
    x, info = lls.solve(Ad, torch.from_numpy(p.b).cuda(), check=False)
    assert info["status_code"] == -2


def test_iteration_cap_reports_not_converged():
    p = synth.svd_lls(1024, 128, "geometric", 1e3, seed=1)
    x, info = run(p, prec="bf16", target="fp64", max_iter=2)
    assert info["status_code"] == 1 and info["iters"] == 2
