"""GPU parity of the least-squares adjoint (lls_backward) and the differentiable solve.

Reference: the oracle's closed-form gradient (oracle.adjoint.lls_grad), itself pinned by FP64
central differences and torch autograd through linalg.lstsq (tests/test_oracle_krylov.py).
Tolerance: the gradient is returned in FP32 and z = (A^T A)^{-1} g is iterated to 1e-13
relative; x from the FP64-target solve carries ~kappa * 1e-12. The normwise relative error of
dL/dA is therefore bounded by ~1e-7 (FP32 rounding) + kappa * 1e-12; the tests use 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint, direct
from paper_1912_05508_gb300 import lls, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_instances_match_closed_form(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((8, 4)).astype(np.float32)
    b = rng.standard_normal(8)
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = lls.lstsq(At, bt, prec="fp16", target="fp64")
    (x * x).sum().backward()
    xs = direct.lls(A, b)
    gA, gb = adjoint.lls_grad(A.astype(np.float64), b, xs, 2 * xs)
    np.testing.assert_allclose(x.detach().cpu().numpy(), xs, rtol=1e-9, atol=1e-12)
    assert rel(At.grad.cpu().numpy(), gA) <= 1e-6
    assert rel(bt.grad.cpu().numpy(), gb) <= 1e-6


def test_config_shape_problem_through_c_abi():
    p = synth.svd_lls(4096, 256, "geometric", 1e3, seed=14)
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    x, info, R = lls.solve(A, b, want_r=True)
    g = 2 * x
    gAs, gbs = lls.backward([A], [b], [x], [R], [g])
    torch.cuda.synchronize()
    xs = direct.lls(p.A, p.b)
    gA, gb = adjoint.lls_grad(p.A.astype(np.float64), p.b, xs, 2 * xs)
    assert rel(gAs[0].cpu().numpy(), gA) <= 1e-6
    assert rel(gbs[0].cpu().numpy(), gb) <= 1e-6


def test_batched_autograd_uneven_spectra():
    probs = [synth.svd_lls(600, 40, k, 1e2, seed=20 + i) for i, k in enumerate(["geometric", "arithmetic", "cluster"])]
    A = torch.stack([torch.from_numpy(q.A) for q in probs]).cuda().requires_grad_(True)
    b = torch.stack([torch.from_numpy(q.b) for q in probs]).cuda().requires_grad_(True)
    x = lls.lstsq(A, b)
    loss = (x * x).sum()
    loss.backward()
    for i, q in enumerate(probs):
        xs = direct.lls(q.A, q.b)
        gA, gb = adjoint.lls_grad(q.A.astype(np.float64), q.b, xs, 2 * xs)
        assert rel(A.grad[i].cpu().numpy(), gA) <= 1e-6
        assert rel(b.grad[i].cpu().numpy(), gb) <= 1e-6


def test_gradient_of_general_loss_matches_finite_differences():
    # L = w . x for a fixed random w: check dL/db against central differences of the GPU solve
    rng = np.random.default_rng(5)
    A = rng.standard_normal((64, 12)).astype(np.float32)
    b = rng.standard_normal(64)
    w = torch.from_numpy(rng.standard_normal(12)).cuda()
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    At = torch.from_numpy(A).cuda()
    (lls.lstsq(At, bt) * w).sum().backward()
    h = 1e-4
    fd = []
    for i in range(5):
        e = np.zeros(64)
        e[i] = h
        xp = lls.lstsq(At, torch.from_numpy(b + e).cuda()).detach()
        xm = lls.lstsq(At, torch.from_numpy(b - e).cuda()).detach()
        fd.append(float(((xp - xm) * w).sum()) / (2 * h))
    np.testing.assert_allclose(bt.grad.cpu().numpy()[:5], fd, rtol=1e-6, atol=1e-9)


def test_batched_adjoint_uneven_shapes_one_launch():
    # a batch of uneven problems: the forward solve and the adjoint each run as one persistent
    # launch (each CTA whole problems); every problem's gradient matches the closed form
    rng = np.random.default_rng(11)
    probs = []
    for i in range(12):
        n = int(rng.integers(20, 200))
        m = int(rng.integers(4 * n, 3000))
        probs.append(synth.svd_lls(m, n, "geometric", 10.0 ** rng.uniform(1, 3), seed=300 + i))
    As = [lls.colmajor(q.A) for q in probs]
    bs = [torch.from_numpy(q.b).cuda() for q in probs]
    xs, infos, Rs = lls.solve_batched(As, bs, target="fp64", want_r=True)
    assert all(i["status"] == 0 for i in infos)
    gxs = [2 * x for x in xs]
    torch.cuda.synchronize()
    c0 = lls.lls_kernel_launch_count()
    gAs, gbs = lls.backward(As, bs, xs, Rs, gxs)
    torch.cuda.synchronize()
    assert lls.lls_kernel_launch_count() - c0 == 1
    for i, q in enumerate(probs):
        xo = direct.lls(q.A, q.b)
        gA, gb = adjoint.lls_grad(q.A.astype(np.float64), q.b, xo, 2 * xo)
        assert rel(gAs[i].cpu().numpy(), gA) <= 1e-6, i
        assert rel(gbs[i].cpu().numpy(), gb) <= 1e-6, i
