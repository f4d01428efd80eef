"""Starting points of the Krylov iteration and non-finite inputs, through lls_solve.

* LLS_X0_DIRECT starts CGLS from the direct solve x0 = R^{-1} Q^T b with the mixed-precision
  factors (Alg. 1's last two steps on the RGSQRF Q and R; Sec. 3.2.2, 4.2.2). The solution is
  the same least-squares solution (checked against the oracle), reached in fewer iterations.
* LLS_X0_GIVEN is a warm start: started from the converged x, the fresh-residual test passes
  at once; started from a nearby problem's solution, the iteration needs fewer steps.
* A NaN or infinity in A, b or a given x0 is reported as LLS_ERR_SINGULAR (status -2), never
  as a converged solve.
* LLS_LOG=1 prints the stop quantity of every iteration; checked in a child process.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import direct, metrics
from parity import kw_bound as parity_kw_bound
from paper_1912_05508_gb300 import lls, synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def prob():
    p = synth.svd_lls(8192, 512, "geometric", 1e3, seed=61)
    return p, direct.lls(p.A, p.b)


def kw_bound(A32, R):
    return parity_kw_bound(A32, R.cpu().numpy())


@pytest.mark.parametrize("krylov", ["cgls", "lsqr"])
def test_direct_start_converges_in_fewer_iterations(prob, krylov):
    p, xs = prob
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    x0, i0, R0 = lls.solve(A, b, krylov=krylov, want_r=True)
    x1, i1, R1 = lls.solve(A, b, krylov=krylov, x0="direct", want_r=True)
    assert i0["status"] == 0 and i1["status"] == 0, (i0, i1)
    assert i0["eta"] <= 1e-12 and i1["eta"] <= 1e-12
    # the direct start never costs iterations (its A-norm error is far smaller, see below; the
    # count saved is small and may round to none at the 1e-12 threshold)
    assert i1["iters"] <= i0["iters"], (i0["iters"], i1["iters"])
    for x, R in ((x0, R0), (x1, R1)):
        xn = x.cpu().numpy()
        assert metrics.eta_kw(p.A, p.b, xn) <= kw_bound(p.A, R)
        assert metrics.forward_error(xn, xs) <= 10 * p.kappa * 1e-12


def test_direct_start_lowers_the_starting_residual(prob):
    # The direct solve with the low-precision factors is inaccurate in x (Sec. 4.2.2), but its
    # residual is close to the optimal one: ||A (x0 - x*)|| is at the level of the factors'
    # loss of orthogonality times ||b|| (the oracle's FP16 recursion gives 0.04 ||b|| here
    # against ||b|| for x = 0), and that A-norm error is what CGLS reduces. After one step from
    # each start, the fresh residual of the direct start is far smaller.
    p, xs = prob
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    _, i_direct = lls.solve(A, b, x0="direct", max_iter=1, tol=1e-300, check=False)
    _, i_zero = lls.solve(A, b, max_iter=1, tol=1e-300, check=False)
    assert i_direct["status"] == 1 and i_zero["status"] == 1 and i_direct["iters"] == 1
    assert i_direct["res_norm"] < 0.5 * i_zero["res_norm"], (i_direct, i_zero)


def test_warm_start_from_the_solution_stops_at_once(prob):
    p, xs = prob
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    x, info = lls.solve(A, b)
    x2, info2 = lls.solve(A, b, x0=x)
    assert info2["status"] == 0 and info2["iters"] <= 1, info2
    assert metrics.forward_error(x2.cpu().numpy(), xs) <= 10 * p.kappa * 1e-12


def test_warm_start_from_a_nearby_problem(prob):
    p, xs = prob
    A = lls.colmajor(p.A)
    b = torch.from_numpy(p.b).cuda()
    bp = b * (1.0 + 1e-4 * torch.randn_like(b))
    xp, _ = lls.solve(A, bp)
    _, cold = lls.solve(A, b)
    xw, warm = lls.solve(A, b, x0=xp)
    assert warm["status"] == 0 and warm["iters"] < cold["iters"], (warm, cold)
    assert metrics.forward_error(xw.cpu().numpy(), xs) <= 10 * p.kappa * 1e-12


@pytest.mark.parametrize("where,value", [("A", np.nan), ("A", np.inf), ("b", np.nan), ("b", -np.inf),
                                         ("x0", np.nan)])
def test_non_finite_input_is_reported_singular(where, value):
    p = synth.svd_lls(3000, 96, "geometric", 1e2, seed=62)
    A = p.A.copy()
    b = p.b.copy()
    x0 = None
    if where == "A":
        A[1234, 50] = value
    elif where == "b":
        b[777] = value
    else:
        x0 = torch.zeros(96, dtype=torch.float64)
        x0[5] = value
    x, info = lls.solve(lls.colmajor(A), torch.from_numpy(b).cuda(), x0=x0, check=False)
    assert info["status_code"] == -2 and info["status"] == -2, info
    # the context stays usable: a clean solve right after converges
    _, ok = lls.solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda())
    assert ok["status"] == 0


def test_iteration_log_prints_the_history():
    code = (
        "import torch\n"
        "from paper_1912_05508_gb300 import lls, synth\n"
        "p = synth.svd_lls(2048, 128, 'geometric', 1e3, seed=63)\n"
        "x, info = lls.solve(lls.colmajor(p.A), torch.from_numpy(p.b).cuda())\n"
        "print('ITERS', info['iters'])\n")
    env = dict(os.environ, LLS_LOG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    iters = int(r.stdout.split("ITERS")[1].split()[0])
    line = [l for l in r.stderr.splitlines() if l.startswith("[lls log]")]
    assert len(line) == 1, r.stderr
    vals = [float(t.split(":")[1]) for t in line[0].split("iteration:")[1].split()]
    assert len(vals) == iters + 1
    assert vals[-1] <= 1e-12 < vals[0]
