"""Host logic of the batched Gauss-Newton driver (nls.gauss_newton_batched) on the CPU.

The batched linear solve is replaced by a NumPy least-squares solve of the same FP32
Jacobians, so the tests exercise the driver alone: step halving, the stopping rules, the
reported reasons and the bookkeeping of problems that stop at different iterations. The GPU
solve itself is checked in test_gpu_nls.py.
"""
import numpy as np
import pytest
import torch

from paper_1912_05508_gb300 import lls, nls


def numpy_solve_batched(fail=()):
    calls = {"n": 0}

    def solve(As, bs, prec="fp16", target="fp64", **kw):
        calls["n"] += 1
        xs, infos = [], []
        for k, (A, b) in enumerate(zip(As, bs)):
            x = np.linalg.lstsq(A.double().numpy(), b.double().numpy(), rcond=None)[0]
            xs.append(torch.from_numpy(x))
            infos.append({"status": -2 if (calls["n"], k) in fail else 0})
        return xs, infos
    return solve


def exp_fits(count, seed):
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(count):
        m = int(rng.integers(50, 200))
        t = np.linspace(0.0, 4.0, m)
        theta = np.array([rng.uniform(0.5, 2.0), rng.uniform(0.3, 1.5), rng.uniform(-0.5, 0.5)])
        y = theta[0] * np.exp(-theta[1] * t) + theta[2] + 1e-3 * rng.standard_normal(m)
        probs.append((torch.from_numpy(t), torch.from_numpy(y), theta * (1.0 + 0.3 * rng.uniform(-1, 1, 3))))
    return probs


def exp_fun(probs, flip_jacobian=()):
    def fun(idx, thetas):
        rs, Js = [], []
        for i, th in zip(idx, thetas):
            t, y, _ = probs[i]
            e = torch.exp(-th[1] * t)
            rs.append(th[0] * e + th[2] - y)
            J = torch.stack([e, -th[0] * t * e, torch.ones_like(e)], dim=1)
            Js.append(-J if i in flip_jacobian else J)
        return rs, Js
    return fun


def test_fits_converge_to_the_minimiser(monkeypatch):
    scipy_opt = pytest.importorskip("scipy.optimize")
    monkeypatch.setattr(lls, "solve_batched", numpy_solve_batched())
    probs = exp_fits(8, seed=3)
    thetas, infos = nls.gauss_newton_batched(exp_fun(probs), [torch.from_numpy(p[2]) for p in probs],
                                             max_iter=60, xtol=1e-13)
    for (t, y, start), th, info in zip(probs, thetas, infos):
        tn, yn = t.numpy(), y.numpy()
        res = lambda q: q[0] * np.exp(-q[1] * tn) + q[2] - yn
        ref = scipy_opt.least_squares(res, start, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
        assert info["reason"] in ("xtol", "ftol", "no_decrease"), info
        J = np.stack([np.exp(-ref.x[1] * tn), -ref.x[0] * tn * np.exp(-ref.x[1] * tn), np.ones_like(tn)], axis=1)
        # FP32 Jacobians: the fixed point moves by about cond(J) u32 (module docstring)
        assert np.linalg.norm(th.numpy() - ref.x) <= 16 * np.linalg.cond(J) * 2.0 ** -24 * np.linalg.norm(ref.x)
        assert info["cost"] <= ref.cost * (1 + 1e-6)


def test_failed_solve_is_not_reported_converged(monkeypatch):
    # the first batched call fails for problem 1; the others carry on to convergence
    monkeypatch.setattr(lls, "solve_batched", numpy_solve_batched(fail={(1, 1)}))
    probs = exp_fits(3, seed=4)
    _, infos = nls.gauss_newton_batched(exp_fun(probs), [torch.from_numpy(p[2]) for p in probs], xtol=1e-12)
    assert infos[1] == {**infos[1], "converged": False, "reason": "solve_failed", "iters": 1}
    assert infos[0]["converged"] and infos[2]["converged"]


def test_ascent_direction_stops_without_convergence(monkeypatch):
    # a Jacobian of the wrong sign makes every Gauss-Newton step an ascent direction: no halving
    # decreases the cost while the linear model predicts a large decrease
    monkeypatch.setattr(lls, "solve_batched", numpy_solve_batched())
    probs = exp_fits(2, seed=5)
    _, infos = nls.gauss_newton_batched(exp_fun(probs, flip_jacobian={0}),
                                        [torch.from_numpy(p[2]) for p in probs], xtol=1e-12)
    assert infos[0]["reason"] == "no_decrease" and not infos[0]["converged"] and infos[0]["iters"] == 1
    assert infos[1]["converged"]


def test_iteration_cap_is_reported(monkeypatch):
    monkeypatch.setattr(lls, "solve_batched", numpy_solve_batched())
    probs = exp_fits(3, seed=6)
    _, infos = nls.gauss_newton_batched(exp_fun(probs), [torch.from_numpy(p[2]) for p in probs],
                                        max_iter=1, xtol=1e-14)
    for info in infos:
        assert info["iters"] == 1 and info["reason"] == "max_iter" and not info["converged"]


def test_step_halving_takes_over_when_the_full_step_overshoots(monkeypatch):
    # r(theta) = atan(theta) from theta = 2: the full Gauss-Newton step lands at -3.5, where
    # |atan| is larger; halving once gives a decrease, and the iteration converges to 0
    monkeypatch.setattr(lls, "solve_batched", numpy_solve_batched())
    calls = {"fun": 0}

    def fun(idx, thetas):
        calls["fun"] += 1
        rs = [torch.atan(th[:1]) for th in thetas]
        Js = [(1.0 / (1.0 + th[:1] ** 2))[:, None] for th in thetas]
        return rs, Js

    thetas, infos = nls.gauss_newton_batched(fun, [torch.tensor([2.0], dtype=torch.float64)], xtol=1e-12)
    assert infos[0]["converged"] and abs(float(thetas[0][0])) < 1e-8
    # one evaluation to start, then at least one per iteration, and more where halving happened
    assert calls["fun"] > 1 + infos[0]["iters"]
