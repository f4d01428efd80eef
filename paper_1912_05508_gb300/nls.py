"""Batched nonlinear least squares as a sequence of batched linear least-squares solves.

The paper names nonlinear least squares as the next application of its solver (Sec. 6): a
Gauss-Newton iteration reduces min_theta ||r(theta)||^2 to one linear least-squares problem
per step, min_delta ||J delta + r||, which is what ``lls_solve_batched`` solves for many
independent problems in one launch (recursive Gram-Schmidt QR with low-precision products,
then R-preconditioned CGLS to FP64 accuracy).

Each step here:
  1. evaluates the residuals r_i and Jacobians J_i of all unconverged problems (the caller's
     function, on the device);
  2. solves every J_i delta_i = -r_i in the least-squares sense with one batched launch;
  3. halves the step until ||r_i(theta_i + t delta_i)|| decreases (at most ``max_halvings``
     times), which keeps Gauss-Newton monotone on problems whose residuals are not small.
A problem stops when its relative step ||t delta|| <= xtol (1 + ||theta||) or when the
Gauss-Newton decrease ||J delta||^2 falls below ftol ||r||^2 (reasons "xtol", "ftol": converged).
It also stops, without counting as converged, when its linear solve fails ("solve_failed"),
when no halving of the step decreases the cost ("no_decrease"), or at max_iter ("max_iter").
"no_decrease" is what a wrong Jacobian gives, but also what the FP32 Jacobian can give near its
fixed point, where the step it yields is no longer a descent direction of the true cost: the
driver cannot tell the two apart, so it reports the stop and leaves the judgement to the caller.

The linear solver takes the Jacobian in FP32 (the paper's setting for A), so the iteration's
fixed point satisfies J~^T r = 0 for the rounded Jacobian J~: it matches the FP64 minimiser
to about cond(J) * 2^-24 relative, while each step itself is solved to FP64 accuracy.
"""
from __future__ import annotations

from . import lls


def gauss_newton_batched(fun, thetas, max_iter=50, xtol=1e-10, ftol=1e-20, max_halvings=30,
                         prec="fp16"):
    """Minimise ||r_i(theta_i)||^2 for every problem i of a batch.

    fun(indices, thetas) -> (rs, Js): for the given problem indices and parameter vectors
        (FP64 device tensors of length n_i), the residuals (FP64, length m_i) and Jacobians
        (FP32 or FP64 (m_i, n_i)); called for the unconverged problems only.
    thetas: list of FP64 device tensors (initial guesses).
    Returns (thetas, infos) with per-problem dicts: iters, cost (||r||^2 / 2), converged and
    reason (see the module docstring).
    """
    torch = lls._torch()
    thetas = [t.clone().to(torch.float64) for t in thetas]
    batch = len(thetas)
    iters = [0] * batch
    reason = ["max_iter"] * batch
    active = list(range(batch))
    rs, Js = fun(active, [thetas[i] for i in active])
    res = {i: r for i, r in zip(active, rs)}
    jac = {i: J for i, J in zip(active, Js)}
    for _ in range(max_iter):
        if not active:
            break
        As = [lls.colmajor(jac[i], dtype=torch.float32, device=jac[i].device) for i in active]
        bs = [-res[i] for i in active]
        deltas, infos = lls.solve_batched(As, bs, prec=prec, target="fp64")
        nxt = []
        for k, i in enumerate(active):
            iters[i] += 1
            if infos[k]["status"] not in (0, 1):
                reason[i] = "solve_failed"
                continue
            d = deltas[k]
            r0 = res[i]
            f0 = float(r0 @ r0)
            pred = float(torch.linalg.norm(As[k].double() @ d) ** 2)
            t = 1.0
            accepted = None
            for _h in range(max_halvings + 1):
                trial = thetas[i] + t * d
                rt, Jt = fun([i], [trial])
                ft = float(rt[0] @ rt[0])
                if ft <= f0:
                    accepted = (trial, rt[0], Jt[0])
                    break
                t *= 0.5
            if accepted is None:                   # no decrease along the Gauss-Newton direction
                reason[i] = "no_decrease"
                continue
            step = float(torch.linalg.norm(t * d))
            thetas[i], res[i], jac[i] = accepted
            if step <= xtol * (1.0 + float(torch.linalg.norm(thetas[i]))):
                reason[i] = "xtol"
            elif pred <= ftol * max(f0, 1e-300):
                reason[i] = "ftol"
            else:
                nxt.append(i)
        active = nxt
    infos = []
    for i in range(batch):
        r = res[i]
        infos.append({"iters": iters[i], "cost": 0.5 * float(r @ r),
                      "converged": reason[i] in ("xtol", "ftol"), "reason": reason[i]})
    return thetas, infos
