"""Reverse mode of the oracle step (TEST INFRASTRUCTURE ONLY, like the rest of
``oracle/``): the exact vector-Jacobian product of one SSP-RK3 step with
respect to the state and the two parameters theta = (dsigma/dT, heat-source
power), obtained by PyTorch autograd through the oracle's own float64
operators.

The projection solve enters through ``_Solve``: its forward is the oracle's
multigrid solve converged to ``rtol`` (not a fixed number of cycles), and its
backward applies the same solve to the incoming gradient -- the operator
L = -D beta G is symmetric for any face coefficients beta, and the mean
removal before and after the solve is an orthogonal projector, so the
adjoint of b -> p is the solve itself.  With unequal phase densities beta
depends on alpha: p = L^+ b gives dp = -L^+ (dL) p, so the gradient of a
face coefficient is -(gb_R - gb_L)(p_R - p_L)/h^2 with gb = L^+ (dJ/dp)
(the bilinear form of L), and autograd carries it on to alpha through
beta = 1/rho_f; every other property of the mixture (mu, lambda, rho c_p)
is differentiated by autograd through the oracle's own operators.  The dt is
fixed.
"""
from __future__ import annotations

import torch

from . import fvm_oracle as O


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, alpha, prm, grid, rtol, beta0, beta1, beta2):
        q = prm.replace(mg_rtol=rtol, mg_fixed_cycles=0, mg_max_cycles=400)
        b = b - b.mean()
        p, _, _ = O.mg_solve(alpha.detach(), b.detach(), torch.zeros_like(b), q, grid)
        ctx.saved = (alpha.detach(), q, grid, p)
        return p

    @staticmethod
    def backward(ctx, gp):
        alpha, q, grid, p = ctx.saved
        g = gp - gp.mean()
        gb, _, _ = O.mg_solve(alpha, g, torch.zeros_like(g), q, grid)
        gb = gb - gb.mean()
        gbeta = []
        for d in range(3):
            if grid.n[d] == 1:
                gbeta.append(torch.zeros_like(p))
                continue
            w = 1.0 / (grid.h * grid.h)
            # low d-face of cell c: L = c - e_d, R = c
            gbeta.append(-(gb - O._roll_dn(gb, d)) * (p - O._roll_dn(p, d)) * w)
        return (gb, None, None, None, None) + tuple(gbeta)


def _projection(vel_star, alpha, prm, grid, dt, rtol):
    h = grid.h
    b = -O.divergence(vel_star, grid) / dt
    beta = O.fine_beta(alpha, prm, grid)
    p = _Solve.apply(b, alpha, prm, grid, rtol, *beta)
    out = []
    for d in range(3):
        u = vel_star[d] - dt * beta[d] * (p - O._roll_dn(p, d)) / h
        if grid.bc[d] == O.WALL:
            u = O._zero_wall_face(u, d)
        out.append(u)
    return out


def differentiable_step(state, prm, step_index, dt, rtol=1e-13):
    """One step with autograd-tracked state tensors and parameters; prm may
    hold 0-d tensors for dsigma_dT and q_power."""
    grid = O.Grid(prm)
    Sn = dict(state)
    for d, k in enumerate(("u", "v", "w")):
        if grid.bc[d] == O.WALL:
            Sn[k] = O._zero_wall_face(Sn[k], d)
    X = Sn
    for a, b, c in O.RK3:
        pr = O.predictor(X, prm, grid, dt, step_index, c)
        vel = _projection(pr["ustar"], X["alpha"], prm, grid, dt, rtol)
        E = {"u": vel[0], "v": vel[1], "w": vel[2], "alpha": pr["alpha"], "T": pr["T"]}
        X = {k: a * Sn[k] + b * E[k] for k in ("u", "v", "w", "alpha", "T")}
    return X


FIELDS = ("u", "v", "w", "alpha", "T")


def step_vjp(state, prm, step_index, dt, lam, rtol=1e-13):
    """(lambda_n, dtheta) with lambda_n = (dS_{n+1}/dS_n)^T lam and
    dtheta = (dS_{n+1}/dtheta)^T lam, theta = (dsigma/dT, q_power)."""
    S = {k: O._t(state[k]).clone().requires_grad_(True) for k in FIELDS}
    th = [torch.tensor(float(prm.dsigma_dT), dtype=O.DT, requires_grad=True),
          torch.tensor(float(prm.q_power), dtype=O.DT, requires_grad=True)]
    q = prm.replace(dsigma_dT=th[0], q_power=th[1])
    out = differentiable_step(S, q, step_index, dt, rtol)
    J = sum((out[k] * O._t(lam[k])).sum() for k in FIELDS)
    grads = torch.autograd.grad(J, [S[k] for k in FIELDS] + th, allow_unused=True)
    lam_n = {k: (g if g is not None else torch.zeros_like(S[k])).detach()
             for k, g in zip(FIELDS, grads[:5])}
    dth = [0.0 if g is None else g.item() for g in grads[5:]]
    return lam_n, dth


def interface_height_objective(alpha, h, target):
    """J = sum over columns (i, j) of (sum_k alpha h - target)^2 h^2 and its
    gradient with respect to alpha."""
    a = O._t(alpha)
    H = a.sum(dim=0) * h
    J = (((H - target) ** 2) * h * h).sum().item()
    g = (2.0 * (H - target) * h * h * h).unsqueeze(0).expand_as(a).clone()
    return J, g
