"""Gradients through a rollout of FP64 steps.

The reverse sweep calls ``fvm_step_adjoint`` once per step (the discrete
adjoint of one SSP-RK3 step with its three projections, run by libfvm); this
module only keeps the checkpoints: the forward rollout stores the state
(u, v, w, alpha, T and the pressure warm start p) every ``every`` steps, and
the reverse sweep recomputes each segment from its checkpoint before walking
it backwards, so device memory holds K/every + every states for K steps.

theta = (dsigma/dT, q_power) are the two model parameters whose gradients
the adjoint returns: the Marangoni coefficient of the surface tension
(Sec. II, the temperature dependence of sigma) and the absorbed power of the
Gaussian surface heat source.
"""
from __future__ import annotations

import math

import torch

from .fvm import FIELDS5

STATE_KEYS = FIELDS5 + ("p",)


def _clone(state):
    return {k: state[k].clone() for k in STATE_KEYS}


def rollout(solver, state, step0, dts):
    """Advance ``state`` in place by len(dts) steps with the given dt."""
    for n, dt in enumerate(dts):
        solver.fvm_step(state, step0 + n, float(dt), info=False)
    return state


def rollout_vjp(solver, state0, step0, dts, lam_final, every=None):
    """(lam_0, [dJ/d dsigma_dT, dJ/d q_power]) for J with dJ/dS_K = lam_final,
    S_K the state after len(dts) steps from ``state0`` (not modified)."""
    K = len(dts)
    if K == 0:
        return {k: lam_final[k].clone() for k in FIELDS5}, [0.0, 0.0]
    every = every or max(1, int(round(math.sqrt(K))))
    ckpt = {}
    s = _clone(state0)
    for n in range(K):
        if n % every == 0:
            ckpt[n] = _clone(s)
        solver.fvm_step(s, step0 + n, float(dts[n]), info=False)
    del s
    lam = {k: lam_final[k].contiguous() for k in FIELDS5}
    dth = [0.0, 0.0]
    for start in reversed(range(0, K, every)):
        stop = min(start + every, K)
        states = [ckpt.pop(start)]
        s = _clone(states[0])
        for n in range(start, stop - 1):
            solver.fvm_step(s, step0 + n, float(dts[n]), info=False)
            states.append(_clone(s))
        for n in reversed(range(start, stop)):
            lam, d = solver.fvm_step_adjoint(states[n - start], step0 + n, float(dts[n]), lam)
            dth[0] += d[0]
            dth[1] += d[1]
    return lam, dth


class Rollout(torch.autograd.Function):
    """S_K = Step^K(S_0; theta) as an autograd node.

    apply(solver, step0, dts, theta, u, v, w, alpha, T, p) -> (u, v, w, alpha, T)
    after len(dts) steps.  theta is a float64 tensor of 2 entries that must
    equal the solver's (dsigma_dT, q_power) (the context holds the values the
    kernels use); its gradient, and those of u, v, w, alpha, T, come from
    ``rollout_vjp``.  p is the pressure warm start and gets no gradient.
    """

    @staticmethod
    def forward(ctx, solver, step0, dts, theta, u, v, w, alpha, T, p):
        prm = solver.params
        want = (float(prm.dsigma_dT), float(prm.q_power))
        got = tuple(float(x) for x in theta.detach().cpu())
        if got != want:
            raise ValueError(f"theta {got} differs from the solver's {want}")
        state0 = {"u": u.detach().clone(), "v": v.detach().clone(), "w": w.detach().clone(),
                  "alpha": alpha.detach().clone(), "T": T.detach().clone(),
                  "p": p.detach().clone()}
        s = rollout(solver, _clone(state0), step0, dts)
        ctx.solver, ctx.step0, ctx.dts, ctx.state0 = solver, step0, list(dts), state0
        ctx.theta_device = theta.device
        return tuple(s[k] for k in FIELDS5)

    @staticmethod
    def backward(ctx, *grads):
        lam_final = {}
        for k, g, ref in zip(FIELDS5, grads, (ctx.state0[k] for k in FIELDS5)):
            lam_final[k] = torch.zeros_like(ref) if g is None else g.contiguous()
        lam0, dth = rollout_vjp(ctx.solver, ctx.state0, ctx.step0, ctx.dts, lam_final)
        gth = torch.tensor(dth, dtype=torch.float64, device=ctx.theta_device)
        return (None, None, None, gth) + tuple(lam0[k] for k in FIELDS5) + (None,)
