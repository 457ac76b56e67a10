"""Pins of the solutal part of Eq. 5: a transported concentration c enters
the surface tension as sigma(c, T) = sigma0 + dsigma/dT (T - T0)
+ dsigma/dc (c - c0), and sigma is differentiated as a cell field (Sec. IV).

* The gradient of the sigma field is the chain rule of Eq. 5 for the
  linear model: dsigma/dT grad T + dsigma/dc grad c.
* Exchanging the roles of T and c leaves the step unchanged: with equal
  unit heat capacities (so that conduction of T and diffusion of c are the
  same operator) and the same WENO5 epsilon, a step driven by
  sigma = sigma0 + s (T - T0) with c passive gives the velocity and
  pressure of a step driven by sigma = sigma0 + s (c - c0) with c = T, and
  the new c of the second equals the new T of the first.  A dropped or sign-
  flipped concentration term, or a different transport of c, fails it.
* c is conserved to round-off under no-flux walls and periodic wrap."""
import numpy as np
import torch

import cases
from oracle import fvm_oracle as O


def _prm(**kw):
    base = dict(nx=16, ny=12, nz=12, h=1.0 / 16, bc=(1, 0, 1), rho=(1.0, 4.0), mu=(0.02, 0.05),
                cp=(1.0, 0.25), lam=(0.03, 0.03), sigma0=0.1, T0=0.2, g=(0.0, 0.0, -0.3),
                weno_scale=(1.0, 1.0, 1.0), weno_scale_c=1.0, concentration=1, c0=0.4,
                diff_c=(0.03, 0.03), mg_fixed_cycles=4)
    base.update(kw)
    return cases.Params(**base)


def test_sigma_field_gradient_is_the_chain_rule():
    p = _prm(dsigma_dT=-0.3, dsigma_dc=0.7)
    grid = O.Grid(p)
    s = cases.random_smooth_state(p)
    T = O.pad_scalar(torch.tensor(s["T"]), grid)
    c = O.pad_scalar(torch.tensor(s["c"]), grid)
    gs = O.central_grad(O.sigma_field(T, c, p), grid)
    gT = O.central_grad(T, grid)
    gc = O.central_grad(c, grid)
    for d in range(3):
        ref = p.dsigma_dT * gT[d] + p.dsigma_dc * gc[d]
        assert (gs[d] - ref).abs().max().item() <= 1e-13 * ref.abs().max().item()


def test_exchanging_temperature_and_concentration_leaves_the_step_unchanged():
    """rho c_p = 1 in both phases makes the T equation's conduction
    div(lambda grad T) / (rho c_p) the concentration's div(D grad c)."""
    pA = _prm(dsigma_dT=-0.4, dsigma_dc=0.0, T0=0.25, c0=0.0)
    pA = pA.replace(cp=(1.0 / pA.rho[0], 1.0 / pA.rho[1]))
    pB = pA.replace(dsigma_dT=0.0, dsigma_dc=-0.4, c0=0.25)
    s = cases.random_smooth_state(pA, amp_u=0.3)
    sA = dict(s)
    sB = dict(s)
    sB["c"] = s["T"].copy()
    outA, infoA = O.step(sA, pA, 2, 0.0)
    outB, infoB = O.step(sB, pB, 2, 0.0)
    assert infoA["dt"] == infoB["dt"]
    for k in ("u", "v", "w", "p", "alpha"):
        scale = outA[k].abs().max().item()
        assert (outA[k] - outB[k]).abs().max().item() <= 1e-12 * scale, k
    assert (outB["c"] - outA["T"]).abs().max().item() <= 1e-12 * outA["T"].abs().max().item()
    # and the concentration term is not inert: without it the flow differs
    outC, _ = O.step(sB, pB.replace(dsigma_dc=0.0), 2, 0.0)
    assert (outC["u"] - outB["u"]).abs().max().item() > 1e-6 * outB["u"].abs().max().item()


def test_concentration_is_conserved():
    for bc in ((1, 0, 1), (0, 0, 0)):
        p = _prm(bc=bc, dsigma_dT=-0.2, dsigma_dc=0.5)
        s = cases.random_smooth_state(p, amp_u=0.5)
        c0 = s["c"].sum()
        st = s
        for n in range(3):
            st, info = O.step(st, p, n)
        assert abs(st["c"].sum().item() - c0) <= 1e-13 * abs(c0), bc
