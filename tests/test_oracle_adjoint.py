"""Pins of the oracle's reverse mode (the reference for the GPU adjoint step):
central finite differences of the oracle step along random state directions
and in each parameter theta = (dsigma/dT, q_power)."""
import torch

import cases
from oracle import fvm_adjoint as A
from oracle import fvm_oracle as O

FIELDS = A.FIELDS


def _inner(a, b):
    return sum(float((O._t(a[k]) * O._t(b[k])).sum()) for k in FIELDS)


def _forward(state, prm, dt):
    S = {k: O._t(state[k]) for k in FIELDS}
    with torch.no_grad():
        return A.differentiable_step(S, prm, 2, dt, rtol=1e-13)


import pytest

CASES = {
    "equal": {},
    # unequal phase densities (the d L / d alpha term of the projection) and
    # unequal viscosity, conductivity and heat capacity
    "density_ratio_10": dict(rho=(1.0, 10.0), mu=(0.5, 1.5), lam=(0.7, 1.3), cp=(2.0, 0.3)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_step_vjp_matches_central_differences(case):
    p, s = cases.adjoint_channel(nx=8, ny=8, nz=8)
    p = p.replace(**CASES[case])
    s["u"][:] = 0.02 * cases.uniform(5, p.shape, -1, 1)
    s["v"][:] = 0.02 * cases.uniform(6, p.shape, -1, 1)
    s["w"][:] = 0.02 * cases.uniform(7, p.shape, -1, 1)
    cases.zero_wall_faces(p, s)
    dt = 0.2 * p.h * p.h
    lam = {k: cases.uniform(20 + i, p.shape, -1, 1) for i, k in enumerate(FIELDS)}
    lam_n, dth = A.step_vjp(s, p, 2, dt, lam)
    # state directions
    for seed in (31, 32):
        delta = {k: cases.uniform(seed * 10 + i, p.shape, -1, 1) for i, k in enumerate(FIELDS)}
        cases.zero_wall_faces(p, delta)
        eps = 1e-6
        sp = {k: s[k] + eps * delta[k] for k in FIELDS}
        sm = {k: s[k] - eps * delta[k] for k in FIELDS}
        fd = (_inner(lam, _forward(sp, p, dt)) - _inner(lam, _forward(sm, p, dt))) / (2 * eps)
        ad = _inner(lam_n, delta)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    # parameters
    for i, name in enumerate(("dsigma_dT", "q_power")):
        v = getattr(p, name)
        # a step of 1e-3 |theta|: O(eps^2) truncation ~1e-7 relative, well above
        # the rounding of J left by the 1e-13 solves
        eps = 1e-3 * abs(v)
        fp = _inner(lam, _forward(s, p.replace(**{name: v + eps}), dt))
        fm = _inner(lam, _forward(s, p.replace(**{name: v - eps}), dt))
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - dth[i]) <= 1e-6 * abs(dth[i]), (name, fd, dth[i])
