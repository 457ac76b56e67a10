"""Pins of the bounded phase-fraction transport option (alpha_scheme = 1):
flux-corrected transport (Zalesak 1979) between the first-order upwind flux
and the WENO5 flux with the bounds 0 and 1, the reading of the paper's
Sec. V-A remark that the divergence is discretised by a mixture of
first-order bounded and high-order WENO schemes.

* a sharp block of alpha advected by a discretely divergence-free vortex
  stays within [0, 1] (WENO5 alone leaves it);
* away from the bounds no flux is limited: the result is the WENO5 one;
* the sum of alpha is conserved to round-off;
* on a tiny 1D case the fluxes equal a scalar loop over faces and cells
  written from Zalesak's formulas."""
import math

import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O


def _vortex_case(n=32, scheme=1, amp=0.6):
    """2D periodic box, equal properties, no capillarity: the projection keeps
    the velocity divergence-free; the velocity is the discrete curl of a
    streamfunction on the cell corners (exactly solenoidal on the MAC grid)."""
    h = 1.0 / n
    p = cases.Params(nx=n, ny=n, nz=1, h=h, bc=(0, 0, 0), rho=(1.0, 1.0), mu=(1e-4, 1e-4),
                     lam=(1e-6, 1e-6), weno_scale=(1.0, 1.0, 1.0), alpha_scheme=scheme,
                     mg_rtol=1e-12)
    xc = np.arange(n) * h                       # corner coordinates (i - 1/2) h + h/2
    X, Y = np.meshgrid(xc, xc, indexing="xy")   # [j, i]
    psi = amp / (2 * math.pi) * np.sin(2 * math.pi * X) * np.sin(2 * math.pi * Y)
    s = cases.zero_state(p)
    s["u"][0] = (np.roll(psi, -1, 0) - psi) / h
    s["v"][0] = -(np.roll(psi, -1, 1) - psi) / h
    a = np.zeros((n, n))
    a[n // 4:n // 2, n // 3:2 * n // 3] = 1.0
    s["alpha"][0] = a
    return p, s


def test_sharp_block_stays_within_bounds():
    p, s = _vortex_case(scheme=1)
    st = s
    for k in range(6):
        st, info = O.step(st, p, k)
    a = st["alpha"]
    assert a.min().item() >= -1e-14 and a.max().item() <= 1.0 + 1e-14, (a.min(), a.max())
    p0, s0 = _vortex_case(scheme=0)
    st0 = s0
    for k in range(6):
        st0, _ = O.step(st0, p0, k)
    a0 = st0["alpha"]
    assert a0.min().item() < -1e-6 or a0.max().item() > 1.0 + 1e-6   # WENO5 alone overshoots


def test_smooth_alpha_away_from_the_bounds_is_plain_weno():
    p, s = _vortex_case(scheme=1, amp=0.3)
    n = p.nx
    x = (np.arange(n) + 0.5) / n
    s["alpha"][0] = 0.5 + 0.2 * np.sin(2 * math.pi * x)[None, :] * np.cos(2 * math.pi * x)[:, None]
    out1, _ = O.step(s, p, 0)
    out0, _ = O.step(s, p.replace(alpha_scheme=0), 0)
    assert (out1["alpha"] - out0["alpha"]).abs().max().item() <= 1e-14


def test_bounded_transport_conserves_alpha():
    p, s = _vortex_case(scheme=1)
    v0 = s["alpha"].sum()
    st = s
    for k in range(4):
        st, _ = O.step(st, p, k)
    assert abs(st["alpha"].sum().item() - v0) <= 1e-13 * v0


def _zalesak_loop(a, U, h, dt, eps):
    """1D periodic, uniform U: face f sits between cells f-1 and f."""
    n = len(a)
    fh, fl = [], []
    for f in range(n):
        vals = [a[(f + k) % n] for k in (-3, -2, -1, 0, 1, 2)]
        if U >= 0:
            hi = O.weno5(*[torch.tensor(v, dtype=torch.float64) for v in vals[:5]], eps).item()
            lo = vals[2]
        else:
            hi = O.weno5(*[torch.tensor(v, dtype=torch.float64) for v in vals[5:0:-1]], eps).item()
            lo = vals[3]
        fh.append(U * hi)
        fl.append(U * lo)
    A = [fh[f] - fl[f] for f in range(n)]
    td = [a[c] - dt * (fl[(c + 1) % n] - fl[c]) / h for c in range(n)]
    Rp, Rm = [], []
    for c in range(n):
        lo_f, hi_f = A[c], A[(c + 1) % n]
        pin = max(0.0, lo_f) + max(0.0, -hi_f)
        pout = max(0.0, -lo_f) + max(0.0, hi_f)
        qin, qout = (1.0 - td[c]) * h / dt, td[c] * h / dt
        Rp.append(min(1.0, max(0.0, qin / pin)) if pin > 0 else 0.0)
        Rm.append(min(1.0, max(0.0, qout / pout)) if pout > 0 else 0.0)
    F = []
    for f in range(n):
        L, R = (f - 1) % n, f
        if A[f] > 0:
            th = min(Rp[R], Rm[L])
        elif A[f] < 0:
            th = min(Rp[L], Rm[R])
        else:
            th = 1.0
        F.append(fl[f] + th * A[f])
    return [-(F[(c + 1) % n] - F[c]) / h for c in range(n)]


@pytest.mark.parametrize("U", [0.8, -0.6])
def test_limited_fluxes_equal_a_scalar_loop(U):
    n, h, dt, eps = 12, 0.1, 0.05, 1e-6
    a = [0.0, 0.0, 0.0, 0.3, 1.0, 1.0, 1.0, 0.95, 0.2, 0.0, 0.0, 0.0]
    p = cases.Params(nx=n, ny=1, nz=1, h=h, bc=(0, 0, 0))
    grid = O.Grid(p)
    vel = [torch.full(p.shape, U, dtype=torch.float64), torch.zeros(p.shape, dtype=torch.float64),
           torch.zeros(p.shape, dtype=torch.float64)]
    velP = [O.pad_velocity(vel[d], grid, d) for d in range(3)]
    Ap = O.pad_scalar(torch.tensor(a, dtype=torch.float64).reshape(p.shape), grid)
    got = O.bounded_alpha_rhs(Ap, velP, grid, eps, dt).reshape(-1).tolist()
    ref = _zalesak_loop(a, U, h, dt, eps)
    assert np.abs(np.array(got) - np.array(ref)).max() <= 1e-13
    new = np.array(a) + dt * np.array(ref)
    assert new.min() >= -1e-15 and new.max() <= 1 + 1e-15
