"""Pins of the capillary terms (Sec. III, Eq. 2-5): the Laplace jump of a
static drop, the curvature of circles and spheres, the Marangoni stress of a
flat interface, sigma as a differentiable field, and the analytic
two-layer thermocapillary channel."""
import math

import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O


def test_static_drop_laplace_jump():
    """One step of the 64 x 64 drop (R = 0.25, sigma = 1): the pressure
    jump p_in - p_out equals sigma / R = 4 within 2 %."""
    p, s = cases.static_drop()
    st, info = O.step(s, p, 0, 0.0)
    assert info["dt_limiter"] == 1
    P = st["p"].numpy()[0]
    x = (np.arange(64) + 0.5) / 64
    X, Y = np.meshgrid(x, x)
    r = np.hypot(X - 0.5, Y - 0.5)
    h = 1 / 64
    dp = P[r < 0.25 - 3 * h].mean() - P[r > 0.25 + 3 * h].mean()
    assert abs(dp - 4.0) < 0.08, dp
    assert info["max_div_dt"] < 1e-10


@pytest.mark.parametrize("dim3", [False, True])
def test_curvature_of_circle_and_sphere(dim3):
    """kappa = div n with n into the alpha = 1 phase: -1/R for a disc and
    -2/R for a ball, averaged with the interface weight |grad alpha|."""
    n = 48
    R = 0.3
    p = cases.Params(nx=n, ny=n, nz=n if dim3 else 1, h=1.0 / n, bc=(1, 1, 1 if dim3 else 0))
    x, y, z = cases.cell_centres(p)
    d = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + ((z - 0.5) ** 2 if dim3 else 0 * z))
    alpha = torch.tensor(np.broadcast_to(0.5 * (1 - np.tanh((d - R) / (1.5 * p.h))), p.shape).copy())
    grid = O.Grid(p)
    kap = O.curvature(O.smooth_alpha(alpha, grid, 2), grid)
    g = O.central_grad(O.pad_scalar(alpha, grid), grid)
    w = torch.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    kmean = (kap * w).sum().item() / w.sum().item()
    expect = -(2.0 if dim3 else 1.0) / R
    assert abs(kmean - expect) < 0.03 * abs(expect), (kmean, expect)


def test_flat_interface_marangoni_integral():
    """For a flat interface the Marangoni force summed across it equals the
    surface-tension gradient d sigma / dx (tangential term of Eq. 4 with
    delta_s = |grad alpha|: sum |g_z| h telescopes to 1), and the normal CSF
    force vanishes (kappa = 0)."""
    p = cases.Params(nx=16, ny=4, nz=24, h=0.05, bc=(0, 0, 1), sigma0=1.0, dsigma_dT=-0.3, T0=0.0)
    x, y, z = cases.cell_centres(p)
    zi = 12 * p.h + 0.37 * p.h
    alpha = 0.5 * (1 - np.tanh((z - zi) / (1.2 * p.h)))
    alpha = np.broadcast_to(alpha, p.shape).copy()
    alpha = (alpha - alpha.min()) / (alpha.max() - alpha.min())
    k = 2 * math.pi / (p.nx * p.h)
    T = np.broadcast_to(0.7 * np.sin(k * x), p.shape).copy()
    grid = O.Grid(p)
    a = torch.tensor(alpha)
    forces, kappa, gn = O.interface_forces(a, O.smooth_alpha(a, grid, 2), torch.tensor(T), p, grid)
    fn_x, fM_x = forces[0]
    colsum = fM_x.sum(dim=0) * p.h                     # sum over z at each (y, x-face)
    xf = np.arange(p.nx) * p.h
    # face value of d sigma/dx: mean of the two cells' central differences of sigma
    ds_c = p.dsigma_dT * 0.7 * (np.sin(k * (x + p.h)) - np.sin(k * (x - p.h))) / (2 * p.h)
    ds_c = ds_c.reshape(-1)
    ds_f = 0.5 * (np.roll(ds_c, 1) + ds_c)
    assert np.abs(colsum.numpy() - ds_f[None, :]).max() < 1e-12 * np.abs(ds_f).max() + 1e-14
    # the unit normal is only defined where grad alpha is not ~0; weighted by
    # the interface delta the curvature, and so the normal force, vanishes
    fn_z = forces[2][0]
    assert fn_x.abs().max().item() < 1e-12
    assert fn_z.abs().max().item() < 1e-6 * abs(p.sigma0) / p.h ** 2


def test_sigma_gradient_as_field_matches_chain_rule():
    """Eq. 5 / Sec. IV: differentiating the cell field sigma(T) equals
    dsigma/dT times the gradient of T for a linear law."""
    p = cases.Params(nx=10, ny=8, nz=6, h=0.1, bc=(1, 0, 1), sigma0=1.9, dsigma_dT=-4.3e-4,
                     T0=1700.0, tbc=(0, 0, 0, 0, 1, 1), tbc_T0=(0, 0, 0, 0, 1800.0, 1700.0))
    T = torch.tensor(1700.0 + 50.0 * cases.uniform(3, p.shape, -1, 1))
    grid = O.Grid(p)
    TP = O.pad_temperature(T, p, grid)
    gs = O.central_grad(O.sigma_of_T(TP, p), grid)
    gT = O.central_grad(TP, grid)
    for d in range(3):
        ref = p.dsigma_dT * gT[d]
        assert (gs[d] - ref).abs().max().item() <= 1e-12 * ref.abs().max().item() + 1e-15


def _channel_analytic(k, zi, H, F0, mu=1.0):
    """Stokes flow of two equal layers between no-slip walls z = 0, H, with
    a flat impermeable interface at zi carrying the tangential stress
    F0 sin(kx): stream function F(z) sin(kx) with
    F = (A + B z) cosh kz + (C + D z) sinh kz in each layer."""
    def basis(z):
        c, s = math.cosh(k * z), math.sinh(k * z)
        F = [c, z * c, s, z * s]
        dF = [k * s, c + z * k * s, k * c, s + z * k * c]
        d2F = [k * k * c, 2 * k * s + z * k * k * c, k * k * s, 2 * k * c + z * k * k * s]
        return np.array(F), np.array(dF), np.array(d2F)
    A = np.zeros((8, 8))
    b = np.zeros(8)
    F, dF, _ = basis(0.0)
    A[0, :4], A[1, :4] = F, dF                 # no slip, no penetration at z = 0
    F, dF, _ = basis(H)
    A[2, 4:], A[3, 4:] = F, dF                 # and at z = H
    F, dF, d2 = basis(zi)
    A[4, :4] = F                               # w = 0 on the interface, both sides
    A[5, 4:] = F
    A[6, :4], A[6, 4:] = dF, -dF               # u continuous
    A[7, :4], A[7, 4:] = -mu * d2, mu * d2     # mu [u_z] = -d sigma / dx
    b[7] = -F0
    c = np.linalg.solve(A, b)

    def fields(z):
        F_, dF_ = [], []
        for zz in z:
            Fb, dFb, _ = basis(zz)
            cc = c[:4] if zz < zi else c[4:]
            F_.append(Fb @ cc)
            dF_.append(dFb @ cc)
        return np.array(F_), np.array(dF_)
    return fields


def _channel_error(nz, T_end=0.1):
    p, s = cases.thermocapillary_channel(nx=2 * nz, ny=1, nz=nz)
    h, H, zi, k = p.h, 1.0, 0.5, math.pi
    F0 = -p.dsigma_dT * 1.0 * k * math.sinh(k * (H - zi)) / math.sinh(k * H)
    fields = _channel_analytic(k, zi, H, F0)
    xf, xc = np.arange(p.nx) * h, (np.arange(p.nx) + 0.5) * h
    zc, zf = (np.arange(nz) + 0.5) * h, np.arange(nz) * h
    _, dF_c = fields(zc)
    F_f, _ = fields(zf)
    s["u"][:, 0, :] = dF_c[:, None] * np.sin(k * xf)[None, :]
    s["w"][:, 0, :] = -k * F_f[:, None] * np.cos(k * xc)[None, :]
    s["w"][0] = 0.0
    ua = s["u"].copy()
    nsteps = int(math.ceil(T_end / (0.25 * h * h)))
    dt = T_end / nsteps
    st = s
    for i in range(nsteps):
        st, info = O.step(st, p, i, dt)
    return math.sqrt(((st["u"].numpy() - ua) ** 2).sum() / (ua ** 2).sum())


def test_thermocapillary_channel_matches_stokes_solution():
    """Two-layer channel with wall temperature cos(kx) (Re, Ma << 1): after
    five viscous e-folding times from the analytic state the discrete flow
    stays within 6 % of the Stokes solution at 16 cells per height and the
    error falls at second order."""
    e8, e16 = _channel_error(8), _channel_error(16)
    assert e16 < 0.06, e16
    assert e8 / e16 > 3.0, (e8, e16)
