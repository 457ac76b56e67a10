"""Pins of the temperature equation (advection-diffusion with the surface
heat flux): exact linear conduction between Dirichlet walls and the energy
deposited by the Gaussian flux through a flat interface."""

import numpy as np

import cases
from oracle import fvm_oracle as O


def test_linear_conduction_is_steady():
    """u = 0, Dirichlet walls 300 / 500 with a jump in lambda: the piecewise
    linear profile with continuous flux is preserved to round-off (harmonic
    face conductivity, wall ghost 2 T_w - T)."""
    nz = 16
    h = 1.0 / nz
    p = cases.Params(nx=4, ny=4, nz=nz, h=h, bc=(0, 0, 1), tbc=(0, 0, 0, 0, 1, 1),
                     tbc_T0=(0, 0, 0, 0, 300.0, 500.0), lam=(1.0, 3.0), rho=(1.0, 1.0),
                     cp=(1.0, 1.0), sigma0=0.0)
    s = cases.zero_state(p)
    x, y, z = cases.cell_centres(p)
    s["alpha"][:] = np.broadcast_to((z < 0.5).astype(float), p.shape)
    # flux q = (500-300)/(0.5/3 + 0.5/1); T(z) piecewise linear
    q = 200.0 / (0.5 / 3.0 + 0.5 / 1.0)
    Ti = 300.0 + q * 0.5 / 3.0
    T = np.where(z < 0.5, 300.0 + q * z / 3.0, Ti + q * (z - 0.5) / 1.0)
    s["T"][:] = np.broadcast_to(T, p.shape)
    st, _ = O.step(s, p, 0, 1e-3)
    assert np.abs(st["T"].numpy() - s["T"]).max() < 1e-10


def test_heat_source_deposits_power():
    """With u = 0 and no conduction, one step raises the heat content
    sum(rho c_p T) h^3 by P dt: the Gaussian integrates to P over the plane
    and sum |d alpha/dz| h = 1 across a flat interface."""
    n = 32
    h = 1e-3
    P = 2.0
    p = cases.Params(nx=n, ny=n, nz=16, h=h, bc=(0, 0, 1), rho=(2.0, 2.0), cp=(3.0, 3.0),
                     lam=(1e-30, 1e-30), sigma0=0.0, q_power=P, q_radius=5 * h,
                     q_x0=10.3 * h, q_y0=17.0 * h, q_speed=0.5)
    s = cases.zero_state(p)
    x, y, z = cases.cell_centres(p)
    s["alpha"][:] = np.broadcast_to(0.5 * (1 - np.tanh((z - 8 * h) / (1.5 * h))), p.shape)
    s["alpha"][-1] = 0.0
    s["alpha"][0] = 1.0
    dt = 1e-4
    st, _ = O.step(s, p, 3, dt)
    dE = ((st["T"].numpy() - s["T"]) * 6.0).sum() * h ** 3
    assert abs(dE - P * dt) < 1e-6 * P * dt, (dE, P * dt)
