"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
the same seeded inputs.  F64 bar: relative L2 <= 1e-11 per field per step
with the same number of multigrid cycles on both sides."""

import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O
from tests.gpu_util import FIELDS, gpu_step, need_gpu, rel_l2

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-11


def _sphere(p, R=0.3, sharp=False):
    x, y, z = cases.cell_centres(p)
    L = np.array([p.nx, p.ny, p.nz]) * p.h
    d = np.sqrt((x - 0.5 * L[0]) ** 2 + (y - 0.5 * L[1]) ** 2 + ((z - 0.5 * L[2]) ** 2 if p.nz > 1 else 0 * z))
    r = R * min(L[0], L[1])
    a = (d < r).astype(float) if sharp else 0.5 * (1 - np.tanh((d - r) / (1.5 * p.h)))
    return np.broadcast_to(a, p.shape).copy()


POISSON_CASES = [
    dict(nx=16, ny=16, nz=16, bc=(1, 1, 1), rho=(1.0, 100.0)),
    dict(nx=20, ny=12, nz=10, bc=(1, 0, 1), rho=(1.0, 7900.0)),      # ragged wall axes
    dict(nx=64, ny=64, nz=1, bc=(1, 1, 0), rho=(1.0, 10.0)),          # 2D
    dict(nx=32, ny=16, nz=8, bc=(0, 0, 0), rho=(1.0, 3.0)),           # fully periodic
]


@pytest.mark.parametrize("case", POISSON_CASES)
def test_poisson_f64_fixed_cycles(case):
    P = need_gpu()
    p = cases.Params(h=1.0 / case["nx"], mg_fixed_cycles=5, **case)
    alpha = _sphere(p, sharp=True)
    rhs = cases.uniform(7, p.shape, -1, 1)
    p0 = cases.uniform(8, p.shape, -0.1, 0.1)
    ref, cyc, rel = O.poisson_solve(alpha, rhs, p0, p)
    s = P.Solver(p)
    da = torch.tensor(alpha, device="cuda")
    dr = torch.tensor(rhs, device="cuda")
    dp = torch.tensor(p0, device="cuda")
    info = s.fvm_poisson_solve(da, dr, dp)
    out = dp.cpu().numpy()
    assert info["vcycles"][0] == 5
    assert rel_l2(out, ref.numpy()) <= TOL_F64
    assert abs(info["rel_residual"][0] - rel) <= 1e-6 * rel + 1e-15


@pytest.mark.parametrize("case", POISSON_CASES[:2])
def test_poisson_f64_to_tolerance(case):
    P = need_gpu()
    p = cases.Params(h=1.0 / case["nx"], mg_rtol=1e-11, **case)
    alpha = _sphere(p)
    rhs = cases.uniform(9, p.shape, -1, 1)
    ref, cyc, rel = O.poisson_solve(alpha, rhs, np.zeros(p.shape), p)
    s = P.Solver(p)
    dp = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    info = s.fvm_poisson_solve(torch.tensor(alpha, device="cuda"), torch.tensor(rhs, device="cuda"), dp)
    assert info["rel_residual"][0] <= 1e-11
    assert abs(info["vcycles"][0] - cyc) <= 1
    assert rel_l2(dp.cpu().numpy(), ref.numpy()) <= 1e-9


def test_poisson_zero_rhs_gives_zero():
    P = need_gpu()
    p = cases.Params(nx=8, ny=8, nz=8, h=0.125, bc=(1, 1, 1))
    s = P.Solver(p)
    dp = torch.ones(p.shape, dtype=torch.float64, device="cuda")
    info = s.fvm_poisson_solve(torch.zeros(p.shape, dtype=torch.float64, device="cuda"),
                               torch.full(p.shape, 3.0, dtype=torch.float64, device="cuda"), dp)
    assert info["vcycles"][0] == 0
    assert dp.abs().max().item() == 0.0


def _compare(out, ref, tol, fields=FIELDS):
    errs = {k: rel_l2(out[k], ref[k].numpy()) for k in fields}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, errs
    return errs


def test_step_f64_static_drop():
    """64 x 64 static drop, one step, dt from the limits, 8 cycles per stage."""
    P = need_gpu()
    p, s = cases.static_drop()
    p = p.replace(mg_fixed_cycles=8)
    ref, rinfo = O.step(s, p, 0, 0.0)
    out, infos = gpu_step(P, p, s)
    assert infos[0]["dt"] == pytest.approx(rinfo["dt"], rel=1e-14)
    assert infos[0]["dt_limiter"] == rinfo["dt_limiter"]
    _compare(out, ref, TOL_F64)
    assert infos[0]["vol_sum"] == pytest.approx(rinfo["vol_sum"], rel=1e-13)
    assert infos[0]["mass_sum"] == pytest.approx(rinfo["mass_sum"], rel=1e-13)


def _physics_case(nx, ny, nz, bc, tbc_axis=2):
    tbc = [0] * 6
    T0 = [0.0] * 6
    amp = [0.0] * 6
    if tbc_axis is not None:
        tbc[2 * tbc_axis] = 1
        tbc[2 * tbc_axis + 1] = 1
        T0[2 * tbc_axis] = 1.3
        T0[2 * tbc_axis + 1] = -0.4
        amp[2 * tbc_axis] = 0.5
    h = 1.0 / 16
    return cases.Params(nx=nx, ny=ny, nz=nz, h=h, bc=bc, tbc=tuple(tbc), tbc_T0=tuple(T0),
                        tbc_dTamp=tuple(amp), rho=(1.0, 6.0), mu=(0.02, 0.05), cp=(1.0, 2.0),
                        lam=(0.01, 0.03), sigma0=0.05, dsigma_dT=-0.02, T0=0.2,
                        g=(0.1, -0.2, -0.5), q_power=0.002, q_radius=3 * h, q_x0=5.2 * h,
                        q_y0=4.7 * h, q_speed=0.5, weno_scale=(1.0, 1.0, 1.0),
                        mg_fixed_cycles=4)


PHYS_CASES = [
    (20, 12, 10, (1, 0, 1), 2),      # ragged sizes, walls x/z, Dirichlet z
    (16, 16, 12, (0, 0, 1), 2),      # channel-like
    (12, 18, 8, (1, 1, 0), 1),       # Dirichlet on y walls
    (16, 8, 8, (0, 0, 0), None),     # fully periodic
]


@pytest.mark.parametrize("nx,ny,nz,bc,tax", PHYS_CASES)
def test_step_f64_all_physics(nx, ny, nz, bc, tax):
    """Random smooth state, every term active (WENO5 transport, CSF,
    Marangoni, Dirichlet walls, gravity, moving heat source)."""
    P = need_gpu()
    p = _physics_case(nx, ny, nz, bc, tax)
    s = cases.random_smooth_state(p, amp_u=0.5)
    ref, rinfo = O.step(s, p, 3, 0.0)
    out, infos = gpu_step(P, p, s, step_index=3)
    assert infos[0]["dt"] == pytest.approx(rinfo["dt"], rel=1e-14)
    _compare(out, ref, TOL_F64)


def test_step_f64_after_ten_gpu_steps():
    """Parity protocol: take the GPU state after 10 steps and step both from it."""
    P = need_gpu()
    p, s = cases.static_drop(n=32)
    p = p.replace(mg_fixed_cycles=6)
    mid, _ = gpu_step(P, p, s, nsteps=10)
    ref, _ = O.step(mid, p, 10, 0.0)
    out, _ = gpu_step(P, p, mid, step_index=10)
    _compare(out, ref, TOL_F64)
