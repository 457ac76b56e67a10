"""Parity at the benchmark's full size (256^3 melt-pool surrogate, the launch
configuration bench.py times) and at the largest configuration, plus the
edge cases of the step.

Full-size checks use what the oracle can compute piece by piece:
* the stage-local operators (smoothing, normals, curvature, Marangoni,
  WENO5 transport, momentum predictor) on sampled interior windows: the
  oracle evaluates a window cropped with a 6-cell halo, wider than the
  predictor's stencil reach (5 cells), and the window's interior is exact;
* the time-step limit and the diagnostic sums from the full arrays;
* properties that hold at any size: the projection residual, conservation
  of sum(alpha), finiteness.
"""

import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O
from tests.gpu_util import FIELDS, need_gpu, rel_l2

pytestmark = pytest.mark.gpu

HALO = 6
W = 8


def _windows(p, count=5, seed=123):
    """Interior windows (z away from the walls) whose x/y distance to the
    heat-source centre is below half the domain, so the crop's direct
    distances equal the periodic nearest-image distances of the full grid."""
    r = cases.uniform(seed, (count, 3), 0.0, 1.0)
    out = []
    for q in range(count):
        z0 = HALO + 2 + int(r[q, 2] * (p.nz - W - 2 * HALO - 4))
        x0 = int(p.q_x0 / p.h) - 40 + int(r[q, 0] * 80)
        y0 = int(p.q_y0 / p.h) - 40 + int(r[q, 1] * 80)
        out.append((x0 % p.nx, y0 % p.ny, z0))
    return out


def _crop(a, x0, y0, z0, n):
    """a[z0-HALO : z0+W+HALO, ...] with wrap in x and y."""
    zi = np.arange(z0 - HALO, z0 + W + HALO)
    yi = np.arange(y0 - HALO, y0 + W + HALO) % n[1]
    xi = np.arange(x0 - HALO, x0 + W + HALO) % n[0]
    return a[np.ix_(zi, yi, xi)]


def _oracle_window(state, p, x0, y0, z0, dt, step_index):
    size = W + 2 * HALO
    q = p.replace(nx=size, ny=size, nz=size, bc=(1, 1, 1),
                  q_x0=p.q_x0 - (x0 - HALO) * p.h, q_y0=p.q_y0 - (y0 - HALO) * p.h)
    X = {k: torch.tensor(_crop(state[k], x0, y0, z0, (p.nx, p.ny, p.nz))) for k in
         ("u", "v", "w", "alpha", "T")}
    pr = O.predictor(X, q, O.Grid(q), dt, step_index, 0.0)
    sl = (slice(HALO, HALO + W),) * 3
    return {"u": pr["ustar"][0][sl].numpy(), "v": pr["ustar"][1][sl].numpy(),
            "w": pr["ustar"][2][sl].numpy(), "alpha": pr["alpha"][sl].numpy(),
            "T": pr["T"][sl].numpy()}


@pytest.mark.parametrize("precision", [cases.MIXED, cases.F64])
def test_stage_predictor_on_full_size_windows(precision):
    P = need_gpu()
    p, s = cases.melt_pool(256, 256, 256, precision=precision)
    if precision == cases.MIXED:
        s = {k: v.astype(np.float32).astype(np.float64) for k, v in s.items()}
    dt = 8.5e-9
    step_index = 7
    solver = P.Solver(p)
    dev = P.to_device(s, precision == cases.MIXED)
    out = solver.fvm_stage_predict(dev, step_index, dt)
    torch.cuda.synchronize()
    host = {k: v.double().cpu().numpy() for k, v in out.items()}
    tol = {"u": 1e-5, "v": 1e-5, "w": 1e-5, "alpha": 1e-6, "T": 1e-6} \
        if precision == cases.MIXED else {k: 1e-11 for k in ("u", "v", "w", "alpha", "T")}
    for (x0, y0, z0) in _windows(p):
        ref = _oracle_window(s, p, x0, y0, z0, dt, step_index)
        xi = np.arange(x0, x0 + W) % p.nx
        yi = np.arange(y0, y0 + W) % p.ny
        zi = np.arange(z0, z0 + W)
        for k in ("u", "v", "w", "alpha", "T"):
            got = host[k][np.ix_(zi, yi, xi)]
            e = rel_l2(got, ref[k])
            assert e <= tol[k], (k, (x0, y0, z0), e)
    solver.close()


def test_full_size_step_properties_mixed():
    """One step of the benchmark configuration: the limits give the oracle's
    dt, every projection reaches 1e-10, sum(alpha) is conserved to float
    rounding, the double diagnostic sums equal the oracle's sums of the
    result, and nothing is non-finite."""
    P = need_gpu()
    p, s = cases.melt_pool(256, 256, 256, precision=cases.MIXED)
    s32 = {k: v.astype(np.float32).astype(np.float64) for k, v in s.items()}
    grid = O.Grid(p)
    dt_ref, lim_ref = O.time_step_limit({k: torch.tensor(v) for k, v in s32.items()}, p, grid)
    solver = P.Solver(p)
    dev = P.to_device(s32, True)
    vol0 = dev["alpha"].double().sum().item()
    info = solver.fvm_step(dev, 0, 0.0)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["nan_flag"] == 0
    assert info["dt_limiter"] == lim_ref
    assert info["dt"] == pytest.approx(dt_ref, rel=1e-6)
    assert max(info["rel_residual"]) <= p.mg_rtol
    alpha = dev["alpha"].double()
    vol1 = alpha.sum().item()
    assert abs(vol1 - vol0) <= 1e-6 * vol0
    h3 = p.h ** 3
    assert info["vol_sum"] == pytest.approx(vol1 * h3, rel=1e-12)
    mass = (O.mix(alpha.cpu(), p.rho).sum() * h3).item()
    assert info["mass_sum"] == pytest.approx(mass, rel=1e-6)
    for k in FIELDS:
        assert torch.isfinite(dev[k]).all()
    solver.close()


def test_full_size_pressure_solve_residual_f64():
    """The FP64 solve at 256^3 on the melt-pool phase field: the oracle's
    operator applied to the GPU solution leaves ||b - L p|| <= 1e-10 ||b||."""
    P = need_gpu()
    p, s = cases.melt_pool(256, 256, 256, precision=cases.F64)
    rhs = cases.uniform(77, p.shape, -1.0, 1.0)
    solver = P.Solver(p)
    dp = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    info = solver.fvm_poisson_solve(torch.tensor(s["alpha"], device="cuda"),
                                    torch.tensor(rhs, device="cuda"), dp)
    assert info["rel_residual"][0] <= 1e-10
    grid = O.Grid(p)
    alpha = torch.tensor(s["alpha"])
    lev = O.Level(grid.n, (grid.h,) * 3, grid.bc, O.fine_beta(alpha, p, grid))
    b = torch.tensor(rhs)
    b = b - b.mean()
    r = b - O.apply_L(dp.cpu(), lev)
    assert (r.norm() / b.norm()).item() <= 2e-10
    assert abs(dp.mean().item()) <= 1e-12 * dp.abs().max().item()
    solver.close()


def test_largest_configuration_step_mixed():
    """512 x 512 x 256 (67 M cells), the largest configuration: one step
    converges and conserves."""
    P = need_gpu()
    p, s = cases.melt_pool(512, 512, 256, precision=cases.MIXED)
    solver = P.Solver(p)
    dev = P.to_device(s, True)
    vol0 = dev["alpha"].double().sum().item()
    info = solver.fvm_step(dev, 0, 0.0)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["nan_flag"] == 0
    assert max(info["rel_residual"]) <= p.mg_rtol
    assert abs(dev["alpha"].double().sum().item() - vol0) <= 1e-6 * vol0
    solver.close()
    del dev
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- edge cases
def test_nonfinite_input_is_reported_not_propagated():
    P = need_gpu()
    p, s = cases.static_drop(n=16)
    s["T"][0, 3, 5] = np.nan
    solver = P.Solver(p)
    dev = P.to_device(s, False)
    info = solver.fvm_step(dev, 0, 1e-3, raise_on_error=False)
    assert info["status"] == P.fvm.FVM_EUNSTABLE
    # the context stays usable
    p2, s2 = cases.static_drop(n=16)
    dev2 = P.to_device(s2, False)
    info2 = solver.fvm_step(dev2, 0, 1e-3, raise_on_error=False)
    assert info2["status"] == 0


def test_cycle_cap_reports_no_convergence():
    P = need_gpu()
    p = cases.Params(nx=16, ny=16, nz=16, h=1 / 16, bc=(1, 1, 1), rho=(1.0, 1000.0),
                     mg_max_cycles=1, mg_rtol=1e-14)
    alpha = np.zeros(p.shape)
    alpha[:8] = 1.0
    solver = P.Solver(p)
    dp = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    info = solver.fvm_poisson_solve(torch.tensor(alpha, device="cuda"),
                                    torch.tensor(cases.uniform(3, p.shape, -1, 1), device="cuda"),
                                    dp, raise_on_error=False)
    assert info["status"] == P.fvm.FVM_ENOCONV
    assert info["vcycles"][0] == 1


def test_single_cell_and_minimum_wall_box():
    """A fully periodic single cell (no coupling at all) steps without error;
    the smallest wall box (4^3) matches the oracle to 1e-11."""
    P = need_gpu()
    p1 = cases.Params(nx=1, ny=1, nz=1, h=0.1, bc=(0, 0, 0))
    s1 = cases.zero_state(p1)
    s1["alpha"][:] = 0.3
    s1["T"][:] = 2.0
    solver = P.Solver(p1)
    dev = P.to_device(s1, False)
    info = solver.fvm_step(dev, 0, 1e-3)
    assert info["status"] == 0
    assert dev["alpha"].item() == pytest.approx(0.3, abs=1e-15)
    p4 = cases.Params(nx=4, ny=4, nz=4, h=0.25, bc=(1, 1, 1), rho=(1.0, 3.0), mu=(0.1, 0.2),
                      sigma0=0.05, dsigma_dT=-0.01, g=(0.0, 0.0, -1.0), mg_fixed_cycles=3)
    s4 = cases.random_smooth_state(p4, amp_u=0.2)
    ref, _ = O.step(s4, p4, 0, 1e-3)
    solver4 = P.Solver(p4)
    dev4 = P.to_device(s4, False)
    solver4.fvm_step(dev4, 0, 1e-3)
    torch.cuda.synchronize()
    for k in FIELDS:
        assert rel_l2(dev4[k].cpu().numpy(), ref[k].numpy()) <= 1e-11, k
