"""V-cycle shapes other than the default V(2,2) against the oracle.

The multigrid folds work into its sweeps: the prolongation into the first
post-smoothing sweep, the coarse level's first sweep into the restriction,
the mixed form's zeroing of the correction into its first sweep (or the
residual kernel), p += e into its last sweep, and it skips a finest-level
sweep that would repeat the previous cycle's last one.  Each fold needs the
sweep it rides on, so a cycle without pre- or post-smoothing on a level, an
odd number of sweeps, or another coarse-level count takes the plain passes
instead.  These cases run those shapes through the FP64 solve (fixed
cycles, against the oracle's V-cycle of the same shape at the FP64 parity
bound) and the mixed solve (to 1e-12, against the oracle's FP64 solution)."""
import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O
from tests.gpu_util import need_gpu, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def _alpha(p):
    x, y, z = cases.cell_centres(p)
    L = np.array([p.nx, p.ny, p.nz]) * p.h
    d = np.sqrt((x - 0.4 * L[0]) ** 2 + (y - 0.55 * L[1]) ** 2 + (z - 0.5 * L[2]) ** 2)
    a = np.clip(0.5 - (d - 0.3 * min(L)) / (2.0 * p.h), 0.0, 1.0)
    return np.broadcast_to(a, p.shape).copy()


# (mg_pre, mg_post, mg_coarse_sweeps); 48 x 32 x 32 has a coarse level of
# 6144 cells that sweeps on its own and a one-CTA tail below it
SHAPES = [(2, 2, 3), (0, 2, 3), (2, 0, 3), (1, 1, 0), (3, 1, 2), (1, 2, 1)]


def _params(pre, post, coarse, precision, **kw):
    return cases.Params(nx=48, ny=32, nz=32, h=1.0 / 48, bc=(1, 0, 1), rho=(1.0, 100.0),
                        mg_pre=pre, mg_post=post, mg_coarse_sweeps=coarse,
                        precision=precision, **kw)


@pytest.mark.parametrize("pre,post,coarse", SHAPES)
def test_f64_solve_of_each_shape_equals_oracle(pre, post, coarse):
    P = need_gpu()
    p = _params(pre, post, coarse, cases.F64, mg_fixed_cycles=4)
    alpha = _alpha(p)
    rhs = cases.uniform(13, p.shape, -1, 1)
    ref, cyc, _ = O.poisson_solve(alpha, rhs, np.zeros(p.shape), p)
    assert cyc == 4
    s = P.Solver(p)
    dp = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    info = s.fvm_poisson_solve(torch.tensor(alpha, device="cuda"), torch.tensor(rhs, device="cuda"),
                               dp)
    assert info["vcycles"][0] == 4
    assert rel_l2(dp.cpu().numpy(), ref.numpy()) <= TOL64
    s.close()


@pytest.mark.parametrize("pre,post,coarse,inner", [s + (2,) for s in SHAPES] +
                         [(2, 2, 3, 1), (2, 2, 3, 3), (1, 2, 3, 1)])
def test_mixed_solve_of_each_shape_reaches_double_tolerance(pre, post, coarse, inner):
    P = need_gpu()
    p = _params(pre, post, coarse, cases.MIXED, mg_rtol=1e-12, mx_inner_cycles=inner,
                mg_max_cycles=200)
    alpha = _alpha(p)
    rhs = cases.uniform(17, p.shape, -1, 1)
    ref, _, _ = O.poisson_solve(alpha, rhs, np.zeros(p.shape),
                                p.replace(precision=cases.F64, mg_rtol=1e-12))
    s = P.Solver(p)
    dp = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    info = s.fvm_poisson_solve(torch.tensor(alpha, dtype=torch.float32, device="cuda"),
                               torch.tensor(rhs, device="cuda"), dp)
    assert info["status"] == 0
    assert info["rel_residual"][0] <= 1e-12
    assert rel_l2(dp.cpu().numpy(), ref.numpy()) <= 1e-6
    s.close()
