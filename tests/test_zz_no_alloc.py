"""The allocation-free pressure solve against the regular one.

fvm_poisson_solve_noalloc() exists for callers that cannot allocate device
memory (a plugin inside a host application that owns the whole device pool,
a real-time loop that must not allocate): it keeps its scratch in a static
device array inside the library.  It must give the same answer as
fvm_poisson_solve() with a caller-allocated workspace, on every call,
although all calls share (and inherit the contents of) that array.  This
file is collected last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest
import torch

import cases
from tests.gpu_util import need_gpu, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-11     # the FP64 parity bound of the GPU tests


def _alpha(p):
    x, y, z = cases.cell_centres(p)
    L = np.array([p.nx, p.ny, p.nz]) * p.h
    d = np.sqrt((x - 0.4 * L[0]) ** 2 + (y - 0.55 * L[1]) ** 2 + (z - 0.5 * L[2]) ** 2)
    return np.broadcast_to((d < 0.3 * min(L)).astype(float), p.shape).copy()


@pytest.mark.parametrize("precision", [cases.F64, cases.MIXED])
def test_noalloc_matches_workspace_solve_twice(precision):
    P = need_gpu()
    p = cases.Params(nx=32, ny=24, nz=16, h=1.0 / 32, bc=(1, 0, 1), rho=(1.0, 100.0),
                     mg_rtol=1e-10, precision=precision)
    dt = torch.float32 if precision == cases.MIXED else torch.float64
    alpha = torch.tensor(_alpha(p), dtype=dt, device="cuda")
    solver = P.Solver(p)
    for call, seed in enumerate((41, 42)):       # two calls in a row
        rhs = torch.tensor(cases.uniform(seed, p.shape, -1, 1), device="cuda")
        p_ref = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
        ref = solver.fvm_poisson_solve(alpha, rhs, p_ref)
        p_na = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
        got = P.fvm.fvm_poisson_solve_noalloc(p, alpha, rhs, p_na)
        torch.cuda.synchronize()
        assert got["status"] == 0, got
        assert got["vcycles"][0] == ref["vcycles"][0]
        assert got["rel_residual"][0] <= p.mg_rtol
        assert rel_l2(p_na.cpu().numpy(), p_ref.cpu().numpy()) <= TOL, call
    solver.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    P = need_gpu()
    p = cases.Params(nx=128, ny=128, nz=128, h=1.0 / 128, bc=(1, 1, 1))
    t = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    got = P.fvm.fvm_poisson_solve_noalloc(p, t, t, t)
    assert got["status"] == P.fvm.FVM_ENOMEM
