"""The pressure solve as a CUDA graph with its stopping test on the device.

On a stream of its own each solve of fvm_step / fvm_poisson_solve runs as one
graph whose conditional loop node repeats the cycle (F64) or refinement
(mixed) until ||b - L p|| <= mg_rtol ||b|| (or mg_fixed_cycles), decided by
a controller kernel, so a step with info == NULL never waits for the device.
The graph launches the same kernels in the same order as the host loop, so
the two give the same bits; a cap reached on the device is reported by
fvm_sync."""
import pytest
import torch

import cases
from tests.gpu_util import FIELDS, need_gpu

pytestmark = pytest.mark.gpu


def _run(P, p, s, nsteps, graph):
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        solver = P.Solver(p, stream=st)
        if not graph:
            solver.fvm_profile(True)     # profiling: eager launches, host loop
        dev = P.to_device(s, p.precision == cases.MIXED)
        solver.fvm_launch_count(reset=True)
        infos = [solver.fvm_step(dev, n, 0.0) for n in range(nsteps)]
        count = solver.fvm_launch_count()
        solver.close()
    torch.cuda.synchronize()
    return dev, infos, count


@pytest.mark.parametrize("precision", [cases.F64, cases.MIXED])
def test_graph_solve_equals_host_loop(precision):
    P = need_gpu()
    p, s = cases.melt_pool(32, 32, 32, precision=precision)
    a, ia, na = _run(P, p, s, 3, graph=True)
    b, ib, nb = _run(P, p, s, 3, graph=False)
    for k in FIELDS:
        assert torch.equal(a[k], b[k]), k
    for x, y in zip(ia, ib):
        assert x["vcycles"] == y["vcycles"]
        assert x["rel_residual"] == y["rel_residual"]
        assert x["dt"] == y["dt"]
    # the graph adds per solve a controller reset, a test before the loop,
    # one test per cycle, the zero-rhs guard and the record store; in FP64 it
    # also launches every cycle's first finest-level sweep, which from the
    # second cycle on does nothing on the device (it would repeat the previous
    # cycle's last sweep), where the host loop does not launch it
    extra = sum(4 + c for info in ia for c in info["vcycles"])
    if precision == cases.F64:
        extra += sum(max(c - 1, 0) for info in ia for c in info["vcycles"])
    assert na == nb + extra


def test_async_step_reports_the_cycle_cap_through_sync():
    P = need_gpu()
    p, s = cases.melt_pool(16, 16, 16, precision=cases.F64)
    p = p.replace(mg_max_cycles=1, mg_rtol=1e-14)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        solver = P.Solver(p, stream=st)
        dev = P.to_device(s, False)
        out = solver.fvm_step(dev, 0, 0.0, info=False)     # does not wait
        assert out["status"] == 0
        assert solver.fvm_sync(raise_on_error=False) == P.fvm.FVM_ENOCONV
        assert solver.fvm_sync(raise_on_error=False) == 0   # cleared
        info = solver.fvm_step(dev, 1, 0.0, raise_on_error=False)
        assert info["status"] == P.fvm.FVM_ENOCONV
        assert info["vcycles"] == [1, 1, 1]
        solver.close()


def test_async_poisson_solve_with_zero_rhs_gives_zero():
    P = need_gpu()
    p = cases.Params(nx=8, ny=8, nz=8, h=0.125, bc=(1, 1, 1))
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        solver = P.Solver(p, stream=st)
        dp = torch.ones(p.shape, dtype=torch.float64, device="cuda")
        info = solver.fvm_poisson_solve(torch.zeros(p.shape, dtype=torch.float64, device="cuda"),
                                        torch.full(p.shape, 3.0, dtype=torch.float64,
                                                   device="cuda"), dp)
        assert info["vcycles"][0] == 0
        assert dp.abs().max().item() == 0.0
        solver.close()
