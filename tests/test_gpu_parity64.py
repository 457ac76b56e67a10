"""Element-wise parity of whole steps on a grid large enough that the
multigrid runs its per-level kernels below the finest level: the 64^3
melt-pool surrogate (walls on z, periodic x and y, density ratio 7900,
Marangoni stress from the seeded temperature field, gravity, the moving
surface heat flux).  Its hierarchy is 64^3, 32^3, 16^3, ..., so the red-black
sweeps, the residual restriction and the prolongation of the 32^3 level run
as their own launches (the one-CTA coarse tail starts at 16^3 = 4096 cells),
unlike the smaller parity grids, whose coarse levels all run in the tail.

FP64: relative L2 <= 1e-11 per field with the same fixed cycle count on both
sides.  Mixed form: the per-field bounds of the mixed-form tests."""

import numpy as np
import pytest

import cases
from oracle import fvm_oracle as O
from tests.gpu_util import FIELDS, gpu_step, need_gpu, rel_l2
from tests.test_gpu_mixed import RTOL_CMP, TOL_MX

pytestmark = pytest.mark.gpu

N = 64
CYCLES = 3


def _case(precision):
    p, s = cases.melt_pool(N, N, N, precision=precision, q_power=0.05)
    return p.replace(mg_fixed_cycles=CYCLES), s


@pytest.mark.parametrize("nsteps_before", [0, 4])
def test_full_step_f64_64cubed(nsteps_before):
    """One FP64 step from the initial state, and one from the GPU's own state
    after four steps (the parity protocol: both sides step the same input)."""
    P = need_gpu()
    p, s = _case(cases.F64)
    if nsteps_before:
        s, _ = gpu_step(P, p, s, nsteps=nsteps_before)
    ref, rinfo = O.step(s, p, nsteps_before, 0.0)
    out, infos = gpu_step(P, p, s, step_index=nsteps_before)
    assert infos[0]["vcycles"] == [CYCLES] * 3
    assert infos[0]["dt"] == pytest.approx(rinfo["dt"], rel=1e-14)
    assert infos[0]["dt_limiter"] == rinfo["dt_limiter"]
    errs = {k: rel_l2(out[k], ref[k].numpy()) for k in FIELDS}
    assert max(errs.values()) <= 1e-11, errs
    assert infos[0]["vol_sum"] == pytest.approx(rinfo["vol_sum"], rel=1e-13)
    assert infos[0]["mass_sum"] == pytest.approx(rinfo["mass_sum"], rel=1e-13)


def test_full_step_mixed_64cubed():
    """The mixed step (float transport, double refinement) against the FP64
    oracle, both solved to RTOL_CMP, from the GPU FP64 state after four steps
    rounded to float."""
    P = need_gpu()
    p, s = _case(cases.F64)
    s, _ = gpu_step(P, p, s, nsteps=4)
    p = p.replace(mg_fixed_cycles=0, mg_rtol=RTOL_CMP)
    s32 = {k: (v if k == "p" else v.astype(np.float32).astype(np.float64)) for k, v in s.items()}
    ref, rinfo = O.step(s32, p, 4, 0.0)
    out, infos = gpu_step(P, p.replace(precision=cases.MIXED), s32, step_index=4)
    assert infos[0]["nan_flag"] == 0
    assert max(infos[0]["rel_residual"]) <= RTOL_CMP
    assert infos[0]["dt"] == pytest.approx(rinfo["dt"], rel=1e-6)
    errs = {k: rel_l2(out[k], ref[k].numpy()) for k in FIELDS}
    bad = {k: (errs[k], TOL_MX[k]) for k in FIELDS if not errs[k] <= TOL_MX[k]}
    assert not bad, errs
