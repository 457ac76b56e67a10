"""GPU parity of the bounded phase-fraction transport (alpha_scheme = 1,
the flux-corrected blend of upwind and WENO5 fluxes with the bounds 0 and
1), through the C ABI against the oracle: FP64 relative L2 <= 1e-11 per
field; the mixed form keeps alpha within [0, 1] up to float rounding and
conserves it."""
import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O
from tests.gpu_util import FIELDS, gpu_step, need_gpu, rel_l2
from tests.test_gpu_parity import _physics_case
from tests.test_oracle_bounded import _vortex_case

pytestmark = pytest.mark.gpu


def test_sharp_block_f64_parity_and_bounds():
    P = need_gpu()
    p, s = _vortex_case(scheme=1)
    p = p.replace(mg_fixed_cycles=5)
    mid, _ = gpu_step(P, p, s, nsteps=3)
    assert mid["alpha"].min() >= -1e-14 and mid["alpha"].max() <= 1 + 1e-14
    ref, rinfo = O.step(mid, p, 3, 0.0)
    out, infos = gpu_step(P, p, mid, step_index=3)
    assert infos[0]["dt"] == pytest.approx(rinfo["dt"], rel=1e-14)
    errs = {k: rel_l2(out[k], ref[k].numpy()) for k in FIELDS}
    assert max(errs.values()) <= 1e-11, errs


@pytest.mark.parametrize("nx,ny,nz,bc,tax", [(20, 12, 10, (1, 0, 1), 2), (16, 8, 8, (0, 0, 0), None)])
def test_all_physics_f64_bounded(nx, ny, nz, bc, tax):
    P = need_gpu()
    p = _physics_case(nx, ny, nz, bc, tax).replace(alpha_scheme=1)
    s = cases.random_smooth_state(p, amp_u=0.5)
    s["alpha"] = (s["alpha"] > 0.5).astype(np.float64)      # a sharp drop: the limiter acts
    ref, rinfo = O.step(s, p, 3, 0.0)
    out, infos = gpu_step(P, p, s, step_index=3)
    errs = {k: rel_l2(out[k], ref[k].numpy()) for k in FIELDS}
    assert max(errs.values()) <= 1e-11, errs
    # the limiter is active here: the WENO5 step differs
    ref0, _ = O.step(s, p.replace(alpha_scheme=0), 3, 0.0)
    assert rel_l2(ref0["alpha"].numpy(), ref["alpha"].numpy()) > 1e-9


def test_sharp_block_mixed_stays_bounded_and_conserves():
    P = need_gpu()
    p, s = _vortex_case(scheme=1)
    p = p.replace(precision=cases.MIXED, mg_rtol=1e-10)
    s32 = {k: (v if k == "p" else v.astype(np.float32).astype(np.float64)) for k, v in s.items()}
    out, _ = gpu_step(P, p, s32, nsteps=6)
    a = out["alpha"]
    assert a.min() >= -1e-6 and a.max() <= 1 + 1e-6, (a.min(), a.max())
    assert abs(a.sum() - s32["alpha"].sum()) <= 1e-5 * s32["alpha"].sum()
