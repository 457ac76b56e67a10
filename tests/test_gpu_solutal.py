"""GPU parity of the solutal Marangoni extension (Eq. 5, second term): a
transported concentration c with sigma(c, T) = sigma0 + dsigma/dT (T - T0)
+ dsigma/dc (c - c0), through the C ABI against the oracle.  FP64: relative
L2 <= 1e-11 per field with the same cycle count; mixed: the mixed-form
bounds, c like alpha and T (1e-6)."""
import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O
from tests.gpu_util import need_gpu, rel_l2
from tests.test_gpu_mixed import RTOL_CMP, TOL_MX
from tests.test_gpu_parity import _physics_case

pytestmark = pytest.mark.gpu

FIELDS_C = ("u", "v", "w", "alpha", "T", "p", "c")


def _case(nx, ny, nz, bc, tax):
    p = _physics_case(nx, ny, nz, bc, tax)
    return p.replace(concentration=1, dsigma_dc=0.03, c0=0.45, diff_c=(0.004, 0.012),
                     weno_scale_c=1.0)


def _gpu(P, p, s, step_index, nsteps=1):
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        solver = P.Solver(p, stream=st)
        dev = P.to_device(s, p.precision == cases.MIXED)
        infos = [solver.fvm_step(dev, step_index + n, 0.0) for n in range(nsteps)]
        solver.close()
    torch.cuda.synchronize()
    return {k: dev[k].double().cpu().numpy() for k in FIELDS_C}, infos


@pytest.mark.parametrize("nx,ny,nz,bc,tax", [(20, 12, 10, (1, 0, 1), 2), (16, 16, 12, (0, 0, 1), 2),
                                             (24, 20, 1, (1, 1, 0), 1)])
def test_step_f64_with_concentration(nx, ny, nz, bc, tax):
    P = need_gpu()
    p = _case(nx, ny, nz, bc, tax)
    s = cases.random_smooth_state(p, amp_u=0.5)
    ref, rinfo = O.step(s, p, 3, 0.0)
    out, infos = _gpu(P, p, s, 3)
    assert infos[0]["dt"] == pytest.approx(rinfo["dt"], rel=1e-14)
    assert infos[0]["dt_limiter"] == rinfo["dt_limiter"]
    errs = {k: rel_l2(out[k], ref[k].numpy()) for k in FIELDS_C}
    assert max(errs.values()) <= 1e-11, errs


def test_concentration_drives_the_flow_on_the_gpu():
    """With dsigma/dc switched off the velocity changes: the solutal term is
    live in the CUDA path, and both agree with the oracle."""
    P = need_gpu()
    p = _case(20, 12, 10, (1, 0, 1), 2)
    s = cases.random_smooth_state(p, amp_u=0.5)
    a, _ = _gpu(P, p, s, 0)
    b, _ = _gpu(P, p.replace(dsigma_dc=0.0), s, 0)
    assert rel_l2(a["u"], b["u"]) > 1e-6
    ref, _ = O.step(s, p.replace(dsigma_dc=0.0), 0, 0.0)
    assert rel_l2(b["u"], ref["u"].numpy()) <= 1e-11


def test_step_mixed_with_concentration():
    P = need_gpu()
    p = _case(20, 12, 10, (1, 0, 1), 2).replace(mg_fixed_cycles=0, mg_rtol=RTOL_CMP)
    s = cases.random_smooth_state(p, amp_u=0.5)
    s32 = {k: (v if k == "p" else v.astype(np.float32).astype(np.float64)) for k, v in s.items()}
    ref, rinfo = O.step(s32, p, 3, 0.0)
    out, infos = _gpu(P, p.replace(precision=cases.MIXED), s32, 3)
    tol = dict(TOL_MX, c=1e-6)
    errs = {k: rel_l2(out[k], ref[k].numpy()) for k in FIELDS_C}
    bad = {k: (errs[k], tol[k]) for k in FIELDS_C if not errs[k] <= tol[k]}
    assert not bad, errs
