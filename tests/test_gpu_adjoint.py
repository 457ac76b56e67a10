"""The GPU reverse-mode step (fvm_step_adjoint) against the oracle's reverse
mode (PyTorch autograd through the FP64 oracle step, itself pinned by central
differences in test_oracle_adjoint.py), and gradients of a multi-step rollout
against central differences of the GPU forward step."""
import numpy as np
import pytest
import torch

import cases
from oracle import fvm_adjoint as A
from tests.gpu_util import need_gpu, rel_l2

pytestmark = pytest.mark.gpu

FIELDS = A.FIELDS
# Both sides are FP64 with every projection converged to 1e-13; what remains
# is the summation order of the two-pass transposes (and of the atomic adds at
# boundaries) against autograd's, a few ulps per term.
TOL = 1e-9


def _case(shape, passes=2, bc=None, vel=0.02, ripple=0.6, density=1.0):
    """The channel physics; density > 1 makes the alpha = 1 phase that much
    denser with its heat capacity per mass lowered in proportion (equal
    rho c_p, viscosity and conductivity: the setting the adjoint supports)."""
    p, s = cases.adjoint_channel(nx=shape[0], ny=shape[1], nz=shape[2], ripple=ripple)
    p = p.replace(mg_rtol=1e-13, adjoint=1, smooth_passes=passes, precision=cases.F64)
    if density != 1.0:
        p = p.replace(rho=(p.rho[0], p.rho[0] * density), cp=(p.cp[0], p.cp[0] / density))
    if bc is not None:
        p = p.replace(bc=bc)
    for i, k in enumerate(("u", "v", "w")):
        s[k][:] = vel * cases.uniform(5 + i, p.shape, -1, 1)
    cases.zero_wall_faces(p, s)
    return p, s


@pytest.mark.parametrize("shape,passes,bc,density", [
    ((16, 16, 8), 2, None, 1.0),
    ((32, 32, 16), 2, None, 1.0),
    ((40, 24, 12), 2, None, 1.0),          # ragged against the 32 x 4 x 4 tiles
    ((16, 16, 8), 1, None, 1.0),
    ((16, 16, 8), 0, None, 1.0),
    ((16, 12, 8), 2, (1, 0, 1), 1.0),      # a second wall axis (x)
    ((16, 16, 8), 2, None, 10.0),          # unequal densities: the d L / d alpha terms
    ((20, 12, 8), 2, (1, 0, 1), 100.0),
])
def test_step_adjoint_matches_oracle(shape, passes, bc, density):
    P = need_gpu()
    p, s = _case(shape, passes, bc, density=density)
    dt = 0.2 * p.h * p.h
    lam = {k: cases.uniform(20 + i, p.shape, -1, 1) for i, k in enumerate(FIELDS)}
    ref, dth_ref = A.step_vjp(s, p, 2, dt, lam, rtol=1e-13)
    solver = P.Solver(p)
    dev = P.to_device(s, False)
    lam_dev = {k: torch.tensor(lam[k], device="cuda") for k in FIELDS}
    got, dth = solver.fvm_step_adjoint(dev, 2, dt, lam_dev)
    torch.cuda.synchronize()
    for k in FIELDS:
        e = rel_l2(got[k].cpu().numpy(), ref[k].numpy())
        assert e <= TOL, (k, e)
    for q in range(2):
        assert abs(dth[q] - dth_ref[q]) <= TOL * abs(dth_ref[q]), (q, dth[q], dth_ref[q])
    # the state is read only
    for k in FIELDS:
        assert np.array_equal(dev[k].cpu().numpy(), s[k])
    solver.close()


def _objective(S, T0, h):
    """J = sum |u|^2 h^3 + 1e-3 sum (T - T0)^2 h^3.  From a flat interface at
    rest both terms start at zero: the velocity comes from the Marangoni
    stress alone (J_u ~ (dsigma/dT)^2) and the temperature change mostly
    from the heat source, and the weight makes the two terms of similar size,
    so that central differences in either parameter keep their digits."""
    Ju = sum((S[k] ** 2).sum() for k in ("u", "v", "w")) * h ** 3
    JT = ((S["T"] - T0) ** 2).sum() * h ** 3
    return Ju + 1e-3 * JT


def _rollout_J(P, p, s, dts, state_delta=None, eps=0.0):
    from paper_2209_09671_gb300 import adjoint as ADJ
    solver = P.Solver(p.replace(adjoint=0))
    dev = P.to_device(s, False)
    T0 = torch.tensor(s["T"], device="cuda")
    if state_delta is not None:
        for k, d in state_delta.items():
            dev[k] += eps * torch.tensor(d, device="cuda")
    ADJ.rollout(solver, dev, 0, dts)
    J = _objective(dev, T0, p.h).item()
    solver.close()
    return J


@pytest.mark.parametrize("density", [1.0, 10.0])
def test_rollout_gradient_matches_central_differences(density):
    """Four steps of the 32 x 32 x 16 channel with a flat interface, starting
    at rest: dJ/dtheta and the directional derivative along a smooth state
    perturbation agree with central differences of the GPU forward to 1e-6
    (equal densities, and a ten times denser lower layer)."""
    P = need_gpu()
    from paper_2209_09671_gb300 import adjoint as ADJ
    p, s = _case((32, 32, 16), vel=0.0, ripple=0.0, density=density)
    dts = [0.25 * p.h * p.h] * 4
    x, y, z = cases.cell_centres(p)
    T0 = torch.tensor(s["T"], device="cuda")
    solver = P.Solver(p)
    dev = P.to_device(s, False)
    theta = torch.tensor([p.dsigma_dT, p.q_power], dtype=torch.float64, device="cuda",
                         requires_grad=True)
    ins = {k: dev[k].clone().requires_grad_(True) for k in FIELDS}
    out = ADJ.Rollout.apply(solver, 0, dts, theta, *(ins[k] for k in FIELDS), dev["p"])
    J = _objective(dict(zip(FIELDS, out)), T0, p.h)
    J.backward()
    gth = theta.grad.cpu().numpy()
    # theta
    for q, name in enumerate(("dsigma_dT", "q_power")):
        v = getattr(p, name)
        eps = 1e-4 * abs(v)
        Jp = _rollout_J(P, p.replace(**{name: v + eps}), s, dts)
        Jm = _rollout_J(P, p.replace(**{name: v - eps}), s, dts)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - gth[q]) <= 1e-6 * abs(gth[q]), (name, fd, gth[q])
    # a smooth perturbation of T and u
    delta = {"T": 0.1 * np.cos(2 * np.pi * x / (p.nx * p.h)) * np.sin(np.pi * z),
             "u": 0.01 * np.sin(2 * np.pi * y / (p.ny * p.h)) * np.sin(np.pi * z)}
    delta = {k: np.ascontiguousarray(np.broadcast_to(v, p.shape)) for k, v in delta.items()}
    ad = sum(float((ins[k].grad.cpu().numpy() * d).sum()) for k, d in delta.items())
    eps = 1e-5
    Jp = _rollout_J(P, p, s, dts, delta, eps)
    Jm = _rollout_J(P, p, s, dts, delta, -eps)
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    solver.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    P = need_gpu()
    from paper_2209_09671_gb300 import adjoint as ADJ
    p, s = _case((16, 16, 8))
    dts = [0.2 * p.h * p.h] * 5
    solver = P.Solver(p)
    dev = P.to_device(s, False)
    lam = {k: torch.tensor(cases.uniform(40 + i, p.shape, -1, 1), device="cuda")
           for i, k in enumerate(FIELDS)}
    l1, d1 = ADJ.rollout_vjp(solver, dev, 3, dts, lam, every=1)
    l5, d5 = ADJ.rollout_vjp(solver, dev, 3, dts, lam, every=5)
    l2, d2 = ADJ.rollout_vjp(solver, dev, 3, dts, lam, every=2)
    for k in FIELDS:
        assert torch.equal(l1[k], l5[k]) or rel_l2(l1[k].cpu(), l5[k].cpu()) <= 1e-13
        assert rel_l2(l1[k].cpu(), l2[k].cpu()) <= 1e-13
    assert d1 == pytest.approx(d5, rel=1e-12) and d1 == pytest.approx(d2, rel=1e-12)
    solver.close()


def test_adjoint_argument_errors():
    P = need_gpu()
    fvm = P.fvm
    p, s = _case((16, 16, 8))
    dt = 0.2 * p.h * p.h
    lam = {k: torch.zeros(p.shape, dtype=torch.float64, device="cuda") for k in FIELDS}
    # a context without the adjoint buffers
    solver = P.Solver(p.replace(adjoint=0))
    dev = P.to_device(s, False)
    with pytest.raises(fvm.FvmError) as e:
        solver.fvm_step_adjoint(dev, 0, dt, lam)
    assert e.value.status == fvm.FVM_EINVAL
    solver.close()
    # unequal viscosities, or unequal densities with unequal rho c_p
    for q in (p.replace(mu=(1.0, 2.0)), p.replace(rho=(1.0, 2.0))):
        solver = P.Solver(q)
        with pytest.raises(fvm.FvmError) as e:
            solver.fvm_step_adjoint(dev, 0, dt, lam)
        assert e.value.status == fvm.FVM_EUNSUPPORTED
        solver.close()
    solver = P.Solver(p)
    # dt must be given
    with pytest.raises(fvm.FvmError) as e:
        solver.fvm_step_adjoint(dev, 0, 0.0, lam)
    assert e.value.status == fvm.FVM_EINVAL
    # lam_n may not alias lam_np1
    with pytest.raises(fvm.FvmError) as e:
        solver.fvm_step_adjoint(dev, 0, dt, lam, lam)
    assert e.value.status == fvm.FVM_EINVAL
    # a zero adjoint stays zero
    out, dth = solver.fvm_step_adjoint(dev, 0, dt, lam)
    assert dth == [0.0, 0.0]
    for k in FIELDS:
        assert not out[k].any()
    solver.close()
