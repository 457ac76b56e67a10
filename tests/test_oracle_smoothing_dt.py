"""Pins of the two oracle pieces that the physics pins leave loose: the
[1, 2, 1]/4 smoothing of the phase fraction used for normals and curvature
(Sec. III, the smoothed alpha behind n and kappa), and the four time-step
limits.

The smoothing is fixed by what a [1, 2, 1]/4 pass does mathematically: it
keeps linear fields, adds exactly h^2/2 of curvature per axis and pass to a
quadratic (the filter's second moment), multiplies a periodic Fourier mode
by cos^2(k h / 2), conserves the sum with wrap or even-mirror boundaries,
and equals a 27-point brute-force stencil with explicit ghost indices.

The time-step limits are checked against hand-computed closed forms on
uniform states, each limit binding in turn: the advective CFL limit, the
capillary limit of Brackbill, Kothe & Zemach (J. Comput. Phys. 100, 1992,
sqrt(rho_mean h^3 / (2 pi sigma)) with rho_mean = (rho0 + rho1)/2), the
explicit viscous and thermal diffusion limits and dt_max."""
import itertools
import math

import numpy as np
import pytest
import torch

import cases
from oracle import fvm_oracle as O


def _grid(n, bc, h=0.1):
    return O.Grid(cases.Params(nx=n[0], ny=n[1], nz=n[2], h=h, bc=bc))


def _brute_smooth(a, n, bc):
    """One pass as a 27-point tensor stencil, ghost indices written out:
    wrap on a periodic axis, mirror (ghost -1 <- 0, ghost n <- n-1) at a
    wall, and no averaging along an axis of one cell."""
    out = np.zeros_like(a)
    w = {-1: 0.25, 0: 0.5, 1: 0.25}

    def idx(c, d):
        m = n[d]
        if bc[d] == 0:
            return c % m
        if c < 0:
            return -1 - c
        if c >= m:
            return 2 * m - 1 - c
        return c

    for k, j, i in itertools.product(range(n[2]), range(n[1]), range(n[0])):
        acc = 0.0
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            wt = 1.0
            for d, o in ((0, dx), (1, dy), (2, dz)):
                if n[d] == 1:
                    wt *= 1.0 if o == 0 else 0.0
                else:
                    wt *= w[o]
            if wt == 0.0:
                continue
            acc += wt * a[idx(k + dz, 2), idx(j + dy, 1), idx(i + dx, 0)]
        out[k, j, i] = acc
    return out


@pytest.mark.parametrize("n,bc", [((5, 4, 6), (1, 0, 1)), ((6, 6, 1), (1, 1, 0)),
                                  ((4, 6, 4), (0, 0, 0)), ((4, 4, 4), (1, 1, 1))])
def test_smoothing_equals_brute_force_stencil(n, bc):
    a = cases.uniform(11, (n[2], n[1], n[0]), -1.0, 2.0)
    grid = _grid(n, bc)
    ref1 = _brute_smooth(a, n, bc)
    ref2 = _brute_smooth(ref1, n, bc)
    t = torch.tensor(a)
    assert np.abs(O.smooth_alpha(t, grid, 0).numpy() - a).max() == 0.0
    assert np.abs(O.smooth_alpha(t, grid, 1).numpy() - ref1).max() <= 1e-15
    assert np.abs(O.smooth_alpha(t, grid, 2).numpy() - ref2).max() <= 1e-15


@pytest.mark.parametrize("passes", [1, 2])
def test_smoothing_keeps_linear_and_adds_half_h2_per_axis_and_pass(passes):
    """Away from the walls (more than `passes` cells) a linear field is
    unchanged, and a x^2 + b y^2 + c z^2 gains (a + b + c) h^2 / 2 per pass:
    the [1, 2, 1]/4 weights have zero mean and second moment h^2 / 2."""
    n = (12, 10, 14)
    h = 0.1
    grid = _grid(n, (1, 1, 1), h)
    p = cases.Params(nx=n[0], ny=n[1], nz=n[2], h=h)
    x, y, z = cases.cell_centres(p)
    lin = np.broadcast_to(0.3 + 1.7 * x - 2.2 * y + 0.9 * z, p.shape)
    a, b, c = 1.3, -0.4, 2.1
    quad = np.broadcast_to(a * x ** 2 + b * y ** 2 + c * z ** 2 + 0.5 * x - y, p.shape)
    m = passes
    core = (slice(m, n[2] - m), slice(m, n[1] - m), slice(m, n[0] - m))
    out_l = O.smooth_alpha(torch.tensor(lin.copy()), grid, passes).numpy()
    out_q = O.smooth_alpha(torch.tensor(quad.copy()), grid, passes).numpy()
    assert np.abs(out_l[core] - lin[core]).max() <= 1e-13
    gain = passes * (a + b + c) * h * h / 2.0
    assert np.abs(out_q[core] - quad[core] - gain).max() <= 1e-13
    # the wall rows are not linear any more: the mirror is even, not odd
    assert np.abs(out_l - lin).max() > 1e-3


def test_smoothing_damps_periodic_modes_by_cos_squared():
    """On periodic axes a mode cos(k.x) is an eigenfunction of one pass with
    eigenvalue prod_d cos^2(k_d h / 2); axes of one cell are left alone."""
    n = (16, 8, 1)
    h = 0.25
    grid = _grid(n, (0, 0, 0), h)
    p = cases.Params(nx=n[0], ny=n[1], nz=n[2], h=h)
    x, y, _ = cases.cell_centres(p)
    kx, ky = 2 * math.pi * 3 / (n[0] * h), 2 * math.pi * 1 / (n[1] * h)
    f = np.broadcast_to(np.cos(kx * x + 0.4) * np.cos(ky * y - 1.1), p.shape).copy()
    lam = math.cos(kx * h / 2) ** 2 * math.cos(ky * h / 2) ** 2
    for passes in (1, 2):
        out = O.smooth_alpha(torch.tensor(f), grid, passes).numpy()
        assert np.abs(out - lam ** passes * f).max() <= 1e-14


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1), (1, 0, 1)])
def test_smoothing_conserves_the_sum(bc):
    n = (8, 6, 10)
    a = torch.tensor(cases.uniform(5, (n[2], n[1], n[0]), 0.0, 1.0))
    grid = _grid(n, bc)
    s0 = a.sum().item()
    for passes in (1, 2):
        s1 = O.smooth_alpha(a, grid, passes).sum().item()
        assert abs(s1 - s0) <= 1e-13 * s0


def test_odd_periodic_axis_is_rejected():
    """(i + j + k) mod 2 is no 2-colouring on a periodic axis of odd size
    n >= 3 (cells 0 and n - 1 are wrap neighbours of one colour), so such
    grids are rejected; one periodic cell (2D) stays allowed."""
    with pytest.raises(ValueError):
        _grid((15, 8, 8), (0, 0, 0))
    with pytest.raises(ValueError):
        _grid((8, 8, 3), (1, 1, 0))
    _grid((8, 8, 1), (1, 1, 0))
    _grid((15, 8, 8), (1, 0, 0))      # an odd wall axis is a valid 2-colouring


# ---------------------------------------------------------------------------
# time-step limits
def _uniform_state(p, u=0.0, v=0.0, w=0.0, alpha=0.0, T=0.0):
    s = cases.zero_state(p)
    s["u"][:] = u
    s["v"][:] = v
    s["w"][:] = w
    s["alpha"][:] = alpha
    s["T"][:] = T
    return {k: torch.tensor(a) for k, a in s.items()}


def _limit(p, **kw):
    grid = O.Grid(p)
    return O.time_step_limit(_uniform_state(p, **kw), p, grid)


BASE = dict(nx=8, ny=8, nz=8, h=0.1, bc=(0, 0, 0), rho=(1.0, 3.0), mu=(1e-9, 1e-9),
            cp=(1.0, 1.0), lam=(1e-9, 1e-9), sigma0=0.0, dsigma_dT=0.0, T0=0.0)


def test_cfl_limit_closed_form():
    p = cases.Params(**BASE)
    dt, lim = _limit(p, u=3.0, v=-1.0, w=0.5, alpha=0.25)
    assert lim == 0
    assert dt == pytest.approx(0.5 * 0.1 / 4.5, rel=1e-15)


def test_capillary_limit_closed_form():
    """Brackbill et al. (1992): dt <= sqrt(rho_mean h^3 / (2 pi sigma)),
    rho_mean = (rho0 + rho1)/2, taken with the factor 0.5."""
    p = cases.Params(**dict(BASE, sigma0=2.0, dsigma_dT=-0.5, T0=1.0))
    dt, lim = _limit(p, T=0.2)            # sigma = 2 - 0.5 (0.2 - 1) = 2.4
    assert lim == 1
    expect = 0.5 * math.sqrt((1.0 + 3.0) / 2.0 * 0.1 ** 3 / (2.0 * math.pi * 2.4))
    assert dt == pytest.approx(expect, rel=1e-14)


def test_viscous_limit_closed_form_on_the_mixture():
    """h^2 / (8 max mu/rho) with mu, rho the arithmetic mixtures of
    clamp(alpha, 0, 1)."""
    p = cases.Params(**dict(BASE, mu=(0.2, 0.9)))
    dt, lim = _limit(p, alpha=0.25)       # mu = 0.375, rho = 1.5
    assert lim == 2
    assert dt == pytest.approx(0.1 ** 2 / 8.0 / (0.375 / 1.5), rel=1e-14)
    dt1, _ = _limit(p, alpha=1.7)         # clamped to 1: mu/rho = 0.3
    assert dt1 == pytest.approx(0.1 ** 2 / 8.0 / 0.3, rel=1e-14)


def test_thermal_limit_closed_form_and_max_over_cells():
    p = cases.Params(**dict(BASE, lam=(0.05, 2.0), cp=(2.0, 0.5)))
    st = _uniform_state(p, alpha=0.0)
    st["alpha"][:, :, :4] = 1.0           # half the cells alpha = 1: lambda/(rho cp) = 4/3
    dt, lim = O.time_step_limit(st, p, O.Grid(p))
    assert lim == 3
    assert dt == pytest.approx(0.1 ** 2 / 8.0 / (2.0 / 1.5), rel=1e-14)


def test_dt_max_and_limiter_order():
    p = cases.Params(**dict(BASE, dt_max=1e-4))
    dt, lim = _limit(p, u=1.0)
    assert (dt, lim) == (1e-4, 4)
    p0 = cases.Params(**BASE)
    dt, lim = _limit(p0)                  # nothing moves and nothing diffuses
    assert lim == 2                       # the smallest finite limit (mu = 1e-9)
    assert dt == pytest.approx(0.1 ** 2 / 8.0 / (1e-9 / 1.0), rel=1e-14)
