"""Pins of the WENO5-JS reconstruction used by the oracle (Sec. IV: high
order WENO face values)."""
import math

import numpy as np
import torch

from oracle import fvm_oracle as O


def _cell_averages_poly(c, x0, h, m):
    """Exact cell averages of sum c_k x^k over cells [x0 + i h, x0 + (i+1) h]."""
    F = lambda x: sum(ck * x ** (k + 1) / (k + 1) for k, ck in enumerate(c))
    xs = x0 + np.arange(m) * h
    return (F(xs + h) - F(xs)) / h


def test_linear_limit_reproduces_quartics():
    """With eps -> infinity the weights are the linear ones and the face value
    of a degree-4 polynomial is exact from its five cell averages."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        c = rng.normal(size=5)
        h = rng.uniform(0.05, 0.3)
        x0 = rng.uniform(-1, 1)
        avg = torch.tensor(_cell_averages_poly(c, x0, h, 5))
        val = O.weno5(*avg, 1e30).item()
        xf = x0 + 3 * h          # right face of the centre cell
        exact = sum(ck * xf ** k for k, ck in enumerate(c))
        assert abs(val - exact) <= 1e-11 * max(1.0, abs(exact))


def test_candidates_exact_for_quadratics_any_weights():
    """Every candidate stencil is exact for quadratics, so the nonlinear
    combination is exact whatever the weights (pins q0, q1, q2)."""
    rng = np.random.default_rng(2)
    for eps in (1e-6, 1e-2, 1.0):
        for _ in range(20):
            c = rng.normal(size=3)
            h = rng.uniform(0.05, 0.3)
            x0 = rng.uniform(-1, 1)
            avg = torch.tensor(_cell_averages_poly(c, x0, h, 5))
            val = O.weno5(*avg, eps).item()
            xf = x0 + 3 * h
            exact = sum(ck * xf ** k for k, ck in enumerate(c))
            assert abs(val - exact) <= 1e-12 * max(1.0, abs(exact))


def test_fifth_order_on_smooth_data():
    """Face values from cell averages of sin(2 pi x + phi): error falls at
    close to fifth order as the grid is refined."""
    errs = []
    Ns = (32, 64, 128, 256)
    phi = 0.3
    for N in Ns:
        h = 1.0 / N
        xs = np.arange(N) * h
        avg = (np.cos(2 * math.pi * xs + phi) - np.cos(2 * math.pi * (xs + h) + phi)) / (2 * math.pi * h)
        a = torch.tensor(avg)
        v = [a.roll(2 - k) for k in range(5)]          # cells i-2 .. i+2
        val = O.weno5(*v, 1e-6)
        exact = torch.tensor(np.sin(2 * math.pi * (xs + h) + phi))
        errs.append((val - exact).abs().max().item())
    slopes = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(errs) - 1)]
    assert slopes[-1] > 4.5, (errs, slopes)
    assert errs[-1] < 5e-9


def test_mirror_and_upwind_choice():
    rng = np.random.default_rng(3)
    v = [torch.tensor(rng.normal(size=16)) for _ in range(6)]
    Upos = torch.full((16,), 2.0)
    f_pos = O.upwind_flux(Upos, v, 1e-6)
    f_neg = O.upwind_flux(-Upos, v, 1e-6)
    left = O.weno5(v[0], v[1], v[2], v[3], v[4], 1e-6)
    right = O.weno5(v[5], v[4], v[3], v[2], v[1], 1e-6)
    assert torch.equal(f_pos, 2.0 * left)
    assert torch.equal(f_neg, -2.0 * right)
    # mirroring the data swaps the biased values
    mir = list(reversed(v))
    assert torch.allclose(O.upwind_flux(-Upos, mir, 1e-6), -2.0 * left, rtol=0, atol=0)


def test_step_is_not_oscillatory():
    """At a jump the reconstruction picks the smooth side: the face value
    stays within the range of the two adjacent cells (up to O(eps))."""
    for pos in range(1, 5):
        data = torch.tensor([0.0] * pos + [1.0] * (6 - pos))
        val = O.weno5(data[0], data[1], data[2], data[3], data[4], 1e-6).item()
        lo, hi = min(data[2].item(), data[3].item()), max(data[2].item(), data[3].item())
        assert lo - 1e-6 <= val <= hi + 1e-6
