"""The window method the full-size GPU tests rely on: the oracle's stage
predictor evaluated on a crop with a 6-cell halo equals, in the crop's
interior, the predictor of the whole grid (the stencil reaches 5 cells)."""
import numpy as np
import torch

import cases
from oracle import fvm_oracle as O
from tests import test_gpu_fullsize as F


def test_cropped_windows_equal_the_full_grid():
    p, s = cases.melt_pool(48, 48, 48, precision=cases.F64)
    p = p.replace(q_x0=20 * p.h, q_y0=24 * p.h)
    for k, seed in (("u", 1), ("v", 2), ("w", 3)):
        s[k][:] = cases.uniform(seed, p.shape, -1, 1)
    cases.zero_wall_faces(p, s)
    X = {k: torch.tensor(v) for k, v in s.items()}
    full = O.predictor(X, p, O.Grid(p), 8.5e-9, 3, 0.0)
    fullh = {"u": full["ustar"][0].numpy(), "v": full["ustar"][1].numpy(),
             "w": full["ustar"][2].numpy(), "alpha": full["alpha"].numpy(), "T": full["T"].numpy()}
    for (x0, y0, z0) in [(1, 40, 10), (30, 5, 20), (44, 20, 26)]:
        ref = F._oracle_window(s, p, x0, y0, z0, 8.5e-9, 3)
        xi = np.arange(x0, x0 + F.W) % p.nx
        yi = np.arange(y0, y0 + F.W) % p.ny
        zi = np.arange(z0, z0 + F.W)
        for k in ref:
            assert np.array_equal(fullh[k][np.ix_(zi, yi, xi)], ref[k]), (k, x0, y0, z0)
