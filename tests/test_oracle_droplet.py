"""The migrating droplet of Sec. V-A (Table 1) in the oracle, at 20 x 20
cells for 60 steps: what the paper states about the case holds — the
Marangoni stress drives two counter-rotating vortices, the droplet moves up
the temperature gradient (dsigma/dT < 0: toward the hot top wall) and the
phase volume is conserved — and the mirror symmetry of the setup about the
vertical centre line is kept."""
import numpy as np

import cases
from oracle import fvm_oracle as O


def _run(n, steps):
    p, s = cases.ma_bothe_droplet(n=n)
    st = {k: v.copy() for k, v in s.items()}
    for q in range(steps):
        st, _ = O.step(st, p, q, 0.0)
    return p, s, {k: np.asarray(v) for k, v in st.items()}


def test_droplet_vortex_pair_upward_migration_and_symmetry():
    p, s, st = _run(20, 60)
    _, y, _ = cases.cell_centres(p)
    yy = np.broadcast_to(y, p.shape)
    a0, a = s["alpha"], st["alpha"]
    # volume of the droplet phase
    assert abs(a.sum() - a0.sum()) <= 1e-12 * a0.sum()
    # centroid moves toward the hot wall (by ~0.05 cells here)
    dy = ((a * yy).sum() / a.sum() - (a0 * yy).sum() / a0.sum()) / p.h
    assert dy > 0.02, dy
    # mirror symmetry about x = L/2: alpha and v even, u odd (x-faces, face n on the wall)
    u, v = st["u"], st["v"]
    scale = max(np.abs(u).max(), np.abs(v).max())
    assert np.abs(a - a[..., ::-1]).max() <= 1e-8
    assert np.abs(v - v[..., ::-1]).max() <= 1e-8 * scale
    uf = np.concatenate([u, np.zeros_like(u[..., :1])], axis=-1)
    assert np.abs(uf + uf[..., ::-1]).max() <= 1e-8 * scale
    # two counter-rotating vortices: the circulation of each half is the flow
    # along the centre line, upward (the droplet's direction of motion)
    w = (np.diff(v, axis=-1)[:, 1:, :] - np.diff(u, axis=-2)[:, :, 1:]) / p.h
    half = w.shape[-1] // 2
    left, right = w[..., :half].sum(), w[..., half:].sum()
    assert left > 0.0 and right < 0.0
    assert abs(left + right) <= 1e-6 * abs(left)


def test_temperature_reference_does_not_change_the_model():
    """Storing temperatures relative to 290 K (what the mixed form wants)
    gives the same flow and phase field, and the same temperature shifted by
    290 K: only T - T0 enters the model."""
    p0, s0 = cases.ma_bothe_droplet(n=16)
    p1, s1 = cases.ma_bothe_droplet(n=16, t_ref=290.0)
    a, b = dict(s0), dict(s1)
    for q in range(4):
        a, _ = O.step(a, p0, q, 0.0)
        b, _ = O.step(b, p1, q, 0.0)
    a = {k: np.asarray(v) for k, v in a.items()}
    b = {k: np.asarray(v) for k, v in b.items()}
    for k in ("u", "v", "alpha", "p"):
        scale = np.abs(a[k]).max()
        assert np.abs(a[k] - b[k]).max() <= 1e-9 * scale, k
    assert np.abs((a["T"] - 290.0) - b["T"]).max() <= 1e-9
