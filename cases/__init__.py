"""Seeded synthetic inputs for the thermocapillary two-phase step.

This module builds parameter sets and initial states (phase fraction,
temperature, velocity, pressure) for the workloads the solver is exercised
on.  It holds none of the method's arithmetic: no flux, force, projection or
time-integration formula appears here, only geometry of the initial data and
a counter-based random generator.  Both the CPU oracle and the CUDA path
read their inputs from here, so the two always see the same bytes.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds and a final xor-shift; a double in [0,1)
is the top 53 bits times 2^-53.

Array layout (shared with the C ABI): every field is a C-contiguous float64
array of shape (nz, ny, nx), x fastest.  Velocity components are stored on
the MAC faces in "low face" form: ``u[k, j, i]`` is the x-velocity on the
face between cells (i-1, j, k) and (i, j, k); along a wall axis the entry at
index 0 is the wall face and is always 0, the face at index n is implied
(0 for a wall, equal to index 0 for a periodic axis).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass

import numpy as np

SEED = 20220919

PERIODIC, WALL = 0, 1
NEUMANN, DIRICHLET = 0, 1
F64, MIXED = 0, 1

# side order for per-side thermal boundary data: -x, +x, -y, +y, -z, +z
SIDES = ("-x", "+x", "-y", "+y", "-z", "+z")


# --------------------------------------------------------------------------
# SplitMix64
# --------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return ``count`` SplitMix64 outputs of the stream ``seed``, starting at
    draw number ``offset`` (counter-based: draw n uses state seed+(n+1)*golden).
    """
    with np.errstate(over="ignore"):
        n = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + n * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, shape, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    count = int(np.prod(shape)) if len(shape) else 1
    return (lo + (hi - lo) * uniform01(seed, count, offset)).reshape(shape)


# --------------------------------------------------------------------------
# Parameters (mirror of the C struct fvm_params)
# --------------------------------------------------------------------------
@dataclass
class Params:
    nx: int = 16
    ny: int = 16
    nz: int = 16
    h: float = 1.0 / 16
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)          # per axis x, y, z
    tbc: tuple = (NEUMANN,) * 6                         # per side (SIDES)
    tbc_T0: tuple = (0.0,) * 6                          # Dirichlet wall temperature ...
    tbc_dTamp: tuple = (0.0,) * 6                       # ... T0 + dTamp*cos(2 pi s / L_s)
    rho: tuple = (1.0, 1.0)                             # [alpha=0 phase, alpha=1 phase]
    mu: tuple = (1.0, 1.0)
    cp: tuple = (1.0, 1.0)
    lam: tuple = (1.0, 1.0)
    sigma0: float = 0.0
    dsigma_dT: float = 0.0
    T0: float = 0.0
    g: tuple = (0.0, 0.0, 0.0)
    q_power: float = 0.0
    q_radius: float = 1.0
    q_x0: float = 0.0
    q_y0: float = 0.0
    q_speed: float = 0.0                                # cells per step along +x
    cfl: float = 0.5
    c_cap: float = 0.5
    c_visc: float = 0.125
    c_therm: float = 0.125
    dt_max: float = 1.0e30
    weno_eps: float = 1.0e-6
    weno_scale: tuple = (1.0, 1.0, 1.0)                 # alpha, T, velocity
    smooth_passes: int = 2
    mg_levels: int = 16
    mg_pre: int = 2
    mg_post: int = 2
    mg_max_cycles: int = 100
    mg_fixed_cycles: int = 0
    mg_rtol: float = 1.0e-10
    coarse_rtol: float = 1.0e-12
    coarse_maxit: int = 1000
    precision: int = F64
    mx_inner_cycles: int = 2
    adjoint: int = 0
    concentration: int = 0                              # 1: transport c, sigma(c, T)
    dsigma_dc: float = 0.0                              # sigma += dsigma_dc (c - c0)
    c0: float = 0.0
    diff_c: tuple = (0.0, 0.0)                          # diffusivity of c per phase
    weno_scale_c: float = 1.0                           # WENO5 eps scale of c
    alpha_scheme: int = 0                               # 0 WENO5, 1 bounded (FCT blend)
    mg_coarse_sweeps: int = 3                           # pre/post sweeps below the finest level

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


def zero_state(p: Params) -> dict:
    keys = ("u", "v", "w", "alpha", "T", "p") + (("c",) if p.concentration else ())
    s = {k: np.zeros(p.shape) for k in keys}
    return s


def cell_centres(p: Params):
    """Cell-centre coordinates broadcast to (nz, ny, nx)."""
    x = (np.arange(p.nx) + 0.5) * p.h
    y = (np.arange(p.ny) + 0.5) * p.h
    z = (np.arange(p.nz) + 0.5) * p.h
    return x[None, None, :], y[None, :, None], z[:, None, None]


def zero_wall_faces(p: Params, s: dict) -> dict:
    """Set the wall-face entries (index 0 along a wall axis) of u, v, w to 0."""
    if p.bc[0] == WALL:
        s["u"][:, :, 0] = 0.0
    if p.bc[1] == WALL:
        s["v"][:, 0, :] = 0.0
    if p.bc[2] == WALL:
        s["w"][0, :, :] = 0.0
    return s


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
def static_drop(n: int = 64, seed: int = SEED, subsamples: int = 16):
    """2D static droplet in the unit box (64 x 64 x 1 by default).

    No-slip walls on x and y, one periodic cell in z.  Drop of the heavy
    phase (alpha = 1) centred at (0.5, 0.5) with radius 0.25 plus a seeded
    perturbation sum_{m=2..8} a_m cos(m theta + phi_m) scaled to a maximum
    of 1e-3.  alpha is the cell area fraction from subsamples^2 points per
    cell.  rho 10/1, mu 0.1/0.01, sigma = 1 constant, T uniform, no gravity.
    """
    h = 1.0 / n
    p = Params(nx=n, ny=n, nz=1, h=h, bc=(WALL, WALL, PERIODIC),
               rho=(1.0, 10.0), mu=(0.01, 0.1), cp=(1.0, 1.0), lam=(1e-6, 1e-6),
               sigma0=1.0, dsigma_dT=0.0, T0=0.0, weno_scale=(1.0, 1.0, 1.0))
    r = uniform(seed, (7, 2), 0.0, 1.0)
    amp = 2.0 * r[:, 0] - 1.0
    phase = 2.0 * math.pi * r[:, 1]
    m = np.arange(2, 9)
    th = np.linspace(0.0, 2.0 * math.pi, 8192, endpoint=False)
    dr = (amp[None, :] * np.cos(m[None, :] * th[:, None] + phase[None, :])).sum(1)
    amp = amp * (1e-3 / np.abs(dr).max())

    sub = (np.arange(subsamples) + 0.5) / subsamples
    xs = ((np.arange(n)[:, None] + sub[None, :]) * h).reshape(-1)   # n*sub points
    X, Y = np.meshgrid(xs, xs, indexing="xy")                        # [y, x]
    dx, dy = X - 0.5, Y - 0.5
    rad = np.hypot(dx, dy)
    theta = np.arctan2(dy, dx)
    R = 0.25 + (amp[None, None, :] * np.cos(m[None, None, :] * theta[..., None]
                                             + phase[None, None, :])).sum(-1)
    inside = (rad < R).astype(np.float64)
    frac = inside.reshape(n, subsamples, n, subsamples).mean(axis=(1, 3))
    s = zero_state(p)
    s["alpha"][0] = frac
    return p, s


def ma_bothe_droplet(n: int = 100, precision: int = F64, subsamples: int = 8,
                     t_ref: float = 0.0):
    """The migrating droplet of Sec. V-A (Table 1): a 2D box of 4a x 4a,
    a = 1.44e-3 m, on n x n x 1 cells; a droplet of radius a (alpha = 1) at
    the centre in a medium (alpha = 0) with rho 250 / 500, c_p 5e-5 / 1e-4,
    mu 0.012 / 0.024, lambda 1.2e-6 / 2.4e-6 (medium / droplet), sigma = 0.1
    and Marangoni coefficient 0.02, read as sigma = 0.1 - 0.02 (T - 290).
    No-slip walls, Neumann temperature on the side walls and Dirichlet on the
    bottom (290 K) and top (290 + 200 K/m * 4a), the initial temperature the
    linear profile between them, the fluid at rest, no gravity.  alpha is the
    cell area fraction from subsamples^2 points per cell.

    Temperatures are stored relative to t_ref (only T - 290 enters the
    model).  The mixed form keeps T in float: at 290 K a float resolves
    3e-5 K, against 0.0115 K between neighbouring cells at n = 100, so it
    wants t_ref = 290."""
    a = 1.44e-3
    L = 4.0 * a
    h = L / n
    grad = 200.0
    p = Params(nx=n, ny=n, nz=1, h=h, bc=(WALL, WALL, PERIODIC),
               tbc=(NEUMANN, NEUMANN, DIRICHLET, DIRICHLET, NEUMANN, NEUMANN),
               tbc_T0=(0.0, 0.0, 290.0 - t_ref, 290.0 - t_ref + grad * L, 0.0, 0.0),
               tbc_dTamp=(0.0,) * 6,
               rho=(250.0, 500.0), mu=(0.012, 0.024), cp=(5e-5, 1e-4), lam=(1.2e-6, 2.4e-6),
               sigma0=0.1, dsigma_dT=-0.02, T0=290.0 - t_ref, g=(0.0, 0.0, 0.0),
               weno_scale=(1.0, grad * L, 0.01), precision=precision)
    sub = (np.arange(subsamples) + 0.5) / subsamples
    xs = ((np.arange(n)[:, None] + sub[None, :]) * h).reshape(-1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")                        # [y, x]
    inside = (np.hypot(X - 0.5 * L, Y - 0.5 * L) < a).astype(np.float64)
    s = zero_state(p)
    s["alpha"][0] = inside.reshape(n, subsamples, n, subsamples).mean(axis=(1, 3))
    _, y, _ = cell_centres(p)
    s["T"][:] = np.broadcast_to(290.0 - t_ref + grad * y, p.shape)
    return p, s


def thermocapillary_channel(nx: int = 128, ny: int = 128, nz: int = 64, dT: float = 1.0,
                            sigmaT: float = 0.01):
    """Two-layer thermocapillary channel (box 2 x 2 x 1 at 128 x 128 x 64).

    Periodic x, y; no-slip walls in z with Dirichlet temperature:
    bottom T0 + dT cos(2 pi x / Lx), top T0.  Flat interface at mid-height
    (alpha = 1 below).  Equal unit properties in both layers,
    sigma(T) = 1 - sigmaT (T - T0).  Initial state at rest with the pure
    conduction temperature field of those walls.
    """
    h = 1.0 / nz
    Lx = nx * h
    p = Params(nx=nx, ny=ny, nz=nz, h=h, bc=(PERIODIC, PERIODIC, WALL),
               tbc=(NEUMANN, NEUMANN, NEUMANN, NEUMANN, DIRICHLET, DIRICHLET),
               tbc_T0=(0.0,) * 6, tbc_dTamp=(0.0, 0.0, 0.0, 0.0, dT, 0.0),
               rho=(1.0, 1.0), mu=(1.0, 1.0), cp=(1.0, 1.0), lam=(1.0, 1.0),
               sigma0=1.0, dsigma_dT=-sigmaT, T0=0.0, weno_scale=(1.0, max(dT, 1e-30), 1.0))
    s = zero_state(p)
    x, y, z = cell_centres(p)
    H = nz * h
    k = 2.0 * math.pi / Lx
    T = dT * np.cos(k * x) * np.sinh(k * (H - z)) / math.sinh(k * H)
    s["T"][:] = np.broadcast_to(T, p.shape)
    s["alpha"][:] = np.broadcast_to((z < 0.5 * H).astype(np.float64), p.shape)
    return p, s


def melt_pool(nx: int = 256, ny: int = 256, nz: int = 256, h: float = 2e-6,
              seed: int = SEED, q_power: float = 5e-3, precision: int = MIXED,
              noise_corr_cells: float = 8.0):
    """Melt-pool surrogate (256^3 by default, h = 2 um).

    Periodic x, y; walls in z (adiabatic).  Liquid 316L-like layer
    (alpha = 1) below z = nz/2 cells: rho 7900, mu 5.85e-3, cp 790,
    lambda 6.6; gas above: rho 1, mu 5.85e-5, cp 1900, lambda 0.02.
    sigma0 1.908 N/m, dsigma/dT = -4.3e-4 N/(m K), T0 = 1700 K with a seeded
    smooth 1 % temperature perturbation (correlation length ~8 cells).  Gaussian surface heat flux of radius 8 cells starting
    at (nx/8, ny/2) cells and moving +x by 0.5 cell per step; gravity -z.
    """
    p = Params(nx=nx, ny=ny, nz=nz, h=h, bc=(PERIODIC, PERIODIC, WALL),
               rho=(1.0, 7900.0), mu=(5.85e-5, 5.85e-3), cp=(1900.0, 790.0),
               lam=(0.02, 6.6), sigma0=1.908, dsigma_dT=-4.3e-4, T0=1700.0,
               g=(0.0, 0.0, -9.81), q_power=q_power, q_radius=8.0 * h,
               q_x0=(nx // 8) * h, q_y0=(ny // 2) * h, q_speed=0.5,
               weno_scale=(1.0, 17.0, 1.0), precision=precision)
    s = zero_state(p)
    x, y, z = cell_centres(p)
    s["alpha"][:] = np.broadcast_to((z < (nz // 2) * h).astype(np.float64), p.shape)
    s["T"][:] = p.T0 * (1.0 + 0.01 * smooth_noise(seed, p.shape, corr_cells=noise_corr_cells))
    return p, s


def smooth_noise(seed: int, shape, corr_cells: float = 8.0) -> np.ndarray:
    """Seeded random field with values in [-1, 1] and a correlation length of
    about ``corr_cells`` cells: uniform white noise low-pass filtered in
    Fourier space by exp(-(k corr/2)^2), then scaled to max |value| = 1."""
    xi = uniform(seed, shape, -1.0, 1.0)
    F = np.fft.rfftn(xi)
    ks = [np.fft.fftfreq(n) for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    K2 = np.zeros(F.shape)
    for ax, k in enumerate(ks):
        sh = [1] * len(shape)
        sh[ax] = k.size
        K2 = K2 + (2 * math.pi * k.reshape(sh)) ** 2
    F *= np.exp(-K2 * (corr_cells / 2.0) ** 2)
    out = np.fft.irfftn(F, s=shape, axes=tuple(range(len(shape))))
    return out / np.abs(out).max()


def adjoint_channel(nx: int = 32, ny: int = 32, nz: int = 16, dT: float = 1.0,
                    sigmaT: float = 0.01, q_power: float = 0.05, ripple: float = 0.6):
    """The thermocapillary channel physics (equal unit properties, Dirichlet
    cos(2 pi x / L) bottom wall) with a stationary Gaussian surface source of
    radius 8 cells at the centre of the interface; the interface (a tanh
    profile 1.2 cells wide) carries a seeded ripple of `ripple` cells so that
    curvature, Marangoni and WENO terms are all active (ripple = 0: the flat
    interface of the channel).  Used for gradients with respect to
    theta = (dsigma/dT, q_power)."""
    p, s = thermocapillary_channel(nx=nx, ny=ny, nz=nz, dT=dT, sigmaT=sigmaT)
    h = p.h
    p = p.replace(q_power=q_power, q_radius=8.0 * h, q_x0=0.5 * nx * h, q_y0=0.5 * ny * h,
                  q_speed=0.0)
    x, y, z = cell_centres(p)
    r = uniform(SEED + 7, (4,), 0.0, 1.0)
    Lx, Ly = nx * h, ny * h
    zi = 0.5 * nz * h + ripple * h * (np.cos(2 * math.pi * x / Lx + 6.283 * r[0]) *
                                    np.cos(2 * math.pi * y / Ly + 6.283 * r[1]))
    s["alpha"][:] = np.broadcast_to(0.5 * (1.0 - np.tanh((z - zi) / (1.2 * h))), p.shape)
    return p, s


def random_smooth_state(p: Params, seed: int = SEED, amp_u: float = 1.0,
                        drop: bool = True, T_amp: float = 1.0, modes: int = 3) -> dict:
    """A seeded smooth test state: a few Fourier modes per velocity component
    and temperature, plus a blurred spherical drop of the alpha = 1 phase.
    Wall-face entries of the velocities are zero."""
    s = zero_state(p)
    x, y, z = cell_centres(p)
    L = (p.nx * p.h, p.ny * p.h, p.nz * p.h)
    off = 0
    for name, a in (("u", amp_u), ("v", amp_u), ("w", amp_u), ("T", T_amp)):
        r = uniform(seed, (modes, 7), 0.0, 1.0, offset=off)
        off += modes * 7
        f = np.zeros(p.shape)
        for mrow in r:
            kx, ky, kz = (1 + int(3 * mrow[0]), 1 + int(3 * mrow[1]), 1 + int(3 * mrow[2]))
            f = f + (2 * mrow[3] - 1) * np.cos(2 * math.pi * kx * x / L[0] + 6.283 * mrow[4]) \
                * np.cos(2 * math.pi * ky * y / L[1] + 6.283 * mrow[5]) \
                * np.cos(2 * math.pi * kz * z / L[2] + 6.283 * mrow[6])
        s[name][:] = a * f
    if p.concentration:
        r = uniform(seed + 11, (modes, 7), 0.0, 1.0)
        f = np.zeros(p.shape)
        for mrow in r:
            kx, ky, kz = (1 + int(3 * mrow[0]), 1 + int(3 * mrow[1]), 1 + int(3 * mrow[2]))
            f = f + (2 * mrow[3] - 1) * np.cos(2 * math.pi * kx * x / L[0] + 6.283 * mrow[4]) \
                * np.cos(2 * math.pi * ky * y / L[1] + 6.283 * mrow[5]) \
                * np.cos(2 * math.pi * kz * z / L[2] + 6.283 * mrow[6])
        s["c"][:] = 0.5 + 0.25 * f
    if p.nz == 1:
        s["w"][:] = 0.0
    if drop:
        c = uniform(seed, (4,), 0.3, 0.7, offset=off)
        cx, cy, cz = c[0] * L[0], c[1] * L[1], c[2] * L[2]
        R = 0.25 * min(L[0], L[1], L[2] if p.nz > 1 else L[0])
        if p.nz == 1:
            d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2) + 0 * z
        else:
            d = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        s["alpha"][:] = 0.5 * (1.0 - np.tanh((d - R) / (1.5 * p.h)))
    zero_wall_faces(p, s)
    return s


def as_float32_state(s: dict) -> dict:
    """Round the transported fields to float32 (pressure stays float64)."""
    out = {}
    for k, v in s.items():
        out[k] = v.copy() if k == "p" else v.astype(np.float32)
    return out
