"""CPU FP64 oracle of one explicit time step of the thermocapillary two-phase
finite-volume method (Zimbrod, Schreter & Schilp, "Efficient Simulation of
Complex Capillary Effects in Advanced Manufacturing Processes using the Finite
Volume Method", 2022).

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library; it
is imported by the tests, by ``__graft_entry__.smoke()`` and by the CPU
baseline / reference arm of ``bench.py``, never by the product path, and it
shares no code with it.  Every operation is plain float64 PyTorch on the CPU,
written as the definition of each discrete operator so that a reader can
check it against the paper line by line:

* Sec. III, Eq. 1 -- conservative phase-fraction transport
  (WENO5 face values, flux differences; ``scalar_rhs``).
* Sec. III, Eq. 2-4 -- capillary stress split into the normal CSF force
  -sigma kappa n delta_s and the tangential Marangoni force
  delta_s (I - n n) grad sigma (``interface_forces``).
* Sec. III, Eq. 5 and Sec. IV -- sigma evaluated cell-wise from T (and from
  a transported concentration c, the solutal term of Eq. 5) and
  differentiated as a field (``sigma_field``, central differences of sigma).
* Sec. III, delta_s = |grad alpha| and n = grad alpha / delta_s.
* Sec. III -- incompressible Navier-Stokes and energy equations, which the
  paper names but does not write out: momentum predictor with WENO5
  advection and variable-viscosity stress, pressure projection with
  beta = 1/rho, geometric multigrid, SSP-RK3 time stepping.

Where the paper is silent the discrete choices are the readings recorded in
the design notes of this repository (time integrator, MAC layout, boundary
ghosts, WENO5-JS epsilon, smoothing of alpha, curvature as the divergence of
face normals, multigrid components, time-step limits); each function below
states the reading it implements.

Field layout: tensors of shape (nz, ny, nx), x fastest.  Velocities are
stored in "low face" form: ``u[k, j, i]`` lives on the x-face between cells
i-1 and i; the face at index n along an axis is implied (0 at a wall, equal
to face 0 on a periodic axis); along a wall axis the stored face 0 is the
wall and is 0.

Parity status: every operator below is pinned by the CPU tests under
``tests/`` (closed forms, conservation, symmetry, brute force, a direct
sparse solve) except where a test file says otherwise.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64
PERIODIC, WALL = 0, 1
NEUMANN, DIRICHLET = 0, 1
G = 3                      # ghost layers: WENO5 reaches three cells across a face
AXIS_DIM = (2, 1, 0)       # direction x, y, z -> tensor dimension


def _t(a):
    return torch.as_tensor(a, dtype=DT)


def norm3(x):
    """sqrt(x) for the squared length of a gradient; equal to torch.sqrt in
    value, with the derivative at x = 0 taken as 0 (|g| has no gradient where
    g vanishes, e.g. away from the interface)."""
    pos = x > 0.0
    return torch.where(pos, torch.sqrt(torch.where(pos, x, torch.ones_like(x))), torch.zeros_like(x))


# ==========================================================================
# Grid helpers
# ==========================================================================
class Grid:
    def __init__(self, prm):
        self.n = (int(prm.nx), int(prm.ny), int(prm.nz))
        self.h = float(prm.h)
        self.bc = tuple(int(b) for b in prm.bc)
        self.L = tuple(n * self.h for n in self.n)
        for d in range(3):
            if self.bc[d] == WALL and self.n[d] < 4:
                raise ValueError("a wall axis needs at least 4 cells")
            # the red-black colour (i + j + k) mod 2 of the smoother is a
            # 2-colouring under wrap only for an even number of cells
            if self.bc[d] == PERIODIC and self.n[d] > 1 and self.n[d] % 2:
                raise ValueError("a periodic axis needs an even number of cells (or one)")

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])


def _coords(grid, d, lo=0, hi=None):
    """Cell-centre coordinate along direction d for indices lo..hi-1."""
    hi = grid.n[d] if hi is None else hi
    return (torch.arange(lo, hi, dtype=DT) + 0.5) * grid.h


def _bshape(d, m):
    s = [1, 1, 1]
    s[AXIS_DIM[d]] = m
    return s


def _cell_index(n, periodic):
    """Source index and ghost mask for extended cell indices -G..n+G-1.

    Periodic: wrap.  Wall: mirror about the boundary face
    (ghost -1-m <- cell m, ghost n+m <- cell n-1-m).
    """
    idx = torch.arange(-G, n + G)
    if periodic:
        return idx % n, torch.zeros_like(idx, dtype=torch.bool)
    src = torch.where(idx < 0, -1 - idx, torch.where(idx >= n, 2 * n - 1 - idx, idx))
    return src, (idx < 0) | (idx >= n)


def pad_cell_axis(a, grid, d, sign=1.0, wall_value=None):
    """Extend a cell-centred field by G ghost layers along direction d.

    Ghost rule at a wall: ghost = sign * mirror (+ 2*T_w for a Dirichlet
    temperature, i.e. the linear extrapolation through the wall value).
    ``wall_value`` is (lo, hi), each None or a tensor broadcastable to one
    layer, giving T_w on that side.
    """
    dim = AXIS_DIM[d]
    n = a.shape[dim]
    periodic = grid.bc[d] == PERIODIC
    src, ghost = _cell_index(n, periodic)
    out = a.index_select(dim, src)
    if periodic:
        return out
    ext = n + 2 * G
    sgn = torch.where(ghost, _t(sign), _t(1.0)).reshape(_bshape(d, ext))
    out = out * sgn
    if wall_value is not None:
        lo_mask = (torch.arange(ext) < G).to(DT).reshape(_bshape(d, ext))
        hi_mask = (torch.arange(ext) >= n + G).to(DT).reshape(_bshape(d, ext))
        if wall_value[0] is not None:
            out = out + lo_mask * 2.0 * wall_value[0]
        if wall_value[1] is not None:
            out = out + hi_mask * 2.0 * wall_value[1]
    return out


def pad_face_axis(a, grid, d):
    """Extend the d-velocity along its own direction to faces -G..n+G.

    Periodic: face n+m is face m.  Wall: faces 0 and n are 0 and the
    velocity is odd about the wall face (face -m <- -face m,
    face n+m <- -face n-m).
    """
    dim = AXIS_DIM[d]
    n = a.shape[dim]
    idx = torch.arange(-G, n + G + 1)
    if grid.bc[d] == PERIODIC:
        return a.index_select(dim, idx % n)
    src = torch.where(idx < 0, -idx, torch.where(idx > n, 2 * n - idx, idx))
    sgn = torch.where((idx < 0) | (idx > n), -1.0, 1.0).to(DT)
    sgn = torch.where((idx == 0) | (idx == n), 0.0, sgn)
    src = torch.where(src >= n, torch.zeros_like(src), src)
    ext = n + 2 * G + 1
    return a.index_select(dim, src) * sgn.reshape(_bshape(d, ext))


def pad_scalar(a, grid, sign=1.0):
    """Ghost-extend a cell field in x, then y, then z (even or odd at walls)."""
    for d in range(3):
        a = pad_cell_axis(a, grid, d, sign)
    return a


def pad_velocity(vel, grid, d):
    """Ghost-extend velocity component d: face-type along d, odd (no-slip)
    cell-type along the two tangential directions."""
    a = vel
    for e in range(3):
        a = pad_face_axis(a, grid, e) if e == d else pad_cell_axis(a, grid, e, -1.0)
    return a


def wall_temperature(prm, grid, side, ext_coords):
    """Dirichlet wall temperature T0 + dTamp cos(2 pi s / L_s) on one side;
    s is x for y- and z-walls and y for x-walls."""
    d = side // 2
    s_dir = 1 if d == 0 else 0
    s = ext_coords[s_dir]
    val = prm.tbc_T0[side] + prm.tbc_dTamp[side] * torch.cos(2.0 * math.pi * s / grid.L[s_dir])
    return val.reshape(_bshape(s_dir, s.numel()))


def pad_temperature(T, prm, grid):
    """Ghost-extend T: wrap, even mirror (Neumann) or 2 T_w - mirror (Dirichlet)."""
    a = T
    ext = []
    for d in range(3):
        ext.append(_coords(grid, d))
    for d in range(3):
        if grid.bc[d] == PERIODIC:
            a = pad_cell_axis(a, grid, d)
        else:
            lo, hi = 2 * d, 2 * d + 1
            if prm.tbc[lo] == DIRICHLET or prm.tbc[hi] == DIRICHLET:
                wv = (wall_temperature(prm, grid, lo, ext) if prm.tbc[lo] == DIRICHLET else None,
                      wall_temperature(prm, grid, hi, ext) if prm.tbc[hi] == DIRICHLET else None)
                a = _pad_T_axis(a, grid, d, prm, wv)
            else:
                a = pad_cell_axis(a, grid, d, 1.0)
        # coordinates along d now include ghosts for later axes
        ext[d] = (torch.arange(-G, grid.n[d] + G, dtype=DT) + 0.5) * grid.h
    return a


def _pad_T_axis(a, grid, d, prm, wv):
    """Wall axis with at least one Dirichlet side."""
    dim = AXIS_DIM[d]
    n = a.shape[dim]
    src, ghost = _cell_index(n, False)
    out = a.index_select(dim, src)
    ext = n + 2 * G
    idx = torch.arange(ext)
    lo_g = (idx < G)
    hi_g = (idx >= n + G)
    sgn = torch.ones(ext, dtype=DT)
    if prm.tbc[2 * d] == DIRICHLET:
        sgn = torch.where(lo_g, -1.0, sgn)
    if prm.tbc[2 * d + 1] == DIRICHLET:
        sgn = torch.where(hi_g, -1.0, sgn)
    out = out * sgn.reshape(_bshape(d, ext))
    if wv[0] is not None:
        out = out + lo_g.to(DT).reshape(_bshape(d, ext)) * 2.0 * wv[0]
    if wv[1] is not None:
        out = out + hi_g.to(DT).reshape(_bshape(d, ext)) * 2.0 * wv[1]
    return out


def S(P, grid, ox=0, oy=0, oz=0):
    """Interior-sized window of a ghost-extended array, shifted by (ox, oy, oz)
    cells/faces.  Index G of the extended array is cell (or face) 0."""
    nx, ny, nz = grid.n
    return P[G + oz:G + oz + nz, G + oy:G + oy + ny, G + ox:G + ox + nx]


def _off(d, s):
    o = [0, 0, 0]
    o[d] = s
    return o


def Sd(P, grid, *shifts):
    """Window shifted by a sum of (direction, amount) pairs."""
    o = [0, 0, 0]
    for d, s in shifts:
        o[d] += s
    return S(P, grid, *o)


# ==========================================================================
# Material properties (Sec. III; mixtures of the two phases)
# ==========================================================================
def clamp01(alpha):
    return torch.clamp(alpha, 0.0, 1.0)


def mix(alpha, pair):
    """Arithmetic mixture a*phi_1 + (1-a)*phi_0 with a = clamp(alpha, 0, 1);
    index 1 is the alpha = 1 phase."""
    a = clamp01(alpha)
    return a * pair[1] + (1.0 - a) * pair[0]


def rho_cp(alpha, prm):
    a = clamp01(alpha)
    return a * (prm.rho[1] * prm.cp[1]) + (1.0 - a) * (prm.rho[0] * prm.cp[0])


def sigma_of_T(T, prm):
    """Surface-tension coefficient as a cell field (Eq. 5, Sec. IV):
    sigma = sigma0 + (dsigma/dT) (T - T0)."""
    return prm.sigma0 + prm.dsigma_dT * (T - prm.T0)


def has_concentration(prm):
    return int(getattr(prm, "concentration", 0)) == 1


def sigma_field(T, c, prm):
    """sigma(c, T) as a cell field (Eq. 5 with the chain rule of its
    gradient; Sec. IV: sigma is formed locally from every field it depends
    on and then differentiated as a field): sigma0 + (dsigma/dT)(T - T0)
    + (dsigma/dc)(c - c0), the concentration term only when a transported
    concentration is present."""
    s = sigma_of_T(T, prm)
    if c is not None:
        s = s + prm.dsigma_dc * (c - prm.c0)
    return s


# ==========================================================================
# WENO5-JS reconstruction (Jiang & Shu 1996), Sec. IV "high order WENO"
# ==========================================================================
def weno5(vm2, vm1, v0, vp1, vp2, eps):
    """Value at the face i+1/2 from cells i-2..i+2, biased to the left.

    Three third-order candidates, smoothness indicators and nonlinear
    weights with linear weights (0.1, 0.6, 0.3).
    """
    q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0
    q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0
    q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0
    b0 = 13.0 / 12.0 * (vm2 - 2.0 * vm1 + v0) ** 2 + 0.25 * (vm2 - 4.0 * vm1 + 3.0 * v0) ** 2
    b1 = 13.0 / 12.0 * (vm1 - 2.0 * v0 + vp1) ** 2 + 0.25 * (vm1 - vp1) ** 2
    b2 = 13.0 / 12.0 * (v0 - 2.0 * vp1 + vp2) ** 2 + 0.25 * (3.0 * v0 - 4.0 * vp1 + vp2) ** 2
    a0 = 0.1 / (eps + b0) ** 2
    a1 = 0.6 / (eps + b1) ** 2
    a2 = 0.3 / (eps + b2) ** 2
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2)


def upwind_flux(U, vals, eps):
    """Flux U * phi_face at a face whose upwind neighbours are given as the six
    values vals = (v[-3], v[-2], v[-1], v[0], v[1], v[2]) relative to the face
    (v[-1] left of it, v[0] right of it).  Left-biased WENO5 when U >= 0,
    right-biased (mirror) otherwise."""
    m3, m2, m1, p0, p1, p2 = vals
    left = weno5(m3, m2, m1, p0, p1, eps)
    right = weno5(p2, p1, p0, m1, m2, eps)
    return torch.where(U >= 0.0, U * left, U * right)


# ==========================================================================
# Stage pieces
# ==========================================================================
def smooth_alpha(alpha, grid, passes):
    """Smoothed phase fraction: ``passes`` applications of the separable
    [1, 2, 1]/4 filter along x, y, z (even mirror at walls, wrap on periodic
    axes; axes of one cell are left alone)."""
    a = alpha
    for _ in range(passes):
        for d in range(3):
            if grid.n[d] == 1:
                continue
            P = pad_cell_axis(a, grid, d, 1.0)
            dim = AXIS_DIM[d]
            n = grid.n[d]
            am = P.narrow(dim, G - 1, n)
            a0 = P.narrow(dim, G, n)
            ap = P.narrow(dim, G + 1, n)
            a = (am + 2.0 * a0 + ap) * 0.25
    return a


def face_normal_component(At, grid, d, eps_n, s=0):
    """Normal component n_d on the low d-face of cell c + s e_d, from the
    smoothed alpha (extended array At): n = grad / (|grad| + eps_n), with the
    normal derivative across the face and each tangential derivative the mean
    of the two adjacent cells' central differences."""
    h = grid.h
    gd = (Sd(At, grid, (d, s)) - Sd(At, grid, (d, s - 1))) / h
    sq = gd * gd
    for t in range(3):
        if t == d:
            continue
        gt = ((Sd(At, grid, (t, 1), (d, s)) - Sd(At, grid, (t, -1), (d, s)))
              + (Sd(At, grid, (t, 1), (d, s - 1)) - Sd(At, grid, (t, -1), (d, s - 1)))) / (4.0 * h)
        sq = sq + gt * gt
    return gd / (norm3(sq) + eps_n)


def curvature(alpha_s, grid):
    """kappa = div n at cell centres from face normals of the smoothed alpha
    (n points into the alpha = 1 phase, so a convex drop has kappa < 0)."""
    h = grid.h
    eps_n = 1e-8 / h
    At = pad_scalar(alpha_s, grid, 1.0)
    kappa = torch.zeros(grid.shape, dtype=DT)
    for d in range(3):
        n_lo = face_normal_component(At, grid, d, eps_n, 0)
        n_hi = face_normal_component(At, grid, d, eps_n, 1)
        kappa = kappa + (n_hi - n_lo) / h
    return kappa


def central_grad(P, grid):
    """Central differences (P[c+e_d] - P[c-e_d]) / 2h of an extended array."""
    h = grid.h
    return [(Sd(P, grid, (d, 1)) - Sd(P, grid, (d, -1))) / (2.0 * h) for d in range(3)]


def marangoni_vector(Ap, Asp, sigP, grid):
    """Cell-centred Marangoni force |g| (grad sigma - nh (nh . grad sigma)),
    the tangential part of Eq. 4 with delta_s = |grad alpha| (raw alpha)
    and the unit normal nh from the smoothed alpha (regularised by eps_n)."""
    h = grid.h
    eps_n = 1e-8 / h
    g = central_grad(Ap, grid)
    t = central_grad(Asp, grid)
    s = central_grad(sigP, grid)
    gn = norm3(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    tn = norm3(t[0] ** 2 + t[1] ** 2 + t[2] ** 2) + eps_n
    nh = [t[d] / tn for d in range(3)]
    ns = nh[0] * s[0] + nh[1] * s[1] + nh[2] * s[2]
    return [gn * (s[d] - nh[d] * ns) for d in range(3)], gn


def heat_source(prm, grid, step_index, c_stage):
    """Gaussian surface flux q_s = 2P/(pi r^2) exp(-2 d^2 / r^2) around the
    moving centre (x0 + speed*h*(n + c), y0); distances use the nearest
    periodic image on periodic axes.  Returned on (1, ny, nx)."""
    if prm.q_power == 0.0:
        return None
    h = grid.h
    xc = prm.q_x0 + prm.q_speed * h * (step_index + c_stage)
    yc = prm.q_y0
    x = _coords(grid, 0).reshape(1, 1, -1)
    y = _coords(grid, 1).reshape(1, -1, 1)
    dx = x - xc
    dy = y - yc
    if grid.bc[0] == PERIODIC:
        dx = dx - grid.L[0] * torch.floor(dx / grid.L[0] + 0.5)
    if grid.bc[1] == PERIODIC:
        dy = dy - grid.L[1] * torch.floor(dy / grid.L[1] + 0.5)
    r2 = prm.q_radius ** 2
    return 2.0 * prm.q_power / (math.pi * r2) * torch.exp(-2.0 * (dx * dx + dy * dy) / r2)


def scalar_rhs(phiP, velP, grid, eps):
    """-div(u phi) by WENO5 face values (Eq. 1 for phi = alpha): the flux
    through the low d-face of cell c+s uses the d-velocity on that face."""
    h = grid.h
    R = torch.zeros(grid.shape, dtype=DT)
    for d in range(3):
        F = []
        for s in (0, 1):
            U = Sd(velP[d], grid, (d, s))
            vals = [Sd(phiP, grid, (d, s + k)) for k in (-3, -2, -1, 0, 1, 2)]
            F.append(upwind_flux(U, vals, eps))
        R = R - (F[1] - F[0]) / h
    return R


def bounded_alpha_rhs(Ap, velP, grid, eps, dt):
    """-div(u alpha) with fluxes kept between the first-order upwind flux and
    the WENO5 flux so that the forward-Euler stage keeps alpha within [0, 1]
    (the bounded option of the transport scheme; the paper's Sec. V-A mixes
    first-order bounded and high-order WENO divergence schemes).  The blend
    is flux-corrected transport (Zalesak, J. Comput. Phys. 31, 1979) with the
    global bounds 0 and 1:

    F_L = U alpha_upwind, A = F_WENO - F_L (antidiffusive part),
    alpha_td = alpha - dt div F_L (bounded for a divergence-free U at the
    CFL limit), per cell P+ / P- = sum of antidiffusive fluxes into / out of
    it, Q+ = (1 - alpha_td) h / dt, Q- = alpha_td h / dt,
    R+- = clamp(Q+- / P+-, 0, 1) (0 where P vanishes); a face with A > 0
    (from its low cell L to its high cell R) takes theta = min(R+_R, R-_L),
    with A < 0 theta = min(R+_L, R-_R); the flux is F_L + theta A."""
    h = grid.h
    n = grid.shape
    FL, AA = [], []
    for d in range(3):
        FLd, Ad = [], []
        for s in (0, 1):
            U = Sd(velP[d], grid, (d, s))
            vals = [Sd(Ap, grid, (d, s + k)) for k in (-3, -2, -1, 0, 1, 2)]
            fh = upwind_flux(U, vals, eps)
            fl = torch.where(U >= 0.0, U * vals[2], U * vals[3])
            FLd.append(fl)
            Ad.append(fh - fl)
        FL.append(FLd)
        AA.append(Ad)
    alpha = S(Ap, grid)
    div_low = torch.zeros(n, dtype=DT)
    Pp = torch.zeros(n, dtype=DT)
    Pm = torch.zeros(n, dtype=DT)
    for d in range(3):
        div_low = div_low + (FL[d][1] - FL[d][0]) / h
        a_lo, a_hi = AA[d][0], AA[d][1]
        Pp = Pp + torch.clamp(a_lo, min=0.0) + torch.clamp(-a_hi, min=0.0)
        Pm = Pm + torch.clamp(-a_lo, min=0.0) + torch.clamp(a_hi, min=0.0)
    a_td = alpha - dt * div_low
    Qp = (1.0 - a_td) * h / dt
    Qm = a_td * h / dt

    def ratio(Q, P):
        pos = P > 0.0
        return torch.where(pos, torch.clamp(Q / torch.where(pos, P, 1.0), 0.0, 1.0), 0.0)

    Rp, Rm = ratio(Qp, Pp), ratio(Qm, Pm)
    RpP, RmP = pad_scalar(Rp, grid, 1.0), pad_scalar(Rm, grid, 1.0)
    out = torch.zeros(n, dtype=DT)
    for d in range(3):
        F = []
        for s in (0, 1):
            a = AA[d][s]
            # the face's low cell L = c + (s-1) e_d, high cell R = c + s e_d
            rpL, rmL = Sd(RpP, grid, (d, s - 1)), Sd(RmP, grid, (d, s - 1))
            rpR, rmR = Sd(RpP, grid, (d, s)), Sd(RmP, grid, (d, s))
            theta = torch.where(a > 0.0, torch.minimum(rpR, rmL),
                                torch.where(a < 0.0, torch.minimum(rpL, rmR), torch.ones_like(a)))
            F.append(FL[d][s] + theta * a)
        out = out - (F[1] - F[0]) / h
    return out


def diffusion_rhs(TP, lamP, grid):
    """div(lambda grad T) with the harmonic mean of lambda on each face (0 on
    a face where lambda vanishes on both sides)."""
    h = grid.h
    R = torch.zeros(grid.shape, dtype=DT)
    for d in range(3):
        D = []
        for s in (0, 1):
            lL, lR = Sd(lamP, grid, (d, s - 1)), Sd(lamP, grid, (d, s))
            den = lL + lR
            lf = torch.where(den > 0.0, 2.0 * lL * lR / torch.where(den > 0.0, den, 1.0), 0.0)
            D.append(lf * (Sd(TP, grid, (d, s)) - Sd(TP, grid, (d, s - 1))) / h)
        R = R + (D[1] - D[0]) / h
    return R


def momentum_predictor(d, velP, prm, grid, dt, props, forces, eps):
    """u_d* = u_d + dt (A + (V + f_n + f_M)/rho_f + g_d) on every low d-face.

    A: conservative WENO5 advection on the MAC control volume; the
    normal flux at the cell centres uses the mean of the two d-faces as
    advecting velocity, the tangential flux at the edge uses the mean of the
    two t-faces there.  V: divergence of mu (grad u + grad u^T) with cell mu
    for the normal stress and the 4-cell mean at edges.  f_n, f_M, rho_f as
    in ``interface_forces``.  Wall faces (index 0 on a wall axis) are 0.
    """
    h = grid.h
    ud = velP[d]
    muP = props["muP"]
    # --- advection -------------------------------------------------------
    A = torch.zeros(grid.shape, dtype=DT)
    Fc = []
    for s in (-1, 0):                      # cell below the face (c = f-e_d) and above (c = f)
        Uc = 0.5 * (Sd(ud, grid, (d, s)) + Sd(ud, grid, (d, s + 1)))
        vals = [Sd(ud, grid, (d, s + k)) for k in (-2, -1, 0, 1, 2, 3)]
        Fc.append(upwind_flux(Uc, vals, eps))
    A = A - (Fc[1] - Fc[0]) / h
    for t in range(3):
        if t == d:
            continue
        Ge = []
        for s in (0, 1):                   # low t-edge of face f and of face f+e_t
            Ue = 0.5 * (Sd(velP[t], grid, (t, s), (d, -1)) + Sd(velP[t], grid, (t, s)))
            vals = [Sd(ud, grid, (t, s + k)) for k in (-3, -2, -1, 0, 1, 2)]
            Ge.append(upwind_flux(Ue, vals, eps))
        A = A - (Ge[1] - Ge[0]) / h
    # --- viscous stress ----------------------------------------------------
    V = torch.zeros(grid.shape, dtype=DT)
    tau = []
    for s in (-1, 0):
        mu_c = Sd(muP, grid, (d, s))
        tau.append(2.0 * mu_c * (Sd(ud, grid, (d, s + 1)) - Sd(ud, grid, (d, s))) / h)
    V = V + (tau[1] - tau[0]) / h
    for t in range(3):
        if t == d:
            continue
        te = []
        for s in (0, 1):
            mu_e = 0.25 * (Sd(muP, grid, (t, s)) + Sd(muP, grid, (t, s), (d, -1))
                           + Sd(muP, grid, (t, s - 1)) + Sd(muP, grid, (t, s - 1), (d, -1)))
            dud_dt = (Sd(ud, grid, (t, s)) - Sd(ud, grid, (t, s - 1))) / h
            dut_dd = (Sd(velP[t], grid, (t, s)) - Sd(velP[t], grid, (t, s), (d, -1))) / h
            te.append(mu_e * (dud_dt + dut_dd))
        V = V + (te[1] - te[0]) / h
    # --- assemble ------------------------------------------------------------
    rho_f = 0.5 * (Sd(props["rhoP"], grid, (d, -1)) + Sd(props["rhoP"], grid))
    fn, fM = forces[d]
    ustar = Sd(ud, grid) + dt * (A + (V + fn + fM) / rho_f + prm.g[d])
    if grid.bc[d] == WALL:
        ustar = _zero_wall_face(ustar, d)
    return ustar


def _zero_wall_face(a, d):
    a = a.clone()
    idx = [slice(None)] * 3
    idx[AXIS_DIM[d]] = 0
    a[tuple(idx)] = 0.0
    return a


def interface_forces(alpha, alpha_s, T, prm, grid, c=None):
    """Face forces from Eq. 4 in balanced-force form, per direction d:

    f_n = -sigma_f kappa_f (alpha_R - alpha_L)/h  (the normal term
          -sigma kappa n delta_s with n delta_s = grad alpha, raw alpha);
    f_M = face mean of the cell Marangoni vector's d-component (the
          tangential term delta_s (I - n n) grad sigma).
    sigma_f, kappa_f are the means of the two cells.
    """
    h = grid.h
    kappa = curvature(alpha_s, grid)
    KP = pad_scalar(kappa, grid, 1.0)
    Ap = pad_scalar(alpha, grid, 1.0)
    Asp = pad_scalar(alpha_s, grid, 1.0)
    TP = pad_temperature(T, prm, grid)
    cP = pad_scalar(c, grid, 1.0) if c is not None else None
    sigP = sigma_field(TP, cP, prm)
    M, gnorm = marangoni_vector(Ap, Asp, sigP, grid)
    MP = [pad_scalar(M[d], grid, 1.0) for d in range(3)]
    out = []
    for d in range(3):
        sig_f = 0.5 * (Sd(sigP, grid, (d, -1)) + Sd(sigP, grid))
        kap_f = 0.5 * (Sd(KP, grid, (d, -1)) + Sd(KP, grid))
        jump = (Sd(Ap, grid) - Sd(Ap, grid, (d, -1))) / h
        fn = -sig_f * kap_f * jump
        fM = 0.5 * (Sd(MP[d], grid, (d, -1)) + Sd(MP[d], grid))
        out.append((fn, fM))
    return out, kappa, gnorm


# ==========================================================================
# Pressure projection and geometric multigrid
# ==========================================================================
class Level:
    """One multigrid level: sizes, spacings, periodicity and face betas
    (beta[d][c] lives on the low d-face of cell c; wall faces are 0)."""

    def __init__(self, n, hs, bc, beta):
        self.n = n
        self.hs = hs
        self.bc = bc
        self.beta = beta

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])


def _roll_up(a, d):
    """a[c + e_d] with wrap (callers mask the wall faces through beta)."""
    return a.roll(-1, AXIS_DIM[d])


def _roll_dn(a, d):
    return a.roll(1, AXIS_DIM[d])


def _beta_hi(lev, d):
    """beta on the high d-face of each cell (0 at the last wall face)."""
    b = _roll_up(lev.beta[d], d)
    if lev.bc[d] == WALL:
        b = b.clone()
        idx = [slice(None)] * 3
        idx[AXIS_DIM[d]] = lev.n[d] - 1
        b[tuple(idx)] = 0.0
    return b


def apply_L(p, lev):
    """(L p)_c = sum over faces beta_f (p_c - p_nb) / h_d^2 = -div(beta grad p);
    axes with a single cell carry no coupling."""
    out = torch.zeros_like(p)
    for d in range(3):
        if lev.n[d] == 1:
            continue
        w = 1.0 / (lev.hs[d] ** 2)
        out = out + (lev.beta[d] * (p - _roll_dn(p, d)) + _beta_hi(lev, d) * (p - _roll_up(p, d))) * w
    return out


def fine_beta(alpha, prm, grid):
    """beta = 1/rho_f with rho_f the mean of the two cells' mixture
    densities; wall faces carry 0."""
    rho = mix(alpha, prm.rho)
    betas = []
    for d in range(3):
        rho_f = 0.5 * (_roll_dn(rho, d) + rho)
        b = 1.0 / rho_f
        if grid.bc[d] == WALL:
            b = _zero_wall_face(b, d)
        betas.append(b)
    return betas


def coarsen_factors(n, bc):
    """Direction d is halved when its size is even and >= 4 and, on a
    periodic axis, the halved size stays even (red-black colouring must
    remain a 2-colouring under wrap)."""
    f = []
    for d in range(3):
        ok = n[d] % 2 == 0 and n[d] >= 4
        if ok and bc[d] == PERIODIC and (n[d] // 2) % 2 != 0:
            ok = False
        f.append(2 if ok else 1)
    return f


def restrict_mean(a, f):
    nz, ny, nx = a.shape
    return a.reshape(nz // f[2], f[2], ny // f[1], f[1], nx // f[0], f[0]).mean(dim=(1, 3, 5))


def coarse_beta(beta, n, f):
    """Coarse face beta = mean of the fine faces it covers: the fine d-faces
    at fine index f_d*I along d, over the children in the two other axes."""
    out = []
    for d in range(3):
        b = beta[d]
        dim = AXIS_DIM[d]
        if f[d] == 2:
            b = b.index_select(dim, torch.arange(0, n[d], 2))
        ff = list(f)
        ff[d] = 1
        out.append(restrict_mean(b, ff))
    return out


def build_hierarchy(beta0, grid, max_levels):
    levels = [Level(grid.n, (grid.h,) * 3, grid.bc, beta0)]
    while len(levels) < max_levels:
        lev = levels[-1]
        f = coarsen_factors(lev.n, lev.bc)
        if f == [1, 1, 1]:
            break
        n = tuple(lev.n[d] // f[d] for d in range(3))
        hs = tuple(lev.hs[d] * f[d] for d in range(3))
        levels.append(Level(n, hs, lev.bc, coarse_beta(lev.beta, lev.n, f)))
    return levels


def colour_mask(lev, colour):
    nx, ny, nz = lev.n
    k = torch.arange(nz).reshape(-1, 1, 1)
    j = torch.arange(ny).reshape(1, -1, 1)
    i = torch.arange(nx).reshape(1, 1, -1)
    return ((i + j + k) % 2) == colour


def gs_colour(p, b, lev, colour):
    """One Gauss-Seidel update of the cells of one colour ((i+j+k) mod 2)."""
    num = b.clone()
    den = torch.zeros_like(p)
    for d in range(3):
        if lev.n[d] == 1:
            continue
        w = 1.0 / (lev.hs[d] ** 2)
        blo = lev.beta[d]
        bhi = _beta_hi(lev, d)
        num = num + (blo * _roll_dn(p, d) + bhi * _roll_up(p, d)) * w
        den = den + (blo + bhi) * w
    return torch.where(colour_mask(lev, colour), num / den, p)


def coarse_cg(b, lev, rtol, maxit):
    """Conjugate gradients on the coarsest level, mean-removed right-hand
    side, x0 = 0, stop at ||r|| <= rtol ||b|| or on breakdown (p.Ap <= 0);
    mean-free result."""
    b = b - b.mean()
    bn = torch.sqrt((b * b).sum())
    x = torch.zeros_like(b)
    if bn.item() == 0.0:
        return x
    r = b.clone()
    d = r.clone()
    rr = (r * r).sum()
    for _ in range(maxit):
        if torch.sqrt(rr).item() <= rtol * bn.item():
            break
        Ad = apply_L(d, lev)
        pAp = (d * Ad).sum()
        if not pAp.item() > 0.0:   # breakdown: the search direction carries no energy
            break
        a = rr / pAp
        x = x + a * d
        r = r - a * Ad
        rr_new = (r * r).sum()
        d = r + (rr_new / rr) * d
        rr = rr_new
    return x - x.mean()


def sweeps(prm, l):
    """Pre- and post-smoothing sweeps of level l: mg_pre, mg_post on the
    finest level; mg_coarse_sweeps each on the coarser ones (0: the finest
    level's counts)."""
    c = int(getattr(prm, "mg_coarse_sweeps", 0))
    if l == 0 or c == 0:
        return prm.mg_pre, prm.mg_post
    return c, c


def vcycle(levels, l, x, b, prm):
    """V(pre, post) cycle: red-black GS (red first) before, residual
    restricted by the mean of the children, piecewise-constant prolongation,
    black-red GS after; CG on the coarsest level.  The coarse levels take
    their own sweep count (``sweeps``)."""
    lev = levels[l]
    if l == len(levels) - 1:
        return coarse_cg(b, lev, prm.coarse_rtol, prm.coarse_maxit)
    pre, post = sweeps(prm, l)
    for _ in range(pre):
        x = gs_colour(x, b, lev, 0)
        x = gs_colour(x, b, lev, 1)
    r = b - apply_L(x, lev)
    f = [levels[l].n[d] // levels[l + 1].n[d] for d in range(3)]
    bc_ = restrict_mean(r, f)
    ec = vcycle(levels, l + 1, torch.zeros_like(bc_), bc_, prm)
    x = x + ec.repeat_interleave(f[2], 0).repeat_interleave(f[1], 1).repeat_interleave(f[0], 2)
    for _ in range(post):
        x = gs_colour(x, b, lev, 1)
        x = gs_colour(x, b, lev, 0)
    return x


def mg_solve(alpha, b, p0, prm, grid, fixed_cycles=None):
    """Solve L p = b (b mean-free) from the guess p0 by V-cycles until
    ||b - L p||_2 <= rtol ||b||_2 (checked before every cycle) or exactly
    ``fixed_cycles`` cycles; returns mean-free p, cycles, relative residual."""
    levels = build_hierarchy(fine_beta(alpha, prm, grid), grid, prm.mg_levels)
    lev = levels[0]
    bn = torch.sqrt((b * b).sum()).item()
    fixed = prm.mg_fixed_cycles if fixed_cycles is None else fixed_cycles
    p = p0.clone()
    if bn == 0.0:
        return torch.zeros_like(p), 0, 0.0
    cycles = 0
    if fixed > 0:
        for _ in range(fixed):
            p = vcycle(levels, 0, p, b, prm)
        cycles = fixed
        rel = torch.sqrt(((b - apply_L(p, lev)) ** 2).sum()).item() / bn
    else:
        while True:
            rel = torch.sqrt(((b - apply_L(p, lev)) ** 2).sum()).item() / bn
            if rel <= prm.mg_rtol or cycles >= prm.mg_max_cycles:
                break
            p = vcycle(levels, 0, p, b, prm)
            cycles += 1
    return p - p.mean(), cycles, rel


def divergence(vel, grid):
    """(D u)_c = sum_d (u_d[c+e_d] - u_d[c]) / h with the implied high face."""
    h = grid.h
    out = torch.zeros(grid.shape, dtype=DT)
    for d in range(3):
        P = pad_face_axis(vel[d], grid, d)
        dim = AXIS_DIM[d]
        n = grid.n[d]
        out = out + (P.narrow(dim, G + 1, n) - P.narrow(dim, G, n)) / h
    return out


def projection(vel_star, alpha, p0, prm, grid, dt, fixed_cycles=None):
    """Density-weighted projection: b = -(D u*)/dt minus its mean, L p = b,
    u = u* - dt beta_f (p_R - p_L)/h on every non-wall face."""
    h = grid.h
    b = -divergence(vel_star, grid) / dt
    b = b - b.mean()
    p, cycles, rel = mg_solve(alpha, b, p0, prm, grid, fixed_cycles)
    beta = fine_beta(alpha, prm, grid)
    out = []
    for d in range(3):
        u = vel_star[d] - dt * beta[d] * (p - _roll_dn(p, d)) / h
        if grid.bc[d] == WALL:
            u = _zero_wall_face(u, d)
        out.append(u)
    return out, p, cycles, rel


# ==========================================================================
# Time step
# ==========================================================================
def time_step_limit(state, prm, grid):
    """dt = min(CFL, capillary, viscous, thermal, dt_max) from max-reductions:
    C_u h / (max|u|+max|v|+max|w|), C_sigma sqrt((rho0+rho1) h^3 / (4 pi max|sigma|)),
    C_nu h^2 / max(mu/rho), C_kappa h^2 / max(lambda/(rho c_p)).
    With a transported concentration, max(mu/rho) is joined in the last limit
    by max(D_c) and |sigma| is that of sigma(c, T).
    Returns (dt, index of the binding limit)."""
    h = grid.h
    umax = sum(state[k].abs().max().item() for k in ("u", "v", "w"))
    a = state["alpha"]
    c = state["c"] if has_concentration(prm) else None
    smax = sigma_field(state["T"], c, prm).abs().max().item()
    numax = (mix(a, prm.mu) / mix(a, prm.rho)).max().item()
    kapmax = (mix(a, prm.lam) / rho_cp(a, prm)).max().item()
    if c is not None:   # the concentration's diffusion shares the diffusive limit
        kapmax = max(kapmax, mix(a, prm.diff_c).max().item())
    lim = [math.inf] * 5
    if umax > 0.0:
        lim[0] = prm.cfl * h / umax
    if smax > 0.0:
        lim[1] = prm.c_cap * math.sqrt((prm.rho[0] + prm.rho[1]) * h ** 3 / (4.0 * math.pi * smax))
    if numax > 0.0:
        lim[2] = prm.c_visc * h * h / numax
    if kapmax > 0.0:
        lim[3] = prm.c_therm * h * h / kapmax
    lim[4] = prm.dt_max
    k = min(range(5), key=lambda i: (lim[i], i))
    return lim[k], k


def predictor(X, prm, grid, dt, step_index, c_stage):
    """Everything of one forward-Euler substep before the projection:
    smoothed alpha, interface forces, scalar updates and u*."""
    h = grid.h
    alpha, T = X["alpha"], X["T"]
    vel = [X["u"], X["v"], X["w"]]
    velP = [pad_velocity(vel[d], grid, d) for d in range(3)]
    c = X["c"] if has_concentration(prm) else None
    alpha_s = smooth_alpha(alpha, grid, prm.smooth_passes)
    forces, kappa, gnorm = interface_forces(alpha, alpha_s, T, prm, grid, c)
    Ap = pad_scalar(alpha, grid, 1.0)
    TP = pad_temperature(T, prm, grid)
    eps = [prm.weno_eps * s * s for s in prm.weno_scale]
    # phase fraction (Eq. 1) and temperature
    if int(getattr(prm, "alpha_scheme", 0)) == 1:
        R_alpha = bounded_alpha_rhs(Ap, velP, grid, eps[0], dt)
    else:
        R_alpha = scalar_rhs(Ap, velP, grid, eps[0])
    lamP = mix(Ap, prm.lam)
    rcp = rho_cp(alpha, prm)
    R_T = scalar_rhs(TP, velP, grid, eps[1]) + diffusion_rhs(TP, lamP, grid) / rcp
    q = heat_source(prm, grid, step_index, c_stage)
    if q is not None:
        R_T = R_T + q * gnorm / rcp
    props = {"muP": mix(Ap, prm.mu), "rhoP": mix(Ap, prm.rho)}
    ustar = [momentum_predictor(d, velP, prm, grid, dt, props, forces, eps[2]) for d in range(3)]
    out = {"alpha": alpha + dt * R_alpha, "T": T + dt * R_T, "ustar": ustar,
           "alpha_s": alpha_s, "kappa": kappa}
    if c is not None:
        # a transported concentration (the solutal part of Eq. 5): WENO5
        # advection like T and diffusion with the harmonic face mean of the
        # mixture diffusivity, even (no-flux) at walls
        cP = pad_scalar(c, grid, 1.0)
        R_c = scalar_rhs(cP, velP, grid, prm.weno_eps * prm.weno_scale_c ** 2) + \
            diffusion_rhs(cP, mix(Ap, prm.diff_c), grid)
        out["c"] = c + dt * R_c
    return out


def substep(X, prm, grid, dt, step_index, c_stage, fixed_cycles=None):
    """E(X): forward-Euler predictor followed by the projection."""
    pr = predictor(X, prm, grid, dt, step_index, c_stage)
    vel, p, cycles, rel = projection(pr["ustar"], X["alpha"], X["p"], prm, grid, dt, fixed_cycles)
    E = {"u": vel[0], "v": vel[1], "w": vel[2], "alpha": pr["alpha"], "T": pr["T"], "p": p}
    if "c" in pr:
        E["c"] = pr["c"]
    return E, cycles, rel


RK3 = ((0.0, 1.0, 0.0), (0.75, 0.25, 1.0), (1.0 / 3.0, 2.0 / 3.0, 0.5))


def step(state, prm, step_index=0, dt=0.0, fixed_cycles=None):
    """One SSP-RK3 (Shu-Osher) step with a projection per stage:
    S1 = E(Sn), S2 = 3/4 Sn + 1/4 E(S1), S(n+1) = 1/3 Sn + 2/3 E(S2).

    ``state`` holds float64 tensors u, v, w, alpha, T, p.  dt <= 0 means
    the limit of ``time_step_limit``.  ``fixed_cycles`` is None (use
    prm.mg_fixed_cycles), an int, or a list of three ints (one per stage).
    Returns (new_state, info).
    """
    grid = Grid(prm)
    Sn = {k: _t(v) for k, v in state.items()}
    # the stored wall faces are not part of the state: they are read as 0
    for d, k in enumerate(("u", "v", "w")):
        if grid.bc[d] == WALL:
            Sn[k] = _zero_wall_face(Sn[k], d)
    limiter = -1
    if dt <= 0.0:
        dt, limiter = time_step_limit(Sn, prm, grid)
    X = Sn
    vcycles, rels = [], []
    for s, (a, b, c) in enumerate(RK3):
        fc = fixed_cycles[s] if isinstance(fixed_cycles, (list, tuple)) else fixed_cycles
        E, cyc, rel = substep(X, prm, grid, dt, step_index, c, fc)
        vcycles.append(cyc)
        rels.append(rel)
        X = {k: a * Sn[k] + b * E[k] for k in transported(prm)}
        X["p"] = E["p"]
    info = diagnostics(X, prm, grid, dt)
    info.update({"dt": dt, "dt_limiter": limiter, "vcycles": vcycles, "rel_residual": rels})
    return X, info


def transported(prm):
    """The fields the time integrator advances (the concentration when present)."""
    return ("u", "v", "w", "alpha", "T") + (("c",) if has_concentration(prm) else ())


def diagnostics(X, prm, grid, dt):
    """Volume sum alpha h^3, mass sum rho(alpha) h^3, max |D u| dt, NaN flag."""
    h3 = grid.h ** 3
    div = divergence([X["u"], X["v"], X["w"]], grid)
    finite = all(torch.isfinite(X[k]).all().item() for k in transported(prm) + ("p",))
    return {"vol_sum": (X["alpha"].sum() * h3).item(),
            "mass_sum": (mix(X["alpha"], prm.rho).sum() * h3).item(),
            "max_div_dt": (div.abs().max() * dt).item(),
            "nan_flag": 0 if finite else 1}


def poisson_solve(alpha, rhs, p0, prm, fixed_cycles=None):
    """The multigrid projection solve alone: rhs is made mean-free first."""
    grid = Grid(prm)
    b = _t(rhs)
    b = b - b.mean()
    return mg_solve(_t(alpha), b, _t(p0), prm, grid, fixed_cycles)
