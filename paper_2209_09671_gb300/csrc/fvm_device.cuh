// Device helpers: boundary-aware loads, material mixtures and the WENO5-JS
// reconstruction.  Boundary conditions are realised by ghost values computed
// inside the loads (no stored ghost layers):
//   periodic axis  -> wrap
//   wall axis      -> cell-centred fields mirror about the wall face
//                     (ghost -1-m <- cell m); even for alpha, kappa, M and
//                     Neumann T, odd for tangential velocity (no slip),
//                     2 T_w - mirror for a Dirichlet temperature side;
//                     the normal velocity is odd about the wall face and 0 on it.
#pragma once

#include <math.h>

#include "fvm_internal.h"

namespace fvm {

__device__ __forceinline__ int wrapi(int c, int n) {
  if (c < 0) {
    c += n;
    if (c < 0) c = ((c % n) + n) % n;
  } else if (c >= n) {
    c -= n;
    if (c >= n) c %= n;
  }
  return c;
}

// cell-type index along one axis; flips `s` on a wall reflection when odd
__device__ __forceinline__ int mapc(int c, int n, int bc, bool odd, int& s) {
  if (bc == PER) return wrapi(c, n);
  if (c < 0) {
    if (odd) s = -s;
    return -1 - c;
  }
  if (c >= n) {
    if (odd) s = -s;
    return 2 * n - 1 - c;
  }
  return c;
}

// face-type index along the velocity's own axis
__device__ __forceinline__ int mapf(int f, int n, int bc, int& s) {
  if (bc == PER) return wrapi(f, n);
  if (f <= 0) {
    if (f == 0) s = 0;
    else s = -s;
    return -f;
  }
  if (f >= n) {
    if (f == n) { s = 0; return 0; }
    s = -s;
    return 2 * n - f;
  }
  return f;
}

__device__ __forceinline__ long long lin(const Geo& g, int i, int j, int k) {
  return (long long)k * g.sz + (long long)j * g.sy + i;
}

// even cell field (alpha, smoothed alpha, kappa, M, properties)
template <typename R>
__device__ __forceinline__ R ld_even(const R* __restrict__ a, const Geo& g, int i, int j, int k) {
  int s = 1;
  i = mapc(i, g.n[0], g.bc[0], false, s);
  j = mapc(j, g.n[1], g.bc[1], false, s);
  k = mapc(k, g.n[2], g.bc[2], false, s);
  return __ldg(a + lin(g, i, j, k));
}

// velocity component C: face-type along C, odd cell-type along the others
template <int C, typename R>
__device__ __forceinline__ R ld_vel(const R* __restrict__ a, const Geo& g, int i, int j, int k) {
  int s = 1;
  i = (C == 0) ? mapf(i, g.n[0], g.bc[0], s) : mapc(i, g.n[0], g.bc[0], true, s);
  j = (C == 1) ? mapf(j, g.n[1], g.bc[1], s) : mapc(j, g.n[1], g.bc[1], true, s);
  k = (C == 2) ? mapf(k, g.n[2], g.bc[2], s) : mapc(k, g.n[2], g.bc[2], true, s);
  R v = __ldg(a + lin(g, i, j, k));
  return s == 1 ? v : (s == 0 ? R(0) : -v);
}

// temperature with Neumann (even) or Dirichlet (2 T_w - mirror) walls
template <typename R>
__device__ __forceinline__ R ld_T(const R* __restrict__ a, const Geo& g, const TBC& tb, int i,
                                  int j, int k) {
  int c[3] = {i, j, k};
  int m[3];
  int side = -1;
  for (int d = 0; d < 3; ++d) {
    int s = 1;
    m[d] = mapc(c[d], g.n[d], g.bc[d], false, s);
    if (d == tb.axis && g.bc[d] == WALL) {
      if (c[d] < 0 && tb.dir[0]) side = 0;
      if (c[d] >= g.n[d] && tb.dir[1]) side = 1;
    }
  }
  R v = __ldg(a + lin(g, m[0], m[1], m[2]));
  if (side >= 0) {
    double sc = (m[tb.s_axis] + 0.5) * g.h;
    double Tw = tb.T0[side] + tb.amp[side] * cos(2.0 * M_PI * sc / tb.Ls);
    v = (R)(2.0 * Tw - (double)v);
  }
  return v;
}

template <typename R>
__device__ __forceinline__ R clamp01(R a) {
  return a < R(0) ? R(0) : (a > R(1) ? R(1) : a);
}

// arithmetic mixture a*p1 + (1-a)*p0 with a = clamp(alpha, 0, 1)
template <typename R>
__device__ __forceinline__ R mixp(R alpha, const double* pair) {
  R a = clamp01(alpha);
  return a * (R)pair[1] + (R(1) - a) * (R)pair[0];
}

template <typename R>
__device__ __forceinline__ R sigma_of_T(R T, const Phys& ph) {
  return (R)ph.sigma0 + (R)ph.dsdT * (T - (R)ph.T0);
}

// Material and source constants in the working precision, so that float
// kernels carry no double arithmetic or conversions.
template <typename R>
struct PhysR {
  R rho[2], mu[2], lam[2], rcp[2];
  R sigma0, dsdT, T0;
  R g[3];
  R eps_a, eps_T, eps_u, eps_n;
  R L[3];
  R h, ih;
  R dsdc, c0, diff_c[2], eps_c;
};

template <typename R>
inline PhysR<R> make_physr(const Phys& ph, const Geo& g) {
  PhysR<R> q;
  for (int k = 0; k < 2; ++k) {
    q.rho[k] = (R)ph.rho[k];
    q.mu[k] = (R)ph.mu[k];
    q.lam[k] = (R)ph.lam[k];
    q.rcp[k] = (R)ph.rcp[k];
  }
  q.sigma0 = (R)ph.sigma0;
  q.dsdT = (R)ph.dsdT;
  q.T0 = (R)ph.T0;
  for (int d = 0; d < 3; ++d) {
    q.g[d] = (R)ph.g[d];
    q.L[d] = (R)ph.L[d];
  }
  q.eps_a = (R)ph.eps_a;
  q.eps_T = (R)ph.eps_T;
  q.eps_u = (R)ph.eps_u;
  q.eps_n = (R)ph.eps_n;
  q.h = (R)g.h;
  q.ih = (R)g.ih;
  q.dsdc = (R)ph.dsdc;
  q.c0 = (R)ph.c0;
  q.diff_c[0] = (R)ph.diff_c[0];
  q.diff_c[1] = (R)ph.diff_c[1];
  q.eps_c = (R)ph.eps_c;
  return q;
}

template <typename R>
__device__ __forceinline__ R mixr(R alpha, const R* pair) {
  R a = clamp01(alpha);
  return a * pair[1] + (R(1) - a) * pair[0];
}

template <typename R>
__device__ __forceinline__ R sigma_r(R T, const PhysR<R>& q) {
  return q.sigma0 + q.dsdT * (T - q.T0);
}

// sigma(c, T) of Eq. 5 with the solutal term
template <typename R>
__device__ __forceinline__ R sigma_rc(R T, R c, const PhysR<R>& q) {
  return q.sigma0 + q.dsdT * (T - q.T0) + q.dsdc * (c - q.c0);
}

// harmonic face mean 2 a b / (a + b), 0 where both vanish
template <typename R>
__device__ __forceinline__ R harmonic(R a, R b) {
  const R s = a + b;
  return s > R(0) ? R(2) * a * b / s : R(0);
}

// WENO5-JS value at the face right of v0 from cells v0-2 .. v0+2 (left bias),
// nonlinear weights a_k = d_k / (eps + beta_k)^2, d = (0.1, 0.6, 0.3).
// In double the weights are combined over a common denominator so that one
// division is needed: with s_k = (eps + beta_k)^2,
//   value = (d0 q0 s1 s2 + d1 q1 s0 s2 + d2 q2 s0 s1) / (d0 s1 s2 + d1 s0 s2 + d2 s0 s1);
// the products grow like beta^2, far inside the double range.  In float they
// would overflow once velocity jumps reach ~1e4, so float keeps the
// reciprocal form (which underflows gracefully instead) with the fast
// approximate division: the weights need only a few correct digits.
template <typename R>
__device__ __forceinline__ R weno5(R vm2, R vm1, R v0, R vp1, R vp2, R eps) {
  const R c6 = R(1) / R(6);
  R q0 = (R(2) * vm2 - R(7) * vm1 + R(11) * v0) * c6;
  R q1 = (-vm1 + R(5) * v0 + R(2) * vp1) * c6;
  R q2 = (R(2) * v0 + R(5) * vp1 - vp2) * c6;
  R t0 = vm2 - R(2) * vm1 + v0, u0 = vm2 - R(4) * vm1 + R(3) * v0;
  R t1 = vm1 - R(2) * v0 + vp1, u1 = vm1 - vp1;
  R t2 = v0 - R(2) * vp1 + vp2, u2 = R(3) * v0 - R(4) * vp1 + vp2;
  const R c1312 = R(13) / R(12);
  R b0 = c1312 * t0 * t0 + R(0.25) * u0 * u0;
  R b1 = c1312 * t1 * t1 + R(0.25) * u1 * u1;
  R b2 = c1312 * t2 * t2 + R(0.25) * u2 * u2;
  R s0 = (eps + b0) * (eps + b0);
  R s1 = (eps + b1) * (eps + b1);
  R s2 = (eps + b2) * (eps + b2);
  if (sizeof(R) == 8) {
    R w0 = R(0.1) * s1 * s2, w1 = R(0.6) * s0 * s2, w2 = R(0.3) * s0 * s1;
    return (w0 * q0 + w1 * q1 + w2 * q2) / (w0 + w1 + w2);
  } else {
    // the weights only need a few correct digits: fast reciprocal division
    R a0 = __fdividef(R(0.1), s0), a1 = __fdividef(R(0.6), s1), a2 = __fdividef(R(0.3), s2);
    return __fdividef(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
  }
}

// flux U * phi_face from the six values v[0..5] = phi at offsets -3..2 of the
// face (v[2] left of it, v[3] right of it): left-biased WENO5 when U >= 0
template <typename R>
__device__ __forceinline__ R upwind_flux(R U, const R* v, R eps) {
  R val = (U >= R(0)) ? weno5(v[0], v[1], v[2], v[3], v[4], eps)
                      : weno5(v[5], v[4], v[3], v[2], v[1], eps);
  return U * val;
}

}  // namespace fvm
