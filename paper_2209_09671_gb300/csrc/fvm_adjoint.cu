// Reverse mode (adjoint) of one forward-Euler stage of the FP64 step, for the
// equal-property setting (one rho, mu, lambda, c_p for both phases, so that
// the projection coefficient is constant and the projection is self-adjoint).
// Each kernel is the transpose of a forward operator written in scatter form:
// a thread takes the adjoint of the outputs it owns, differentiates its local
// stencil arithmetic (the same arithmetic as the forward kernels) and adds the
// products to the adjoints of the inputs with atomic adds, following the
// boundary rules of the forward loads (a mirrored value passes its adjoint to
// the mirror cell with the mirror's sign; wall faces carry none).
//   k_adj_momentum   transpose of the momentum predictor (WENO5 advection on
//                    the MAC control volumes, viscous stress, CSF and Marangoni
//                    face forces; Sec. III, Eq. 4)
//   k_adj_scalars    transpose of the alpha / T update (Eq. 1 transport,
//                    conduction, surface heat flux)
//   k_adj_interface  transpose of the face normals, curvature and Marangoni
//                    vector (Eq. 2-5 with delta_s = |grad alpha|)
//   k_adj_smooth     transpose of one [1,2,1]/4 smoothing pass
// The derivative of |g| at g = 0 is taken as 0.
#include "fvm_adjoint.h"
#include "fvm_device.cuh"

namespace fvm {

namespace {

struct Ref {
  int idx;
  double s;     // 0: the value is a constant (wall face), +-1: mirror sign
  double off;   // constant part (Dirichlet ghost 2 T_w)
};

__device__ __forceinline__ int lin3(const Geo& g, int i, int j, int k) {
  return (k * g.n[1] + j) * g.n[0] + i;
}

__device__ __forceinline__ Ref r_even(const Geo& g, int i, int j, int k) {
  int s = 1;
  i = mapc(i, g.n[0], g.bc[0], false, s);
  j = mapc(j, g.n[1], g.bc[1], false, s);
  k = mapc(k, g.n[2], g.bc[2], false, s);
  return {lin3(g, i, j, k), 1.0, 0.0};
}

template <int C>
__device__ __forceinline__ Ref r_vel(const Geo& g, int i, int j, int k) {
  int s = 1;
  i = (C == 0) ? mapf(i, g.n[0], g.bc[0], s) : mapc(i, g.n[0], g.bc[0], true, s);
  j = (C == 1) ? mapf(j, g.n[1], g.bc[1], s) : mapc(j, g.n[1], g.bc[1], true, s);
  k = (C == 2) ? mapf(k, g.n[2], g.bc[2], s) : mapc(k, g.n[2], g.bc[2], true, s);
  return {lin3(g, i, j, k), (double)s, 0.0};
}

__device__ __forceinline__ Ref r_T(const Geo& g, const TBC& tb, int i, int j, int k) {
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
  Ref r{lin3(g, m[0], m[1], m[2]), 1.0, 0.0};
  if (side >= 0) {
    double sc = (m[tb.s_axis] + 0.5) * g.h;
    r.s = -1.0;
    r.off = 2.0 * (tb.T0[side] + tb.amp[side] * cos(2.0 * M_PI * sc / tb.Ls));
  }
  return r;
}

__device__ __forceinline__ double val(const double* __restrict__ a, const Ref& r) {
  return r.s == 0.0 ? r.off : r.s * a[r.idx] + r.off;
}

__device__ __forceinline__ void scat(double* la, const Ref& r, double v) {
  if (r.s != 0.0 && v != 0.0) atomicAdd(la + r.idx, r.s * v);
}

template <int A>
__device__ __forceinline__ void off3(int& i, int& j, int& k, int s) {
  if (A == 0) i += s;
  if (A == 1) j += s;
  if (A == 2) k += s;
}

__device__ __forceinline__ double mixd(double a, const double* pair) {
  double c = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
  return c * pair[1] + (1.0 - c) * pair[0];
}

// WENO5-JS value from v[0..4] (left-biased, face right of v[2]) and its
// gradient with respect to the five values:
//   value = sum a_k q_k / S, a_k = d_k/(eps+beta_k)^2, S = sum a_k
//   d value = sum_k [a_k dq_k + (q_k - value) da_k] / S,
//   da_k = -2 a_k/(eps+beta_k) dbeta_k
__device__ double weno5_grad(const double* v, double eps, double* gr) {
  const double vm2 = v[0], vm1 = v[1], v0 = v[2], vp1 = v[3], vp2 = v[4];
  const double q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
  const double q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
  const double q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
  const double t0 = vm2 - 2.0 * vm1 + v0, u0 = vm2 - 4.0 * vm1 + 3.0 * v0;
  const double t1 = vm1 - 2.0 * v0 + vp1, u1 = vm1 - vp1;
  const double t2 = v0 - 2.0 * vp1 + vp2, u2 = 3.0 * v0 - 4.0 * vp1 + vp2;
  const double c1312 = 13.0 / 12.0;
  const double b0 = c1312 * t0 * t0 + 0.25 * u0 * u0;
  const double b1 = c1312 * t1 * t1 + 0.25 * u1 * u1;
  const double b2 = c1312 * t2 * t2 + 0.25 * u2 * u2;
  const double s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  const double a0 = 0.1 / (s0 * s0), a1 = 0.6 / (s1 * s1), a2 = 0.3 / (s2 * s2);
  const double S = a0 + a1 + a2;
  const double value = (a0 * q0 + a1 * q1 + a2 * q2) / S;
  const double dq0[5] = {2.0 / 6.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0};
  const double dq1[5] = {0.0, -1.0 / 6.0, 5.0 / 6.0, 2.0 / 6.0, 0.0};
  const double dq2[5] = {0.0, 0.0, 2.0 / 6.0, 5.0 / 6.0, -1.0 / 6.0};
  const double dt0[5] = {1, -2, 1, 0, 0}, du0[5] = {1, -4, 3, 0, 0};
  const double dt1[5] = {0, 1, -2, 1, 0}, du1[5] = {0, 1, 0, -1, 0};
  const double dt2[5] = {0, 0, 1, -2, 1}, du2[5] = {0, 0, 3, -4, 1};
  const double c0 = -2.0 * a0 / s0, c1 = -2.0 * a1 / s1, c2 = -2.0 * a2 / s2;
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const double db0 = 2.0 * c1312 * t0 * dt0[m] + 0.5 * u0 * du0[m];
    const double db1 = 2.0 * c1312 * t1 * dt1[m] + 0.5 * u1 * du1[m];
    const double db2 = 2.0 * c1312 * t2 * dt2[m] + 0.5 * u2 * du2[m];
    gr[m] = (a0 * dq0[m] + a1 * dq1[m] + a2 * dq2[m] + (q0 - value) * c0 * db0 +
             (q1 - value) * c1 * db1 + (q2 - value) * c2 * db2) / S;
  }
  return value;
}

// flux U * WENO5 (upwind by the sign of U) from v[0..5] (offsets -3..2 of the
// face); dU = dF/dU, gv[m] = dF/dv[m]
__device__ double upwind_grad(double U, const double* v, double eps, double* dU, double* gv) {
  double g5[5];
  for (int m = 0; m < 6; ++m) gv[m] = 0.0;
  double w;
  if (U >= 0.0) {
    const double in[5] = {v[0], v[1], v[2], v[3], v[4]};
    w = weno5_grad(in, eps, g5);
    for (int m = 0; m < 5; ++m) gv[m] = U * g5[m];
  } else {
    const double in[5] = {v[5], v[4], v[3], v[2], v[1]};
    w = weno5_grad(in, eps, g5);
    gv[5] = U * g5[0];
    gv[4] = U * g5[1];
    gv[3] = U * g5[2];
    gv[2] = U * g5[3];
    gv[1] = U * g5[4];
  }
  *dU = w;
  return U * w;
}

__device__ __forceinline__ double warp_sum_a(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void add_theta(double* dth, int q, double v) {
  v = warp_sum_a(v);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dth + q, v);
}

template <int D>
struct TangA {
  static constexpr int t1 = D == 0 ? 1 : 0;
  static constexpr int t2 = D == 2 ? 1 : 2;
};

// --------------------------------------------------------------------------
// momentum predictor: u*_D = u_D + dt (A + (V + f_n + f_M)/rho_f + g_D)
template <int D, int T_>
__device__ void adj_edge(const AdjArgs& A, int i, int j, int k, double coefA, double coefV) {
  const Geo& g = A.g;
  const double ih = g.ih;
  // low T_-edge of the D-face at (i, j, k)
  Ref rv[6];
  double v[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, c = k;
    off3<T_>(a, b, c, m - 3);
    rv[m] = r_vel<D>(g, a, b, c);
    v[m] = val(A.X[D], rv[m]);
  }
  int a2 = i, b2 = j, c2 = k;
  off3<D>(a2, b2, c2, -1);
  const Ref rt_hi = r_vel<T_>(g, i, j, k), rt_lo = r_vel<T_>(g, a2, b2, c2);
  const double Ue = 0.5 * (val(A.X[T_], rt_lo) + val(A.X[T_], rt_hi));
  if (coefA != 0.0) {
    double dU, gv[6];
    upwind_grad(Ue, v, A.eps_u, &dU, gv);
    for (int m = 0; m < 6; ++m) scat(A.lu[D], rv[m], coefA * gv[m]);
    scat(A.lu[T_], rt_lo, coefA * 0.5 * dU);
    scat(A.lu[T_], rt_hi, coefA * 0.5 * dU);
  }
  if (coefV != 0.0) {
    int a3 = i, b3 = j, c3 = k;
    off3<T_>(a3, b3, c3, -1);
    int a4 = a3, b4 = b3, c4 = c3;
    off3<D>(a4, b4, c4, -1);
    const double mue = 0.25 * (mixd(val(A.X[3], r_even(g, i, j, k)), A.mu) +
                               mixd(val(A.X[3], r_even(g, a2, b2, c2)), A.mu) +
                               mixd(val(A.X[3], r_even(g, a3, b3, c3)), A.mu) +
                               mixd(val(A.X[3], r_even(g, a4, b4, c4)), A.mu));
    const double w = coefV * mue * ih;
    scat(A.lu[D], rv[3], w);      // u_D at the face
    scat(A.lu[D], rv[2], -w);     // u_D at face - e_T
    scat(A.lu[T_], rt_hi, w);
    scat(A.lu[T_], rt_lo, -w);
  }
}

template <int D>
__device__ void adj_centre(const AdjArgs& A, int i, int j, int k, double coefA, double coefV) {
  const Geo& g = A.g;
  const double ih = g.ih;
  // centre of cell (i, j, k): faces (cell) + (m-2) e_D
  Ref rv[6];
  double v[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, c = k;
    off3<D>(a, b, c, m - 2);
    rv[m] = r_vel<D>(g, a, b, c);
    v[m] = val(A.X[D], rv[m]);
  }
  if (coefA != 0.0) {
    const double Uc = 0.5 * (v[2] + v[3]);
    double dU, gv[6];
    upwind_grad(Uc, v, A.eps_u, &dU, gv);
    for (int m = 0; m < 6; ++m) scat(A.lu[D], rv[m], coefA * gv[m]);
    scat(A.lu[D], rv[2], coefA * 0.5 * dU);
    scat(A.lu[D], rv[3], coefA * 0.5 * dU);
  }
  if (coefV != 0.0) {
    const double muc = mixd(val(A.X[3], r_even(g, i, j, k)), A.mu);
    const double w = coefV * 2.0 * muc * ih;
    scat(A.lu[D], rv[3], w);
    scat(A.lu[D], rv[2], -w);
  }
}

template <int D>
__device__ void adj_momentum_comp(const AdjArgs& A, int i, int j, int k, int c, double& dth1) {
  const Geo& g = A.g;
  const int gi[3] = {i, j, k};
  if (g.bc[D] == WALL && gi[D] == 0) return;
  const double lam = A.lus[D][c];
  if (lam == 0.0) return;
  constexpr int t1 = TangA<D>::t1, t2 = TangA<D>::t2;
  const double ih = g.ih, dt = A.dt;
  atomicAdd(A.lu[D] + c, lam);                    // u*_D = u_D + ...
  int a = i, b = j, cc = k;
  off3<D>(a, b, cc, -1);                          // cell L = c - e_D
  const Ref rL = r_even(g, a, b, cc);
  const double alL = val(A.X[3], rL), alR = A.X[3][c];
  const double rho_f = 0.5 * (mixd(alL, A.rho) + mixd(alR, A.rho));
  const double lA = dt * lam;                     // adjoint of the advection A
  const double lF = dt * lam / rho_f;             // adjoint of V + f_n + f_M
  // A = -(F_c(c) - F_c(c - e_D)) ih - sum_t (G_t(f + e_t) - G_t(f)) ih
  adj_centre<D>(A, i, j, k, -lA * ih, lF * ih);
  adj_centre<D>(A, a, b, cc, lA * ih, -lF * ih);
  {
    int x = i, y = j, z = k;
    off3<t1>(x, y, z, 1);
    adj_edge<D, t1>(A, i, j, k, lA * ih, -lF * ih);
    adj_edge<D, t1>(A, x, y, z, -lA * ih, lF * ih);
  }
  {
    int x = i, y = j, z = k;
    off3<t2>(x, y, z, 1);
    adj_edge<D, t2>(A, i, j, k, lA * ih, -lF * ih);
    adj_edge<D, t2>(A, x, y, z, -lA * ih, lF * ih);
  }
  // forces on the face between L and R = c
  const Ref tL = r_T(g, A.tb, a, b, cc);
  const double TL = val(A.X[4], tL), TR = A.X[4][c];
  const double sL = A.sigma0 + A.dsdT * (TL - A.T0), sR = A.sigma0 + A.dsdT * (TR - A.T0);
  const Ref kL = r_even(g, a, b, cc);
  const double kapL = val(A.kappa, kL), kapR = A.kappa[c];
  const double jump = (alR - alL) * ih;
  const double sf = 0.5 * (sL + sR), kf = 0.5 * (kapL + kapR);
  const double ls = lF * (-0.5 * kf * jump);      // d f_n / d sigma_L (= d / d sigma_R)
  scat(A.lu[4], tL, A.dsdT * ls);
  atomicAdd(A.lu[4] + c, A.dsdT * ls);
  dth1 += (TL - A.T0) * ls + (TR - A.T0) * ls;
  const double lk = lF * (-0.5 * sf * jump);
  scat(A.lkap, kL, lk);
  atomicAdd(A.lkap + c, lk);
  scat(A.lu[3], rL, lF * sf * kf * ih);            // alpha_L
  atomicAdd(A.lu[3] + c, -lF * sf * kf * ih);      // alpha_R
  scat(A.lM[D], kL, 0.5 * lF);
  atomicAdd(A.lM[D] + c, 0.5 * lF);
}

__global__ void k_adj_momentum(AdjArgs A) {
  const Geo& g = A.g;
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dth1 = 0.0;
  if (cl < g.N) {
    const int c = (int)cl;
    const int i = c % g.n[0], q = c / g.n[0], j = q % g.n[1], k = q / g.n[1];
    adj_momentum_comp<0>(A, i, j, k, c, dth1);
    adj_momentum_comp<1>(A, i, j, k, c, dth1);
    adj_momentum_comp<2>(A, i, j, k, c, dth1);
  }
  add_theta(A.dth, 0, dth1);
}

// --------------------------------------------------------------------------
// scalar update: alpha' = alpha + dt R_alpha, T' = T + dt R_T
template <int D>
__device__ void adj_scalar_face(const AdjArgs& A, int i, int j, int k, int c) {
  const Geo& g = A.g;
  const double ih = g.ih, dt = A.dt;
  const int gi[3] = {i, j, k};
  const bool wallface = g.bc[D] == WALL && gi[D] == 0;
  int a = i, b = j, cc = k;
  off3<D>(a, b, cc, -1);
  const Ref rLc = r_even(g, a, b, cc);            // cell left of the face (mirror at a wall)
  const double laR = A.laE[c], lTR = A.lTE[c];
  const double laL = wallface ? 0.0 : A.laE[rLc.idx];
  const double lTL = wallface ? 0.0 : A.lTE[rLc.idx];
  // advection through the face (none through a wall face)
  if (!wallface) {
    const double lFa = dt * ih * (laR - laL);
    const double lFT = dt * ih * (lTR - lTL);
    Ref ra[6], rt[6];
    double av[6], tv[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      int x = i, y = j, z = k;
      off3<D>(x, y, z, m - 3);
      ra[m] = r_even(g, x, y, z);
      rt[m] = r_T(g, A.tb, x, y, z);
      av[m] = val(A.X[3], ra[m]);
      tv[m] = val(A.X[4], rt[m]);
    }
    const double U = A.X[D][c];
    double dUa, dUT, ga[6], gt[6];
    upwind_grad(U, av, A.eps_a, &dUa, ga);
    upwind_grad(U, tv, A.eps_T, &dUT, gt);
    atomicAdd(A.lu[D] + c, lFa * dUa + lFT * dUT);
    for (int m = 0; m < 6; ++m) {
      scat(A.lu[3], ra[m], lFa * ga[m]);
      scat(A.lu[4], rt[m], lFT * gt[m]);
    }
  }
  // conduction D(f) = lambda_f (T_R - T_L) / h, T' += dt/(rho c_p) (D(f+e) - D(f)) / h
  {
    const Ref rTL = r_T(g, A.tb, a, b, cc);
    const double alR = A.X[3][c], alL = val(A.X[3], rLc);
    const double lR = mixd(alR, A.lam), lL = mixd(alL, A.lam);
    const double lf = 2.0 * lL * lR / (lL + lR);
    const double rcR = mixd(alR, A.rcp);
    double lD = -dt * ih * lTR / rcR;
    if (!wallface) lD += dt * ih * lTL / mixd(alL, A.rcp);
    const double w = lD * lf * ih;
    atomicAdd(A.lu[4] + c, w);
    scat(A.lu[4], rTL, -w);
  }
  // the implied high wall face of the last cell along a wall axis
  if (g.bc[D] == WALL && gi[D] == g.n[D] - 1) {
    int x = i, y = j, z = k;
    off3<D>(x, y, z, 1);
    const Ref rTH = r_T(g, A.tb, x, y, z);
    const double alR = A.X[3][c];
    const double alH = val(A.X[3], r_even(g, x, y, z));
    const double l0 = mixd(alR, A.lam), l1 = mixd(alH, A.lam);
    const double lf = 2.0 * l0 * l1 / (l0 + l1);
    const double lD = dt * ih * lTR / mixd(alR, A.rcp);
    const double w = lD * lf * ih;
    scat(A.lu[4], rTH, w);
    atomicAdd(A.lu[4] + c, -w);
  }
}

__global__ void k_adj_scalars(AdjArgs A) {
  const Geo& g = A.g;
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dth2 = 0.0;
  if (cl < g.N) {
    const int c = (int)cl;
    const int i = c % g.n[0], q = c / g.n[0], j = q % g.n[1], k = q / g.n[1];
    atomicAdd(A.lu[3] + c, A.laE[c]);
    atomicAdd(A.lu[4] + c, A.lTE[c]);
    adj_scalar_face<0>(A, i, j, k, c);
    adj_scalar_face<1>(A, i, j, k, c);
    adj_scalar_face<2>(A, i, j, k, c);
    // surface heat flux q |grad alpha| / (rho c_p)
    if (A.qunit != 0.0 && A.lTE[c] != 0.0) {
      const double ih = g.ih;
      const double x = (i + 0.5) * g.h, y = (j + 0.5) * g.h;
      double dx = x - A.xc, dy = y - A.yc;
      if (g.bc[0] == PER) dx = dx - A.L[0] * floor(dx / A.L[0] + 0.5);
      if (g.bc[1] == PER) dy = dy - A.L[1] * floor(dy / A.L[1] + 0.5);
      const double q1 = A.qunit * exp(-2.0 * (dx * dx + dy * dy) * A.ir2);   // per watt
      const double qv = A.qpower * q1;
      Ref rp[3], rm[3];
      double gv[3];
      rp[0] = r_even(g, i + 1, j, k); rm[0] = r_even(g, i - 1, j, k);
      rp[1] = r_even(g, i, j + 1, k); rm[1] = r_even(g, i, j - 1, k);
      rp[2] = r_even(g, i, j, k + 1); rm[2] = r_even(g, i, j, k - 1);
      for (int d = 0; d < 3; ++d) gv[d] = (val(A.X[3], rp[d]) - val(A.X[3], rm[d])) * (0.5 * ih);
      const double gn2 = gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2];
      const double gn = gn2 > 0.0 ? sqrt(gn2) : 0.0;
      const double rc = mixd(A.X[3][c], A.rcp);
      const double lgn = A.dt * qv / rc * A.lTE[c];
      if (gn > 0.0 && qv != 0.0) {
        for (int d = 0; d < 3; ++d) {
          const double w = lgn * gv[d] / gn * 0.5 * ih;
          scat(A.lu[3], rp[d], w);
          scat(A.lu[3], rm[d], -w);
        }
      }
      dth2 += A.dt * q1 * gn / rc * A.lTE[c];
    }
  }
  add_theta(A.dth, 1, dth2);
}

// --------------------------------------------------------------------------
// interface: kappa(c) = sum_D (N_D(c + e_D) - N_D(c)) / h, N = g_D/(|g|+eps)
// from the smoothed alpha; M = |g| (s - n (n.s)) at cells
template <int D>
__device__ void adj_normal(const AdjArgs& A, int i, int j, int k, double lam) {
  if (lam == 0.0) return;
  const Geo& g = A.g;
  const double ih = g.ih;
  int a = i, b = j, c = k;
  off3<D>(a, b, c, -1);
  const Ref r1 = r_even(g, i, j, k), r0 = r_even(g, a, b, c);
  const double gd = (val(A.at, r1) - val(A.at, r0)) * ih;
  Ref rt[2][4];
  double gt[2];
  int q = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t == D) continue;
    const int ox = t == 0, oy = t == 1, oz = t == 2;
    rt[q][0] = r_even(g, i + ox, j + oy, k + oz);
    rt[q][1] = r_even(g, i - ox, j - oy, k - oz);
    rt[q][2] = r_even(g, a + ox, b + oy, c + oz);
    rt[q][3] = r_even(g, a - ox, b - oy, c - oz);
    gt[q] = ((val(A.at, rt[q][0]) - val(A.at, rt[q][1])) +
             (val(A.at, rt[q][2]) - val(A.at, rt[q][3]))) * (0.25 * ih);
    ++q;
  }
  const double sq = gd * gd + gt[0] * gt[0] + gt[1] * gt[1];
  const double nrm = sq > 0.0 ? sqrt(sq) : 0.0;
  const double Dn = nrm + A.eps_n;
  const double dgd = nrm > 0.0 ? 1.0 / Dn - gd * gd / (nrm * Dn * Dn) : 1.0 / Dn;
  const double wd = lam * dgd * ih;
  scat(A.lat, r1, wd);
  scat(A.lat, r0, -wd);
  for (int p2 = 0; p2 < 2; ++p2) {
    const double dgt = nrm > 0.0 ? -gd * gt[p2] / (nrm * Dn * Dn) : 0.0;
    const double w = lam * dgt * 0.25 * ih;
    scat(A.lat, rt[p2][0], w);
    scat(A.lat, rt[p2][1], -w);
    scat(A.lat, rt[p2][2], w);
    scat(A.lat, rt[p2][3], -w);
  }
}

__global__ void k_adj_interface(AdjArgs A) {
  const Geo& g = A.g;
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dth1 = 0.0;
  if (cl < g.N) {
    const int c = (int)cl;
    const int i = c % g.n[0], q = c / g.n[0], j = q % g.n[1], k = q / g.n[1];
    const double ih = g.ih;
    const double lk = A.lkap[c];
    if (lk != 0.0) {
      adj_normal<0>(A, i + 1, j, k, lk * ih);
      adj_normal<0>(A, i, j, k, -lk * ih);
      adj_normal<1>(A, i, j + 1, k, lk * ih);
      adj_normal<1>(A, i, j, k, -lk * ih);
      adj_normal<2>(A, i, j, k + 1, lk * ih);
      adj_normal<2>(A, i, j, k, -lk * ih);
    }
    const double lm[3] = {A.lM[0][c], A.lM[1][c], A.lM[2][c]};
    if (lm[0] != 0.0 || lm[1] != 0.0 || lm[2] != 0.0) {
      Ref ap[3], am[3], tp[3], tm[3];
      double gv[3], tv[3], sv[3], Tp[3], Tm[3];
      for (int d = 0; d < 3; ++d) {
        const int ox = d == 0, oy = d == 1, oz = d == 2;
        ap[d] = r_even(g, i + ox, j + oy, k + oz);
        am[d] = r_even(g, i - ox, j - oy, k - oz);
        tp[d] = r_T(g, A.tb, i + ox, j + oy, k + oz);
        tm[d] = r_T(g, A.tb, i - ox, j - oy, k - oz);
        gv[d] = (val(A.X[3], ap[d]) - val(A.X[3], am[d])) * (0.5 * ih);
        tv[d] = (val(A.at, ap[d]) - val(A.at, am[d])) * (0.5 * ih);
        Tp[d] = val(A.X[4], tp[d]);
        Tm[d] = val(A.X[4], tm[d]);
        sv[d] = ((A.sigma0 + A.dsdT * (Tp[d] - A.T0)) - (A.sigma0 + A.dsdT * (Tm[d] - A.T0))) *
                (0.5 * ih);
      }
      const double gn2 = gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2];
      const double gn = gn2 > 0.0 ? sqrt(gn2) : 0.0;
      const double tn2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
      const double tnr = tn2 > 0.0 ? sqrt(tn2) : 0.0;
      const double Dt = tnr + A.eps_n;
      double nh[3];
      for (int d = 0; d < 3; ++d) nh[d] = tv[d] / Dt;
      const double ns = nh[0] * sv[0] + nh[1] * sv[1] + nh[2] * sv[2];
      const double lmn = lm[0] * nh[0] + lm[1] * nh[1] + lm[2] * nh[2];
      double ls[3], lnh[3];
      double lgn = 0.0;
      for (int d = 0; d < 3; ++d) {
        ls[d] = gn * (lm[d] - nh[d] * lmn);
        lnh[d] = -gn * (lm[d] * ns + sv[d] * lmn);
        lgn += lm[d] * (sv[d] - nh[d] * ns);
      }
      const double lnt = lnh[0] * tv[0] + lnh[1] * tv[1] + lnh[2] * tv[2];
      for (int d = 0; d < 3; ++d) {
        // smoothed alpha (unit normal)
        double lt = lnh[d] / Dt;
        if (tnr > 0.0) lt -= tv[d] * lnt / (tnr * Dt * Dt);
        scat(A.lat, ap[d], lt * 0.5 * ih);
        scat(A.lat, am[d], -lt * 0.5 * ih);
        // raw alpha (|grad alpha|)
        if (gn > 0.0) {
          const double lg = lgn * gv[d] / gn;
          scat(A.lu[3], ap[d], lg * 0.5 * ih);
          scat(A.lu[3], am[d], -lg * 0.5 * ih);
        }
        // sigma(T) central difference
        const double w = ls[d] * 0.5 * ih;
        scat(A.lu[4], tp[d], A.dsdT * w);
        scat(A.lu[4], tm[d], -A.dsdT * w);
        dth1 += w * ((Tp[d] - A.T0) - (Tm[d] - A.T0));
      }
    }
  }
  add_theta(A.dth, 0, dth1);
}

// transpose of one [1,2,1]/4 tensor pass: out(c) = sum w in(map(c + o))
__global__ void k_adj_smooth(Geo g, const double* __restrict__ lout, double* lin) {
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cl >= g.N) return;
  const int c = (int)cl;
  const double l = lout[c];
  if (l == 0.0) return;
  const int i = c % g.n[0], q = c / g.n[0], j = q % g.n[1], k = q / g.n[1];
  const int lo0 = g.n[0] > 1 ? -1 : 0, lo1 = g.n[1] > 1 ? -1 : 0, lo2 = g.n[2] > 1 ? -1 : 0;
  for (int dz = lo2; dz <= -lo2; ++dz) {
    const double wz = lo2 ? (dz == 0 ? 0.5 : 0.25) : 1.0;
    for (int dy = lo1; dy <= -lo1; ++dy) {
      const double wy = lo1 ? (dy == 0 ? 0.5 : 0.25) : 1.0;
      for (int dx = lo0; dx <= -lo0; ++dx) {
        const double wx = lo0 ? (dx == 0 ? 0.5 : 0.25) : 1.0;
        scat(lin, r_even(g, i + dx, j + dy, k + dz), wx * wy * wz * l);
      }
    }
  }
}

__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b,
                        double* __restrict__ y) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) y[c] = b == 0.0 ? a * x[c] : a * x[c] + b * y[c];
}

// zero the wall faces (index 0 along a wall axis) of a face field triple
__global__ void k_zero_wall_faces(Geo g, double* u0, double* u1, double* u2) {
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cl >= g.N) return;
  const int c = (int)cl;
  const int i = c % g.n[0], q = c / g.n[0], j = q % g.n[1], k = q / g.n[1];
  if (g.bc[0] == WALL && i == 0) u0[c] = 0.0;
  if (g.bc[1] == WALL && j == 0) u1[c] = 0.0;
  if (g.bc[2] == WALL && k == 0) u2[c] = 0.0;
}

}  // namespace

static inline unsigned g1(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_adj_momentum(const AdjArgs& A, cudaStream_t s) {
  k_adj_momentum<<<g1(A.g.N, 128), 128, 0, s>>>(A);
}
void launch_adj_scalars(const AdjArgs& A, cudaStream_t s) {
  k_adj_scalars<<<g1(A.g.N, 128), 128, 0, s>>>(A);
}
void launch_adj_interface(const AdjArgs& A, cudaStream_t s) {
  k_adj_interface<<<g1(A.g.N, 128), 128, 0, s>>>(A);
}
void launch_adj_smooth(const Geo& g, const double* lout, double* lin, cudaStream_t s) {
  k_adj_smooth<<<g1(g.N, 256), 256, 0, s>>>(g, lout, lin);
}
void launch_zero_wall_faces(const Geo& g, double* const* u, cudaStream_t s) {
  k_zero_wall_faces<<<g1(g.N, 256), 256, 0, s>>>(g, u[0], u[1], u[2]);
}
// y = a x + b y (y is not read when b == 0)
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby<<<g1(n, 256), 256, 0, s>>>(n, a, x, b, y);
}

}  // namespace fvm
