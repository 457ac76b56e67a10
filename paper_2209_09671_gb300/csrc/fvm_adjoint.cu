// Reverse mode (adjoint) of one forward-Euler stage of the FP64 step, for
// phases of equal viscosity, conductivity and volumetric heat capacity rho
// c_p (the transport coefficients are then constant); the densities may
// differ, which makes the face coefficient beta = 1/rho_f of the momentum
// predictor and of the projection depend on alpha (k_adj_density).
//
// Form of the work.  Every stencil flux is differentiated once, by the thread
// that owns its location (a cell centre, a face or an edge), in two passes:
//   pass 1  the thread computes the flux's adjoint weight from the adjoints
//           of the outputs the flux feeds, differentiates the flux with
//           respect to each value it reads and stores each product in a
//           coefficient slot K[q][location]; slot q has a fixed offset from
//           the location to the value it belongs to;
//   pass 2  one thread per cell adds, in a fixed order, the slots of the
//           locations whose offset lands on it.
// A value read through a boundary rule (a wrap, a mirror with its sign, a
// Dirichlet ghost, a wall face) is not at a fixed offset: pass 1 adds that
// product with an atomic add to the mapped cell and stores 0 in the slot.
// Only fluxes within three cells of a boundary do so, and the fluxes that lie
// outside the slot index space (the edges and faces on a high wall) use
// atomic adds throughout.  Two-point terms (face forces, conduction) are
// gathered directly by the cells they touch.
//   momentum   WENO5 advection on the MAC control volumes and the viscous
//              stress (centre and edge fluxes of each component), then the
//              CSF and Marangoni face forces (Sec. III, Eq. 4)
//   scalars    WENO5 transport of alpha (Eq. 1) and T, conduction, surface
//              heat flux
//   interface  face normals of the smoothed alpha (curvature) and the cell
//              Marangoni vector (Eq. 2-5 with delta_s = |grad alpha|)
// The [1,2,1]/4 smoothing pass is a symmetric matrix (the mirror and the
// wrap are symmetric), so its transpose is the forward smoothing kernel.
// The derivative of |g| at g = 0 is taken as 0.
#include "fvm_adjoint.h"
#include "fvm_device.cuh"

namespace fvm {

namespace {

struct Ref {
  int idx;
  double s;     // 0: the value is a constant (wall face), +-1: mirror sign
  double off;   // constant part (Dirichlet ghost 2 T_w)
  bool direct;  // the value is the unmapped cell at the requested offset
};

__device__ __forceinline__ int lin3(const Geo& g, int i, int j, int k) {
  return (k * g.n[1] + j) * g.n[0] + i;
}

__device__ __forceinline__ bool inr(const Geo& g, int i, int j, int k) {
  return (unsigned)i < (unsigned)g.n[0] && (unsigned)j < (unsigned)g.n[1] &&
         (unsigned)k < (unsigned)g.n[2];
}

__device__ __forceinline__ void decode3(const Geo& g, int c, int& i, int& j, int& k) {
  const int q = c / g.n[0];
  i = c - q * g.n[0];
  k = q / g.n[1];
  j = q - k * g.n[1];
}

__device__ __forceinline__ Ref r_even(const Geo& g, int i, int j, int k) {
  const bool d = inr(g, i, j, k);
  int s = 1;
  i = mapc(i, g.n[0], g.bc[0], false, s);
  j = mapc(j, g.n[1], g.bc[1], false, s);
  k = mapc(k, g.n[2], g.bc[2], false, s);
  return {lin3(g, i, j, k), 1.0, 0.0, d};
}

template <int C>
__device__ __forceinline__ Ref r_vel(const Geo& g, int i, int j, int k) {
  const bool d = inr(g, i, j, k);
  int s = 1;
  i = (C == 0) ? mapf(i, g.n[0], g.bc[0], s) : mapc(i, g.n[0], g.bc[0], true, s);
  j = (C == 1) ? mapf(j, g.n[1], g.bc[1], s) : mapc(j, g.n[1], g.bc[1], true, s);
  k = (C == 2) ? mapf(k, g.n[2], g.bc[2], s) : mapc(k, g.n[2], g.bc[2], true, s);
  return {lin3(g, i, j, k), (double)s, 0.0, d && s == 1};
}

__device__ __forceinline__ Ref r_T(const Geo& g, const TBC& tb, int i, int j, int k) {
  const bool dir = inr(g, i, j, k);
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
  Ref r{lin3(g, m[0], m[1], m[2]), 1.0, 0.0, dir};
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

// atomic add of d value * v into the adjoint la of the referenced value
__device__ __forceinline__ void scat(double* la, const Ref& r, double v) {
  if (r.s != 0.0 && v != 0.0) atomicAdd(la + r.idx, r.s * v);
}

// pass-1 output of one product: into slot q at location l when the value is
// at the slot's offset, else (and always when ATOMIC) straight to the target
template <bool ATOMIC>
__device__ __forceinline__ void emit(double* __restrict__ K, long long N, int q, int l,
                                     const Ref& r, double v, double* tgt) {
  if (!ATOMIC) {
    if (r.direct) {
      K[q * N + l] = v;
      return;
    }
    K[q * N + l] = 0.0;
  }
  scat(tgt, r, v);
}

// pass-2 input: slot q of location (i, j, k), 0 outside the grid
__device__ __forceinline__ double take(const double* __restrict__ K, long long N, int q,
                                       const Geo& g, int i, int j, int k) {
  return inr(g, i, j, k) ? K[q * N + lin3(g, i, j, k)] : 0.0;
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
  const double i6 = 1.0 / 6.0;
  const double q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) * i6;
  const double q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) * i6;
  const double q2 = (2.0 * v0 + 5.0 * vp1 - vp2) * i6;
  const double t0 = vm2 - 2.0 * vm1 + v0, u0 = vm2 - 4.0 * vm1 + 3.0 * v0;
  const double t1 = vm1 - 2.0 * v0 + vp1, u1 = vm1 - vp1;
  const double t2 = v0 - 2.0 * vp1 + vp2, u2 = 3.0 * v0 - 4.0 * vp1 + vp2;
  const double c1312 = 13.0 / 12.0;
  const double b0 = c1312 * t0 * t0 + 0.25 * u0 * u0;
  const double b1 = c1312 * t1 * t1 + 0.25 * u1 * u1;
  const double b2 = c1312 * t2 * t2 + 0.25 * u2 * u2;
  const double s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  // 1/s_k from one reciprocal of the product
  const double iP = 1.0 / (s0 * s1 * s2);
  const double r0 = s1 * s2 * iP, r1 = s0 * s2 * iP, r2 = s0 * s1 * iP;
  const double a0 = 0.1 * r0 * r0, a1 = 0.6 * r1 * r1, a2 = 0.3 * r2 * r2;
  const double iS = 1.0 / (a0 + a1 + a2);
  const double w0 = a0 * iS, w1 = a1 * iS, w2 = a2 * iS;
  const double value = w0 * q0 + w1 * q1 + w2 * q2;
  const double dq0[5] = {2.0 / 6.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0};
  const double dq1[5] = {0.0, -1.0 / 6.0, 5.0 / 6.0, 2.0 / 6.0, 0.0};
  const double dq2[5] = {0.0, 0.0, 2.0 / 6.0, 5.0 / 6.0, -1.0 / 6.0};
  const double dt0[5] = {1, -2, 1, 0, 0}, du0[5] = {1, -4, 3, 0, 0};
  const double dt1[5] = {0, 1, -2, 1, 0}, du1[5] = {0, 1, 0, -1, 0};
  const double dt2[5] = {0, 0, 1, -2, 1}, du2[5] = {0, 0, 3, -4, 1};
  // (q_k - value) (da_k / dbeta_k) / S
  const double e0 = -2.0 * (q0 - value) * w0 * r0;
  const double e1 = -2.0 * (q1 - value) * w1 * r1;
  const double e2 = -2.0 * (q2 - value) * w2 * r2;
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const double db0 = 2.0 * c1312 * t0 * dt0[m] + 0.5 * u0 * du0[m];
    const double db1 = 2.0 * c1312 * t1 * dt1[m] + 0.5 * u1 * du1[m];
    const double db2 = 2.0 * c1312 * t2 * dt2[m] + 0.5 * u2 * du2[m];
    gr[m] = w0 * dq0[m] + w1 * dq1[m] + w2 * dq2[m] + e0 * db0 + e1 * db1 + e2 * db2;
  }
  return value;
}

// flux U * WENO5 (upwind by the sign of U) from v[0..5] (offsets -3..2 of the
// face): *dU = dF/dU, gv[m] = dF/dv[m].  The upwind stencil is selected
// before one reconstruction (one inlined copy of the derivative code: the
// kernels that call this several times are bound by instruction fetch).
__device__ void upwind_grad(double U, const double* v, double eps, double* dU, double* gv) {
  const bool pos = U >= 0.0;
  double in[5], g5[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) in[m] = pos ? v[m] : v[5 - m];
  *dU = weno5_grad(in, eps, g5);
  gv[0] = pos ? U * g5[0] : 0.0;
  gv[5] = pos ? 0.0 : U * g5[0];
#pragma unroll
  for (int m = 1; m < 5; ++m) gv[m] = U * (pos ? g5[m] : g5[5 - m]);
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

#define ADJ_CELL(A, c, i, j, k)                                           \
  const long long cl_ = blockIdx.x * (long long)blockDim.x + threadIdx.x; \
  if (cl_ >= (A).g.N) return;                                             \
  const int c = (int)cl_;                                                 \
  int i, j, k;                                                            \
  decode3((A).g, c, i, j, k)

// --------------------------------------------------------------------------
// momentum predictor, component D on its faces:
//   u*_D(f) = u_D(f) + dt [A(f) + (V(f) + f_n(f) + f_M(f)) / rho_f + g_D]
//   A(f) = -(Fc(cell f) - Fc(cell f - e_D)) / h - sum_t (G_t(f + e_t) - G_t(f)) / h
// with Fc the centre flux (advecting velocity = mean of the cell's two D-faces)
// and G_t the flux through the low t-edge of face f (advecting velocity =
// mean of the two t-faces beside the edge); V has the same two-flux form.

// adjoint of the advection (lA = dt lambda) and of the stress (lF = dt
// lambda / rho_f) at the D-face (i, j, k); ghost faces and wall faces carry
// none.
template <int D>
__device__ __forceinline__ void face_weights(const AdjArgs& A, int i, int j, int k, double& lA,
                                             double& lF) {
  const Geo& g = A.g;
  int c[3] = {i, j, k};
  lA = 0.0;
  lF = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (c[d] < 0 || c[d] >= g.n[d]) {
      if (g.bc[d] == WALL) return;
      c[d] = wrapi(c[d], g.n[d]);
    }
  }
  if (g.bc[D] == WALL && c[D] == 0) return;
  const int f = lin3(g, c[0], c[1], c[2]);
  lA = A.dt * A.lus[D][f];
  lF = lA * A.beta[D][f];
}

// centre flux of component D at cell (i, j, k): slots q0 + m <- u_D at
// (i, j, k) + (m - 2) e_D
template <int D>
__device__ void centre_flux(const AdjArgs& A, int i, int j, int k, int l, int q0) {
  const Geo& g = A.g;
  const double ih = g.ih;
  double lAlo, lFlo, lAhi, lFhi;
  face_weights<D>(A, i, j, k, lAlo, lFlo);
  {
    int a = i, b = j, c = k;
    off3<D>(a, b, c, 1);
    face_weights<D>(A, a, b, c, lAhi, lFhi);
  }
  const double coefA = ih * (lAhi - lAlo), coefV = ih * (lFlo - lFhi);
  Ref rv[6];
  double v[6], out[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, c = k;
    off3<D>(a, b, c, m - 2);
    rv[m] = r_vel<D>(g, a, b, c);
    v[m] = val(A.X[D], rv[m]);
    out[m] = 0.0;
  }
  if (coefA != 0.0) {
    const double Uc = 0.5 * (v[2] + v[3]);
    double dU, gv[6];
    upwind_grad(Uc, v, A.eps_u, &dU, gv);
#pragma unroll
    for (int m = 0; m < 6; ++m) out[m] = coefA * gv[m];
    out[2] += coefA * 0.5 * dU;
    out[3] += coefA * 0.5 * dU;
  }
  if (coefV != 0.0) {
    const double w = coefV * 2.0 * mixd(A.X[3][l], A.mu) * ih;
    out[3] += w;
    out[2] -= w;
  }
#pragma unroll
  for (int m = 0; m < 6; ++m) emit<false>(A.K, A.g.N, q0 + m, l, rv[m], out[m], A.lu[D]);
}

// flux through the low T_-edge of the D-face (i, j, k): slots q0 + m <- u_D at
// (i, j, k) + (m - 3) e_T; q0 + 6 <- u_T at (i, j, k); q0 + 7 <- u_T at
// (i, j, k) - e_D.  ATOMIC: an edge outside the slot index space.
template <int D, int T_, bool ATOMIC>
__device__ void edge_flux(const AdjArgs& A, int i, int j, int k, int l, int q0) {
  const Geo& g = A.g;
  const double ih = g.ih;
  double lA0, lF0, lA1, lF1;
  face_weights<D>(A, i, j, k, lA0, lF0);
  {
    int a = i, b = j, c = k;
    off3<T_>(a, b, c, -1);
    face_weights<D>(A, a, b, c, lA1, lF1);
  }
  const double coefA = ih * (lA0 - lA1), coefV = ih * (lF1 - lF0);
  Ref rv[6];
  double v[6], out[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, c = k;
    off3<T_>(a, b, c, m - 3);
    rv[m] = r_vel<D>(g, a, b, c);
    v[m] = val(A.X[D], rv[m]);
    out[m] = 0.0;
  }
  int a2 = i, b2 = j, c2 = k;
  off3<D>(a2, b2, c2, -1);
  const Ref rt_hi = r_vel<T_>(g, i, j, k), rt_lo = r_vel<T_>(g, a2, b2, c2);
  double chi = 0.0, clo = 0.0;
  if (coefA != 0.0) {
    const double Ue = 0.5 * (val(A.X[T_], rt_lo) + val(A.X[T_], rt_hi));
    double dU, gv[6];
    upwind_grad(Ue, v, A.eps_u, &dU, gv);
#pragma unroll
    for (int m = 0; m < 6; ++m) out[m] = coefA * gv[m];
    chi = clo = coefA * 0.5 * dU;
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
    out[3] += w;
    out[2] -= w;
    chi += w;
    clo -= w;
  }
#pragma unroll
  for (int m = 0; m < 6; ++m) emit<ATOMIC>(A.K, A.g.N, q0 + m, l, rv[m], out[m], A.lu[D]);
  emit<ATOMIC>(A.K, A.g.N, q0 + 6, l, rt_hi, chi, A.lu[T_]);
  emit<ATOMIC>(A.K, A.g.N, q0 + 7, l, rt_lo, clo, A.lu[T_]);
}

// pass 1 of component D: centre flux (slots 0-5), t1-edge (6-13), t2-edge (14-21)
template <int D>
__global__ void k_adj_mom_flux(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  constexpr int t1 = TangA<D>::t1, t2 = TangA<D>::t2;
  const Geo& g = A.g;
  centre_flux<D>(A, i, j, k, c, 0);
  edge_flux<D, t1, false>(A, i, j, k, c, 6);
  edge_flux<D, t2, false>(A, i, j, k, c, 14);
  const int gi[3] = {i, j, k};
  if (g.bc[t1] == WALL && gi[t1] == g.n[t1] - 1) {
    int a = i, b = j, e = k;
    off3<t1>(a, b, e, 1);
    edge_flux<D, t1, true>(A, a, b, e, c, 6);
  }
  if (g.bc[t2] == WALL && gi[t2] == g.n[t2] - 1) {
    int a = i, b = j, e = k;
    off3<t2>(a, b, e, 1);
    edge_flux<D, t2, true>(A, a, b, e, c, 14);
  }
}

// pass 2 of component D, and the identity u*_D = u_D + ...
template <int D>
__global__ void k_adj_mom_gather(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  constexpr int t1 = TangA<D>::t1, t2 = TangA<D>::t2;
  const Geo& g = A.g;
  const long long N = g.N;
  const double* K = A.K;
  double aD = A.lus[D][c];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, e = k;
    off3<D>(a, b, e, 2 - m);
    aD += take(K, N, m, g, a, b, e);
  }
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, e = k;
    off3<t1>(a, b, e, 3 - m);
    aD += take(K, N, 6 + m, g, a, b, e);
  }
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, e = k;
    off3<t2>(a, b, e, 3 - m);
    aD += take(K, N, 14 + m, g, a, b, e);
  }
  int a = i, b = j, e = k;
  off3<D>(a, b, e, 1);
  const double a1 = K[12 * N + c] + take(K, N, 13, g, a, b, e);
  const double a2 = K[20 * N + c] + take(K, N, 21, g, a, b, e);
  A.lu[D][c] += aD;
  A.lu[t1][c] += a1;
  A.lu[t2][c] += a2;
}

// CSF and Marangoni face forces: f = -sigma_f kappa_f (alpha_R - alpha_L)/h
// + (M_D(L) + M_D(R))/2 on every D-face, each cell gathering the two faces
// it touches (its own low face as R, the next face as L), scaled by 1/rho_f
__global__ void k_adj_forces(AdjArgs A) {
  const Geo& g = A.g;
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dth1 = 0.0;
  if (cl < g.N) {
    const int c = (int)cl;
    int i, j, k;
    decode3(g, c, i, j, k);
    const double ih = g.ih, dt = A.dt;
    const int gi[3] = {i, j, k};
    double aT = 0.0, ak = 0.0, aa = 0.0, aM[3] = {0.0, 0.0, 0.0};
    const double alC = A.X[3][c], TC = A.X[4][c], kC = A.kappa[c];
    const double sC = A.sigma0 + A.dsdT * (TC - A.T0);
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      const int ox = D == 0, oy = D == 1, oz = D == 2;
      // own low face: this cell is R
      if (!(g.bc[D] == WALL && gi[D] == 0)) {
        const double lam = A.lus[D][c];
        if (lam != 0.0) {
          const Ref rL = r_even(g, i - ox, j - oy, k - oz);
          const Ref tL = r_T(g, A.tb, i - ox, j - oy, k - oz);
          const double alL = val(A.X[3], rL), TL = val(A.X[4], tL), kL = val(A.kappa, rL);
          const double lF = dt * lam * A.beta[D][c];
          const double sL = A.sigma0 + A.dsdT * (TL - A.T0);
          const double jump = (alC - alL) * ih;
          const double sf = 0.5 * (sL + sC), kf = 0.5 * (kL + kC);
          const double ls = lF * (-0.5 * kf * jump);
          aT += A.dsdT * ls;
          dth1 += ((TL - A.T0) + (TC - A.T0)) * ls;
          ak += lF * (-0.5 * sf * jump);
          aa -= lF * sf * kf * ih;
          aM[D] += 0.5 * lF;
        }
      }
      // next face: this cell is L
      const Ref rf = D == 0 ? r_vel<0>(g, i + 1, j, k)
                            : (D == 1 ? r_vel<1>(g, i, j + 1, k) : r_vel<2>(g, i, j, k + 1));
      if (rf.s != 0.0) {
        const double lam = A.lus[D][rf.idx];
        if (lam != 0.0) {
          const int R = rf.idx;
          const double alR = A.X[3][R], TR = A.X[4][R], kR = A.kappa[R];
          const double lF = dt * lam * A.beta[D][R];
          const double sR = A.sigma0 + A.dsdT * (TR - A.T0);
          const double jump = (alR - alC) * ih;
          const double sf = 0.5 * (sC + sR), kf = 0.5 * (kC + kR);
          const double ls = lF * (-0.5 * kf * jump);
          aT += A.dsdT * ls;
          ak += lF * (-0.5 * sf * jump);
          aa += lF * sf * kf * ih;
          aM[D] += 0.5 * lF;
        }
      }
    }
    A.lu[4][c] += aT;
    A.lu[3][c] += aa;
    A.lkap[c] += ak;
    A.lM[0][c] += aM[0];
    A.lM[1][c] += aM[1];
    A.lM[2][c] += aM[2];
  }
  add_theta(A.dth, 0, dth1);
}

// --------------------------------------------------------------------------
// scalar update: alpha' = alpha + dt R_alpha, T' = T + dt R_T with
// R = -(F(f + e_D) - F(f)) / h summed over D, F = U_f WENO5 (upwind)

// pass 1 along D: slots 0-5 <- alpha at f + (m - 3) e_D, 6-11 <- T there; the
// face velocity's adjoint is added in place (its own face)
template <int D>
__global__ void k_adj_scal_flux(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  const Geo& g = A.g;
  const double ih = g.ih, dt = A.dt;
  const int gi[3] = {i, j, k};
  const bool wallface = g.bc[D] == WALL && gi[D] == 0;
  double outa[6] = {0, 0, 0, 0, 0, 0}, outT[6] = {0, 0, 0, 0, 0, 0};
  Ref ra[6], rt[6];
  double av[6], tv[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int x = i, y = j, z = k;
    off3<D>(x, y, z, m - 3);
    ra[m] = r_even(g, x, y, z);
    rt[m] = r_T(g, A.tb, x, y, z);
  }
  if (!wallface) {
    const int L = ra[2].idx;   // the cell left of the face (wrapped on a periodic axis)
    const double lFa = dt * ih * (A.laE[c] - A.laE[L]);
    const double lFT = dt * ih * (A.lTE[c] - A.lTE[L]);
    if (lFa != 0.0 || lFT != 0.0) {
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        av[m] = val(A.X[3], ra[m]);
        tv[m] = val(A.X[4], rt[m]);
      }
      const double U = A.X[D][c];
      double dUa, dUT, ga[6], gt[6];
      upwind_grad(U, av, A.eps_a, &dUa, ga);
      upwind_grad(U, tv, A.eps_T, &dUT, gt);
      A.lu[D][c] += lFa * dUa + lFT * dUT;
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        outa[m] = lFa * ga[m];
        outT[m] = lFT * gt[m];
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    emit<false>(A.K, g.N, m, c, ra[m], outa[m], A.lu[3]);
    emit<false>(A.K, g.N, 6 + m, c, rt[m], outT[m], A.lu[4]);
  }
}

// pass 2 along D (D = 0 also adds the identity alpha' = alpha + ...)
template <int D>
__global__ void k_adj_scal_gather(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  const Geo& g = A.g;
  const long long N = g.N;
  double aa = D == 0 ? A.laE[c] : 0.0, aT = D == 0 ? A.lTE[c] : 0.0;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = i, b = j, e = k;
    off3<D>(a, b, e, 3 - m);
    aa += take(A.K, N, m, g, a, b, e);
    aT += take(A.K, N, 6 + m, g, a, b, e);
  }
  A.lu[3][c] += aa;
  A.lu[4][c] += aT;
}

// conduction: T' += dt/(rho c_p) (Q(f + e_D) - Q(f)) / h, Q = lambda_f (T_R - T_L)/h
// with the harmonic face conductivity; each cell gathers its two faces per
// axis (a wall ghost of either side maps back onto the cell itself)
__global__ void k_adj_conduction(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  const Geo& g = A.g;
  const double ih = g.ih, dt = A.dt;
  const int gi[3] = {i, j, k};
  const double alC = A.X[3][c];
  const double lC = mixd(alC, A.lam);
  const double qC = A.lTE[c] / mixd(alC, A.rcp);
  double aT = 0.0;
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    const int ox = D == 0, oy = D == 1, oz = D == 2;
    {   // low face: this cell is R; L is a ghost on a low wall
      const bool ghost = g.bc[D] == WALL && gi[D] == 0;
      const Ref rL = r_even(g, i - ox, j - oy, k - oz);
      const double lL = mixd(val(A.X[3], rL), A.lam);
      const double lf = 2.0 * lL * lC / (lL + lC);
      double mu = -dt * ih * qC;
      if (!ghost) mu += dt * ih * A.lTE[rL.idx] / mixd(A.X[3][rL.idx], A.rcp);
      const double w = mu * lf * ih;
      aT += w;
      if (ghost) aT -= r_T(g, A.tb, i - ox, j - oy, k - oz).s * w;
    }
    {   // high face: this cell is L; R is a ghost on a high wall
      const bool ghost = g.bc[D] == WALL && gi[D] == g.n[D] - 1;
      const Ref rR = r_even(g, i + ox, j + oy, k + oz);
      const double lR = mixd(val(A.X[3], rR), A.lam);
      const double lf = 2.0 * lC * lR / (lC + lR);
      double mu = dt * ih * qC;
      if (!ghost) mu -= dt * ih * A.lTE[rR.idx] / mixd(A.X[3][rR.idx], A.rcp);
      const double w = mu * lf * ih;
      aT -= w;
      if (ghost) aT += r_T(g, A.tb, i + ox, j + oy, k + oz).s * w;
    }
  }
  A.lu[4][c] += aT;
}

// surface heat flux q |grad alpha| / (rho c_p) (central grad alpha; nonzero
// only near the interface, so the products go out with atomic adds)
__global__ void k_adj_source(AdjArgs A) {
  const Geo& g = A.g;
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dth2 = 0.0;
  if (cl < g.N && A.qunit != 0.0) {
    const int c = (int)cl;
    int i, j, k;
    decode3(g, c, i, j, k);
    const double lT = A.lTE[c];
    if (lT != 0.0) {
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
      if (gn > 0.0 && qv != 0.0) {
        const double lgn = A.dt * qv / rc * lT;
        for (int d = 0; d < 3; ++d) {
          const double w = lgn * gv[d] / gn * 0.5 * ih;
          scat(A.lu[3], rp[d], w);
          scat(A.lu[3], rm[d], -w);
        }
      }
      dth2 = A.dt * q1 * gn / rc * lT;
    }
  }
  add_theta(A.dth, 1, dth2);
}

// --------------------------------------------------------------------------
// interface: kappa(c) = sum_D (N_D(c + e_D) - N_D(c)) / h with the face
// normal N_D = g_D / (|g| + eps) of the smoothed alpha; M = |grad alpha|
// (s - n (n.s)) at cells, n from the smoothed alpha, s = grad sigma(T)

// face normal N_D at the D-face (i, j, k) with adjoint lam: slot 0 <- at
// (i,j,k), 1 <- at (i,j,k) - e_D, then per tangential axis t (in order)
// 2+4q .. 5+4q <- at +e_t, -e_t, -e_D+e_t, -e_D-e_t
template <int D, bool ATOMIC>
__device__ void normal_flux(const AdjArgs& A, int i, int j, int k, int l, double lam) {
  const Geo& g = A.g;
  const double ih = g.ih;
  int a = i, b = j, c = k;
  off3<D>(a, b, c, -1);
  const Ref r1 = r_even(g, i, j, k), r0 = r_even(g, a, b, c);
  Ref rt[2][4];
  int q = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t == D) continue;
    const int ox = t == 0, oy = t == 1, oz = t == 2;
    rt[q][0] = r_even(g, i + ox, j + oy, k + oz);
    rt[q][1] = r_even(g, i - ox, j - oy, k - oz);
    rt[q][2] = r_even(g, a + ox, b + oy, c + oz);
    rt[q][3] = r_even(g, a - ox, b - oy, c - oz);
    ++q;
  }
  double o1 = 0.0, o0 = 0.0, ot[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  if (lam != 0.0) {
    const double gd = (val(A.at, r1) - val(A.at, r0)) * ih;
    double gt[2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
      gt[p] = ((val(A.at, rt[p][0]) - val(A.at, rt[p][1])) +
               (val(A.at, rt[p][2]) - val(A.at, rt[p][3]))) * (0.25 * ih);
    const double sq = gd * gd + gt[0] * gt[0] + gt[1] * gt[1];
    const double nrm = sq > 0.0 ? sqrt(sq) : 0.0;
    const double Dn = nrm + A.eps_n;
    const double dgd = nrm > 0.0 ? 1.0 / Dn - gd * gd / (nrm * Dn * Dn) : 1.0 / Dn;
    const double wd = lam * dgd * ih;
    o1 = wd;
    o0 = -wd;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const double dgt = nrm > 0.0 ? -gd * gt[p] / (nrm * Dn * Dn) : 0.0;
      const double w = lam * dgt * 0.25 * ih;
      ot[p][0] = w;
      ot[p][1] = -w;
      ot[p][2] = w;
      ot[p][3] = -w;
    }
  }
  emit<ATOMIC>(A.K, g.N, 0, l, r1, o1, A.lat);
  emit<ATOMIC>(A.K, g.N, 1, l, r0, o0, A.lat);
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int s = 0; s < 4; ++s) emit<ATOMIC>(A.K, g.N, 2 + 4 * p + s, l, rt[p][s], ot[p][s], A.lat);
}

// pass 1 of the D-normals: adjoint of N_D(f) = (lkap(cell f - e_D) -
// lkap(cell f)) / h; a high wall face (outside the slot index space) goes out
// with atomic adds
template <int D>
__global__ void k_adj_normal_flux(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  const Geo& g = A.g;
  const double ih = g.ih;
  const int gi[3] = {i, j, k};
  double lam = -A.lkap[c] * ih;
  if (!(g.bc[D] == WALL && gi[D] == 0)) {
    int a = i, b = j, e = k;
    off3<D>(a, b, e, -1);
    lam += A.lkap[r_even(g, a, b, e).idx] * ih;
  }
  normal_flux<D, false>(A, i, j, k, c, lam);
  if (g.bc[D] == WALL && gi[D] == g.n[D] - 1) {
    int a = i, b = j, e = k;
    off3<D>(a, b, e, 1);
    normal_flux<D, true>(A, a, b, e, c, A.lkap[c] * ih);
  }
}

template <int D>
__global__ void k_adj_normal_gather(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  const Geo& g = A.g;
  const long long N = g.N;
  const double* K = A.K;
  int a = i, b = j, e = k;
  off3<D>(a, b, e, 1);
  double acc = K[c] + take(K, N, 1, g, a, b, e);
  int q = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t == D) continue;
    const int ox = t == 0, oy = t == 1, oz = t == 2;
    acc += take(K, N, 2 + 4 * q, g, i - ox, j - oy, k - oz);
    acc += take(K, N, 3 + 4 * q, g, i + ox, j + oy, k + oz);
    acc += take(K, N, 4 + 4 * q, g, a - ox, b - oy, e - oz);
    acc += take(K, N, 5 + 4 * q, g, a + ox, b + oy, e + oz);
    ++q;
  }
  A.lat[c] += acc;
}

// Marangoni vector, pass 1: slots 2d / 2d+1 <- alpha at c + e_d / c - e_d,
// 6+2d / 7+2d <- smoothed alpha there, 12+2d / 13+2d <- T there
__global__ void k_adj_marangoni_flux(AdjArgs A) {
  const Geo& g = A.g;
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dth1 = 0.0;
  if (cl < g.N) {
    const int c = (int)cl;
    int i, j, k;
    decode3(g, c, i, j, k);
    const double ih = g.ih;
    const double lm[3] = {A.lM[0][c], A.lM[1][c], A.lM[2][c]};
    Ref ap[3], am[3], tp[3], tm[3];
    double oa[6] = {0, 0, 0, 0, 0, 0}, ot[6] = {0, 0, 0, 0, 0, 0}, oT[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int ox = d == 0, oy = d == 1, oz = d == 2;
      ap[d] = r_even(g, i + ox, j + oy, k + oz);
      am[d] = r_even(g, i - ox, j - oy, k - oz);
      tp[d] = r_T(g, A.tb, i + ox, j + oy, k + oz);
      tm[d] = r_T(g, A.tb, i - ox, j - oy, k - oz);
    }
    if (lm[0] != 0.0 || lm[1] != 0.0 || lm[2] != 0.0) {
      double gv[3], tv[3], sv[3], Tp[3], Tm[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
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
#pragma unroll
      for (int d = 0; d < 3; ++d) nh[d] = tv[d] / Dt;
      const double ns = nh[0] * sv[0] + nh[1] * sv[1] + nh[2] * sv[2];
      const double lmn = lm[0] * nh[0] + lm[1] * nh[1] + lm[2] * nh[2];
      double ls[3], lnh[3];
      double lgn = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ls[d] = gn * (lm[d] - nh[d] * lmn);
        lnh[d] = -gn * (lm[d] * ns + sv[d] * lmn);
        lgn += lm[d] * (sv[d] - nh[d] * ns);
      }
      const double lnt = lnh[0] * tv[0] + lnh[1] * tv[1] + lnh[2] * tv[2];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double lt = lnh[d] / Dt;
        if (tnr > 0.0) lt -= tv[d] * lnt / (tnr * Dt * Dt);
        ot[2 * d] = lt * 0.5 * ih;
        ot[2 * d + 1] = -lt * 0.5 * ih;
        if (gn > 0.0) {
          const double lg = lgn * gv[d] / gn;
          oa[2 * d] = lg * 0.5 * ih;
          oa[2 * d + 1] = -lg * 0.5 * ih;
        }
        const double w = ls[d] * 0.5 * ih;
        oT[2 * d] = A.dsdT * w;
        oT[2 * d + 1] = -A.dsdT * w;
        dth1 += w * (Tp[d] - Tm[d]);
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      emit<false>(A.K, g.N, 2 * d, c, ap[d], oa[2 * d], A.lu[3]);
      emit<false>(A.K, g.N, 2 * d + 1, c, am[d], oa[2 * d + 1], A.lu[3]);
      emit<false>(A.K, g.N, 6 + 2 * d, c, ap[d], ot[2 * d], A.lat);
      emit<false>(A.K, g.N, 7 + 2 * d, c, am[d], ot[2 * d + 1], A.lat);
      emit<false>(A.K, g.N, 12 + 2 * d, c, tp[d], oT[2 * d], A.lu[4]);
      emit<false>(A.K, g.N, 13 + 2 * d, c, tm[d], oT[2 * d + 1], A.lu[4]);
    }
  }
  add_theta(A.dth, 0, dth1);
}

__global__ void k_adj_marangoni_gather(AdjArgs A) {
  ADJ_CELL(A, c, i, j, k);
  const Geo& g = A.g;
  const long long N = g.N;
  double aa = 0.0, at = 0.0, aT = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ox = d == 0, oy = d == 1, oz = d == 2;
    aa += take(A.K, N, 2 * d, g, i - ox, j - oy, k - oz) +
          take(A.K, N, 2 * d + 1, g, i + ox, j + oy, k + oz);
    at += take(A.K, N, 6 + 2 * d, g, i - ox, j - oy, k - oz) +
          take(A.K, N, 7 + 2 * d, g, i + ox, j + oy, k + oz);
    aT += take(A.K, N, 12 + 2 * d, g, i - ox, j - oy, k - oz) +
          take(A.K, N, 13 + 2 * d, g, i + ox, j + oy, k + oz);
  }
  A.lu[3][c] += aa;
  A.lat[c] += at;
  A.lu[4][c] += aT;
}

// d/d alpha of the two 1/rho_f = beta_f factors of the stage.  With
// mu = lus the adjoint of u*, the momentum predictor's dt (V + f) beta_f and
// the projection's -dt beta_f (G p)_f give, per face, dt mu_f (Phi_f - (G p)_f)
// d beta_f, where Phi_f = V + f_n + f_M and p is the stage's forward
// pressure (the projection's adjoint is u* -> P^T; its derivative in beta is
// -dt P (d beta G p)); d beta_f / d alpha_L,R = -beta_f^2 / 2 (rho_1 - rho_0)
// on [0, 1] (the clamp of the mixture passes its bounds).  Each cell gathers
// its low face (as R) and the next face (as L) in every direction.
__global__ void k_adj_density(AdjArgs A, double drho) {
  const Geo& g = A.g;
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cl >= g.N) return;
  const int c = (int)cl;
  const double al = A.X[3][c];
  if (!(al >= 0.0 && al <= 1.0)) return;
  int i, j, k;
  decode3(g, c, i, j, k);
  const int gi[3] = {i, j, k};
  const int st[3] = {1, g.n[0], g.n[0] * g.n[1]};
  double acc = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int n = g.n[d];
    if (n == 1) continue;
    // own low face f = c (skipped on a wall), then the next face (the low face
    // of the neighbour above, wrapped; none above the last cell of a wall axis)
    for (int side = 0; side < 2; ++side) {
      int f;
      if (side == 0) {
        if (g.bc[d] == WALL && gi[d] == 0) continue;
        f = c;
      } else {
        if (gi[d] == n - 1) {
          if (g.bc[d] == WALL) continue;
          f = c - (n - 1) * st[d];
        } else {
          f = c + st[d];
        }
      }
      int fi, fj, fk;
      decode3(g, f, fi, fj, fk);
      const int fidx[3] = {fi, fj, fk};
      const int lo = fidx[d] == 0 ? f + (n - 1) * st[d] : f - st[d];
      const double gp = (A.pfw[f] - A.pfw[lo]) * g.ih;
      const double b = A.beta[d][f];
      acc += A.lus[d][f] * b * b * (A.phi[d][f] - gp);
    }
  }
  A.lu[3][c] += -0.5 * drho * A.dt * acc;
}


__global__ void k_sub_grad(Geo g, const double* __restrict__ u0, const double* __restrict__ u1,
                           const double* __restrict__ u2, const double* __restrict__ p,
                           const double* __restrict__ dtp, double* __restrict__ o0,
                           double* __restrict__ o1, double* __restrict__ o2) {
  const long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cl >= g.N) return;
  const int c = (int)cl;
  int i, j, k;
  decode3(g, c, i, j, k);
  const int gi[3] = {i, j, k};
  const int st[3] = {1, g.n[0], g.n[0] * g.n[1]};
  const double* u[3] = {u0, u1, u2};
  double* o[3] = {o0, o1, o2};
  const double dth = dtp[0] * g.ih;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (g.bc[d] == WALL && gi[d] == 0) {
      o[d][c] = 0.0;
      continue;
    }
    const int lo = gi[d] == 0 ? c + (g.n[d] - 1) * st[d] : c - st[d];
    o[d][c] = u[d][c] - (p[c] - p[lo]) * dth;
  }
}


__global__ void k_face_mul(long long n, const double* __restrict__ b0, const double* __restrict__ b1,
                           const double* __restrict__ b2, const double* __restrict__ u0,
                           const double* __restrict__ u1, const double* __restrict__ u2,
                           double* __restrict__ o0, double* __restrict__ o1, double* __restrict__ o2) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= n) return;
  o0[c] = b0[c] * u0[c];
  o1[c] = b1[c] * u1[c];
  o2[c] = b2[c] * u2[c];
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
  int i, j, k;
  decode3(g, c, i, j, k);
  if (g.bc[0] == WALL && i == 0) u0[c] = 0.0;
  if (g.bc[1] == WALL && j == 0) u1[c] = 0.0;
  if (g.bc[2] == WALL && k == 0) u2[c] = 0.0;
}

}  // namespace

int launch_adj_density(const AdjArgs& A, cudaStream_t s) {
  k_adj_density<<<(unsigned)((A.g.N + 127) / 128), 128, 0, s>>>(A, A.rho[1] - A.rho[0]);
  return 1;
}

void launch_sub_grad(const Geo& g, double* const* u, const double* p, const double* dt,
                     double* const* out, cudaStream_t s) {
  k_sub_grad<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g, u[0], u[1], u[2], p, dt, out[0],
                                                           out[1], out[2]);
}

void launch_face_mul(const Geo& g, double* const* beta, double* const* u, double* const* out,
                     cudaStream_t s) {
  k_face_mul<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(g.N, beta[0], beta[1], beta[2], u[0],
                                                           u[1], u[2], out[0], out[1], out[2]);
}

static inline unsigned g1(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

int launch_adj_momentum(const AdjArgs& A, cudaStream_t s) {
  const unsigned gb = g1(A.g.N, 128);
  k_adj_mom_flux<0><<<gb, 128, 0, s>>>(A);
  k_adj_mom_gather<0><<<gb, 128, 0, s>>>(A);
  k_adj_mom_flux<1><<<gb, 128, 0, s>>>(A);
  k_adj_mom_gather<1><<<gb, 128, 0, s>>>(A);
  k_adj_mom_flux<2><<<gb, 128, 0, s>>>(A);
  k_adj_mom_gather<2><<<gb, 128, 0, s>>>(A);
  k_adj_forces<<<gb, 128, 0, s>>>(A);
  return 7;
}
int launch_adj_scalars(const AdjArgs& A, cudaStream_t s) {
  const unsigned gb = g1(A.g.N, 128);
  k_adj_scal_flux<0><<<gb, 128, 0, s>>>(A);
  k_adj_scal_gather<0><<<gb, 128, 0, s>>>(A);
  k_adj_scal_flux<1><<<gb, 128, 0, s>>>(A);
  k_adj_scal_gather<1><<<gb, 128, 0, s>>>(A);
  k_adj_scal_flux<2><<<gb, 128, 0, s>>>(A);
  k_adj_scal_gather<2><<<gb, 128, 0, s>>>(A);
  k_adj_conduction<<<gb, 128, 0, s>>>(A);
  k_adj_source<<<gb, 128, 0, s>>>(A);
  return 8;
}
int launch_adj_interface(const AdjArgs& A, cudaStream_t s) {
  const unsigned gb = g1(A.g.N, 128);
  k_adj_normal_flux<0><<<gb, 128, 0, s>>>(A);
  k_adj_normal_gather<0><<<gb, 128, 0, s>>>(A);
  k_adj_normal_flux<1><<<gb, 128, 0, s>>>(A);
  k_adj_normal_gather<1><<<gb, 128, 0, s>>>(A);
  k_adj_normal_flux<2><<<gb, 128, 0, s>>>(A);
  k_adj_normal_gather<2><<<gb, 128, 0, s>>>(A);
  k_adj_marangoni_flux<<<gb, 128, 0, s>>>(A);
  k_adj_marangoni_gather<<<gb, 128, 0, s>>>(A);
  return 8;
}
void launch_zero_wall_faces(const Geo& g, double* const* u, cudaStream_t s) {
  k_zero_wall_faces<<<g1(g.N, 256), 256, 0, s>>>(g, u[0], u[1], u[2]);
}
// y = a x + b y (y is not read when b == 0)
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby<<<g1(n, 256), 256, 0, s>>>(n, a, x, b, y);
}

}  // namespace fvm
