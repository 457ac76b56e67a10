// Kernels of one forward-Euler stage E(X) of the thermocapillary two-phase
// step and its SSP-RK3 combination Y = a*S^n + b*E(X):
//   k_smooth      smoothed phase fraction ([1,2,1]/4 tensor filter)
//   k_interface   curvature kappa = div n from face normals of the smoothed
//                 alpha, and the cell Marangoni vector |grad alpha|(I - n n) grad sigma
//                 (Sec. III, Eq. 4 with delta_s = |grad alpha|, Eq. 5 with sigma a field)
//   k_scalars     WENO5 transport of alpha (Eq. 1) and T, conduction with
//                 harmonic face conductivity, Gaussian surface heat flux,
//                 stage update and RK combination
//   k_momentum    u* on every MAC face: conservative WENO5 advection,
//                 variable-viscosity stress, balanced-force CSF (normal term of
//                 Eq. 4) and face-averaged Marangoni force, gravity
//   k_div_rhs     b = -(D u*)/dt in double, with block partial sums
//   k_beta        beta = 1/rho_f on the fine faces
//   k_correct     u = u* - dt beta grad p and the RK combination
//   k_dt_reduce   maxima for the time-step limits; k_dt_final combines them
//   k_diagnostics volume / mass sums, max |D u| dt, NaN flag
#include "fvm_device.cuh"

namespace fvm {

static inline unsigned grid1d(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__device__ __forceinline__ void decode(const Geo& g, long long c, int& i, int& j, int& k) {
  long long q = c / g.n[0];
  i = (int)(c - q * g.n[0]);
  k = (int)(q / g.n[1]);
  j = (int)(q - (long long)k * g.n[1]);
}

template <int D>
__device__ __forceinline__ void shift(int& i, int& j, int& k, int s) {
  if (D == 0) i += s;
  if (D == 1) j += s;
  if (D == 2) k += s;
}

// ---------------------------------------------------------------------------
// smoothing: one pass of the separable [1,2,1]/4 filter in all axes with
// more than one cell, as a 27-point tensor product
template <typename R>
__global__ void k_smooth(Geo g, const R* __restrict__ in, R* __restrict__ out) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  decode(g, c, i, j, k);
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = g.n[d] > 1 ? -1 : 0;
    hi[d] = g.n[d] > 1 ? 1 : 0;
  }
  R acc = 0;
  for (int dz = lo[2]; dz <= hi[2]; ++dz) {
    R wz = g.n[2] > 1 ? (dz == 0 ? R(0.5) : R(0.25)) : R(1);
    R accy = 0;
    for (int dy = lo[1]; dy <= hi[1]; ++dy) {
      R wy = g.n[1] > 1 ? (dy == 0 ? R(0.5) : R(0.25)) : R(1);
      R accx = 0;
      for (int dx = lo[0]; dx <= hi[0]; ++dx) {
        R wx = g.n[0] > 1 ? (dx == 0 ? R(0.5) : R(0.25)) : R(1);
        accx += wx * ld_even(in, g, i + dx, j + dy, k + dz);
      }
      accy += wy * accx;
    }
    acc += wz * accy;
  }
  out[c] = acc;
}

template <typename R>
void launch_smooth(const Geo& g, const R* in, R* out, cudaStream_t s) {
  k_smooth<R><<<grid1d(g.N, 256), 256, 0, s>>>(g, in, out);
}

// ---------------------------------------------------------------------------
// interface geometry
template <typename R>
__device__ __forceinline__ R at_s(const R* a, const Geo& g, int i, int j, int k) {
  return ld_even(a, g, i, j, k);
}

// n_D on the low D-face of cell (i,j,k) + s e_D, from the smoothed alpha
template <int D, typename R>
__device__ __forceinline__ R face_normal(const R* __restrict__ as, const Geo& g, int i, int j,
                                         int k, int s, R ih, R epsn) {
  int i1 = i, j1 = j, k1 = k, i0 = i, j0 = j, k0 = k;
  shift<D>(i1, j1, k1, s);
  shift<D>(i0, j0, k0, s - 1);
  R gd = (at_s(as, g, i1, j1, k1) - at_s(as, g, i0, j0, k0)) * ih;
  R sq = gd * gd;
  const R q = ih * R(0.25);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t == D) continue;
    int a1 = i1, b1 = j1, c1 = k1, a2 = i1, b2 = j1, c2 = k1;
    int a3 = i0, b3 = j0, c3 = k0, a4 = i0, b4 = j0, c4 = k0;
    if (t == 0) { a1 += 1; a2 -= 1; a3 += 1; a4 -= 1; }
    if (t == 1) { b1 += 1; b2 -= 1; b3 += 1; b4 -= 1; }
    if (t == 2) { c1 += 1; c2 -= 1; c3 += 1; c4 -= 1; }
    R gt = ((at_s(as, g, a1, b1, c1) - at_s(as, g, a2, b2, c2)) +
            (at_s(as, g, a3, b3, c3) - at_s(as, g, a4, b4, c4))) * q;
    sq += gt * gt;
  }
  return gd / (sqrt(sq) + epsn);
}

template <typename R>
__global__ void k_interface(Geo g, Phys ph, TBC tb, const R* __restrict__ alpha,
                            const R* __restrict__ as, const R* __restrict__ T,
                            R* __restrict__ kappa, R* __restrict__ M0, R* __restrict__ M1,
                            R* __restrict__ M2) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  decode(g, c, i, j, k);
  const R ih = R(1.0 / g.h);
  const R epsn = (R)ph.eps_n;
  R kap = 0;
  kap += (face_normal<0>(as, g, i, j, k, 1, ih, epsn) - face_normal<0>(as, g, i, j, k, 0, ih, epsn)) * ih;
  kap += (face_normal<1>(as, g, i, j, k, 1, ih, epsn) - face_normal<1>(as, g, i, j, k, 0, ih, epsn)) * ih;
  kap += (face_normal<2>(as, g, i, j, k, 1, ih, epsn) - face_normal<2>(as, g, i, j, k, 0, ih, epsn)) * ih;
  kappa[c] = kap;

  // Marangoni vector from central differences
  const R i2h = R(0.5) * ih;
  R gv[3], tv[3], sv[3];
  gv[0] = (ld_even(alpha, g, i + 1, j, k) - ld_even(alpha, g, i - 1, j, k)) * i2h;
  gv[1] = (ld_even(alpha, g, i, j + 1, k) - ld_even(alpha, g, i, j - 1, k)) * i2h;
  gv[2] = (ld_even(alpha, g, i, j, k + 1) - ld_even(alpha, g, i, j, k - 1)) * i2h;
  tv[0] = (ld_even(as, g, i + 1, j, k) - ld_even(as, g, i - 1, j, k)) * i2h;
  tv[1] = (ld_even(as, g, i, j + 1, k) - ld_even(as, g, i, j - 1, k)) * i2h;
  tv[2] = (ld_even(as, g, i, j, k + 1) - ld_even(as, g, i, j, k - 1)) * i2h;
  sv[0] = (sigma_of_T(ld_T(T, g, tb, i + 1, j, k), ph) - sigma_of_T(ld_T(T, g, tb, i - 1, j, k), ph)) * i2h;
  sv[1] = (sigma_of_T(ld_T(T, g, tb, i, j + 1, k), ph) - sigma_of_T(ld_T(T, g, tb, i, j - 1, k), ph)) * i2h;
  sv[2] = (sigma_of_T(ld_T(T, g, tb, i, j, k + 1), ph) - sigma_of_T(ld_T(T, g, tb, i, j, k - 1), ph)) * i2h;
  R gn = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
  R tn = sqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]) + epsn;
  R n0 = tv[0] / tn, n1 = tv[1] / tn, n2 = tv[2] / tn;
  R ns = n0 * sv[0] + n1 * sv[1] + n2 * sv[2];
  M0[c] = gn * (sv[0] - n0 * ns);
  M1[c] = gn * (sv[1] - n1 * ns);
  M2[c] = gn * (sv[2] - n2 * ns);
}

template <typename R>
void launch_interface(const Geo& g, const Phys& ph, const TBC& tb, const R* alpha,
                      const R* alpha_s, const R* T, R* kappa, R* M0, R* M1, R* M2,
                      cudaStream_t s) {
  k_interface<R><<<grid1d(g.N, 128), 128, 0, s>>>(g, ph, tb, alpha, alpha_s, T, kappa, M0, M1, M2);
}

// ---------------------------------------------------------------------------
// scalar transport (alpha, T) and stage update
template <int D, typename R>
__device__ __forceinline__ void scalar_axis(const Geo& g, const Phys& ph, const TBC& tb,
                                            const Fields<R>& X, int i, int j, int k, R ih,
                                            R& Ra, R& RT, R& Dif, R& gcomp) {
  R av[7], tv[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    int a = i, b = j, c = k;
    shift<D>(a, b, c, m - 3);
    av[m] = ld_even(X.alpha, g, a, b, c);
    tv[m] = ld_T(X.T, g, tb, a, b, c);
  }
  const R* U = X.u[D];
  R Fa[2], FT[2], Df[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    int a = i, b = j, c = k;
    shift<D>(a, b, c, s);
    R Uf = ld_vel<D>(U, g, a, b, c);
    Fa[s] = upwind_flux(Uf, av + s, (R)ph.eps_a);
    FT[s] = upwind_flux(Uf, tv + s, (R)ph.eps_T);
    R lL = mixp(av[2 + s], ph.lam), lR = mixp(av[3 + s], ph.lam);
    R lf = R(2) * lL * lR / (lL + lR);
    Df[s] = lf * (tv[3 + s] - tv[2 + s]) * ih;
  }
  Ra -= (Fa[1] - Fa[0]) * ih;
  RT -= (FT[1] - FT[0]) * ih;
  Dif += (Df[1] - Df[0]) * ih;
  gcomp = (av[4] - av[2]) * (R(0.5) * ih);
}

template <typename R>
__global__ void k_scalars(Geo g, Phys ph, TBC tb, Fields<R> X, Fields<R> Sn, Fields<R> Y,
                          const double* __restrict__ dtp, R a, R b, double xc) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  decode(g, c, i, j, k);
  const R ih = R(1.0 / g.h);
  const R dt = (R)(*dtp);
  R Ra = 0, RT = 0, Dif = 0, gx, gy, gz;
  scalar_axis<0>(g, ph, tb, X, i, j, k, ih, Ra, RT, Dif, gx);
  scalar_axis<1>(g, ph, tb, X, i, j, k, ih, Ra, RT, Dif, gy);
  scalar_axis<2>(g, ph, tb, X, i, j, k, ih, Ra, RT, Dif, gz);
  R al = X.alpha[c];
  R rcp = mixp(al, ph.rcp);
  RT += Dif / rcp;
  if (ph.q_power != 0.0) {
    double x = (i + 0.5) * g.h, y = (j + 0.5) * g.h;
    double dx = x - xc, dy = y - ph.q_y0;
    if (g.bc[0] == PER) dx = dx - ph.L[0] * floor(dx / ph.L[0] + 0.5);
    if (g.bc[1] == PER) dy = dy - ph.L[1] * floor(dy / ph.L[1] + 0.5);
    double r2 = ph.q_radius * ph.q_radius;
    double q = 2.0 * ph.q_power / (M_PI * r2) * exp(-2.0 * (dx * dx + dy * dy) / r2);
    R gn = sqrt(gx * gx + gy * gy + gz * gz);
    RT += (R)q * gn / rcp;
  }
  R Ea = al + dt * Ra;
  R ET = X.T[c] + dt * RT;
  Y.alpha[c] = a * Sn.alpha[c] + b * Ea;
  Y.T[c] = a * Sn.T[c] + b * ET;
}

template <typename R>
void launch_scalars(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, Fields<R> Sn,
                    Fields<R> Y, const double* dt, double a, double b, double xc, cudaStream_t s) {
  k_scalars<R><<<grid1d(g.N, 128), 128, 0, s>>>(g, ph, tb, X, Sn, Y, dt, (R)a, (R)b, xc);
}

// ---------------------------------------------------------------------------
// momentum predictor for component D on the low D-face of cell (i,j,k)
template <int D, typename R>
__device__ __forceinline__ R ldv(const Fields<R>& X, int comp, const Geo& g, int i, int j, int k) {
  (void)D;
  if (comp == 0) return ld_vel<0>(X.u[0], g, i, j, k);
  if (comp == 1) return ld_vel<1>(X.u[1], g, i, j, k);
  return ld_vel<2>(X.u[2], g, i, j, k);
}

template <int D, typename R>
__device__ __forceinline__ R mu_at(const Fields<R>& X, const Geo& g, const Phys& ph, int i, int j,
                                   int k) {
  return mixp(ld_even(X.alpha, g, i, j, k), ph.mu);
}

template <int D, int T_, typename R>
__device__ __forceinline__ void tangential(const Fields<R>& X, const Geo& g, const Phys& ph, int i,
                                           int j, int k, R ih, R& A, R& V) {
  const R* ud = X.u[D];
  const R* ut = X.u[T_];
  R vals[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    int a = i, b = j, c = k;
    shift<T_>(a, b, c, m - 3);
    vals[m] = ld_vel<D>(ud, g, a, b, c);
  }
  R Ge[2], te[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    int a = i, b = j, c = k;           // f + s e_t
    shift<T_>(a, b, c, s);
    int a2 = a, b2 = b, c2 = c;        // f + s e_t - e_d
    shift<D>(a2, b2, c2, -1);
    R ut_hi = ld_vel<T_>(ut, g, a, b, c);
    R ut_lo = ld_vel<T_>(ut, g, a2, b2, c2);
    R Ue = R(0.5) * (ut_lo + ut_hi);
    Ge[s] = upwind_flux(Ue, vals + s, (R)ph.eps_u);
    int a3 = i, b3 = j, c3 = k;        // f + (s-1) e_t
    shift<T_>(a3, b3, c3, s - 1);
    int a4 = a3, b4 = b3, c4 = c3;     // f + (s-1) e_t - e_d
    shift<D>(a4, b4, c4, -1);
    R mue = R(0.25) * (mu_at<D>(X, g, ph, a, b, c) + mu_at<D>(X, g, ph, a2, b2, c2) +
                       mu_at<D>(X, g, ph, a3, b3, c3) + mu_at<D>(X, g, ph, a4, b4, c4));
    R dud_dt = (vals[3 + s] - vals[2 + s]) * ih;
    R dut_dd = (ut_hi - ut_lo) * ih;
    te[s] = mue * (dud_dt + dut_dd);
  }
  A -= (Ge[1] - Ge[0]) * ih;
  V += (te[1] - te[0]) * ih;
}

template <int D, typename R>
__device__ __forceinline__ R momentum_face(const Fields<R>& X, const Geo& g, const Phys& ph,
                                           const TBC& tb, const R* __restrict__ kappa,
                                           const R* __restrict__ MD, int i, int j, int k, R dt) {
  const R ih = R(1.0 / g.h);
  const R* ud = X.u[D];
  R nv[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    int a = i, b = j, c = k;
    shift<D>(a, b, c, m - 3);
    nv[m] = ld_vel<D>(ud, g, a, b, c);
  }
  // normal advection at the cell centres below (s=-1) and above (s=0) the face
  R Fc[2], tau[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int s = q - 1;
    R Uc = R(0.5) * (nv[3 + s] + nv[4 + s]);
    Fc[q] = upwind_flux(Uc, nv + 1 + s, (R)ph.eps_u);
    int a = i, b = j, c = k;
    shift<D>(a, b, c, s);
    R muc = mu_at<D>(X, g, ph, a, b, c);
    tau[q] = R(2) * muc * (nv[4 + s] - nv[3 + s]) * ih;
  }
  R A = R(0) - (Fc[1] - Fc[0]) * ih;
  R V = R(0) + (tau[1] - tau[0]) * ih;
  if (D == 0) {
    tangential<0, 1>(X, g, ph, i, j, k, ih, A, V);
    tangential<0, 2>(X, g, ph, i, j, k, ih, A, V);
  } else if (D == 1) {
    tangential<1, 0>(X, g, ph, i, j, k, ih, A, V);
    tangential<1, 2>(X, g, ph, i, j, k, ih, A, V);
  } else {
    tangential<2, 0>(X, g, ph, i, j, k, ih, A, V);
    tangential<2, 1>(X, g, ph, i, j, k, ih, A, V);
  }
  // forces on the face between cell L = c - e_D and R = c
  int a = i, b = j, c = k;
  shift<D>(a, b, c, -1);
  R alL = ld_even(X.alpha, g, a, b, c), alR = ld_even(X.alpha, g, i, j, k);
  R rho_f = R(0.5) * (mixp(alL, ph.rho) + mixp(alR, ph.rho));
  R sig_f = R(0.5) * (sigma_of_T(ld_T(X.T, g, tb, a, b, c), ph) + sigma_of_T(ld_T(X.T, g, tb, i, j, k), ph));
  R kap_f = R(0.5) * (ld_even(kappa, g, a, b, c) + ld_even(kappa, g, i, j, k));
  R jump = (alR - alL) * ih;
  R fn = -sig_f * kap_f * jump;
  R fM = R(0.5) * (ld_even(MD, g, a, b, c) + ld_even(MD, g, i, j, k));
  return nv[3] + dt * (A + (V + fn + fM) / rho_f + (R)ph.g[D]);
}

template <typename R>
__global__ void k_momentum(Geo g, Phys ph, TBC tb, Fields<R> X, const R* __restrict__ kappa,
                           const R* __restrict__ M0, const R* __restrict__ M1,
                           const R* __restrict__ M2, R* __restrict__ us0, R* __restrict__ us1,
                           R* __restrict__ us2, const double* __restrict__ dtp) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  decode(g, c, i, j, k);
  const R dt = (R)(*dtp);
  us0[c] = (g.bc[0] == WALL && i == 0) ? R(0) : momentum_face<0>(X, g, ph, tb, kappa, M0, i, j, k, dt);
  us1[c] = (g.bc[1] == WALL && j == 0) ? R(0) : momentum_face<1>(X, g, ph, tb, kappa, M1, i, j, k, dt);
  us2[c] = (g.bc[2] == WALL && k == 0) ? R(0) : momentum_face<2>(X, g, ph, tb, kappa, M2, i, j, k, dt);
}

template <typename R>
void launch_momentum(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, const R* kappa,
                     const R* M0, const R* M1, const R* M2, R* us0, R* us1, R* us2,
                     const double* dt, cudaStream_t s) {
  k_momentum<R><<<grid1d(g.N, 128), 128, 0, s>>>(g, ph, tb, X, kappa, M0, M1, M2, us0, us1, us2, dt);
}

// ---------------------------------------------------------------------------
// block reduction helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double sh[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;   // valid in thread 0
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// projection right-hand side b = -(D u*)/dt in double; grid-stride with a
// fixed number of blocks so that the partial sums have a fixed order
template <typename R>
__global__ void k_div_rhs(Geo g, const R* __restrict__ u0, const R* __restrict__ u1,
                          const R* __restrict__ u2, const double* __restrict__ dtp,
                          double* __restrict__ b, double* __restrict__ partial) {
  const double ih = 1.0 / g.h;
  const double dt = *dtp;
  double acc = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.N;
       c += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    double dv = 0.0;
    dv += ((double)ld_vel<0>(u0, g, i + 1, j, k) - (double)ld_vel<0>(u0, g, i, j, k)) * ih;
    dv += ((double)ld_vel<1>(u1, g, i, j + 1, k) - (double)ld_vel<1>(u1, g, i, j, k)) * ih;
    dv += ((double)ld_vel<2>(u2, g, i, j, k + 1) - (double)ld_vel<2>(u2, g, i, j, k)) * ih;
    double v = -dv / dt;
    b[c] = v;
    acc += v;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename R>
void launch_div_rhs(const Geo& g, R* const* us, const double* dt, double* b, double* partial,
                    cudaStream_t s) {
  k_div_rhs<R><<<kRedBlocks, 256, 0, s>>>(g, us[0], us[1], us[2], dt, b, partial);
}

// ---------------------------------------------------------------------------
// beta = 1 / rho_f on the low faces, rho_f = (rho_L + rho_R)/2; 0 on walls
template <typename R, typename B>
__global__ void k_beta(Geo g, Phys ph, const R* __restrict__ alpha, B* __restrict__ b0,
                       B* __restrict__ b1, B* __restrict__ b2) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  decode(g, c, i, j, k);
  B rc = (B)mixp(alpha[c], ph.rho);
  B rx = (B)mixp(ld_even(alpha, g, i - 1, j, k), ph.rho);
  B ry = (B)mixp(ld_even(alpha, g, i, j - 1, k), ph.rho);
  B rz = (B)mixp(ld_even(alpha, g, i, j, k - 1), ph.rho);
  b0[c] = (g.bc[0] == WALL && i == 0) ? B(0) : B(1) / (B(0.5) * (rx + rc));
  b1[c] = (g.bc[1] == WALL && j == 0) ? B(0) : B(1) / (B(0.5) * (ry + rc));
  b2[c] = (g.bc[2] == WALL && k == 0) ? B(0) : B(1) / (B(0.5) * (rz + rc));
}

template <typename R, typename B>
void launch_beta(const Geo& g, const Phys& ph, const R* alpha, B* b0, B* b1, B* b2,
                 cudaStream_t s) {
  k_beta<R, B><<<grid1d(g.N, 256), 256, 0, s>>>(g, ph, alpha, b0, b1, b2);
}

// ---------------------------------------------------------------------------
// velocity correction and RK combination
template <typename R, typename B>
__global__ void k_correct(Geo g, Fields<R> Sn, Fields<R> Y, const R* __restrict__ us0,
                          const R* __restrict__ us1, const R* __restrict__ us2,
                          const double* __restrict__ p, const B* __restrict__ b0,
                          const B* __restrict__ b1, const B* __restrict__ b2,
                          const double* __restrict__ dtp, double a, double bb) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  decode(g, c, i, j, k);
  const double dt = *dtp;
  const double ih = 1.0 / g.h;
  const double pc = p[c];
  const R* us[3] = {us0, us1, us2};
  const B* be[3] = {b0, b1, b2};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int idx[3] = {i, j, k};
    bool wall_face = (g.bc[d] == WALL && idx[d] == 0);
    int m[3] = {i, j, k};
    m[d] = wrapi(m[d] - 1, g.n[d]);
    double pl = p[lin(g, m[0], m[1], m[2])];
    double ucorr = (double)us[d][c] - dt * (double)be[d][c] * (pc - pl) * ih;
    double un = (double)Sn.u[d][c];
    double out = wall_face ? 0.0 : a * un + bb * ucorr;
    Y.u[d][c] = (R)out;
  }
}

template <typename R, typename B>
void launch_correct(const Geo& g, Fields<R> Sn, Fields<R> Y, R* const* us, const double* p,
                    B* const* beta, const double* dt, double a, double b, cudaStream_t s) {
  k_correct<R, B><<<grid1d(g.N, 256), 256, 0, s>>>(g, Sn, Y, us[0], us[1], us[2], p, beta[0],
                                                   beta[1], beta[2], dt, a, b);
}

// ---------------------------------------------------------------------------
// time-step limits: maxima of |u|, |v|, |w|, |sigma|, mu/rho, lambda/(rho cp)
// as IEEE bit patterns (non-negative doubles order like unsigned integers)
template <typename R>
__global__ void k_dt_reduce(Geo g, Phys ph, Fields<R> X, unsigned long long* __restrict__ maxbits,
                            int* __restrict__ nanflag) {
  unsigned long long m[6] = {0, 0, 0, 0, 0, 0};
  int bad = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.N;
       c += (long long)gridDim.x * blockDim.x) {
    double v[6];
    v[0] = fabs((double)X.u[0][c]);
    v[1] = fabs((double)X.u[1][c]);
    v[2] = fabs((double)X.u[2][c]);
    R al = X.alpha[c];
    R T = X.T[c];
    v[3] = fabs((double)sigma_of_T(T, ph));
    v[4] = (double)(mixp(al, ph.mu) / mixp(al, ph.rho));
    v[5] = (double)(mixp(al, ph.lam) / mixp(al, ph.rcp));
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (!(v[q] <= 1.7976931348623157e308)) bad = 1;
      unsigned long long bits = (unsigned long long)__double_as_longlong(v[q]);
      m[q] = bits > m[q] ? bits : m[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    unsigned long long w = warp_max_u64(m[q]);
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits + q, w);
  }
  if (bad) atomicOr(nanflag, 1);
}

template <typename R>
void launch_dt_reduce(const Geo& g, const Phys& ph, Fields<R> X, unsigned long long* maxbits,
                      int* nanflag, cudaStream_t s) {
  cudaMemsetAsync(maxbits, 0, 6 * sizeof(unsigned long long), s);
  cudaMemsetAsync(nanflag, 0, sizeof(int), s);
  k_dt_reduce<R><<<kRedBlocks, 256, 0, s>>>(g, ph, X, maxbits, nanflag);
}

__global__ void k_dt_final(double h, double rho_sum, double cfl, double c_cap, double c_visc,
                           double c_therm, double dt_max, const unsigned long long* maxbits,
                           double* dt, int* limiter) {
  double mx[6];
  for (int q = 0; q < 6; ++q) mx[q] = __longlong_as_double((long long)maxbits[q]);
  double umax = ((0.0 + mx[0]) + mx[1]) + mx[2];
  double lim[5];
  for (int q = 0; q < 5; ++q) lim[q] = __longlong_as_double(0x7ff0000000000000LL);
  if (umax > 0.0) lim[0] = cfl * h / umax;
  if (mx[3] > 0.0) lim[1] = c_cap * sqrt(rho_sum * (h * h * h) / (4.0 * M_PI * mx[3]));
  if (mx[4] > 0.0) lim[2] = c_visc * h * h / mx[4];
  if (mx[5] > 0.0) lim[3] = c_therm * h * h / mx[5];
  lim[4] = dt_max;
  int kk = 0;
  for (int q = 1; q < 5; ++q)
    if (lim[q] < lim[kk]) kk = q;
  *dt = lim[kk];
  *limiter = kk;
}

void launch_dt_final(const Geo& g, const Phys& ph, double cfl, double c_cap, double c_visc,
                     double c_therm, double dt_max, const unsigned long long* maxbits,
                     double* dt, int* limiter, cudaStream_t s) {
  k_dt_final<<<1, 1, 0, s>>>(g.h, ph.rho[0] + ph.rho[1], cfl, c_cap, c_visc, c_therm, dt_max,
                             maxbits, dt, limiter);
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

void launch_set_scalar(double* dst, double v, cudaStream_t s) { k_set_scalar<<<1, 1, 0, s>>>(dst, v); }

// ---------------------------------------------------------------------------
// diagnostics: partial sums of alpha and rho(alpha) (two slots per block),
// max |D u| as bits in maxbits[0], NaN flag
template <typename R>
__global__ void k_diagnostics(Geo g, Phys ph, Fields<R> X, const double* __restrict__ p,
                              double* __restrict__ partial, unsigned long long* __restrict__ maxbits,
                              int* __restrict__ nanflag) {
  const double ih = 1.0 / g.h;
  double sa = 0.0, sm = 0.0;
  unsigned long long mdiv = 0;
  int bad = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.N;
       c += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    R al = X.alpha[c];
    sa += (double)al;
    sm += (double)mixp(al, ph.rho);
    double dv = 0.0;
    dv += ((double)ld_vel<0>(X.u[0], g, i + 1, j, k) - (double)ld_vel<0>(X.u[0], g, i, j, k)) * ih;
    dv += ((double)ld_vel<1>(X.u[1], g, i, j + 1, k) - (double)ld_vel<1>(X.u[1], g, i, j, k)) * ih;
    dv += ((double)ld_vel<2>(X.u[2], g, i, j, k + 1) - (double)ld_vel<2>(X.u[2], g, i, j, k)) * ih;
    double adv = fabs(dv);
    unsigned long long bits = (unsigned long long)__double_as_longlong(adv);
    mdiv = bits > mdiv ? bits : mdiv;
    double chk = (double)X.u[0][c] + (double)X.u[1][c] + (double)X.u[2][c] + (double)al +
                 (double)X.T[c] + p[c];
    if (!(fabs(chk) <= 1.7976931348623157e308) || !(adv <= 1.7976931348623157e308)) bad = 1;
  }
  double s1 = block_sum(sa);
  __syncthreads();
  double s2 = block_sum(sm);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s1;
    partial[kRedBlocks + blockIdx.x] = s2;
  }
  unsigned long long w = warp_max_u64(mdiv);
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, w);
  if (bad) atomicOr(nanflag, 1);
}

template <typename R>
void launch_diagnostics(const Geo& g, const Phys& ph, Fields<R> X, const double* p,
                        const double* dt, double* partial, unsigned long long* maxbits,
                        int* nanflag, cudaStream_t s) {
  (void)dt;
  cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(nanflag, 0, sizeof(int), s);
  k_diagnostics<R><<<kRedBlocks, 256, 0, s>>>(g, ph, X, p, partial, maxbits, nanflag);
}

// ---------------------------------------------------------------------------
#define FVM_INST(R)                                                                              \
  template void launch_smooth<R>(const Geo&, const R*, R*, cudaStream_t);                        \
  template void launch_interface<R>(const Geo&, const Phys&, const TBC&, const R*, const R*,     \
                                    const R*, R*, R*, R*, R*, cudaStream_t);                     \
  template void launch_scalars<R>(const Geo&, const Phys&, const TBC&, Fields<R>, Fields<R>,     \
                                  Fields<R>, const double*, double, double, double,              \
                                  cudaStream_t);                                                 \
  template void launch_momentum<R>(const Geo&, const Phys&, const TBC&, Fields<R>, const R*,     \
                                   const R*, const R*, const R*, R*, R*, R*, const double*,      \
                                   cudaStream_t);                                                \
  template void launch_div_rhs<R>(const Geo&, R* const*, const double*, double*, double*,        \
                                  cudaStream_t);                                                 \
  template void launch_dt_reduce<R>(const Geo&, const Phys&, Fields<R>, unsigned long long*,     \
                                    int*, cudaStream_t);                                         \
  template void launch_diagnostics<R>(const Geo&, const Phys&, Fields<R>, const double*,         \
                                      const double*, double*, unsigned long long*, int*,         \
                                      cudaStream_t);

FVM_INST(double)
FVM_INST(float)

#define FVM_INST2(R, B)                                                                         \
  template void launch_beta<R, B>(const Geo&, const Phys&, const R*, B*, B*, B*, cudaStream_t); \
  template void launch_correct<R, B>(const Geo&, Fields<R>, Fields<R>, R* const*, const double*, \
                                     B* const*, const double*, double, double, cudaStream_t);

FVM_INST2(double, double)
FVM_INST2(double, float)
FVM_INST2(float, double)
FVM_INST2(float, float)

}  // namespace fvm
