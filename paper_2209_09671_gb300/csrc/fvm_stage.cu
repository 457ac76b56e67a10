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
//
// Layout of the work: a CTA owns a kBX x kBY x kBZ tile of cells on a 3D grid.
// Every face flux (and every edge flux of the momentum control volumes) is
// evaluated once, by the thread owning the face, and exchanged through shared
// memory; the threads on the high (or low) side of the tile evaluate the one
// extra layer the divergence needs.  Tiles whose stencil reach (3 cells)
// stays inside the domain take loads without boundary handling; the others
// go through the wrap/mirror loaders.
#include "fvm_device.cuh"

namespace fvm {

static inline unsigned grid1d(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }
static inline dim3 tile_grid(const Geo& g) {
  return dim3((unsigned)((g.n[0] + kBX - 1) / kBX), (unsigned)((g.n[1] + kBY - 1) / kBY),
              (unsigned)((g.n[2] + kBZ - 1) / kBZ));
}

__device__ __forceinline__ void decode(const Geo& g, long long c, int& i, int& j, int& k) {
  int cc = (int)c;
  int q = cc / g.n[0];
  i = cc - q * g.n[0];
  k = q / g.n[1];
  j = q - k * g.n[1];
}

template <int D>
__device__ __forceinline__ void shift(int& i, int& j, int& k, int s) {
  if (D == 0) i += s;
  if (D == 1) j += s;
  if (D == 2) k += s;
}

// loads with (IN = false) or without (IN = true) boundary handling
template <bool IN>
struct Ld {
  template <typename R>
  static __device__ __forceinline__ R even(const R* __restrict__ a, const Geo& g, int i, int j,
                                           int k) {
    if (IN) return __ldg(a + ((k * (int)g.n[1] + j) * (int)g.n[0] + i));
    return ld_even(a, g, i, j, k);
  }
  template <int C, typename R>
  static __device__ __forceinline__ R vel(const R* __restrict__ a, const Geo& g, int i, int j,
                                          int k) {
    if (IN) return __ldg(a + ((k * (int)g.n[1] + j) * (int)g.n[0] + i));
    return ld_vel<C>(a, g, i, j, k);
  }
  template <typename R>
  static __device__ __forceinline__ R T(const R* __restrict__ a, const Geo& g, const TBC& tb,
                                        int i, int j, int k) {
    if (IN) return __ldg(a + ((k * (int)g.n[1] + j) * (int)g.n[0] + i));
    return ld_T(a, g, tb, i, j, k);
  }
};

// the tile and its stencil reach H stay inside the domain on every axis
__device__ __forceinline__ bool tile_interior(const Geo& g, int H) {
  const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * kBZ;
  return x0 - H >= 0 && x0 + kBX - 1 + H < g.n[0] && y0 - H >= 0 &&
         y0 + kBY - 1 + H < g.n[1] && z0 - H >= 0 && z0 + kBZ - 1 + H < g.n[2];
}

// ---------------------------------------------------------------------------
// smoothing: one pass of the separable [1,2,1]/4 filter in all axes with
// more than one cell, as a 27-point tensor product
template <bool IN, typename R>
__device__ __forceinline__ void smooth_body(const Geo& g, const R* __restrict__ in,
                                            R* __restrict__ out, int i, int j, int k) {
  const int lo0 = g.n[0] > 1 ? -1 : 0, lo1 = g.n[1] > 1 ? -1 : 0, lo2 = g.n[2] > 1 ? -1 : 0;
  R acc = 0;
  for (int dz = lo2; dz <= -lo2; ++dz) {
    R wz = lo2 ? (dz == 0 ? R(0.5) : R(0.25)) : R(1);
    R accy = 0;
    for (int dy = lo1; dy <= -lo1; ++dy) {
      R wy = lo1 ? (dy == 0 ? R(0.5) : R(0.25)) : R(1);
      R accx = 0;
      for (int dx = lo0; dx <= -lo0; ++dx) {
        R wx = lo0 ? (dx == 0 ? R(0.5) : R(0.25)) : R(1);
        accx += wx * Ld<IN>::even(in, g, i + dx, j + dy, k + dz);
      }
      accy += wy * accx;
    }
    acc += wz * accy;
  }
  out[(k * g.n[1] + j) * g.n[0] + i] = acc;
}

template <typename R>
__global__ void __launch_bounds__(kBX * kBY * kBZ) k_smooth(Geo g, const R* __restrict__ in,
                                                            R* __restrict__ out) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y,
            k = blockIdx.z * kBZ + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
  if (tile_interior(g, 1)) smooth_body<true>(g, in, out, i, j, k);
  else smooth_body<false>(g, in, out, i, j, k);
}

template <typename R>
void launch_smooth(const Geo& g, const R* in, R* out, cudaStream_t s) {
  k_smooth<R><<<tile_grid(g), dim3(kBX, kBY, kBZ), 0, s>>>(g, in, out);
}

// ---------------------------------------------------------------------------
// shared-memory tiles: a field staged with a halo of H cells around the CTA's
// tile; local coordinates run from -H to kB*+H-1
constexpr int kThreads = kBX * kBY * kBZ;

template <int H>
struct Tile {
  static constexpr int SX = kBX + 2 * H, SY = kBY + 2 * H, SZ = kBZ + 2 * H;
  static constexpr int N = SX * SY * SZ;
  static __device__ __forceinline__ int at(int lx, int ly, int lz) {
    return ((lz + H) * SY + (ly + H)) * SX + (lx + H);
  }
};

__device__ __forceinline__ int flat_tid() {
  return threadIdx.x + kBX * (threadIdx.y + kBY * threadIdx.z);
}

enum { F_EVEN = 0, F_VEL = 1, F_TEMP = 2 };

// stage one field into s: the boundary rules of the loaders are applied once
// per staged point; points more than H cells outside the domain (ragged
// tiles) are never read and hold 0.  Threads walk rows of the tile: x from
// threadIdx.x, one row (y, z) per (threadIdx.y, threadIdx.z) step.
template <int H, int KIND, int C, typename R>
__device__ __forceinline__ void stage(R* __restrict__ s, const R* __restrict__ a, const Geo& g,
                                      const TBC& tb) {
  constexpr int SX = Tile<H>::SX, SY = Tile<H>::SY, SZ = Tile<H>::SZ;
  const bool in = tile_interior(g, H);
  const int x0 = blockIdx.x * kBX - H, y0 = blockIdx.y * kBY - H, z0 = blockIdx.z * kBZ - H;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int tx = threadIdx.x;
  for (int row = threadIdx.y + kBY * threadIdx.z; row < SY * SZ; row += kBY * kBZ) {
    const int ly = row % SY, lz = row / SY;
    const int j = y0 + ly, k = z0 + lz;
    R* __restrict__ srow = s + row * SX;
    if (in) {
      const R* __restrict__ arow = a + ((k * ny + j) * nx + x0);
#pragma unroll
      for (int lx = tx; lx < SX; lx += kBX) srow[lx] = __ldg(arow + lx);
    } else {
      const bool rowout = j < -H || j > ny - 1 + H || k < -H || k > nz - 1 + H;
      for (int lx = tx; lx < SX; lx += kBX) {
        const int i = x0 + lx;
        R v;
        if (rowout || i < -H || i > nx - 1 + H) v = R(0);
        else if (KIND == F_EVEN) v = ld_even(a, g, i, j, k);
        else if (KIND == F_VEL) v = ld_vel<C>(a, g, i, j, k);
        else v = ld_T(a, g, tb, i, j, k);
        srow[lx] = v;
      }
    }
  }
}

// single loads for the few values a kernel does not stage: direct in an
// interior tile, through the boundary loaders otherwise
template <typename R>
__device__ __forceinline__ R g_even(const R* __restrict__ a, const Geo& g, bool in, int i, int j,
                                    int k) {
  return in ? __ldg(a + ((k * g.n[1] + j) * g.n[0] + i)) : ld_even(a, g, i, j, k);
}
template <int C, typename R>
__device__ __forceinline__ R g_vel(const R* __restrict__ a, const Geo& g, bool in, int i, int j,
                                   int k) {
  return in ? __ldg(a + ((k * g.n[1] + j) * g.n[0] + i)) : ld_vel<C>(a, g, i, j, k);
}
template <typename R>
__device__ __forceinline__ R g_T(const R* __restrict__ a, const Geo& g, const TBC& tb, bool in,
                                 int i, int j, int k) {
  return in ? __ldg(a + ((k * g.n[1] + j) * g.n[0] + i)) : ld_T(a, g, tb, i, j, k);
}

template <int A>
__device__ __forceinline__ int tsel(int tx, int ty, int tz) {
  return A == 0 ? tx : (A == 1 ? ty : tz);
}

// ---------------------------------------------------------------------------
// interface geometry: two smoothing passes, face normals, curvature and the
// Marangoni vector in one kernel (the smoothed alpha never leaves the SM)
template <typename R>
struct IfaceShared {
  R a[Tile<3>::N];          // alpha
  R s1[Tile<2>::N];         // after the first [1,2,1]/4 pass
  R s2[Tile<1>::N];         // smoothed alpha
  R T[Tile<1>::N];
  R c[Tile<1>::N];          // concentration (when transported)
  R nx[kBZ][kBY][kBX + 1];  // face normals
  R ny[kBZ][kBY + 1][kBX];
  R nz[kBZ + 1][kBY][kBX];
};

// one [1,2,1]/4 tensor pass from a tile of halo HI onto the tile of halo HO
template <int HI, int HO, typename R>
__device__ __forceinline__ void smooth_pass(const Geo& g, const R* __restrict__ in,
                                            R* __restrict__ out) {
  const bool sx = g.n[0] > 1, sy = g.n[1] > 1, sz = g.n[2] > 1;
  constexpr int SX = Tile<HO>::SX, SY = Tile<HO>::SY, SZ = Tile<HO>::SZ;
  for (int row = threadIdx.y + kBY * threadIdx.z; row < SY * SZ; row += kBY * kBZ) {
    const int ly = row % SY - HO, lz = row / SY - HO;
    for (int ex = threadIdx.x; ex < SX; ex += kBX) {
      const int lx = ex - HO;
      R acc = 0;
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        if (!sz && dz != 0) continue;
        const R wz = sz ? (dz == 0 ? R(0.5) : R(0.25)) : R(1);
        R accy = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          if (!sy && dy != 0) continue;
          const R wy = sy ? (dy == 0 ? R(0.5) : R(0.25)) : R(1);
          R accx = 0;
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            if (!sx && dx != 0) continue;
            const R wx = sx ? (dx == 0 ? R(0.5) : R(0.25)) : R(1);
            accx += wx * in[Tile<HI>::at(lx + dx, ly + dy, lz + dz)];
          }
          accy += wy * accx;
        }
        acc += wz * accy;
      }
      out[row * SX + ex] = acc;
    }
  }
}

template <int HI, int HO, typename R>
__device__ __forceinline__ void copy_tile(const R* __restrict__ in, R* __restrict__ out) {
  constexpr int SX = Tile<HO>::SX, SY = Tile<HO>::SY, SZ = Tile<HO>::SZ;
  for (int row = threadIdx.y + kBY * threadIdx.z; row < SY * SZ; row += kBY * kBZ) {
    const int ly = row % SY - HO, lz = row / SY - HO;
    for (int ex = threadIdx.x; ex < SX; ex += kBX)
      out[row * SX + ex] = in[Tile<HI>::at(ex - HO, ly, lz)];
  }
}

// n_D on the low D-face of local cell (lx,ly,lz), from the smoothed alpha:
// grad / (|grad| + eps_n) with the normal derivative across the face and each
// tangential derivative the mean of the two cells' central differences
template <int D, typename R>
__device__ __forceinline__ R face_normal(const R* __restrict__ s2, int lx, int ly, int lz, R ih,
                                         R epsn) {
  const int dx = D == 0, dy = D == 1, dz = D == 2;
  R gd = (s2[Tile<1>::at(lx, ly, lz)] - s2[Tile<1>::at(lx - dx, ly - dy, lz - dz)]) * ih;
  R sq = gd * gd;
  const R q = ih * R(0.25);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t == D) continue;
    const int ox = t == 0, oy = t == 1, oz = t == 2;
    R gt = ((s2[Tile<1>::at(lx + ox, ly + oy, lz + oz)] - s2[Tile<1>::at(lx - ox, ly - oy, lz - oz)]) +
            (s2[Tile<1>::at(lx - dx + ox, ly - dy + oy, lz - dz + oz)] -
             s2[Tile<1>::at(lx - dx - ox, ly - dy - oy, lz - dz - oz)])) * q;
    sq += gt * gt;
  }
  return gd / (sqrt(sq) + epsn);
}

template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 4 : 1)
    k_interface(Geo g, PhysR<R> ph, TBC tb, int passes, const R* __restrict__ alpha,
                const R* __restrict__ T, const R* __restrict__ conc, R* __restrict__ kappa,
                R* __restrict__ M0, R* __restrict__ M1, R* __restrict__ M2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  IfaceShared<R>& S = *reinterpret_cast<IfaceShared<R>*>(smem_raw);
  stage<3, F_EVEN, 0>(S.a, alpha, g, tb);
  stage<1, F_TEMP, 0>(S.T, T, g, tb);
  if (conc) stage<1, F_EVEN, 0>(S.c, conc, g, tb);
  __syncthreads();
  if (passes >= 1) {
    smooth_pass<3, 2>(g, S.a, S.s1);
    __syncthreads();
    if (passes >= 2) smooth_pass<2, 1>(g, S.s1, S.s2);
    else copy_tile<2, 1>(S.s1, S.s2);
  } else {
    copy_tile<3, 1>(S.a, S.s2);
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int i = blockIdx.x * kBX + tx, j = blockIdx.y * kBY + ty, k = blockIdx.z * kBZ + tz;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const R ih = ph.ih;
  const R epsn = ph.eps_n;
  if (i <= nx && j < ny && k < nz) {
    S.nx[tz][ty][tx] = face_normal<0>(S.s2, tx, ty, tz, ih, epsn);
    if (tx == kBX - 1 && i + 1 <= nx) S.nx[tz][ty][tx + 1] = face_normal<0>(S.s2, tx + 1, ty, tz, ih, epsn);
  }
  if (i < nx && j <= ny && k < nz) {
    S.ny[tz][ty][tx] = face_normal<1>(S.s2, tx, ty, tz, ih, epsn);
    if (ty == kBY - 1 && j + 1 <= ny) S.ny[tz][ty + 1][tx] = face_normal<1>(S.s2, tx, ty + 1, tz, ih, epsn);
  }
  if (i < nx && j < ny && k <= nz) {
    S.nz[tz][ty][tx] = face_normal<2>(S.s2, tx, ty, tz, ih, epsn);
    if (tz == kBZ - 1 && k + 1 <= nz) S.nz[tz + 1][ty][tx] = face_normal<2>(S.s2, tx, ty, tz + 1, ih, epsn);
  }
  __syncthreads();
  if (i >= nx || j >= ny || k >= nz) return;
  const int c = (k * ny + j) * nx + i;
  R kap = 0;
  kap += (S.nx[tz][ty][tx + 1] - S.nx[tz][ty][tx]) * ih;
  kap += (S.ny[tz][ty + 1][tx] - S.ny[tz][ty][tx]) * ih;
  kap += (S.nz[tz + 1][ty][tx] - S.nz[tz][ty][tx]) * ih;
  kappa[c] = kap;
  // Marangoni vector from central differences of alpha, smoothed alpha, sigma(T)
  const R i2h = R(0.5) * ih;
  R gv[3], tv[3], sv[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int ox = d == 0, oy = d == 1, oz = d == 2;
    gv[d] = (S.a[Tile<3>::at(tx + ox, ty + oy, tz + oz)] - S.a[Tile<3>::at(tx - ox, ty - oy, tz - oz)]) * i2h;
    tv[d] = (S.s2[Tile<1>::at(tx + ox, ty + oy, tz + oz)] - S.s2[Tile<1>::at(tx - ox, ty - oy, tz - oz)]) * i2h;
    const R Tp = S.T[Tile<1>::at(tx + ox, ty + oy, tz + oz)];
    const R Tm = S.T[Tile<1>::at(tx - ox, ty - oy, tz - oz)];
    // central difference of the sigma field (Eq. 5 as a cell field).  In
    // float it is taken as dsigma/dT (T+ - T-), the same number for the
    // linear sigma(T): the difference of two neighbouring temperatures is
    // exact, while sigma0 + dsigma/dT (T - T0) rounded to float at
    // sigma ~ 1.9 keeps only ~4 digits of a variation of ~1e-3
    if (conc) {
      // sigma(c, T) of Eq. 5: in float the exact neighbour differences
      // again, in double the difference of the two cells' sigma values
      const R cp = S.c[Tile<1>::at(tx + ox, ty + oy, tz + oz)];
      const R cm = S.c[Tile<1>::at(tx - ox, ty - oy, tz - oz)];
      if (sizeof(R) == 4) sv[d] = (ph.dsdT * (Tp - Tm) + ph.dsdc * (cp - cm)) * i2h;
      else sv[d] = (sigma_rc(Tp, cp, ph) - sigma_rc(Tm, cm, ph)) * i2h;
    } else if (sizeof(R) == 4) {
      sv[d] = ph.dsdT * (Tp - Tm) * i2h;
    } else {
      sv[d] = (sigma_r(Tp, ph) - sigma_r(Tm, ph)) * i2h;
    }
  }
  R gn = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
  R tn = sqrt(tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2]) + epsn;
  R n0 = tv[0] / tn, n1 = tv[1] / tn, n2 = tv[2] / tn;
  R ns = n0 * sv[0] + n1 * sv[1] + n2 * sv[2];
  M0[c] = gn * (sv[0] - n0 * ns);
  M1[c] = gn * (sv[1] - n1 * ns);
  M2[c] = gn * (sv[2] - n2 * ns);
}

template <typename R>
void launch_interface(const Geo& g, const Phys& ph, const TBC& tb, int passes, const R* alpha,
                      const R* T, const R* c, R* kappa, R* M0, R* M1, R* M2, cudaStream_t s) {
  const int smem = (int)sizeof(IfaceShared<R>);
  cudaFuncSetAttribute(k_interface<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_interface<R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  k_interface<R><<<tile_grid(g), dim3(kBX, kBY, kBZ), smem, s>>>(
      g, make_physr<R>(ph, g), tb, passes, alpha, T, c, kappa, M0, M1, M2);
}

// ---------------------------------------------------------------------------
// scalar transport (alpha, T) and stage update

// face fluxes of one tile: [0] alpha advection, [1] T advection, [2] T conduction
template <typename R>
struct ScalFlux {
  R x[3][kBZ][kBY][kBX + 1];
  R y[3][kBZ][kBY + 1][kBX];
  R z[3][kBZ + 1][kBY][kBX];
};

template <typename R>
struct ScalShared {
  R a[Tile<3>::N];
  R T[Tile<3>::N];
  ScalFlux<R> F;
};

// advective fluxes of alpha and T and the conductive flux of T through the
// low D-face of local cell (lx,ly,lz)
// limiter ratios of the bounded phase-fraction option (null: plain WENO5)
template <typename R>
struct FctRatios {
  const R* Rp;   // R+ per cell: fraction of the incoming antidiffusive flux allowed
  const R* Rm;   // R- per cell: fraction of the outgoing antidiffusive flux allowed
};

// flux-corrected alpha flux through the low D-face of global cell (i,j,k)
// (Zalesak 1979 with the bounds 0 and 1): between the upwind flux F_L and
// the WENO5 flux F_H, F = F_L + theta (F_H - F_L) with theta from the
// limiter ratios of the face's two cells
template <int D, typename R>
__device__ __forceinline__ R fct_flux(const FctRatios<R>& f, const Geo& g, bool in, int i, int j,
                                      int k, R U, R aL, R aR, R FH) {
  const R FL = U >= R(0) ? U * aL : U * aR;
  const R A = FH - FL;
  int li = i, lj = j, lk = k;
  shift<D>(li, lj, lk, -1);
  R th = R(1);
  if (A > R(0)) {
    const R rpR = g_even(f.Rp, g, in, i, j, k), rmL = g_even(f.Rm, g, in, li, lj, lk);
    th = rpR < rmL ? rpR : rmL;
  } else if (A < R(0)) {
    const R rpL = g_even(f.Rp, g, in, li, lj, lk), rmR = g_even(f.Rm, g, in, i, j, k);
    th = rpL < rmR ? rpL : rmR;
  }
  return FL + th * A;
}

template <int D, typename R>
__device__ __forceinline__ void scalar_face(const ScalShared<R>& S, const PhysR<R>& ph, const R Uf,
                                            int lx, int ly, int lz, R& Fa, R& FT, R& Df,
                                            const FctRatios<R>& fct, const Geo& g, bool in,
                                            int gi, int gj, int gk) {
  const int dx = D == 0, dy = D == 1, dz = D == 2;
  R av[6], tv[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int o = m - 3;
    av[m] = S.a[Tile<3>::at(lx + o * dx, ly + o * dy, lz + o * dz)];
    tv[m] = S.T[Tile<3>::at(lx + o * dx, ly + o * dy, lz + o * dz)];
  }
  Fa = upwind_flux(Uf, av, ph.eps_a);
  if (fct.Rp) Fa = fct_flux<D>(fct, g, in, gi, gj, gk, Uf, av[2], av[3], Fa);
  FT = upwind_flux(Uf, tv, ph.eps_T);
  R lL = mixr(av[2], ph.lam), lR = mixr(av[3], ph.lam);
  R lf = R(2) * lL * lR / (lL + lR);
  Df = lf * (tv[3] - tv[2]) * ph.ih;
}

template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 4 : 1)
    k_scalars(Geo g, PhysR<R> ph, TBC tb, Fields<R> X, Fields<R> Sn, Fields<R> Y,
              const double* __restrict__ dtp, R a, R b, R xc, R yc, R qamp, R ir2,
              FctRatios<R> fct) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScalShared<R>& S = *reinterpret_cast<ScalShared<R>*>(smem_raw);
  stage<3, F_EVEN, 0>(S.a, X.alpha, g, tb);
  stage<3, F_TEMP, 0>(S.T, X.T, g, tb);
  const bool in = tile_interior(g, 3);
  __syncthreads();
  const R dt = (R)dtp[0];
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int i = blockIdx.x * kBX + tx, j = blockIdx.y * kBY + ty, k = blockIdx.z * kBZ + tz;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const R ih = ph.ih;
  ScalFlux<R>& F = S.F;
  if (i <= nx && j < ny && k < nz) {
    scalar_face<0>(S, ph, g_vel<0>(X.u[0], g, in, i, j, k), tx, ty, tz, F.x[0][tz][ty][tx], F.x[1][tz][ty][tx], F.x[2][tz][ty][tx],
                   fct, g, in, i, j, k);
    if (tx == kBX - 1 && i + 1 <= nx)
      scalar_face<0>(S, ph, g_vel<0>(X.u[0], g, in, i + 1, j, k), tx + 1, ty, tz, F.x[0][tz][ty][tx + 1], F.x[1][tz][ty][tx + 1],
                     F.x[2][tz][ty][tx + 1], fct, g, in, i + 1, j, k);
  }
  if (i < nx && j <= ny && k < nz) {
    scalar_face<1>(S, ph, g_vel<1>(X.u[1], g, in, i, j, k), tx, ty, tz, F.y[0][tz][ty][tx], F.y[1][tz][ty][tx], F.y[2][tz][ty][tx],
                   fct, g, in, i, j, k);
    if (ty == kBY - 1 && j + 1 <= ny)
      scalar_face<1>(S, ph, g_vel<1>(X.u[1], g, in, i, j + 1, k), tx, ty + 1, tz, F.y[0][tz][ty + 1][tx], F.y[1][tz][ty + 1][tx],
                     F.y[2][tz][ty + 1][tx], fct, g, in, i, j + 1, k);
  }
  if (i < nx && j < ny && k <= nz) {
    scalar_face<2>(S, ph, g_vel<2>(X.u[2], g, in, i, j, k), tx, ty, tz, F.z[0][tz][ty][tx], F.z[1][tz][ty][tx], F.z[2][tz][ty][tx],
                   fct, g, in, i, j, k);
    if (tz == kBZ - 1 && k + 1 <= nz)
      scalar_face<2>(S, ph, g_vel<2>(X.u[2], g, in, i, j, k + 1), tx, ty, tz + 1, F.z[0][tz + 1][ty][tx], F.z[1][tz + 1][ty][tx],
                     F.z[2][tz + 1][ty][tx], fct, g, in, i, j, k + 1);
  }
  __syncthreads();
  if (i >= nx || j >= ny || k >= nz) return;
  const int c = (k * ny + j) * nx + i;
  R Ra = 0, RT = 0, Dif = 0;
  Ra -= (F.x[0][tz][ty][tx + 1] - F.x[0][tz][ty][tx]) * ih;
  RT -= (F.x[1][tz][ty][tx + 1] - F.x[1][tz][ty][tx]) * ih;
  Dif += (F.x[2][tz][ty][tx + 1] - F.x[2][tz][ty][tx]) * ih;
  Ra -= (F.y[0][tz][ty + 1][tx] - F.y[0][tz][ty][tx]) * ih;
  RT -= (F.y[1][tz][ty + 1][tx] - F.y[1][tz][ty][tx]) * ih;
  Dif += (F.y[2][tz][ty + 1][tx] - F.y[2][tz][ty][tx]) * ih;
  Ra -= (F.z[0][tz + 1][ty][tx] - F.z[0][tz][ty][tx]) * ih;
  RT -= (F.z[1][tz + 1][ty][tx] - F.z[1][tz][ty][tx]) * ih;
  Dif += (F.z[2][tz + 1][ty][tx] - F.z[2][tz][ty][tx]) * ih;
  const R al = S.a[Tile<3>::at(tx, ty, tz)];
  const R rcp = mixr(al, ph.rcp);
  RT += Dif / rcp;
  if (qamp != R(0)) {
    const R i2h = R(0.5) * ih;
    R gx = (S.a[Tile<3>::at(tx + 1, ty, tz)] - S.a[Tile<3>::at(tx - 1, ty, tz)]) * i2h;
    R gy = (S.a[Tile<3>::at(tx, ty + 1, tz)] - S.a[Tile<3>::at(tx, ty - 1, tz)]) * i2h;
    R gz = (S.a[Tile<3>::at(tx, ty, tz + 1)] - S.a[Tile<3>::at(tx, ty, tz - 1)]) * i2h;
    R dx = (R(i) + R(0.5)) * ph.h - xc, dy = (R(j) + R(0.5)) * ph.h - yc;
    if (g.bc[0] == PER) dx = dx - ph.L[0] * floor(dx / ph.L[0] + R(0.5));
    if (g.bc[1] == PER) dy = dy - ph.L[1] * floor(dy / ph.L[1] + R(0.5));
    R q = qamp * exp(R(-2) * (dx * dx + dy * dy) * ir2);
    R gn = sqrt(gx * gx + gy * gy + gz * gz);
    RT += q * gn / rcp;
  }
  R Ea = al + dt * Ra;
  R ET = S.T[Tile<3>::at(tx, ty, tz)] + dt * RT;
  Y.alpha[c] = a * Sn.alpha[c] + b * Ea;
  Y.T[c] = a * Sn.T[c] + b * ET;
}

template <typename R>
void launch_scalars(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, Fields<R> Sn,
                    Fields<R> Y, const double* dt, double a, double b, double xc, const R* fct_p,
                    const R* fct_m, cudaStream_t s) {
  // source amplitude 2P/(pi r^2) and 1/r^2 formed once on the host
  double r2 = ph.q_radius * ph.q_radius;
  double qamp = ph.q_power != 0.0 ? 2.0 * ph.q_power / (M_PI * r2) : 0.0;
  double ir2 = ph.q_power != 0.0 ? 1.0 / r2 : 0.0;
  const int smem = (int)sizeof(ScalShared<R>);
  cudaFuncSetAttribute(k_scalars<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_scalars<R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  k_scalars<R><<<tile_grid(g), dim3(kBX, kBY, kBZ), smem, s>>>(
      g, make_physr<R>(ph, g), tb, X, Sn, Y, dt, (R)a, (R)b, (R)xc, (R)ph.q_y0, (R)qamp, (R)ir2,
      FctRatios<R>{fct_p, fct_m});
}

// limiter ratios of the bounded alpha transport for one stage: per cell the
// upwind (low-order) update alpha_td and the antidiffusive fluxes of its six
// faces give R+ = clamp((1 - alpha_td) h / dt / P+, 0, 1) and
// R- = clamp(alpha_td h / dt / P-, 0, 1) (0 where P vanishes), P+- the sums
// of antidiffusive fluxes into and out of the cell
template <int D, typename R>
__device__ __forceinline__ void fct_cell_face(const Geo& g, const PhysR<R>& ph, const R* alpha,
                                              const R* u, int i, int j, int k, int s, R& FLo,
                                              R& Ao) {
  int fi = i, fj = j, fk = k;
  shift<D>(fi, fj, fk, s);                   // the low face of cell c + s e_D
  const R U = ld_vel<D>(u, g, fi, fj, fk);
  R v[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int a = fi, b = fj, cc = fk;
    shift<D>(a, b, cc, m - 3);
    v[m] = ld_even(alpha, g, a, b, cc);
  }
  const R FH = upwind_flux(U, v, ph.eps_a);
  FLo = U >= R(0) ? U * v[2] : U * v[3];
  Ao = FH - FLo;
}

template <typename R>
__global__ void k_fct_ratios(Geo g, PhysR<R> ph, Fields<R> X, const double* __restrict__ dtp,
                             R* __restrict__ Rp, R* __restrict__ Rm) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y,
            k = blockIdx.z * kBZ + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
  const R dt = (R)dtp[0];
  R div = 0, Pp = 0, Pm = 0;
  R FL0, A0, FL1, A1;
  fct_cell_face<0>(g, ph, X.alpha, X.u[0], i, j, k, 0, FL0, A0);
  fct_cell_face<0>(g, ph, X.alpha, X.u[0], i, j, k, 1, FL1, A1);
  div += (FL1 - FL0) * ph.ih;
  Pp += (A0 > R(0) ? A0 : R(0)) + (-A1 > R(0) ? -A1 : R(0));
  Pm += (-A0 > R(0) ? -A0 : R(0)) + (A1 > R(0) ? A1 : R(0));
  fct_cell_face<1>(g, ph, X.alpha, X.u[1], i, j, k, 0, FL0, A0);
  fct_cell_face<1>(g, ph, X.alpha, X.u[1], i, j, k, 1, FL1, A1);
  div += (FL1 - FL0) * ph.ih;
  Pp += (A0 > R(0) ? A0 : R(0)) + (-A1 > R(0) ? -A1 : R(0));
  Pm += (-A0 > R(0) ? -A0 : R(0)) + (A1 > R(0) ? A1 : R(0));
  fct_cell_face<2>(g, ph, X.alpha, X.u[2], i, j, k, 0, FL0, A0);
  fct_cell_face<2>(g, ph, X.alpha, X.u[2], i, j, k, 1, FL1, A1);
  div += (FL1 - FL0) * ph.ih;
  Pp += (A0 > R(0) ? A0 : R(0)) + (-A1 > R(0) ? -A1 : R(0));
  Pm += (-A0 > R(0) ? -A0 : R(0)) + (A1 > R(0) ? A1 : R(0));
  const long long c = lin(g, i, j, k);
  const R atd = X.alpha[c] - dt * div;
  const R Qp = (R(1) - atd) * ph.h / dt, Qm = atd * ph.h / dt;
  R rp = R(0), rm = R(0);
  if (Pp > R(0)) rp = fmin(R(1), fmax(R(0), Qp / Pp));
  if (Pm > R(0)) rm = fmin(R(1), fmax(R(0), Qm / Pm));
  Rp[c] = rp;
  Rm[c] = rm;
}

template <typename R>
void launch_fct_ratios(const Geo& g, const Phys& ph, Fields<R> X, const double* dt, R* Rp, R* Rm,
                       cudaStream_t s) {
  k_fct_ratios<R><<<tile_grid(g), dim3(kBX, kBY, kBZ), 0, s>>>(g, make_physr<R>(ph, g), X, dt, Rp,
                                                                 Rm);
}

// ---------------------------------------------------------------------------
// transport of a concentration c (the solutal field of Eq. 5): WENO5
// advection with the face velocity, diffusion with the harmonic face mean of
// the mixture diffusivity, no flux through walls (even ghosts), stage update
template <typename R>
struct ConcShared {
  R c[Tile<3>::N];
  R D[Tile<1>::N];                       // mixture diffusivity of the cells
  R fx[2][kBZ][kBY][kBX + 1];            // [0] advective, [1] diffusive face fluxes
  R fy[2][kBZ][kBY + 1][kBX];
  R fz[2][kBZ + 1][kBY][kBX];
};

template <int D, typename R>
__device__ __forceinline__ void conc_face(const ConcShared<R>& S, const PhysR<R>& ph, const R Uf,
                                          int lx, int ly, int lz, R& Fa, R& Fd) {
  const int dx = D == 0, dy = D == 1, dz = D == 2;
  R v[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int o = m - 3;
    v[m] = S.c[Tile<3>::at(lx + o * dx, ly + o * dy, lz + o * dz)];
  }
  Fa = upwind_flux(Uf, v, ph.eps_c);
  const R dL = S.D[Tile<1>::at(lx - dx, ly - dy, lz - dz)], dR = S.D[Tile<1>::at(lx, ly, lz)];
  Fd = harmonic(dL, dR) * (v[3] - v[2]) * ph.ih;
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_concentration(Geo g, PhysR<R> ph, Fields<R> X, Fields<R> Sn, Fields<R> Y,
                    const double* __restrict__ dtp, R a, R b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ConcShared<R>& S = *reinterpret_cast<ConcShared<R>*>(smem_raw);
  TBC tb;
  tb.axis = -1;
  stage<3, F_EVEN, 0>(S.c, X.c, g, tb);
  stage<1, F_EVEN, 0>(S.D, X.alpha, g, tb);
  __syncthreads();
  for (int e = flat_tid(); e < Tile<1>::N; e += kThreads) S.D[e] = mixr(S.D[e], ph.diff_c);
  const bool in = tile_interior(g, 3);
  __syncthreads();
  const R dt = (R)dtp[0];
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int i = blockIdx.x * kBX + tx, j = blockIdx.y * kBY + ty, k = blockIdx.z * kBZ + tz;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  if (i <= nx && j < ny && k < nz) {
    conc_face<0>(S, ph, g_vel<0>(X.u[0], g, in, i, j, k), tx, ty, tz, S.fx[0][tz][ty][tx], S.fx[1][tz][ty][tx]);
    if (tx == kBX - 1 && i + 1 <= nx)
      conc_face<0>(S, ph, g_vel<0>(X.u[0], g, in, i + 1, j, k), tx + 1, ty, tz, S.fx[0][tz][ty][tx + 1],
                   S.fx[1][tz][ty][tx + 1]);
  }
  if (i < nx && j <= ny && k < nz) {
    conc_face<1>(S, ph, g_vel<1>(X.u[1], g, in, i, j, k), tx, ty, tz, S.fy[0][tz][ty][tx], S.fy[1][tz][ty][tx]);
    if (ty == kBY - 1 && j + 1 <= ny)
      conc_face<1>(S, ph, g_vel<1>(X.u[1], g, in, i, j + 1, k), tx, ty + 1, tz, S.fy[0][tz][ty + 1][tx],
                   S.fy[1][tz][ty + 1][tx]);
  }
  if (i < nx && j < ny && k <= nz) {
    conc_face<2>(S, ph, g_vel<2>(X.u[2], g, in, i, j, k), tx, ty, tz, S.fz[0][tz][ty][tx], S.fz[1][tz][ty][tx]);
    if (tz == kBZ - 1 && k + 1 <= nz)
      conc_face<2>(S, ph, g_vel<2>(X.u[2], g, in, i, j, k + 1), tx, ty, tz + 1, S.fz[0][tz + 1][ty][tx],
                   S.fz[1][tz + 1][ty][tx]);
  }
  __syncthreads();
  if (i >= nx || j >= ny || k >= nz) return;
  const int c = (k * ny + j) * nx + i;
  const R ih = ph.ih;
  R Ra = 0, Dif = 0;
  Ra -= (S.fx[0][tz][ty][tx + 1] - S.fx[0][tz][ty][tx]) * ih;
  Dif += (S.fx[1][tz][ty][tx + 1] - S.fx[1][tz][ty][tx]) * ih;
  Ra -= (S.fy[0][tz][ty + 1][tx] - S.fy[0][tz][ty][tx]) * ih;
  Dif += (S.fy[1][tz][ty + 1][tx] - S.fy[1][tz][ty][tx]) * ih;
  Ra -= (S.fz[0][tz + 1][ty][tx] - S.fz[0][tz][ty][tx]) * ih;
  Dif += (S.fz[1][tz + 1][ty][tx] - S.fz[1][tz][ty][tx]) * ih;
  const R Ec = S.c[Tile<3>::at(tx, ty, tz)] + dt * (Ra + Dif);
  Y.c[c] = a * Sn.c[c] + b * Ec;
}

template <typename R>
void launch_concentration(const Geo& g, const Phys& ph, Fields<R> X, Fields<R> Sn, Fields<R> Y,
                          const double* dt, double a, double b, cudaStream_t s) {
  const int smem = (int)sizeof(ConcShared<R>);
  cudaFuncSetAttribute(k_concentration<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_concentration<R><<<tile_grid(g), dim3(kBX, kBY, kBZ), smem, s>>>(
      g, make_physr<R>(ph, g), X, Sn, Y, dt, (R)a, (R)b);
}

// ---------------------------------------------------------------------------
// momentum predictor

// flux arrays for one component: [0] centre, [1] edge along t1, [2] edge along
// t2; advective (a) and viscous (v) parts.  Extents kBZ+1 x kBY+1 x kBX+1
// cover the one extra layer on any axis.
template <typename R>
struct MomFlux {
  R a[3][kBZ + 1][kBY + 1][kBX + 1];
  R v[3][kBZ + 1][kBY + 1][kBX + 1];
};

template <typename R>
struct MomShared {
  R u[3][Tile<3>::N];     // velocity components
  R mu[Tile<1>::N];       // cell viscosity mu(alpha)
  MomFlux<R> F;
};

template <int D>
struct Tang {
  static constexpr int t1 = D == 0 ? 1 : 0;
  static constexpr int t2 = D == 2 ? 1 : 2;
};

template <int A>
__device__ __forceinline__ void sh1(int& x, int& y, int& z, int s) {
  if (A == 0) x += s;
  if (A == 1) y += s;
  if (A == 2) z += s;
}

// normal momentum fluxes of component D at the centre of local cell
// (lx,ly,lz): advective U_c WENO5(u_D) with U_c the mean of the two D-faces,
// viscous normal stress 2 mu du_D/dx_D
template <int D, typename R>
__device__ __forceinline__ void centre_flux(const MomShared<R>& S, const PhysR<R>& ph, int lx,
                                            int ly, int lz, R& Fa, R& Fv) {
  R v[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int x = lx, y = ly, z = lz;
    sh1<D>(x, y, z, m - 2);
    v[m] = S.u[D][Tile<3>::at(x, y, z)];
  }
  const R Uc = R(0.5) * (v[2] + v[3]);
  Fa = upwind_flux(Uc, v, ph.eps_u);
  Fv = R(2) * S.mu[Tile<1>::at(lx, ly, lz)] * (v[3] - v[2]) * ph.ih;
}

// tangential fluxes of component D along T_ at the low T_-edge of the D-face
// of local cell (lx,ly,lz): advective U_e WENO5(u_D along T_) with U_e the
// mean of the two T_-faces at the edge, viscous mu_e (du_D/dx_T + du_T/dx_D)
// with mu_e the mean of the four cells around the edge
template <int D, int T_, typename R>
__device__ __forceinline__ void edge_flux(const MomShared<R>& S, const PhysR<R>& ph, int lx,
                                          int ly, int lz, R& Fa, R& Fv) {
  R v[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    int x = lx, y = ly, z = lz;
    sh1<T_>(x, y, z, m - 3);
    v[m] = S.u[D][Tile<3>::at(x, y, z)];
  }
  int x2 = lx, y2 = ly, z2 = lz;   // f - e_D
  sh1<D>(x2, y2, z2, -1);
  const R ut_hi = S.u[T_][Tile<3>::at(lx, ly, lz)];
  const R ut_lo = S.u[T_][Tile<3>::at(x2, y2, z2)];
  const R Ue = R(0.5) * (ut_lo + ut_hi);
  Fa = upwind_flux(Ue, v, ph.eps_u);
  int x3 = lx, y3 = ly, z3 = lz;   // f - e_T
  sh1<T_>(x3, y3, z3, -1);
  int x4 = x3, y4 = y3, z4 = z3;   // f - e_T - e_D
  sh1<D>(x4, y4, z4, -1);
  const R mue = R(0.25) * (S.mu[Tile<1>::at(lx, ly, lz)] + S.mu[Tile<1>::at(x2, y2, z2)] +
                           S.mu[Tile<1>::at(x3, y3, z3)] + S.mu[Tile<1>::at(x4, y4, z4)]);
  const R dud_dt = (v[3] - v[2]) * ph.ih;
  const R dut_dd = (ut_hi - ut_lo) * ph.ih;
  Fv = mue * (dud_dt + dut_dd);
}

template <int D, typename R>
__device__ __forceinline__ void momentum_component(const Geo& g, const PhysR<R>& ph, const TBC& tb,
                                                   const Fields<R>& X, const R* __restrict__ kappa,
                                                   const R* __restrict__ MD, bool in,
                                                   MomShared<R>& S, R* __restrict__ us, R dt,
                                                   R* __restrict__ phi) {
  constexpr int t1 = Tang<D>::t1, t2 = Tang<D>::t2;
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int i = blockIdx.x * kBX + tx, j = blockIdx.y * kBY + ty, k = blockIdx.z * kBZ + tz;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int gi[3] = {i, j, k};
  const bool inside = i < nx && j < ny && k < nz;
  MomFlux<R>& F = S.F;
  // centre fluxes: cell c at index t_D + 1; the low extra (c - e_D) at index 0
  if (inside) {
    int ci = tx, cj = ty, ck = tz;
    sh1<D>(ci, cj, ck, 1);
    centre_flux<D>(S, ph, tx, ty, tz, F.a[0][ck][cj][ci], F.v[0][ck][cj][ci]);
    if (tsel<D>(tx, ty, tz) == 0) {
      int x = tx, y = ty, z = tz;
      sh1<D>(x, y, z, -1);
      centre_flux<D>(S, ph, x, y, z, F.a[0][tz][ty][tx], F.v[0][tz][ty][tx]);
    }
  }
  // edge fluxes along t1 and t2: low edge of face c at index t_T; the high
  // extra at t_T + 1 (a thread one past the domain on T computes its own low
  // edge, which is the high edge of the last cell)
  if (inside || (gi[t1] == g.n[t1] && gi[D] < g.n[D] && gi[t2] < g.n[t2])) {
    edge_flux<D, t1>(S, ph, tx, ty, tz, F.a[1][tz][ty][tx], F.v[1][tz][ty][tx]);
    if (inside && tsel<t1>(tx, ty, tz) == tsel<t1>(kBX, kBY, kBZ) - 1) {
      int x = tx, y = ty, z = tz;
      sh1<t1>(x, y, z, 1);
      edge_flux<D, t1>(S, ph, x, y, z, F.a[1][z][y][x], F.v[1][z][y][x]);
    }
  }
  if (inside || (gi[t2] == g.n[t2] && gi[D] < g.n[D] && gi[t1] < g.n[t1])) {
    edge_flux<D, t2>(S, ph, tx, ty, tz, F.a[2][tz][ty][tx], F.v[2][tz][ty][tx]);
    if (inside && tsel<t2>(tx, ty, tz) == tsel<t2>(kBX, kBY, kBZ) - 1) {
      int x = tx, y = ty, z = tz;
      sh1<t2>(x, y, z, 1);
      edge_flux<D, t2>(S, ph, x, y, z, F.a[2][z][y][x], F.v[2][z][y][x]);
    }
  }
  __syncthreads();
  if (inside) {
    const int c = (k * ny + j) * nx + i;
    if (g.bc[D] == WALL && gi[D] == 0) {
      us[c] = R(0);
      if (phi) phi[c] = R(0);
    } else {
      const R ih = ph.ih;
      int ci = tx, cj = ty, ck = tz;
      sh1<D>(ci, cj, ck, 1);
      R A = R(0) - (F.a[0][ck][cj][ci] - F.a[0][tz][ty][tx]) * ih;
      R V = R(0) + (F.v[0][ck][cj][ci] - F.v[0][tz][ty][tx]) * ih;
      {
        int x = tx, y = ty, z = tz;
        sh1<t1>(x, y, z, 1);
        A -= (F.a[1][z][y][x] - F.a[1][tz][ty][tx]) * ih;
        V += (F.v[1][z][y][x] - F.v[1][tz][ty][tx]) * ih;
      }
      {
        int x = tx, y = ty, z = tz;
        sh1<t2>(x, y, z, 1);
        A -= (F.a[2][z][y][x] - F.a[2][tz][ty][tx]) * ih;
        V += (F.v[2][z][y][x] - F.v[2][tz][ty][tx]) * ih;
      }
      // forces on the face between cell L = c - e_D and R = c
      int a = i, b = j, cc = k;
      sh1<D>(a, b, cc, -1);
      const R alL = g_even(X.alpha, g, in, a, b, cc), alR = X.alpha[c];
      const R rho_f = R(0.5) * (mixr(alL, ph.rho) + mixr(alR, ph.rho));
      const R TL = g_T(X.T, g, tb, in, a, b, cc), TR = X.T[c];
      const R sig_f = X.c ? R(0.5) * (sigma_rc(TL, g_even(X.c, g, in, a, b, cc), ph) +
                                      sigma_rc(TR, X.c[c], ph))
                          : R(0.5) * (sigma_r(TL, ph) + sigma_r(TR, ph));
      const R kap_f = R(0.5) * (g_even(kappa, g, in, a, b, cc) + kappa[c]);
      const R jump = (alR - alL) * ih;
      const R fn = -sig_f * kap_f * jump;
      const R fM = R(0.5) * (g_even(MD, g, in, a, b, cc) + MD[c]);
      us[c] = S.u[D][Tile<3>::at(tx, ty, tz)] + dt * (A + (V + fn + fM) / rho_f + ph.g[D]);
      if (phi) phi[c] = V + fn + fM;   // the force sum before 1/rho_f (the adjoint's density term)
    }
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 1)
    k_momentum(Geo g, PhysR<R> ph, TBC tb, Fields<R> X, const R* __restrict__ kappa,
               const R* __restrict__ M0, const R* __restrict__ M1, const R* __restrict__ M2,
               R* __restrict__ us0, R* __restrict__ us1, R* __restrict__ us2,
               const double* __restrict__ dtp, R* __restrict__ ph0, R* __restrict__ ph1,
               R* __restrict__ ph2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MomShared<R>& S = *reinterpret_cast<MomShared<R>*>(smem_raw);
  stage<3, F_VEL, 0>(S.u[0], X.u[0], g, tb);
  stage<3, F_VEL, 1>(S.u[1], X.u[1], g, tb);
  stage<3, F_VEL, 2>(S.u[2], X.u[2], g, tb);
  stage<1, F_EVEN, 0>(S.mu, X.alpha, g, tb);
  __syncthreads();
  for (int e = flat_tid(); e < Tile<1>::N; e += kThreads) S.mu[e] = mixr(S.mu[e], ph.mu);
  __syncthreads();
  const R dt = (R)dtp[0];
  const bool in = tile_interior(g, 3);
  momentum_component<0>(g, ph, tb, X, kappa, M0, in, S, us0, dt, ph0);
  momentum_component<1>(g, ph, tb, X, kappa, M1, in, S, us1, dt, ph1);
  momentum_component<2>(g, ph, tb, X, kappa, M2, in, S, us2, dt, ph2);
}

template <typename R>
void launch_momentum(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, const R* kappa,
                     const R* M0, const R* M1, const R* M2, R* us0, R* us1, R* us2,
                     const double* dt, cudaStream_t s, R* const* phi) {
  const int smem = (int)sizeof(MomShared<R>);
  cudaFuncSetAttribute(k_momentum<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // float tiles (71 KB) fit three CTAs per SM when the L1/shared split favours shared memory
  cudaFuncSetAttribute(k_momentum<R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  k_momentum<R><<<tile_grid(g), dim3(kBX, kBY, kBZ), smem, s>>>(
      g, make_physr<R>(ph, g), tb, X, kappa, M0, M1, M2, us0, us1, us2, dt,
      phi ? phi[0] : nullptr, phi ? phi[1] : nullptr, phi ? phi[2] : nullptr);
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
  const double ih = g.ih;
  const double idt = dtp[1];
  double acc = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.N;
       c += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    double dv = 0.0;
    dv += ((double)ld_vel<0>(u0, g, i + 1, j, k) - (double)u0[c]) * ih;
    dv += ((double)ld_vel<1>(u1, g, i, j + 1, k) - (double)u1[c]) * ih;
    dv += ((double)ld_vel<2>(u2, g, i, j, k + 1) - (double)u2[c]) * ih;
    double v = -dv * idt;
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
// velocity correction and RK combination.  The pressure difference is taken
// in double; in the mixed form the rest is float arithmetic.
template <typename R, typename B>
__global__ void k_correct(Geo g, Fields<R> Sn, Fields<R> Y, const R* __restrict__ us0,
                          const R* __restrict__ us1, const R* __restrict__ us2,
                          const double* __restrict__ p, const B* __restrict__ b0,
                          const B* __restrict__ b1, const B* __restrict__ b2,
                          const double* __restrict__ dtp, R a, R bb) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.N) return;
  int i, j, k;
  decode(g, c, i, j, k);
  const double dtih = dtp[0] * g.ih;
  const double pc = p[c];
  const R* us[3] = {us0, us1, us2};
  const B* be[3] = {b0, b1, b2};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int idx[3] = {i, j, k};
    bool wall_face = (g.bc[d] == WALL && idx[d] == 0);
    int m[3] = {i, j, k};
    m[d] = wrapi(m[d] - 1, g.n[d]);
    double pl = p[(m[2] * g.n[1] + m[1]) * g.n[0] + m[0]];
    R gp = (R)((pc - pl) * dtih);
    R ucorr = us[d][c] - (R)be[d][c] * gp;
    R out = wall_face ? R(0) : a * Sn.u[d][c] + bb * ucorr;
    Y.u[d][c] = out;
  }
}

template <typename R, typename B>
void launch_correct(const Geo& g, Fields<R> Sn, Fields<R> Y, R* const* us, const double* p,
                    B* const* beta, const double* dt, double a, double b, cudaStream_t s) {
  k_correct<R, B><<<grid1d(g.N, 256), 256, 0, s>>>(g, Sn, Y, us[0], us[1], us[2], p, beta[0],
                                                   beta[1], beta[2], dt, (R)a, (R)b);
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
    R sg = sigma_of_T(T, ph);
    if (X.c) sg += (R)ph.dsdc * (X.c[c] - (R)ph.c0);
    v[3] = fabs((double)sg);
    v[4] = (double)(mixp(al, ph.mu) / mixp(al, ph.rho));
    v[5] = (double)(mixp(al, ph.lam) / mixp(al, ph.rcp));
    if (X.c) {   // the concentration's diffusion shares the diffusive limit
      const double dc = (double)mixp(al, ph.diff_c);
      v[5] = dc > v[5] ? dc : v[5];
    }
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

// dt[0] = step, dt[1] = 1/step
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
  dt[0] = lim[kk];
  dt[1] = 1.0 / lim[kk];
  *limiter = kk;
}

void launch_dt_final(const Geo& g, const Phys& ph, double cfl, double c_cap, double c_visc,
                     double c_therm, double dt_max, const unsigned long long* maxbits,
                     double* dt, int* limiter, cudaStream_t s) {
  k_dt_final<<<1, 1, 0, s>>>(g.h, ph.rho[0] + ph.rho[1], cfl, c_cap, c_visc, c_therm, dt_max,
                             maxbits, dt, limiter);
}

__global__ void k_set_scalar(double* dst, double v, double iv) {
  dst[0] = v;
  dst[1] = iv;
}

void launch_set_scalar(double* dst, double v, cudaStream_t s) {
  k_set_scalar<<<1, 1, 0, s>>>(dst, v, 1.0 / v);
}

// ---------------------------------------------------------------------------
// diagnostics: partial sums of alpha and rho(alpha) (two slots per block),
// max |D u| as bits in maxbits[0], NaN flag
template <typename R>
__global__ void k_diagnostics(Geo g, Phys ph, Fields<R> X, const double* __restrict__ p,
                              double* __restrict__ partial, unsigned long long* __restrict__ maxbits,
                              int* __restrict__ nanflag) {
  const double ih = g.ih;
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
                 (double)X.T[c] + p[c] + (X.c ? (double)X.c[c] : 0.0);
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
  template void launch_interface<R>(const Geo&, const Phys&, const TBC&, int, const R*,          \
                                    const R*, const R*, R*, R*, R*, R*, cudaStream_t);           \
  template void launch_concentration<R>(const Geo&, const Phys&, Fields<R>, Fields<R>,           \
                                        Fields<R>, const double*, double, double, cudaStream_t); \
  template void launch_scalars<R>(const Geo&, const Phys&, const TBC&, Fields<R>, Fields<R>,     \
                                  Fields<R>, const double*, double, double, double, const R*,    \
                                  const R*, cudaStream_t);                                       \
  template void launch_fct_ratios<R>(const Geo&, const Phys&, Fields<R>, const double*, R*, R*,  \
                                     cudaStream_t);                                              \
  template void launch_momentum<R>(const Geo&, const Phys&, const TBC&, Fields<R>, const R*,     \
                                   const R*, const R*, const R*, R*, R*, R*, const double*,      \
                                   cudaStream_t, R* const*);                                     \
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
