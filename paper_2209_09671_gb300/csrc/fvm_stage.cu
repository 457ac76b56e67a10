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
// Layout of the work: k_interface, k_scalars and k_momentum march along z: a
// CTA of kZX x kZY threads owns one (x, y) column of cells per thread and a
// run of planes; each plane of a field is staged once in shared memory with
// its x-y halo (copied asynchronously one step ahead), the z stencils come
// from rings of planes or per-thread register windows, and every face flux
// (and every edge flux of the momentum control volumes) is evaluated once.
// The other stage kernels (concentration, flux-corrected ratios, smoothing)
// own a kBX x kBY x kBZ tile of cells with a halo staged in shared memory.
// Points whose stored value is what the boundary rule gives are read
// directly; ghost points go through the wrap/mirror loaders.
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
// z-marching layout shared by the stage kernels: a
// CTA of kZX x kZY threads owns one (x, y) column of cells per thread and
// walks a run of planes upward.  Fields are staged one plane at a time in
// shared memory with the x-y halo the stencil needs; what the z-direction
// stencil needs stays in rings of planes (or in each thread's registers), so
// the z halo is read once per column run rather than once per tile.
constexpr int kZX = 32, kZY = 8;
constexpr int kZT = kZX * kZY;

template <int H>
struct Plane {
  static constexpr int PX = kZX + 2 * H, PY = kZY + 2 * H, N = PX * PY;
  static __device__ __forceinline__ int at(int lx, int ly) { return (ly + H) * PX + lx + H; }
};

static inline dim3 zmarch_grid(const Geo& g, int kz) {
  return dim3((unsigned)((g.n[0] + kZX - 1) / kZX), (unsigned)((g.n[1] + kZY - 1) / kZY),
              (unsigned)((g.n[2] + kz - 1) / kz));
}

// the CTA's columns and their x-y reach H stay inside the domain
__device__ __forceinline__ bool zcols_interior(const Geo& g, int H) {
  const int x0 = blockIdx.x * kZX, y0 = blockIdx.y * kZY;
  return x0 - H >= 0 && x0 + kZX - 1 + H < g.n[0] && y0 - H >= 0 && y0 + kZY - 1 + H < g.n[1];
}

// direct loads of plane k are valid in an interior run of columns: a cell
// plane inside the domain, a plane of z-faces strictly inside it (the wall
// faces take the boundary rule)
template <int KIND, int C>
__device__ __forceinline__ bool plane_direct(const Geo& g, bool in, int k) {
  return in && k >= ((KIND == F_VEL && C == 2) ? 1 : 0) && k < g.n[2];
}

// a point of plane k whose stored value is the value the boundary rule gives
template <int KIND, int C>
__device__ __forceinline__ bool point_direct(const Geo& g, int i, int j, int k) {
  const bool vel = KIND == F_VEL;
  return k >= ((vel && C == 2) ? 1 : 0) && k < g.n[2] && i >= ((vel && C == 0) ? 1 : 0) &&
         i < g.n[0] && j >= ((vel && C == 1) ? 1 : 0) && j < g.n[1];
}

template <int KIND, int C, typename R>
__device__ __forceinline__ R ld_rule(const R* __restrict__ a, const Geo& g, const TBC& tb, int i,
                                     int j, int k) {
  if (KIND == F_EVEN) return ld_even(a, g, i, j, k);
  if (KIND == F_VEL) return ld_vel<C>(a, g, i, j, k);
  return ld_T(a, g, tb, i, j, k);
}

// stage plane k of a field with an x-y halo of H (ghost planes k < 0 or
// k >= nz through the boundary rules); points more than H cells outside the
// domain (ragged tiles) are never read and hold 0
template <int H, int KIND, int C = 0, typename R>
__device__ __forceinline__ void stage_plane(R* __restrict__ s, const R* __restrict__ a,
                                            const Geo& g, const TBC& tb, bool in, int k) {
  using P = Plane<H>;
  const int x0 = blockIdx.x * kZX - H, y0 = blockIdx.y * kZY - H;
  const int nx = g.n[0], ny = g.n[1];
  if (plane_direct<KIND, C>(g, in, k)) {
    const R* __restrict__ ak = a + ((k * ny + y0) * nx + x0);
    for (int ly = threadIdx.y; ly < P::PY; ly += kZY) {
#pragma unroll
      for (int lx = threadIdx.x; lx < P::PX; lx += kZX) s[ly * P::PX + lx] = __ldg(ak + ly * nx + lx);
    }
    return;
  }
  for (int ly = threadIdx.y; ly < P::PY; ly += kZY) {
    const int j = y0 + ly;
    for (int lx = threadIdx.x; lx < P::PX; lx += kZX) {
      const int i = x0 + lx;
      R v;
      if (i > nx - 1 + H || j > ny - 1 + H) v = R(0);
      else if (point_direct<KIND, C>(g, i, j, k)) v = __ldg(a + ((k * ny + j) * nx + i));
      else v = ld_rule<KIND, C>(a, g, tb, i, j, k);
      s[ly * P::PX + lx] = v;
    }
  }
}

// asynchronous staging of a plane: in an interior run of columns each point
// is one cp.async copy from global to shared memory (4 or 8 bytes), so that
// the next plane is in flight while the current one is used; near the
// boundary the points go through the loaders and are stored directly.  The
// consumer waits with cp_async_wait_all() followed by __syncthreads().
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename R>
__device__ __forceinline__ void cp_async_elem(R* smem, const R* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(R) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <int H, int KIND, int C = 0, typename R>
__device__ __forceinline__ void plane_async(R* __restrict__ s, const R* __restrict__ a,
                                            const Geo& g, const TBC& tb, bool in, int k) {
  using P = Plane<H>;
  const int x0 = blockIdx.x * kZX - H, y0 = blockIdx.y * kZY - H;
  const int nx = g.n[0], ny = g.n[1];
  if (plane_direct<KIND, C>(g, in, k)) {
    const R* __restrict__ ak = a + ((k * ny + y0) * nx + x0);
    for (int ly = threadIdx.y; ly < P::PY; ly += kZY) {
#pragma unroll
      for (int lx = threadIdx.x; lx < P::PX; lx += kZX) cp_async_elem(s + ly * P::PX + lx, ak + ly * nx + lx);
    }
    return;
  }
  for (int ly = threadIdx.y; ly < P::PY; ly += kZY) {
    const int j = y0 + ly;
    for (int lx = threadIdx.x; lx < P::PX; lx += kZX) {
      const int i = x0 + lx;
      R* d = s + ly * P::PX + lx;
      if (i > nx - 1 + H || j > ny - 1 + H) *d = R(0);
      else if (point_direct<KIND, C>(g, i, j, k)) cp_async_elem(d, a + ((k * ny + j) * nx + i));
      else *d = ld_rule<KIND, C>(a, g, tb, i, j, k);
    }
  }
}

// ---------------------------------------------------------------------------
// interface geometry: smoothed alpha, face normals, curvature and the
// Marangoni vector in one kernel (the smoothed alpha never leaves the SM).
// K passes of the [1,2,1]/4 filter along an axis are one binomial filter of
// 2K+1 taps ([1,4,6,4,1]/16 for K = 2), and the passes along different axes
// commute, so the smoothing is applied as one 5-tap pass per axis: x and y
// on each staged plane, z across a ring of x-y-smoothed planes.
constexpr int kZKI = 32;   // planes per CTA

template <typename R>
struct IfaceZ {
  R ar[6][Plane<3>::N];      // alpha, ring of planes (m mod 6)
  R xp[Plane<3>::PY][kZX + 2];   // x-smoothed plane, x halo 1, y halo 3
  R xy[5][Plane<1>::N];      // x-y-smoothed planes (m mod 5)
  R s2[3][Plane<1>::N];      // smoothed alpha (m mod 3)
  R T[4][Plane<1>::N];       // temperature (m mod 4)
  R c[4][Plane<1>::N];       // concentration (m mod 4), when transported
  R nx[kZY][kZX + 1];        // face normals of the current plane
  R ny[kZY + 1][kZX];
};

// smooth the staged alpha plane m in x and y into xy[m mod 5] (the caller
// synchronises after staging and after this)
template <typename R>
__device__ __forceinline__ void iface_plane_xy(IfaceZ<R>& S, int m, const R* wx, const R* wy) {
  using P3 = Plane<3>;
  using P1 = Plane<1>;
  const R* __restrict__ ar = S.ar[(m % 6 + 6) % 6];
  for (int ly = threadIdx.y - 3; ly < kZY + 3; ly += kZY)
    for (int lx = threadIdx.x - 1; lx < kZX + 1; lx += kZX) {
      const int e = P3::at(lx, ly);
      S.xp[ly + 3][lx + 1] = wx[0] * ar[e - 2] + wx[1] * ar[e - 1] + wx[2] * ar[e] +
                             wx[3] * ar[e + 1] + wx[4] * ar[e + 2];
    }
  __syncthreads();
  R* __restrict__ xy = S.xy[(m % 5 + 5) % 5];
  for (int ly = threadIdx.y - 1; ly < kZY + 1; ly += kZY)
    for (int lx = threadIdx.x - 1; lx < kZX + 1; lx += kZX)
      xy[P1::at(lx, ly)] = wy[0] * S.xp[ly + 1][lx + 1] + wy[1] * S.xp[ly + 2][lx + 1] +
                           wy[2] * S.xp[ly + 3][lx + 1] + wy[3] * S.xp[ly + 4][lx + 1] +
                           wy[4] * S.xp[ly + 5][lx + 1];
}

// smoothed plane m from the x-y-smoothed planes m-2 .. m+2
template <typename R>
__device__ __forceinline__ void iface_plane_z(IfaceZ<R>& S, int m, const R* wz) {
  const R* __restrict__ q0 = S.xy[((m - 2) % 5 + 5) % 5];
  const R* __restrict__ q1 = S.xy[((m - 1) % 5 + 5) % 5];
  const R* __restrict__ q2 = S.xy[(m % 5 + 5) % 5];
  const R* __restrict__ q3 = S.xy[((m + 1) % 5 + 5) % 5];
  const R* __restrict__ q4 = S.xy[((m + 2) % 5 + 5) % 5];
  R* __restrict__ o = S.s2[(m % 3 + 3) % 3];
  for (int e = threadIdx.x + kZX * threadIdx.y; e < Plane<1>::N; e += kZT)
    o[e] = wz[0] * q0[e] + wz[1] * q1[e] + wz[2] * q2[e] + wz[3] * q3[e] + wz[4] * q4[e];
}

// normal on the low x-face (D = 0) or y-face (D = 1) of local cell (lx, ly)
// of plane c, with the planes below (m) and above (p): grad / (|grad| + eps_n),
// the normal derivative across the face and each tangential derivative the
// mean of the two cells' central differences
template <int D, typename R>
__device__ __forceinline__ R plane_normal(const R* __restrict__ m, const R* __restrict__ c,
                                          const R* __restrict__ p, int lx, int ly, R ih, R epsn) {
  using P1 = Plane<1>;
  const int e = P1::at(lx, ly);
  const int sd = D == 0 ? 1 : P1::PX;   // stride along the face normal
  const int st = D == 0 ? P1::PX : 1;   // stride along the in-plane tangent
  const R q = ih * R(0.25);
  const R gd = (c[e] - c[e - sd]) * ih;
  const R gt = ((c[e + st] - c[e - st]) + (c[e - sd + st] - c[e - sd - st])) * q;
  const R gz = ((p[e] - m[e]) + (p[e - sd] - m[e - sd])) * q;
  // tangential terms in axis order, as for the z-face
  const R sq = gd * gd + gt * gt + gz * gz;
  return gd / (sqrt(sq) + epsn);
}

// normal on the face between plane c (below) and plane p (above)
template <typename R>
__device__ __forceinline__ R z_normal(const R* __restrict__ c, const R* __restrict__ p, int lx,
                                      int ly, R ih, R epsn) {
  using P1 = Plane<1>;
  const int e = P1::at(lx, ly);
  const R q = ih * R(0.25);
  const R gd = (p[e] - c[e]) * ih;
  const R gx = ((p[e + 1] - p[e - 1]) + (c[e + 1] - c[e - 1])) * q;
  const R gy = ((p[e + P1::PX] - p[e - P1::PX]) + (c[e + P1::PX] - c[e - P1::PX])) * q;
  const R sq = gd * gd + gx * gx + gy * gy;
  return gd / (sqrt(sq) + epsn);
}

// binomial weights of K passes of [1,2,1]/4 on an axis of n cells (identity
// on an axis of one cell)
template <typename R>
__device__ __forceinline__ void binomial5(int K, int n, R* w) {
  const bool id = n == 1 || K == 0;
  w[0] = (!id && K == 2) ? R(0.0625) : R(0);
  w[1] = id ? R(0) : (K == 2 ? R(0.25) : R(0.25));
  w[2] = id ? R(1) : (K == 2 ? R(0.375) : R(0.5));
  w[3] = w[1];
  w[4] = w[0];
}

template <typename R>
__global__ void __launch_bounds__(kZT, sizeof(R) == 4 ? 4 : 2)
    k_interface(Geo g, PhysR<R> ph, TBC tb, int passes, const R* __restrict__ alpha,
                const R* __restrict__ T, const R* __restrict__ conc, R* __restrict__ kappa,
                R* __restrict__ M0, R* __restrict__ M1, R* __restrict__ M2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  IfaceZ<R>& S = *reinterpret_cast<IfaceZ<R>*>(smem_raw);
  using P1 = Plane<1>;
  using P3 = Plane<3>;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * kZX + tx, j = blockIdx.y * kZY + ty;
  const int z0 = blockIdx.z * kZKI;
  const int z1 = min(z0 + kZKI, nz);
  const bool in = zcols_interior(g, 3);
  const bool col = i < nx && j < ny;
  const R ih = ph.ih, i2h = R(0.5) * ph.ih, epsn = ph.eps_n;
  const int K = passes < 2 ? passes : 2;
  R wx[5], wy[5], wz[5];
  binomial5(K, nx, wx);
  binomial5(K, ny, wy);
  binomial5(K, nz, wz);
  // warm-up: alpha planes z0-3 .. z0+2 smoothed in x and y, smoothed planes
  // z0-1 and z0, temperature (and concentration) planes z0-1 and z0
  for (int m = z0 - 3; m <= z0 + 2; ++m) {
    if (m == z0 - 1 || m == z0) {
      stage_plane<1, F_TEMP>(S.T[(m % 4 + 4) % 4], T, g, tb, in, m);
      if (conc) stage_plane<1, F_EVEN>(S.c[(m % 4 + 4) % 4], conc, g, tb, in, m);
    }
    stage_plane<3, F_EVEN>(S.ar[(m % 6 + 6) % 6], alpha, g, tb, in, m);
    __syncthreads();
    iface_plane_xy(S, m, wx, wy);
    __syncthreads();
    if (m == z0 + 1 || m == z0 + 2) {
      iface_plane_z(S, m - 2, wz);
      __syncthreads();
    }
  }
  R nzl = R(0);   // normal on the low z-face of the current plane
  if (col) nzl = z_normal(S.s2[((z0 - 1) % 3 + 3) % 3], S.s2[z0 % 3], tx, ty, ih, epsn);
  // the planes a step needs first are copied one step ahead
  plane_async<3, F_EVEN>(S.ar[(z0 + 3) % 6], alpha, g, tb, in, z0 + 3);
  plane_async<1, F_TEMP>(S.T[(z0 + 1) % 4], T, g, tb, in, z0 + 1);
  if (conc) plane_async<1, F_EVEN>(S.c[(z0 + 1) % 4], conc, g, tb, in, z0 + 1);
  cp_async_commit();
  for (int k = z0; k < z1; ++k) {
    cp_async_wait_all();
    __syncthreads();
    // the slots of alpha k - 2 and T k - 2, last read by the previous step
    if (k + 1 < z1) {
      plane_async<3, F_EVEN>(S.ar[(k + 4) % 6], alpha, g, tb, in, k + 4);
      plane_async<1, F_TEMP>(S.T[(k + 2) % 4], T, g, tb, in, k + 2);
      if (conc) plane_async<1, F_EVEN>(S.c[(k + 2) % 4], conc, g, tb, in, k + 2);
      cp_async_commit();
    }
    iface_plane_xy(S, k + 3, wx, wy);
    __syncthreads();
    iface_plane_z(S, k + 1, wz);
    __syncthreads();
    const R* __restrict__ sm = S.s2[((k - 1) % 3 + 3) % 3];
    const R* __restrict__ sc = S.s2[k % 3];
    const R* __restrict__ sp = S.s2[(k + 1) % 3];
    if (i <= nx && j < ny) S.nx[ty][tx] = plane_normal<0>(sm, sc, sp, tx, ty, ih, epsn);
    if (i < nx && j <= ny) S.ny[ty][tx] = plane_normal<1>(sm, sc, sp, tx, ty, ih, epsn);
    if (ty == 0) {
      if (i < nx && blockIdx.y * kZY + kZY <= ny)
        S.ny[kZY][tx] = plane_normal<1>(sm, sc, sp, tx, kZY, ih, epsn);
    } else if (ty == 1 && tx < kZY) {
      if (blockIdx.x * kZX + kZX <= nx && blockIdx.y * kZY + tx < ny)
        S.nx[tx][kZX] = plane_normal<0>(sm, sc, sp, kZX, tx, ih, epsn);
    }
    R nzh = R(0);
    if (col) nzh = z_normal(sc, sp, tx, ty, ih, epsn);
    __syncthreads();
    if (col) {
      const int c = (k * ny + j) * nx + i;
      R kap = 0;
      kap += (S.nx[ty][tx + 1] - S.nx[ty][tx]) * ih;
      kap += (S.ny[ty + 1][tx] - S.ny[ty][tx]) * ih;
      kap += (nzh - nzl) * ih;
      kappa[c] = kap;
      // Marangoni vector from central differences of alpha, smoothed alpha, sigma(T)
      const R* __restrict__ am = S.ar[((k - 1) % 6 + 6) % 6];
      const R* __restrict__ ac = S.ar[k % 6];
      const R* __restrict__ ap = S.ar[(k + 1) % 6];
      const R* __restrict__ Tm = S.T[((k - 1) % 4 + 4) % 4];
      const R* __restrict__ Tc = S.T[k % 4];
      const R* __restrict__ Tp = S.T[(k + 1) % 4];
      const int e3 = P3::at(tx, ty), e1 = P1::at(tx, ty);
      R gv[3], tv[3], sv[3], cP[3], cM[3], TP[3], TM[3];
      gv[0] = (ac[e3 + 1] - ac[e3 - 1]) * i2h;
      gv[1] = (ac[e3 + P3::PX] - ac[e3 - P3::PX]) * i2h;
      gv[2] = (ap[e3] - am[e3]) * i2h;
      tv[0] = (sc[e1 + 1] - sc[e1 - 1]) * i2h;
      tv[1] = (sc[e1 + P1::PX] - sc[e1 - P1::PX]) * i2h;
      tv[2] = (sp[e1] - sm[e1]) * i2h;
      TP[0] = Tc[e1 + 1];      TM[0] = Tc[e1 - 1];
      TP[1] = Tc[e1 + P1::PX]; TM[1] = Tc[e1 - P1::PX];
      TP[2] = Tp[e1];          TM[2] = Tm[e1];
      if (conc) {
        const R* __restrict__ cm_ = S.c[((k - 1) % 4 + 4) % 4];
        const R* __restrict__ cc_ = S.c[k % 4];
        const R* __restrict__ cp_ = S.c[(k + 1) % 4];
        cP[0] = cc_[e1 + 1];      cM[0] = cc_[e1 - 1];
        cP[1] = cc_[e1 + P1::PX]; cM[1] = cc_[e1 - P1::PX];
        cP[2] = cp_[e1];          cM[2] = cm_[e1];
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        // central difference of the sigma field (Eq. 5 as a cell field).  In
        // float it is taken as dsigma/dT (T+ - T-), the same number for the
        // linear sigma(T): the difference of two neighbouring temperatures is
        // exact, while sigma0 + dsigma/dT (T - T0) rounded to float at
        // sigma ~ 1.9 keeps only ~4 digits of a variation of ~1e-3
        if (conc) {
          // sigma(c, T) of Eq. 5: in float the exact neighbour differences
          // again, in double the difference of the two cells' sigma values
          if (sizeof(R) == 4) sv[d] = (ph.dsdT * (TP[d] - TM[d]) + ph.dsdc * (cP[d] - cM[d])) * i2h;
          else sv[d] = (sigma_rc(TP[d], cP[d], ph) - sigma_rc(TM[d], cM[d], ph)) * i2h;
        } else if (sizeof(R) == 4) {
          sv[d] = ph.dsdT * (TP[d] - TM[d]) * i2h;
        } else {
          sv[d] = (sigma_r(TP[d], ph) - sigma_r(TM[d], ph)) * i2h;
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
    nzl = nzh;
  }
}

template <typename R>
void launch_interface(const Geo& g, const Phys& ph, const TBC& tb, int passes, const R* alpha,
                      const R* T, const R* c, R* kappa, R* M0, R* M1, R* M2, cudaStream_t s) {
  const int smem = (int)sizeof(IfaceZ<R>);
  cudaFuncSetAttribute(k_interface<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_interface<R><<<zmarch_grid(g, kZKI), dim3(kZX, kZY), smem, s>>>(
      g, make_physr<R>(ph, g), tb, passes, alpha, T, c, kappa, M0, M1, M2);
}

// ---------------------------------------------------------------------------
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

// scalar transport (alpha, T) and stage update
//
// Plane k of alpha and T is staged with an x-y halo of 3 (the WENO5 reach);
// the z-direction stencil lives in each thread's registers (a window of its
// column from k-3 to k+3), and the flux through the face between planes k
// and k+1 is evaluated once and carried to the next plane.  Every x- and
// y-face flux is evaluated once per plane: each thread takes the low face of
// its cell, one warp the high y-faces of the tile's last row, another the
// high x-faces of its last column.
constexpr int kZKS = 16;   // planes per CTA

// one cell of column (i, j) at height k (any k: ghost planes go through the
// boundary rules)
template <int KIND, typename R>
__device__ __forceinline__ R col_ld(const R* __restrict__ a, const Geo& g, const TBC& tb, int i,
                                    int j, int k) {
  if (k >= 0 && k < g.n[2]) return __ldg(a + ((k * g.n[1] + j) * g.n[0] + i));
  return KIND == F_EVEN ? ld_even(a, g, i, j, k) : ld_T(a, g, tb, i, j, k);
}

// velocity on the low D-face of cell (i, j, k): direct for a face strictly
// inside the domain along D, through the boundary rules otherwise
template <int D, typename R>
__device__ __forceinline__ R face_u(const R* __restrict__ u, const Geo& g, bool in, int i, int j,
                                    int k) {
  const int f = D == 0 ? i : (D == 1 ? j : k);
  if (in || (f >= 1 && f <= g.n[D] - 1)) return __ldg(u + ((k * g.n[1] + j) * g.n[0] + i));
  return ld_vel<D>(u, g, i, j, k);
}

// advective fluxes of alpha and T and the conductive flux of T through one
// face from the six values of each field around it (av[2] left, av[3] right)
template <typename R>
__device__ __forceinline__ void scal_flux(const R* av, const R* tv, R U, const PhysR<R>& ph,
                                          R& Fa, R& FT, R& Df) {
  Fa = upwind_flux(U, av, ph.eps_a);
  FT = upwind_flux(U, tv, ph.eps_T);
  const R lL = mixr(av[2], ph.lam), lR = mixr(av[3], ph.lam);
  const R lf = R(2) * lL * lR / (lL + lR);
  Df = lf * (tv[3] - tv[2]) * ph.ih;
}

template <typename R>
struct ScalZ {
  R a[2][Plane<3>::N];   // alpha, planes k and k + 1 (k mod 2)
  R T[2][Plane<3>::N];
  R fx[3][kZY][kZX + 1];   // [0] alpha advection, [1] T advection, [2] T conduction
  R fy[3][kZY + 1][kZX];
};

// x- or y-face (D = 0, 1) fluxes of the staged plane through the low face of
// local cell (lx, ly), global cell (i, j, k)
template <int D, typename R>
__device__ __forceinline__ void plane_face(const R* __restrict__ sa, const R* __restrict__ sT,
                                           const PhysR<R>& ph, const Geo& g,
                                           const Fields<R>& X, const FctRatios<R>& fct, bool in,
                                           int lx, int ly, int i, int j, int k, R& Fa, R& FT,
                                           R& Df) {
  using P = Plane<3>;
  R av[6], tv[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const int e = D == 0 ? P::at(lx + m - 3, ly) : P::at(lx, ly + m - 3);
    av[m] = sa[e];
    tv[m] = sT[e];
  }
  const R U = face_u<D>(X.u[D], g, in, i, j, k);
  scal_flux(av, tv, U, ph, Fa, FT, Df);
  if (fct.Rp) Fa = fct_flux<D>(fct, g, in, i, j, k, U, av[2], av[3], Fa);
}

template <typename R>
__global__ void __launch_bounds__(kZT, sizeof(R) == 4 ? 4 : 2)
    k_scalars(Geo g, PhysR<R> ph, TBC tb, Fields<R> X, Fields<R> Sn, Fields<R> Y,
              const double* __restrict__ dtp, R a, R b, R xc, R yc, R qamp, R ir2,
              FctRatios<R> fct) {
  __shared__ ScalZ<R> S;
  using P = Plane<3>;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * kZX + tx, j = blockIdx.y * kZY + ty;
  const int z0 = blockIdx.z * kZKS;
  const int z1 = min(z0 + kZKS, nz);
  const bool in = zcols_interior(g, 3);
  const bool col = i < nx && j < ny;
  const R dt = (R)dtp[0];
  const R ih = ph.ih, i2h = R(0.5) * ph.ih;
  // the Gaussian surface flux depends on (i, j) only
  R qcol = R(0);
  if (qamp != R(0) && col) {
    R dx = (R(i) + R(0.5)) * ph.h - xc, dy = (R(j) + R(0.5)) * ph.h - yc;
    if (g.bc[0] == PER) dx = dx - ph.L[0] * floor(dx / ph.L[0] + R(0.5));
    if (g.bc[1] == PER) dy = dy - ph.L[1] * floor(dy / ph.L[1] + R(0.5));
    qcol = qamp * exp(R(-2) * (dx * dx + dy * dy) * ir2);
  }
  // column window: wa[m], wt[m] = alpha, T at height k - 3 + m
  R wa[7], wt[7];
  R fz0[3] = {R(0), R(0), R(0)};   // fluxes through the low z-face of plane k
  if (col) {
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      wa[m] = col_ld<F_EVEN>(X.alpha, g, tb, i, j, z0 - 3 + m);
      wt[m] = col_ld<F_TEMP>(X.T, g, tb, i, j, z0 - 3 + m);
    }
    const R U = face_u<2>(X.u[2], g, false, i, j, z0);
    scal_flux(wa, wt, U, ph, fz0[0], fz0[1], fz0[2]);
    if (fct.Rp) fz0[0] = fct_flux<2>(fct, g, z0 >= 1, i, j, z0, U, wa[2], wa[3], fz0[0]);
  }
  // the next plane and the next column values, loaded one step ahead
  plane_async<3, F_EVEN>(S.a[z0 & 1], X.alpha, g, tb, in, z0);
  plane_async<3, F_TEMP>(S.T[z0 & 1], X.T, g, tb, in, z0);
  cp_async_commit();
  R na = R(0), nt = R(0);
  for (int k = z0; k < z1; ++k) {
    cp_async_wait_all();
    __syncthreads();
    // the other buffer held plane k - 1, last read before the previous step's
    // second barrier
    if (k + 1 < z1) {
      plane_async<3, F_EVEN>(S.a[(k + 1) & 1], X.alpha, g, tb, in, k + 1);
      plane_async<3, F_TEMP>(S.T[(k + 1) & 1], X.T, g, tb, in, k + 1);
      cp_async_commit();
      if (col) {
        na = col_ld<F_EVEN>(X.alpha, g, tb, i, j, k + 4);
        nt = col_ld<F_TEMP>(X.T, g, tb, i, j, k + 4);
      }
    }
    const R* __restrict__ sa = S.a[k & 1];
    const R* __restrict__ sT = S.T[k & 1];
    if (i <= nx && j < ny)
      plane_face<0>(sa, sT, ph, g, X, fct, in, tx, ty, i, j, k, S.fx[0][ty][tx], S.fx[1][ty][tx],
                    S.fx[2][ty][tx]);
    if (i < nx && j <= ny)
      plane_face<1>(sa, sT, ph, g, X, fct, in, tx, ty, i, j, k, S.fy[0][ty][tx], S.fy[1][ty][tx],
                    S.fy[2][ty][tx]);
    if (ty == 0) {
      // high y-faces of the tile's last row
      const int jj = blockIdx.y * kZY + kZY;
      if (i < nx && jj <= ny)
        plane_face<1>(sa, sT, ph, g, X, fct, in, tx, kZY, i, jj, k, S.fy[0][kZY][tx], S.fy[1][kZY][tx],
                      S.fy[2][kZY][tx]);
    } else if (ty == 1 && tx < kZY) {
      // high x-faces of the tile's last column, one row per lane
      const int ii = blockIdx.x * kZX + kZX, jj = blockIdx.y * kZY + tx;
      if (ii <= nx && jj < ny)
        plane_face<0>(sa, sT, ph, g, X, fct, in, kZX, tx, ii, jj, k, S.fx[0][tx][kZX],
                      S.fx[1][tx][kZX], S.fx[2][tx][kZX]);
    }
    R fz1[3] = {R(0), R(0), R(0)};   // fluxes through the face between k and k + 1
    R gx = R(0), gy = R(0);
    if (col) {
      const R U = face_u<2>(X.u[2], g, false, i, j, k + 1);
      scal_flux(wa + 1, wt + 1, U, ph, fz1[0], fz1[1], fz1[2]);
      if (fct.Rp) fz1[0] = fct_flux<2>(fct, g, k + 1 <= nz - 1, i, j, k + 1, U, wa[3], wa[4], fz1[0]);
      if (qamp != R(0)) {
        gx = (sa[P::at(tx + 1, ty)] - sa[P::at(tx - 1, ty)]) * i2h;
        gy = (sa[P::at(tx, ty + 1)] - sa[P::at(tx, ty - 1)]) * i2h;
      }
    }
    __syncthreads();
    if (col) {
      const int c = (k * ny + j) * nx + i;
      R Ra = -((S.fx[0][ty][tx + 1] - S.fx[0][ty][tx]) * ih +
               (S.fy[0][ty + 1][tx] - S.fy[0][ty][tx]) * ih + (fz1[0] - fz0[0]) * ih);
      R RT = -((S.fx[1][ty][tx + 1] - S.fx[1][ty][tx]) * ih +
               (S.fy[1][ty + 1][tx] - S.fy[1][ty][tx]) * ih + (fz1[1] - fz0[1]) * ih);
      const R Dif = (S.fx[2][ty][tx + 1] - S.fx[2][ty][tx]) * ih +
                    (S.fy[2][ty + 1][tx] - S.fy[2][ty][tx]) * ih + (fz1[2] - fz0[2]) * ih;
      const R al = wa[3];
      const R rcp = mixr(al, ph.rcp);
      RT += Dif / rcp;
      if (qamp != R(0)) {
        const R gz = (wa[4] - wa[2]) * i2h;
        const R gn = sqrt(gx * gx + gy * gy + gz * gz);
        RT += qcol * gn / rcp;
      }
      const R Ea = al + dt * Ra;
      const R ET = wt[3] + dt * RT;
      Y.alpha[c] = a * Sn.alpha[c] + b * Ea;
      Y.T[c] = a * Sn.T[c] + b * ET;
    }
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      wa[m] = wa[m + 1];
      wt[m] = wt[m + 1];
    }
    wa[6] = na;
    wt[6] = nt;
#pragma unroll
    for (int q = 0; q < 3; ++q) fz0[q] = fz1[q];
  }
}

template <typename R>
void launch_scalars(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, Fields<R> Sn,
                    Fields<R> Y, const double* dt, double a, double b, double xc, const R* fct_p,
                    const R* fct_m, cudaStream_t s) {
  // source amplitude 2P/(pi r^2) and 1/r^2 formed once on the host
  double r2 = ph.q_radius * ph.q_radius;
  double qamp = ph.q_power != 0.0 ? 2.0 * ph.q_power / (M_PI * r2) : 0.0;
  double ir2 = ph.q_power != 0.0 ? 1.0 / r2 : 0.0;
  k_scalars<R><<<zmarch_grid(g, kZKS), dim3(kZX, kZY), 0, s>>>(
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
//
// For component D on its MAC faces: conservative WENO5 advection and the
// variable-viscosity stress through the sides of the face-centred control
// volume (normal fluxes at the two cell centres along D, tangential fluxes at
// the four edges), the balanced-force CSF normal force (Eq. 4 normal term),
// the face-averaged Marangoni force and gravity.  z-marching: per plane k the
// velocity planes are staged with an x-y halo of 3 (u and v at k - 1 and k,
// w at k and k + 1) and alpha with a halo of 1 (k - 1 .. k + 1), with the cell
// viscosity mu(alpha) formed once per staged plane; the z-direction stencils
// of u, v and w are register windows of the thread's column, and the fluxes
// through the z-facing sides of a control volume are carried from one plane
// to the next.  Every flux is evaluated once: each thread takes those of its
// own faces, four warps the ones on the tile's high (or low) side.
constexpr int kZKM = 16;   // planes per CTA

template <typename R>
struct MomZ {
  R u[3][Plane<3>::N];    // u planes (m mod 3)
  R v[3][Plane<3>::N];    // v planes (m mod 3)
  R w[3][Plane<3>::N];    // w planes (m mod 3)
  R al[4][Plane<1>::N];   // alpha (m mod 4)
  R mu[3][Plane<1>::N];   // mu(alpha) (m mod 3)
  // fluxes of the current plane, [0] advective, [1] viscous
  R c0[2][kZY][kZX + 1];    // u: centre fluxes of cells x0-1 .. x0+31
  R e0y[2][kZY + 1][kZX];   // u: low y-edges of the faces, rows y0 .. y0+8
  R c1[2][kZY + 1][kZX];    // v: centre fluxes of cells y0-1 .. y0+7
  R e1x[2][kZY][kZX + 1];   // v: low x-edges of the faces, columns x0 .. x0+32
  R e2x[2][kZY][kZX + 1];   // w: low x-edges
  R e2y[2][kZY + 1][kZX];   // w: low y-edges
};

__device__ __forceinline__ int mod3(int m) { return (m % 3 + 3) % 3; }
__device__ __forceinline__ int mod4(int m) { return m & 3; }

// a velocity component at face (i, j, k) of the thread's own column: direct
// inside the domain away from the faces the boundary rule fixes
template <int C, typename R>
__device__ __forceinline__ R col_vel(const R* __restrict__ a, const Geo& g, int i, int j, int k) {
  if (point_direct<F_VEL, C>(g, i, j, k)) return __ldg(a + ((k * g.n[1] + j) * g.n[0] + i));
  return ld_vel<C>(a, g, i, j, k);
}

// a cell value at (i, j, k), any index within the stencil reach
template <int KIND, typename R>
__device__ __forceinline__ R cell_at(const R* __restrict__ a, const Geo& g, const TBC& tb, int i,
                                     int j, int k) {
  if (point_direct<KIND, 0>(g, i, j, k)) return __ldg(a + ((k * g.n[1] + j) * g.n[0] + i));
  return ld_rule<KIND, 0>(a, g, tb, i, j, k);
}

// normal flux of a component at the centre of local cell (lx, ly) along the
// in-plane axis A: WENO5 of the six faces around it with the mean of the
// cell's two faces as the advecting velocity; viscous 2 mu du/dx_A
template <int A, typename R>
__device__ __forceinline__ void mz_centre(const R* __restrict__ q, const R* __restrict__ mu,
                                          const PhysR<R>& ph, int lx, int ly, R& Fa, R& Fv) {
  using P3 = Plane<3>;
  R v[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) v[m] = q[A == 0 ? P3::at(lx + m - 2, ly) : P3::at(lx, ly + m - 2)];
  const R Uc = R(0.5) * (v[2] + v[3]);
  Fa = upwind_flux(Uc, v, ph.eps_u);
  Fv = R(2) * mu[Plane<1>::at(lx, ly)] * (v[3] - v[2]) * ph.ih;
}

// the same along z from the column window v[0..5] (faces k-2 .. k+3 of cell k)
template <typename R>
__device__ __forceinline__ void mz_centre_col(const R* v, R mu_c, const PhysR<R>& ph, R& Fa,
                                              R& Fv) {
  const R Uc = R(0.5) * (v[2] + v[3]);
  Fa = upwind_flux(Uc, v, ph.eps_u);
  Fv = R(2) * mu_c * (v[3] - v[2]) * ph.ih;
}

// tangential flux at an edge: v[0..5] the advected component at offsets -3..2
// across the edge (v[2] below, v[3] above), ut_lo / ut_hi the crossing
// component on the two faces meeting there, mue the mean viscosity of the
// four cells around the edge
template <typename R>
__device__ __forceinline__ void mz_edge(const R* v, R ut_lo, R ut_hi, R mue, const PhysR<R>& ph,
                                        R& Fa, R& Fv) {
  const R Ue = R(0.5) * (ut_lo + ut_hi);
  Fa = upwind_flux(Ue, v, ph.eps_u);
  const R dud_dt = (v[3] - v[2]) * ph.ih;
  const R dut_dd = (ut_hi - ut_lo) * ph.ih;
  Fv = mue * (dud_dt + dut_dd);
}

template <int T, typename R>
__device__ __forceinline__ void mz_gather(const R* __restrict__ q, int lx, int ly, R* v) {
  using P3 = Plane<3>;
#pragma unroll
  for (int m = 0; m < 6; ++m) v[m] = q[T == 0 ? P3::at(lx + m - 3, ly) : P3::at(lx, ly + m - 3)];
}

// u's low y-edge at face (lx, ly) of plane k
template <typename R>
__device__ __forceinline__ void mz_e0y(const R* U, const R* V, const R* mu, const PhysR<R>& ph,
                                       int lx, int ly, R* F) {
  using P3 = Plane<3>;
  using P1 = Plane<1>;
  R v[6];
  mz_gather<1>(U, lx, ly, v);
  const R mue = R(0.25) * (mu[P1::at(lx, ly)] + mu[P1::at(lx - 1, ly)] + mu[P1::at(lx, ly - 1)] +
                           mu[P1::at(lx - 1, ly - 1)]);
  mz_edge(v, V[P3::at(lx - 1, ly)], V[P3::at(lx, ly)], mue, ph, F[0], F[1]);
}

// v's low x-edge at face (lx, ly) of plane k
template <typename R>
__device__ __forceinline__ void mz_e1x(const R* U, const R* V, const R* mu, const PhysR<R>& ph,
                                       int lx, int ly, R* F) {
  using P3 = Plane<3>;
  using P1 = Plane<1>;
  R v[6];
  mz_gather<0>(V, lx, ly, v);
  const R mue = R(0.25) * (mu[P1::at(lx, ly)] + mu[P1::at(lx, ly - 1)] + mu[P1::at(lx - 1, ly)] +
                           mu[P1::at(lx - 1, ly - 1)]);
  mz_edge(v, U[P3::at(lx, ly - 1)], U[P3::at(lx, ly)], mue, ph, F[0], F[1]);
}

// w's low x-edge (T = 0) or y-edge (T = 1) at z-face (lx, ly) of height k;
// Qk, Qm: the crossing component (u or v) in planes k and k - 1
template <int T, typename R>
__device__ __forceinline__ void mz_e2(const R* W, const R* Qk, const R* Qm, const R* muk,
                                      const R* mum, const PhysR<R>& ph, int lx, int ly, R* F) {
  using P3 = Plane<3>;
  using P1 = Plane<1>;
  R v[6];
  mz_gather<T>(W, lx, ly, v);
  const int e = P1::at(lx, ly), et = T == 0 ? P1::at(lx - 1, ly) : P1::at(lx, ly - 1);
  const R mue = R(0.25) * (muk[e] + mum[e] + muk[et] + mum[et]);
  mz_edge(v, Qm[P3::at(lx, ly)], Qk[P3::at(lx, ly)], mue, ph, F[0], F[1]);
}

// u's (D = 0) or v's (D = 1) z-edge at the face column (lx, ly) between
// heights kd (below) and ku = kd + 1 (above): v[0..5] the column window at
// ku-3 .. ku+2, Wu the w plane at ku, muu / mud the viscosity at ku / kd
template <int D, typename R>
__device__ __forceinline__ void mz_ez(const R* v, const R* Wu, const R* muu, const R* mud,
                                      const PhysR<R>& ph, int lx, int ly, R* F) {
  using P3 = Plane<3>;
  using P1 = Plane<1>;
  const int e = P1::at(lx, ly), ed = D == 0 ? P1::at(lx - 1, ly) : P1::at(lx, ly - 1);
  const R mue = R(0.25) * (muu[e] + muu[ed] + mud[e] + mud[ed]);
  const int w1 = P3::at(lx, ly), w0 = D == 0 ? P3::at(lx - 1, ly) : P3::at(lx, ly - 1);
  mz_edge(v, Wu[w0], Wu[w1], mue, ph, F[0], F[1]);
}

// the forces on a D-face between cell L and cell R and the new face velocity
template <int D, typename R>
__device__ __forceinline__ void mz_update(const PhysR<R>& ph, bool conc, R A, R V, R alL, R alR,
                                          R TL, R TR, R cL, R cR, R kL, R kR, R ML, R MR, R uf,
                                          R dt, R& us, R& phi) {
  const R ih = ph.ih;
  const R rho_f = R(0.5) * (mixr(alL, ph.rho) + mixr(alR, ph.rho));
  const R sig_f = conc ? R(0.5) * (sigma_rc(TL, cL, ph) + sigma_rc(TR, cR, ph))
                       : R(0.5) * (sigma_r(TL, ph) + sigma_r(TR, ph));
  const R kap_f = R(0.5) * (kL + kR);
  const R jump = (alR - alL) * ih;
  const R fn = -sig_f * kap_f * jump;
  const R fM = R(0.5) * (ML + MR);
  us = uf + dt * (A + (V + fn + fM) / rho_f + ph.g[D]);
  phi = V + fn + fM;   // the force sum before 1/rho_f (the adjoint's density term)
}

template <typename R>
__global__ void __launch_bounds__(kZT, sizeof(R) == 4 ? 3 : 2)
    k_momentum(Geo g, PhysR<R> ph, TBC tb, Fields<R> X, const R* __restrict__ kappa,
               const R* __restrict__ M0, const R* __restrict__ M1, const R* __restrict__ M2,
               R* __restrict__ us0, R* __restrict__ us1, R* __restrict__ us2,
               const double* __restrict__ dtp, R* __restrict__ ph0, R* __restrict__ ph1,
               R* __restrict__ ph2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MomZ<R>& S = *reinterpret_cast<MomZ<R>*>(smem_raw);
  using P1 = Plane<1>;
  using P3 = Plane<3>;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * kZX + tx, j = blockIdx.y * kZY + ty;
  const int x0 = blockIdx.x * kZX, y0 = blockIdx.y * kZY;
  const int z0 = blockIdx.z * kZKM;
  const int z1 = min(z0 + kZKM, nz);
  const bool in = zcols_interior(g, 3);
  const bool col = i < nx && j < ny;
  const bool conc = X.c != nullptr;
  const R dt = (R)dtp[0];
  const R ih = ph.ih;
  // warm-up: u, v at z0-1 and z0; w at z0 and z0+1; alpha at z0-1 .. z0+1
  for (int m = z0 - 1; m <= z0; ++m) {
    stage_plane<3, F_VEL, 0>(S.u[mod3(m)], X.u[0], g, tb, in, m);
    stage_plane<3, F_VEL, 1>(S.v[mod3(m)], X.u[1], g, tb, in, m);
  }
  for (int m = z0; m <= z0 + 1; ++m) stage_plane<3, F_VEL, 2>(S.w[mod3(m)], X.u[2], g, tb, in, m);
  for (int m = z0 - 1; m <= z0 + 1; ++m) stage_plane<1, F_EVEN>(S.al[mod4(m)], X.alpha, g, tb, in, m);
  __syncthreads();
  for (int m = z0 - 1; m <= z0; ++m)
    for (int e = tx + kZX * ty; e < P1::N; e += kZT) S.mu[mod3(m)][e] = mixr(S.al[mod4(m)][e], ph.mu);
  __syncthreads();
  // column windows: after the warm-up cu[0..5] = u at heights k-2 .. k+3
  R cu[7], cv[7], cw[7];
  R ez0[2] = {R(0), R(0)}, ez1[2] = {R(0), R(0)}, cc2[2] = {R(0), R(0)};
  R TL2 = R(0), kL2 = R(0), cL2 = R(0), ML2 = R(0);   // the cell below the w-face
  if (col) {
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      cu[m] = col_vel<0>(X.u[0], g, i, j, z0 - 3 + m);
      cv[m] = col_vel<1>(X.u[1], g, i, j, z0 - 3 + m);
      cw[m] = col_vel<2>(X.u[2], g, i, j, z0 - 3 + m);
    }
    // fluxes through the z-facing sides below plane z0
    mz_ez<0>(cu, S.w[mod3(z0)], S.mu[mod3(z0)], S.mu[mod3(z0 - 1)], ph, tx, ty, ez0);
    mz_ez<1>(cv, S.w[mod3(z0)], S.mu[mod3(z0)], S.mu[mod3(z0 - 1)], ph, tx, ty, ez1);
    mz_centre_col(cw, S.mu[mod3(z0 - 1)][P1::at(tx, ty)], ph, cc2[0], cc2[1]);
    TL2 = cell_at<F_TEMP>(X.T, g, tb, i, j, z0 - 1);
    kL2 = cell_at<F_EVEN>(kappa, g, tb, i, j, z0 - 1);
    if (conc) cL2 = cell_at<F_EVEN>(X.c, g, tb, i, j, z0 - 1);
    ML2 = cell_at<F_EVEN>(M2, g, tb, i, j, z0 - 1);
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      cu[m] = cu[m + 1];
      cv[m] = cv[m + 1];
      cw[m] = cw[m + 1];
    }
  }
  R nu = R(0), nv = R(0), nw = R(0);
  for (int k = z0; k < z1; ++k) {
    cp_async_wait_all();
    __syncthreads();
    // the slots refilled here held u, v at k - 2, w at k - 1 and alpha at
    // k - 2, last read by the previous step
    if (k + 1 < z1) {
      plane_async<3, F_VEL, 0>(S.u[mod3(k + 1)], X.u[0], g, tb, in, k + 1);
      plane_async<3, F_VEL, 1>(S.v[mod3(k + 1)], X.u[1], g, tb, in, k + 1);
      plane_async<3, F_VEL, 2>(S.w[mod3(k + 2)], X.u[2], g, tb, in, k + 2);
      plane_async<1, F_EVEN>(S.al[mod4(k + 2)], X.alpha, g, tb, in, k + 2);
      cp_async_commit();
      if (col) {
        nu = col_vel<0>(X.u[0], g, i, j, k + 4);
        nv = col_vel<1>(X.u[1], g, i, j, k + 4);
        nw = col_vel<2>(X.u[2], g, i, j, k + 4);
      }
    }
    // mu of plane k + 1 (alpha k + 1 arrived with the previous step's copies)
    {
      const R* __restrict__ a1 = S.al[mod4(k + 1)];
      R* __restrict__ m1 = S.mu[mod3(k + 1)];
      for (int e = tx + kZX * ty; e < P1::N; e += kZT) m1[e] = mixr(a1[e], ph.mu);
    }
    __syncthreads();
    const R* __restrict__ Uk = S.u[mod3(k)];
    const R* __restrict__ Um = S.u[mod3(k - 1)];
    const R* __restrict__ Vk = S.v[mod3(k)];
    const R* __restrict__ Vm = S.v[mod3(k - 1)];
    const R* __restrict__ Wk = S.w[mod3(k)];
    const R* __restrict__ Wp = S.w[mod3(k + 1)];
    const R* __restrict__ mk = S.mu[mod3(k)];
    const R* __restrict__ mm = S.mu[mod3(k - 1)];
    const R* __restrict__ mp = S.mu[mod3(k + 1)];
    R F[2];
    if (col) {
      mz_centre<0>(Uk, mk, ph, tx, ty, F[0], F[1]);
      S.c0[0][ty][tx + 1] = F[0];
      S.c0[1][ty][tx + 1] = F[1];
      mz_centre<1>(Vk, mk, ph, tx, ty, F[0], F[1]);
      S.c1[0][ty + 1][tx] = F[0];
      S.c1[1][ty + 1][tx] = F[1];
    }
    if (i < nx && j <= ny) {
      mz_e0y(Uk, Vk, mk, ph, tx, ty, F);
      S.e0y[0][ty][tx] = F[0];
      S.e0y[1][ty][tx] = F[1];
      mz_e2<1>(Wk, Vk, Vm, mk, mm, ph, tx, ty, F);
      S.e2y[0][ty][tx] = F[0];
      S.e2y[1][ty][tx] = F[1];
    }
    if (i <= nx && j < ny) {
      mz_e1x(Uk, Vk, mk, ph, tx, ty, F);
      S.e1x[0][ty][tx] = F[0];
      S.e1x[1][ty][tx] = F[1];
      mz_e2<0>(Wk, Uk, Um, mk, mm, ph, tx, ty, F);
      S.e2x[0][ty][tx] = F[0];
      S.e2x[1][ty][tx] = F[1];
    }
    // the tile's high (or low) sides
    if (ty == 0) {
      if (i < nx && y0 + kZY <= ny) {
        mz_e0y(Uk, Vk, mk, ph, tx, kZY, F);
        S.e0y[0][kZY][tx] = F[0];
        S.e0y[1][kZY][tx] = F[1];
      }
    } else if (ty == 1) {
      if (i < nx) {
        mz_centre<1>(Vk, mk, ph, tx, -1, F[0], F[1]);
        S.c1[0][0][tx] = F[0];
        S.c1[1][0][tx] = F[1];
      }
    } else if (ty == 2) {
      if (i < nx && y0 + kZY <= ny) {
        mz_e2<1>(Wk, Vk, Vm, mk, mm, ph, tx, kZY, F);
        S.e2y[0][kZY][tx] = F[0];
        S.e2y[1][kZY][tx] = F[1];
      }
    } else if (ty == 3) {
      const int r = tx & 7, q = tx >> 3;
      if (q == 0) {
        if (y0 + r < ny) {
          mz_centre<0>(Uk, mk, ph, -1, r, F[0], F[1]);
          S.c0[0][r][0] = F[0];
          S.c0[1][r][0] = F[1];
        }
      } else if (q == 1) {
        if (x0 + kZX <= nx && y0 + r < ny) {
          mz_e1x(Uk, Vk, mk, ph, kZX, r, F);
          S.e1x[0][r][kZX] = F[0];
          S.e1x[1][r][kZX] = F[1];
        }
      } else if (q == 2) {
        if (x0 + kZX <= nx && y0 + r < ny) {
          mz_e2<0>(Wk, Uk, Um, mk, mm, ph, kZX, r, F);
          S.e2x[0][r][kZX] = F[0];
          S.e2x[1][r][kZX] = F[1];
        }
      }
    }
    // z-direction fluxes above plane k
    R ez0h[2] = {R(0), R(0)}, ez1h[2] = {R(0), R(0)}, cc2h[2] = {R(0), R(0)};
    if (col) {
      mz_ez<0>(cu, Wp, mp, mk, ph, tx, ty, ez0h);
      mz_ez<1>(cv, Wp, mp, mk, ph, tx, ty, ez1h);
      mz_centre_col(cw, mk[P1::at(tx, ty)], ph, cc2h[0], cc2h[1]);
    }
    __syncthreads();
    if (col) {
      const int c = (k * ny + j) * nx + i;
      const R* __restrict__ ak = S.al[mod4(k)];
      const R* __restrict__ am = S.al[mod4(k - 1)];
      const int e1 = P1::at(tx, ty), e3 = P3::at(tx, ty);
      const R alR = ak[e1], TR = X.T[c], kR = kappa[c], cR = conc ? X.c[c] : R(0);
      R us, phv;
      // u on the x-face (i, j, k)
      if (g.bc[0] == WALL && i == 0) {
        us0[c] = R(0);
        if (ph0) ph0[c] = R(0);
      } else {
        R A = R(0) - (S.c0[0][ty][tx + 1] - S.c0[0][ty][tx]) * ih;
        R V = R(0) + (S.c0[1][ty][tx + 1] - S.c0[1][ty][tx]) * ih;
        A -= (S.e0y[0][ty + 1][tx] - S.e0y[0][ty][tx]) * ih;
        V += (S.e0y[1][ty + 1][tx] - S.e0y[1][ty][tx]) * ih;
        A -= (ez0h[0] - ez0[0]) * ih;
        V += (ez0h[1] - ez0[1]) * ih;
        const bool d = i >= 1;
        const R TL = d ? X.T[c - 1] : ld_T(X.T, g, tb, i - 1, j, k);
        const R kL = d ? kappa[c - 1] : ld_even(kappa, g, i - 1, j, k);
        const R cL = conc ? (d ? X.c[c - 1] : ld_even(X.c, g, i - 1, j, k)) : R(0);
        const R ML = d ? M0[c - 1] : ld_even(M0, g, i - 1, j, k);
        mz_update<0>(ph, conc, A, V, ak[e1 - 1], alR, TL, TR, cL, cR, kL, kR, ML, M0[c], Uk[e3],
                     dt, us, phv);
        us0[c] = us;
        if (ph0) ph0[c] = phv;
      }
      // v on the y-face (i, j, k)
      if (g.bc[1] == WALL && j == 0) {
        us1[c] = R(0);
        if (ph1) ph1[c] = R(0);
      } else {
        R A = R(0) - (S.c1[0][ty + 1][tx] - S.c1[0][ty][tx]) * ih;
        R V = R(0) + (S.c1[1][ty + 1][tx] - S.c1[1][ty][tx]) * ih;
        A -= (S.e1x[0][ty][tx + 1] - S.e1x[0][ty][tx]) * ih;
        V += (S.e1x[1][ty][tx + 1] - S.e1x[1][ty][tx]) * ih;
        A -= (ez1h[0] - ez1[0]) * ih;
        V += (ez1h[1] - ez1[1]) * ih;
        const bool d = j >= 1;
        const R TL = d ? X.T[c - nx] : ld_T(X.T, g, tb, i, j - 1, k);
        const R kL = d ? kappa[c - nx] : ld_even(kappa, g, i, j - 1, k);
        const R cL = conc ? (d ? X.c[c - nx] : ld_even(X.c, g, i, j - 1, k)) : R(0);
        const R ML = d ? M1[c - nx] : ld_even(M1, g, i, j - 1, k);
        mz_update<1>(ph, conc, A, V, ak[e1 - P1::PX], alR, TL, TR, cL, cR, kL, kR, ML, M1[c],
                     Vk[e3], dt, us, phv);
        us1[c] = us;
        if (ph1) ph1[c] = phv;
      }
      // w on the z-face (i, j, k)
      const R M2R = M2[c];
      if (g.bc[2] == WALL && k == 0) {
        us2[c] = R(0);
        if (ph2) ph2[c] = R(0);
      } else {
        R A = R(0) - (cc2h[0] - cc2[0]) * ih;
        R V = R(0) + (cc2h[1] - cc2[1]) * ih;
        A -= (S.e2x[0][ty][tx + 1] - S.e2x[0][ty][tx]) * ih;
        V += (S.e2x[1][ty][tx + 1] - S.e2x[1][ty][tx]) * ih;
        A -= (S.e2y[0][ty + 1][tx] - S.e2y[0][ty][tx]) * ih;
        V += (S.e2y[1][ty + 1][tx] - S.e2y[1][ty][tx]) * ih;
        mz_update<2>(ph, conc, A, V, am[e1], alR, TL2, TR, cL2, cR, kL2, kR, ML2, M2R, Wk[e3], dt,
                     us, phv);
        us2[c] = us;
        if (ph2) ph2[c] = phv;
      }
      TL2 = TR;
      kL2 = kR;
      cL2 = cR;
      ML2 = M2R;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      ez0[q] = ez0h[q];
      ez1[q] = ez1h[q];
      cc2[q] = cc2h[q];
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      cu[m] = cu[m + 1];
      cv[m] = cv[m + 1];
      cw[m] = cw[m + 1];
    }
    cu[5] = nu;
    cv[5] = nv;
    cw[5] = nw;
  }
}

template <typename R>
void launch_momentum(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, const R* kappa,
                     const R* M0, const R* M1, const R* M2, R* us0, R* us1, R* us2,
                     const double* dt, cudaStream_t s, R* const* phi) {
  const int smem = (int)sizeof(MomZ<R>);
  cudaFuncSetAttribute(k_momentum<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_momentum<R><<<zmarch_grid(g, kZKM), dim3(kZX, kZY), smem, s>>>(
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
