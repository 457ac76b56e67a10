// Geometric multigrid for the density-weighted pressure operator
//   (L x)_c = sum_faces beta_f (x_c - x_nb) / h_d^2
// and the deterministic reductions the solver and the step use.
//   k_gs                red-black Gauss-Seidel sweep of one colour (i+j+k mod 2)
//   k_residual_restrict residual on the fine level, mean over the children
//   k_prolong           piecewise-constant prolongation, added to the fine level
//   k_gs_prolong        the first sweep after the correction with the prolongation folded in
//   k_gs_zero, k_gs_addp the first sweep from x = 0 and the last one adding x to p (mixed form)
//   k_beta_coarsen      coarse face beta = mean of the fine faces it covers
//   k_coarse_cg         conjugate gradients on the coarsest level, one CTA
//   k_residual_norm2    ||b - L x||^2 partial sums
//   k_residual64        mixed form: r = b - L p in double, stored as float
// The paper names no linear solver; this is the reading used throughout the
// library: V(pre, post) cycles, red first before and black first after the
// coarse correction so that the cycle is a symmetric operator.
#include "fvm_device.cuh"

namespace fvm {

// three float weights passed by value to a kernel
struct W3 {
  float w[3];
};

static inline unsigned grid1d(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block sum, result broadcast to every thread
__device__ double block_sum_all(double v, double* sh) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    double t = (lane < nw) ? sh[lane] : 0.0;
    t = warp_sum_d(t);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_sum_field(const T* __restrict__ a, long long n, int squares,
                            double* __restrict__ partial) {
  __shared__ double sh[33];
  double acc = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double v = (double)a[c];
    acc += squares ? v * v : v;
  }
  double s = block_sum_all(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nparts,
                               double* __restrict__ out) {
  __shared__ double sh[33];
  double acc = 0.0;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc += partial[q];
  double s = block_sum_all(acc, sh);
  if (threadIdx.x == 0) *out = s;
}

void launch_sum_partials(const double* partial, int nparts, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 1024, 0, s>>>(partial, nparts, out);
}

template <typename T>
void launch_sum_field(const T* a, long long n, bool squares, double* partial, double* out,
                      cudaStream_t s) {
  k_sum_field<T><<<kRedBlocks, 256, 0, s>>>(a, n, squares ? 1 : 0, partial);
  launch_sum_partials(partial, kRedBlocks, out, s);
}

// a -= sum / n, with the mean formed once per block (one double division per
// block instead of per element)
__global__ void k_sub_mean(double* __restrict__ a, long long n, const double* __restrict__ sum) {
  __shared__ double mean;
  if (threadIdx.x == 0) mean = (*sum) / (double)n;
  __syncthreads();
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= n) return;
  a[c] = a[c] - mean;
}

void launch_sub_mean(double* a, long long n, const double* sum, cudaStream_t s) {
  k_sub_mean<<<grid1d(n, 256), 256, 0, s>>>(a, n, sum);
}

template <typename T>
__global__ void k_zero(T* __restrict__ a, long long n) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) a[c] = T(0);
}

template <typename T>
void launch_zero(T* a, long long n, cudaStream_t s) {
  k_zero<T><<<grid1d(n, 256), 256, 0, s>>>(a, n);
}

// ---------------------------------------------------------------------------
// operator pieces on a level
template <typename T>
struct OpNb {
  int lo[3], hi[3];
  T blo[3], bhi[3];
};

template <typename T>
__device__ __forceinline__ void neighbours(const MGLevel<T>& L, int i, int j, int k, int c,
                                           OpNb<T>& nb) {
  const Geo& g = L.geo;
  const int idx[3] = {i, j, k};
  const int st[3] = {1, g.n[0], g.n[0] * g.n[1]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int n = g.n[d];
    const int lo = idx[d] == 0 ? c + (n - 1) * st[d] : c - st[d];
    const int hi = idx[d] == n - 1 ? c - (n - 1) * st[d] : c + st[d];
    nb.lo[d] = lo;
    nb.hi[d] = hi;
    nb.blo[d] = L.beta[d][c];
    nb.bhi[d] = (g.bc[d] == WALL && idx[d] == n - 1) ? T(0) : L.beta[d][hi];
  }
}

template <typename T, typename X>
__device__ __forceinline__ X apply_L_at(const MGLevel<T>& L, const X* __restrict__ x, int c,
                                        const OpNb<T>& nb) {
  const Geo& g = L.geo;
  X xc = x[c];
  X out = X(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (g.n[d] == 1) continue;
    out += ((X)nb.blo[d] * (xc - x[nb.lo[d]]) + (X)nb.bhi[d] * (xc - x[nb.hi[d]])) * (X)L.w[d];
  }
  return out;
}

__device__ __forceinline__ void decode_lv(const Geo& g, long long c, int& i, int& j, int& k) {
  const int cc = (int)c;
  const int q = cc / g.n[0];
  i = cc - q * g.n[0];
  k = q / g.n[1];
  j = q - k * g.n[1];
}

// ---------------------------------------------------------------------------
// Gauss-Seidel value of one cell from its right-hand side, the face betas
// and the neighbour values on the low and high side of each axis (axes of
// one cell carry no coupling)
template <typename T>
__device__ __forceinline__ T gs_formula(const Geo& g, const T* w, T b, const T* blo, const T* bhi,
                                        const T* xlo, const T* xhi) {
  T num = b;
  T den = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (g.n[d] == 1) continue;
    num += (blo[d] * xlo[d] + bhi[d] * xhi[d]) * w[d];
    den += (blo[d] + bhi[d]) * w[d];
  }
  return num / den;
}

// Gauss-Seidel update of one cell (its colour's neighbours are fixed)
template <typename T>
__device__ __forceinline__ void gs_point(const MGLevel<T>& L, int i, int j, int k) {
  const Geo& g = L.geo;
  const int c = (k * g.n[1] + j) * g.n[0] + i;
  OpNb<T> nb;
  neighbours(L, i, j, k, c, nb);
  T xlo[3], xhi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xlo[d] = L.x[nb.lo[d]];
    xhi[d] = L.x[nb.hi[d]];
  }
  L.x[c] = gs_formula(g, L.w, L.b[c], nb.blo, nb.bhi, xlo, xhi);
}

// gate (optional): the sweep does nothing once *gate >= gate_min (the FP64
// solve graph skips the first sweep of every cycle after the first, which
// would repeat the previous cycle's last sweep)
template <typename T>
__global__ void k_gs(MGLevel<T> L, int colour, const int* __restrict__ gate, int gate_min) {
  if (gate && *gate >= gate_min) return;
  const Geo& g = L.geo;
  const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (j >= g.n[1] || k >= g.n[2]) return;
  const int i = 2 * i2 + ((colour + j + k) & 1);
  if (i >= g.n[0]) return;
  gs_point(L, i, j, k);
}

template <typename T>
void launch_gs(const MGLevel<T>& L, int colour, cudaStream_t s, const int* gate, int gate_min) {
  const int hx = (L.geo.n[0] + 1) / 2;
  dim3 bs(32, 4, 2);
  dim3 gs((hx + 31) / 32, (L.geo.n[1] + 3) / 4, (L.geo.n[2] + 1) / 2);
  k_gs<T><<<gs, bs, 0, s>>>(L, colour, gate, gate_min);
}

// coarse b = mean over children of (b - L x) on the fine level; coarse x = 0
template <typename T>
__device__ __forceinline__ void restrict_point(const MGLevel<T>& F, const MGLevel<T>& C, int I,
                                               int J, int K) {
  const long long cc = lin(C.geo, I, J, K);
  T acc = T(0);
  int cnt = 0;
  for (int dz = 0; dz < F.f[2]; ++dz)
    for (int dy = 0; dy < F.f[1]; ++dy)
      for (int dx = 0; dx < F.f[0]; ++dx) {
        int i = I * F.f[0] + dx, j = J * F.f[1] + dy, k = K * F.f[2] + dz;
        const int c = (k * F.geo.n[1] + j) * F.geo.n[0] + i;
        OpNb<T> nb;
        neighbours(F, i, j, k, c, nb);
        acc += F.b[c] - apply_L_at<T, T>(F, F.x, c, nb);
        ++cnt;
      }
  C.b[cc] = acc / (T)cnt;
  C.x[cc] = T(0);
}

template <typename T>
__device__ __forceinline__ void restrict_point(const MGLevel<T>& F, const MGLevel<T>& C,
                                               long long cc) {
  int I, J, K;
  decode_lv(C.geo, cc, I, J, K);
  restrict_point(F, C, I, J, K);
}

// one thread per coarse cell on a 3D grid (no index division per thread)
template <typename T>
__global__ void k_residual_restrict(MGLevel<T> F, MGLevel<T> C, int sweep) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  if (I >= C.geo.n[0] || J >= C.geo.n[1] || K >= C.geo.n[2]) return;
  restrict_point(F, C, I, J, K);
  if (sweep && ((I + J + K) & 1) == 0) {
    // the coarse level's first sweep (colour 0 from x = 0) needs only the
    // cell's own right-hand side: taken here, with k_gs's arithmetic
    const int cc = (int)lin(C.geo, I, J, K);
    OpNb<T> nb;
    neighbours(C, I, J, K, cc, nb);
    const T z[3] = {T(0), T(0), T(0)};
    C.x[cc] = gs_formula(C.geo, C.w, C.b[cc], nb.blo, nb.bhi, z, z);
  }
}

// sweep: also take the coarse level's first Gauss-Seidel sweep from x = 0
template <typename T>
void launch_residual_restrict(const MGLevel<T>& F, const MGLevel<T>& C, cudaStream_t s, bool sweep) {
  const dim3 bs(32, 4, 2);
  const dim3 gs((C.geo.n[0] + 31) / 32, (C.geo.n[1] + 3) / 4, (C.geo.n[2] + 1) / 2);
  k_residual_restrict<T><<<gs, bs, 0, s>>>(F, C, sweep ? 1 : 0);
}

// the coarsening factor of an axis is 1 or 2
__device__ __forceinline__ int coarse_index(int i, int f) { return f == 2 ? (i >> 1) : i; }

template <typename T>
__device__ __forceinline__ void prolong_point(const MGLevel<T>& F, const MGLevel<T>& C, int i,
                                              int j, int k) {
  const long long c = lin(F.geo, i, j, k);
  const long long p = lin(C.geo, coarse_index(i, F.f[0]), coarse_index(j, F.f[1]),
                          coarse_index(k, F.f[2]));
  F.x[c] = F.x[c] + C.x[p];
}

template <typename T>
__device__ __forceinline__ void prolong_point(const MGLevel<T>& F, const MGLevel<T>& C,
                                              long long c) {
  int i, j, k;
  decode_lv(F.geo, c, i, j, k);
  prolong_point(F, C, i, j, k);
}

// one thread per fine cell on a 3D grid (no index division per thread)
template <typename T>
__global__ void k_prolong(MGLevel<T> F, MGLevel<T> C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= F.geo.n[0] || j >= F.geo.n[1] || k >= F.geo.n[2]) return;
  prolong_point(F, C, i, j, k);
}

template <typename T>
void launch_prolong(const MGLevel<T>& F, const MGLevel<T>& C, cudaStream_t s) {
  const dim3 bs(32, 4, 2);
  const dim3 gs((F.geo.n[0] + 31) / 32, (F.geo.n[1] + 3) / 4, (F.geo.n[2] + 1) / 2);
  k_prolong<T><<<gs, bs, 0, s>>>(F, C);
}

// The first colour sweep after the coarse correction with the
// piecewise-constant prolongation folded in.  A sweep of one colour reads
// only the other colour, so it takes those cells' values plus the coarse
// correction of their parent cells on the fly; the other colour's stored
// values are then overwritten by the next sweep without being read.  The
// pair of sweeps therefore leaves x as k_prolong followed by two k_gs
// launches would, bit for bit, without the prolongation's pass over x.
template <typename T>
__global__ void k_gs_prolong(MGLevel<T> F, MGLevel<T> C, int colour) {
  const Geo& g = F.geo;
  const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (j >= g.n[1] || k >= g.n[2]) return;
  const int i = 2 * i2 + ((colour + j + k) & 1);
  if (i >= g.n[0]) return;
  const int c = (k * g.n[1] + j) * g.n[0] + i;
  OpNb<T> nb;
  neighbours(F, i, j, k, c, nb);
  const int idx[3] = {i, j, k};
  T xlo[3], xhi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int n = g.n[d];
    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
    lo[d] = idx[d] == 0 ? n - 1 : idx[d] - 1;
    hi[d] = idx[d] == n - 1 ? 0 : idx[d] + 1;
    const long long pl = lin(C.geo, coarse_index(lo[0], F.f[0]), coarse_index(lo[1], F.f[1]),
                             coarse_index(lo[2], F.f[2]));
    const long long ph = lin(C.geo, coarse_index(hi[0], F.f[0]), coarse_index(hi[1], F.f[1]),
                             coarse_index(hi[2], F.f[2]));
    xlo[d] = F.x[nb.lo[d]] + C.x[pl];
    xhi[d] = F.x[nb.hi[d]] + C.x[ph];
  }
  F.x[c] = gs_formula(g, F.w, F.b[c], nb.blo, nb.bhi, xlo, xhi);
}

// The first sweep of a solve that starts from x = 0 (the mixed form's inner
// correction): the other colour's values are 0, so the swept cells take
// gs_formula with zero neighbours and the cells of the other colour are set
// to 0 by the same thread (the pair 2 i2, 2 i2 + 1 of its row), which
// replaces zeroing x in a pass of its own.
template <typename T>
__global__ void k_gs_zero(MGLevel<T> L, int colour) {
  const Geo& g = L.geo;
  const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (j >= g.n[1] || k >= g.n[2]) return;
  const int i = 2 * i2 + ((colour + j + k) & 1), io = i ^ 1;
  const int row = (k * g.n[1] + j) * g.n[0];
  if (io < g.n[0]) L.x[row + io] = T(0);
  if (i >= g.n[0]) return;
  OpNb<T> nb;
  neighbours(L, i, j, k, row + i, nb);
  const T z[3] = {T(0), T(0), T(0)};
  L.x[row + i] = gs_formula(g, L.w, L.b[row + i], nb.blo, nb.bhi, z, z);
}

// The last sweep of the mixed form's inner correction with p += e folded in:
// the thread adds the new value of its cell and the final value of the other
// colour's cell beside it (not written in this sweep) to the double p.  The
// correction e itself is not stored again; the next refinement starts it
// from 0.
__global__ void k_gs_addp(MGLevel<float> L, int colour, double* __restrict__ p) {
  const Geo& g = L.geo;
  const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (j >= g.n[1] || k >= g.n[2]) return;
  const int i = 2 * i2 + ((colour + j + k) & 1), io = i ^ 1;
  const int row = (k * g.n[1] + j) * g.n[0];
  if (io < g.n[0]) p[row + io] = p[row + io] + (double)L.x[row + io];
  if (i >= g.n[0]) return;
  OpNb<float> nb;
  neighbours(L, i, j, k, row + i, nb);
  float xlo[3], xhi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xlo[d] = L.x[nb.lo[d]];
    xhi[d] = L.x[nb.hi[d]];
  }
  const float e = gs_formula(g, L.w, L.b[row + i], nb.blo, nb.bhi, xlo, xhi);
  p[row + i] = p[row + i] + (double)e;
}

template <typename T>
void launch_gs_zero(const MGLevel<T>& L, int colour, cudaStream_t s) {
  const int hx = (L.geo.n[0] + 1) / 2;
  dim3 bs(32, 4, 2);
  dim3 gs((hx + 31) / 32, (L.geo.n[1] + 3) / 4, (L.geo.n[2] + 1) / 2);
  k_gs_zero<T><<<gs, bs, 0, s>>>(L, colour);
}

void launch_gs_addp(const MGLevel<float>& L, int colour, double* p, cudaStream_t s) {
  const int hx = (L.geo.n[0] + 1) / 2;
  dim3 bs(32, 4, 2);
  dim3 gs((hx + 31) / 32, (L.geo.n[1] + 3) / 4, (L.geo.n[2] + 1) / 2);
  k_gs_addp<<<gs, bs, 0, s>>>(L, colour, p);
}

template <typename T>
void launch_gs_prolong(const MGLevel<T>& F, const MGLevel<T>& C, int colour, cudaStream_t s) {
  const int hx = (F.geo.n[0] + 1) / 2;
  dim3 bs(32, 4, 2);
  dim3 gs((hx + 31) / 32, (F.geo.n[1] + 3) / 4, (F.geo.n[2] + 1) / 2);
  k_gs_prolong<T><<<gs, bs, 0, s>>>(F, C, colour);
}

template <typename T>
__global__ void k_beta_coarsen(MGLevel<T> F, MGLevel<T> C) {
  long long cc = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cc >= C.geo.N) return;
  int I, J, K;
  decode_lv(C.geo, cc, I, J, K);
  int base[3] = {I * F.f[0], J * F.f[1], K * F.f[2]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int cnt[3] = {F.f[0], F.f[1], F.f[2]};
    cnt[d] = 1;
    T acc = T(0);
    for (int dz = 0; dz < cnt[2]; ++dz)
      for (int dy = 0; dy < cnt[1]; ++dy)
        for (int dx = 0; dx < cnt[0]; ++dx)
          acc += F.beta[d][lin(F.geo, base[0] + dx, base[1] + dy, base[2] + dz)];
    C.beta[d][cc] = acc / (T)(cnt[0] * cnt[1] * cnt[2]);
  }
}

template <typename T>
void launch_beta_coarsen(const MGLevel<T>& F, const MGLevel<T>& C, cudaStream_t s) {
  k_beta_coarsen<T><<<grid1d(C.geo.N, 128), 128, 0, s>>>(F, C);
}

// ---------------------------------------------------------------------------
// conjugate gradients on the coarsest level in one CTA: mean-free rhs,
// x0 = 0, stop at ||r|| <= rtol ||b|| or on breakdown, mean-free result.
// The vectors are double in both precisions.
template <typename T>
__device__ void coarse_cg_block(const MGLevel<T>& L, double* __restrict__ r,
                                double* __restrict__ dd, double* __restrict__ Ad, double rtol,
                                int maxit, double* sh) {
  const Geo& g = L.geo;
  const int N = (int)g.N;
  double acc = 0.0;
  for (int c = threadIdx.x; c < N; c += blockDim.x) acc += (double)L.b[c];
  double mean = block_sum_all(acc, sh) / (double)N;
  acc = 0.0;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    double v = (double)L.b[c] - mean;
    r[c] = v;
    dd[c] = v;
    Ad[c] = 0.0;      // Ad doubles as the solution accumulator x until the end
    acc += v * v;
  }
  double rr = block_sum_all(acc, sh);
  double bn = sqrt(rr);
  double* x = Ad + N;
  for (int c = threadIdx.x; c < N; c += blockDim.x) x[c] = 0.0;
  if (bn != 0.0) {
    for (int it = 0; it < maxit; ++it) {
      if (sqrt(rr) <= rtol * bn) break;
      __syncthreads();
      acc = 0.0;
      for (int c = threadIdx.x; c < N; c += blockDim.x) {
        int i, j, k;
        decode_lv(g, c, i, j, k);
        OpNb<T> nb;
        neighbours(L, i, j, k, c, nb);
        double a = apply_L_at<T, double>(L, dd, c, nb);
        Ad[c] = a;
        acc += dd[c] * a;
      }
      double pAp = block_sum_all(acc, sh);
      if (!(pAp > 0.0)) break;   // breakdown (exhausted search direction or rounding)
      double a = rr / pAp;
      acc = 0.0;
      for (int c = threadIdx.x; c < N; c += blockDim.x) {
        x[c] = x[c] + a * dd[c];
        double rv = r[c] - a * Ad[c];
        r[c] = rv;
        acc += rv * rv;
      }
      double rr_new = block_sum_all(acc, sh);
      double beta = rr_new / rr;
      for (int c = threadIdx.x; c < N; c += blockDim.x) dd[c] = r[c] + beta * dd[c];
      rr = rr_new;
    }
  }
  __syncthreads();
  acc = 0.0;
  for (int c = threadIdx.x; c < N; c += blockDim.x) acc += x[c];
  double xm = block_sum_all(acc, sh) / (double)N;
  for (int c = threadIdx.x; c < N; c += blockDim.x) L.x[c] = (T)(x[c] - xm);
}

// The coarsest-level CG of a single CTA is bound by the latency of every
// iteration's dependent phases (operator, two reductions, updates); when the
// level is small its vectors and face coefficients are kept in shared
// memory instead of global memory (the same arithmetic in the same order).
constexpr int kCgSmemCells = 640;
struct CgSmem {
  double v[4][kCgSmemCells];   // r, d, Ad, x
  double beta[3][kCgSmemCells];
};

template <typename T>
__device__ void coarse_cg_dispatch(const MGLevel<T>& L, double* r, double* dd, double* Ad,
                                   double rtol, int maxit, double* sh, CgSmem& cs) {
  const int N = (int)L.geo.N;
  if (N > kCgSmemCells || sizeof(T) > sizeof(double)) {
    coarse_cg_block(L, r, dd, Ad, rtol, maxit, sh);
    return;
  }
  // face coefficients staged in the level's precision T; the operator then
  // reads them through a copy of the level whose beta points to them
  T* bs = reinterpret_cast<T*>(&cs.beta[0][0]);
  MGLevel<T> S = L;
  for (int q = 0; q < 3; ++q) {
    S.beta[q] = bs + q * kCgSmemCells;
    for (int c = threadIdx.x; c < N; c += blockDim.x) S.beta[q][c] = L.beta[q][c];
  }
  __syncthreads();
  coarse_cg_block(S, cs.v[0], cs.v[1], cs.v[2], rtol, maxit, sh);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cg(MGLevel<T> L, double* __restrict__ r,
                                                    double* __restrict__ dd,
                                                    double* __restrict__ Ad, double rtol,
                                                    int maxit) {
  __shared__ double sh[33];
  __shared__ CgSmem cs;
  coarse_cg_dispatch(L, r, dd, Ad, rtol, maxit, sh, cs);
}

// The coarse tail of a V-cycle in one CTA: levels small enough that a kernel
// launch per sweep costs more than the sweep.  The same point updates as the
// per-level kernels, in the same order of phases (pre-sweeps red first,
// residual restriction, ..., CG on the coarsest level, ..., prolongation,
// post-sweeps black first), separated by block barriers; within one colour
// sweep (and within restriction and prolongation) the points are
// independent, so the result equals that of the per-level kernels bit for bit.
// one colour sweep of a tail level by the CTA: thread t takes the t-th cell
// of the colour (rows of ceil(nx/2) such cells); the row and plane indices
// come from float reciprocals, exact for the at most 4096 cells of a tail
// level, instead of integer divisions
template <typename T>
__device__ __forceinline__ void tail_colour(const MGLevel<T>& L, int col) {
  const Geo& g = L.geo;
  const int hx = (g.n[0] + 1) >> 1;
  const int half = hx * g.n[1] * g.n[2];
  const float ihx = 1.0f / (float)hx, iny = 1.0f / (float)g.n[1];
  for (int t = threadIdx.x; t < half; t += blockDim.x) {
    const int q = (int)(((float)t + 0.5f) * ihx);   // row j + ny k
    const int i2 = t - q * hx;
    const int k = (int)(((float)q + 0.5f) * iny);
    const int j = q - k * g.n[1];
    const int i = 2 * i2 + ((col + j + k) & 1);
    if (i < g.n[0]) gs_point(L, i, j, k);
  }
}

template <typename T>
__device__ void tail_body(const MGLevel<T>* Ls, int nl, double* r, double* d, double* Ad,
                          double rtol, int maxit, int pre, int post, double* sh, CgSmem& cs) {
  const int last = nl - 1;
  for (int l = 0; l < last; ++l) {
    const MGLevel<T>& L = Ls[l];
    for (int it = 0; it < pre; ++it)
      for (int col = 0; col < 2; ++col) {
        tail_colour(L, col);
        __syncthreads();
      }
    for (int cc = threadIdx.x; cc < (int)Ls[l + 1].geo.N; cc += blockDim.x)
      restrict_point(L, Ls[l + 1], cc);
    __syncthreads();
  }
  coarse_cg_dispatch(Ls[last], r, d, Ad, rtol, maxit, sh, cs);
  __syncthreads();
  for (int l = last - 1; l >= 0; --l) {
    const MGLevel<T>& L = Ls[l];
    const Geo& g = L.geo;
    for (int c = threadIdx.x; c < (int)g.N; c += blockDim.x) prolong_point(L, Ls[l + 1], c);
    __syncthreads();
    for (int it = 0; it < post; ++it)
      for (int col = 0; col < 2; ++col) {
        tail_colour(L, 1 - col);
        __syncthreads();
      }
  }
}

// staged: the tail levels' x, b and betas are copied into dynamic shared
// memory first (x and b of the top level, the betas of every level; the
// lower levels' x and b are set by the restrictions inside the tail), the
// tail runs on those copies, and the top level's x is copied back for the
// prolongation.  The arithmetic is the same as on the global arrays; only the
// latency of each sweep's loads changes.
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_tail(TailArgs<T> A, int staged) {
  __shared__ double sh[33];
  __shared__ CgSmem cs;
  extern __shared__ __align__(16) unsigned char tail_smem[];
  if (!staged) {
    tail_body(A.L, A.nl, A.r, A.d, A.Ad, A.rtol, A.maxit, A.pre, A.post, sh, cs);
    return;
  }
  MGLevel<T> L[kTailLevels];
  T* base = reinterpret_cast<T*>(tail_smem);
  for (int q = 0; q < A.nl; ++q) {
    L[q] = A.L[q];
    const int n = (int)L[q].geo.N;
    L[q].x = base;
    L[q].b = base + n;
    for (int d = 0; d < 3; ++d) L[q].beta[d] = base + (2 + d) * n;
    base += 5 * n;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      for (int d = 0; d < 3; ++d) L[q].beta[d][c] = A.L[q].beta[d][c];
      if (q == 0) {
        L[0].x[c] = A.L[0].x[c];
        L[0].b[c] = A.L[0].b[c];
      }
    }
  }
  __syncthreads();
  tail_body(L, A.nl, A.r, A.d, A.Ad, A.rtol, A.maxit, A.pre, A.post, sh, cs);
  __syncthreads();
  for (int c = threadIdx.x; c < (int)L[0].geo.N; c += blockDim.x) A.L[0].x[c] = L[0].x[c];
}

template <typename T>
void launch_coarse_tail(const TailArgs<T>& A, cudaStream_t s) {
  // stage the levels of the FP64 form when they fit beside the kernel's
  // static shared memory (the float tail was slower staged, 112 -> 124 us per
  // call at 256^3, and reads the global arrays)
  size_t bytes = 0;
  for (int q = 0; q < A.nl; ++q) bytes += 5 * (size_t)A.L[q].geo.N * sizeof(T);
  const size_t limit = 227 * 1024 - sizeof(CgSmem) - 33 * sizeof(double) - 1024;
  const bool staged = sizeof(T) == sizeof(double) && bytes <= limit;
  if (staged)
    cudaFuncSetAttribute(k_coarse_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_coarse_tail<T><<<1, 1024, staged ? bytes : 0, s>>>(A, staged ? 1 : 0);
}

template <typename T>
void launch_coarse_cg(const MGLevel<T>& L, double* r, double* d, double* Ad, double rtol,
                      int maxit, cudaStream_t s) {
  k_coarse_cg<T><<<1, 1024, 0, s>>>(L, r, d, Ad, rtol, maxit);
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_residual_norm2(MGLevel<T> L, double* __restrict__ partial) {
  __shared__ double sh[33];
  double acc = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < L.geo.N;
       c += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode_lv(L.geo, c, i, j, k);
    OpNb<T> nb;
    neighbours(L, i, j, k, (int)c, nb);
    double r = (double)(L.b[c] - apply_L_at<T, T>(L, L.x, (int)c, nb));
    acc += r * r;
  }
  double s = block_sum_all(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename T>
void launch_residual_norm2(const MGLevel<T>& L, double* partial, double* out, cudaStream_t s) {
  k_residual_norm2<T><<<kRedBlocks, 256, 0, s>>>(L, partial);
  launch_sum_partials(partial, kRedBlocks, out, s);
}

// float -> double for a finite beta >= 0 (normal or zero) with integer
// operations only: sign and mantissa move over, the exponent is rebiased
// (127 -> 1023).  GB300 issues FP64 work (conversions included) at a small
// fraction of the FP32 and integer rates, and this kernel is bound by it.
__device__ __forceinline__ double beta_to_double(float f) {
  const unsigned fb = __float_as_uint(f);
  const unsigned mag = fb & 0x7fffffffu;
  const unsigned hi = (fb & 0x80000000u) | (((mag >> 23) + 896u) << 20) | ((mag & 0x7fffffu) >> 3);
  const unsigned lo = fb << 29;
  return mag == 0u ? 0.0 : __hiloint2double((int)hi, (int)lo);
}

// With e32: the first Gauss-Seidel sweep of the next inner solve (colour 0
// from e = 0, the other colour 0) is taken here, from the float residual just
// stored, with the same arithmetic as k_gs_zero: the inner solve then starts
// at its second sweep.  w32: the finest level's float 1/h^2 per axis.
__global__ void k_residual64(Geo g, const double* __restrict__ p, const double* __restrict__ b,
                             const float* __restrict__ b0, const float* __restrict__ b1,
                             const float* __restrict__ b2, float* __restrict__ r32,
                             double* __restrict__ partial, float* __restrict__ e32, W3 w32) {
  __shared__ double sh[33];
  const float* be[3] = {b0, b1, b2};
  const int st[3] = {1, g.n[0], g.n[0] * g.n[1]};
  const double wu = g.n[0] > 1 ? g.w[0] : (g.n[1] > 1 ? g.w[1] : g.w[2]);
  double acc = 0.0;
  for (long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x; cl < g.N;
       cl += (long long)gridDim.x * blockDim.x) {
    const int c = (int)cl;
    int i, j, k;
    decode_lv(g, c, i, j, k);
    const int idx[3] = {i, j, k};
    const double pc = p[c];
    float blo[3] = {0.f, 0.f, 0.f}, bhi[3] = {0.f, 0.f, 0.f};
    // the fine level has cubic cells: one weight 1/h^2 for every coupled axis
    double lsum = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int n = g.n[d];
      if (n == 1) continue;
      const int clo = idx[d] == 0 ? c + (n - 1) * st[d] : c - st[d];
      const int chi = idx[d] == n - 1 ? c - (n - 1) * st[d] : c + st[d];
      blo[d] = be[d][c];
      bhi[d] = (g.bc[d] == WALL && idx[d] == n - 1) ? 0.f : be[d][chi];
      lsum = fma(beta_to_double(blo[d]), pc - p[clo], lsum);
      lsum = fma(beta_to_double(bhi[d]), pc - p[chi], lsum);
    }
    const double r = fma(-wu, lsum, b[c]);
    const float rf = (float)r;
    r32[c] = rf;
    if (e32) {
      const float z[3] = {0.f, 0.f, 0.f};
      e32[c] = ((i + j + k) & 1) == 0 ? gs_formula(g, w32.w, rf, blo, bhi, z, z) : 0.f;
    }
    acc += r * r;
  }
  double s = block_sum_all(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

void launch_residual64(const Geo& g, const double* p, const double* b, float* const* beta,
                       float* r32, double* partial, double* out, cudaStream_t s, float* e32,
                       const float* w32) {
  W3 w = {{0.f, 0.f, 0.f}};
  if (w32)
    for (int d = 0; d < 3; ++d) w.w[d] = w32[d];
  k_residual64<<<kRedBlocks, 256, 0, s>>>(g, p, b, beta[0], beta[1], beta[2], r32, partial, e32, w);
  launch_sum_partials(partial, kRedBlocks, out, s);
}

__global__ void k_add_correction(long long n, double* __restrict__ p, const float* __restrict__ e) {
  long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < n) p[c] = p[c] + (double)e[c];
}

void launch_add_correction(long long n, double* p, const float* e, cudaStream_t s) {
  k_add_correction<<<grid1d(n, 256), 256, 0, s>>>(n, p, e);
}

// ---------------------------------------------------------------------------
// device-side control of the pressure solve (one thread each)
__global__ void k_ctl_reset(SolveCtl* ctl) {
  ctl->iters = 0;
  ctl->status = 0;
  ctl->zero = 0;
  ctl->rel = 0.0;
}

void launch_ctl_reset(SolveCtl* ctl, cudaStream_t s) { k_ctl_reset<<<1, 1, 0, s>>>(ctl); }

// the stopping rule of the host loop, on the device: stop on a non-finite
// norm (EUNSTABLE), a zero right-hand side, after `fixed` cycles, at
// rel <= rtol, or at maxit cycles above rtol (ENOCONV)
__global__ void k_ctl_step(cudaGraphConditionalHandle h, SolveCtl* ctl, const double* bn2p,
                           const double* r2p, double rtol, int maxit, int fixed,
                           unsigned long long* runs_total) {
  const double bn2 = *bn2p;
  unsigned go = 0;
  if (!isfinite(bn2)) {
    ctl->status = FVM_EUNSTABLE;
  } else if (bn2 == 0.0) {
    ctl->zero = 1;
    ctl->rel = 0.0;
  } else {
    const double rel = sqrt(*r2p) / sqrt(bn2);
    ctl->rel = rel;
    if (!isfinite(rel)) {
      ctl->status = FVM_EUNSTABLE;
    } else if (fixed > 0) {
      go = ctl->iters < fixed;
    } else {
      go = rel > rtol && ctl->iters < maxit;
      if (!go && rel > rtol) ctl->status = FVM_ENOCONV;
    }
  }
  if (go) {
    ctl->iters += 1;
    *runs_total += 1ull;
  }
  cudaGraphSetConditional(h, go);
}

void launch_ctl_step(cudaGraphConditionalHandle h, SolveCtl* ctl, const double* bn2,
                     const double* r2, double rtol, int maxit, int fixed,
                     unsigned long long* runs_total, cudaStream_t s) {
  k_ctl_step<<<1, 1, 0, s>>>(h, ctl, bn2, r2, rtol, maxit, fixed, runs_total);
}

__global__ void k_zero_if_rhs_zero(const SolveCtl* __restrict__ ctl, double* __restrict__ p,
                                   long long n) {
  if (!ctl->zero) return;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x)
    p[c] = 0.0;
}

void launch_zero_if_rhs_zero(const SolveCtl* ctl, double* p, long long n, cudaStream_t s) {
  k_zero_if_rhs_zero<<<kRedBlocks, 256, 0, s>>>(ctl, p, n);
}

__global__ void k_ctl_store(const SolveCtl* ctl, SolveCtl* rec, int* sticky) {
  *rec = *ctl;
  if (ctl->status) atomicMax(sticky, ctl->status);
}

void launch_ctl_store(const SolveCtl* ctl, SolveCtl* rec, int* sticky, cudaStream_t s) {
  k_ctl_store<<<1, 1, 0, s>>>(ctl, rec, sticky);
}

#define FVM_MG_INST(T)                                                                       \
  template void launch_sum_field<T>(const T*, long long, bool, double*, double*,             \
                                    cudaStream_t);                                           \
  template void launch_zero<T>(T*, long long, cudaStream_t);                                 \
  template void launch_gs<T>(const MGLevel<T>&, int, cudaStream_t, const int*, int);        \
  template void launch_residual_restrict<T>(const MGLevel<T>&, const MGLevel<T>&, cudaStream_t, bool); \
  template void launch_prolong<T>(const MGLevel<T>&, const MGLevel<T>&, cudaStream_t);       \
  template void launch_gs_prolong<T>(const MGLevel<T>&, const MGLevel<T>&, int, cudaStream_t); \
  template void launch_gs_zero<T>(const MGLevel<T>&, int, cudaStream_t);                      \
  template void launch_beta_coarsen<T>(const MGLevel<T>&, const MGLevel<T>&, cudaStream_t);  \
  template void launch_coarse_tail<T>(const TailArgs<T>&, cudaStream_t);                     \
  template void launch_coarse_cg<T>(const MGLevel<T>&, double*, double*, double*, double,  \
                                    int, cudaStream_t);                                      \
  template void launch_residual_norm2<T>(const MGLevel<T>&, double*, double*, cudaStream_t);

FVM_MG_INST(double)
FVM_MG_INST(float)

}  // namespace fvm
