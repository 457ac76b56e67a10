// C ABI and host runtime of libfvm: parameter checks, workspace plan,
// multigrid hierarchy, the SSP-RK3 stage sequence and the pressure solvers.
// All device memory comes from the caller's workspace; the context itself
// lives in host memory.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "fvm_adjoint.h"
#include "fvm_internal.h"

using namespace fvm;

namespace {

constexpr size_t kAlign = 256;

struct Plan {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + kAlign - 1) / kAlign * kAlign;
    return o;
  }
};

struct LevelShape {
  int n[3];
  double hd[3];
  int f[3];
};

int build_levels(const fvm_params& p, LevelShape* lv) {
  int nl = 0;
  LevelShape cur;
  cur.n[0] = p.nx; cur.n[1] = p.ny; cur.n[2] = p.nz;
  for (int d = 0; d < 3; ++d) { cur.hd[d] = p.h; cur.f[d] = 1; }
  lv[nl++] = cur;
  while (nl < p.mg_levels && nl < kMaxLevels) {
    LevelShape& L = lv[nl - 1];
    int f[3];
    bool any = false;
    for (int d = 0; d < 3; ++d) {
      bool ok = L.n[d] % 2 == 0 && L.n[d] >= 4;
      if (ok && p.bc[d] == PER && (L.n[d] / 2) % 2 != 0) ok = false;
      f[d] = ok ? 2 : 1;
      any = any || ok;
    }
    if (!any) break;
    LevelShape nx;
    for (int d = 0; d < 3; ++d) {
      L.f[d] = f[d];
      nx.n[d] = L.n[d] / f[d];
      nx.hd[d] = L.hd[d] * f[d];
      nx.f[d] = 1;
    }
    lv[nl++] = nx;
  }
  return nl;
}

Geo make_geo(const fvm_params& p, const LevelShape& s) {
  Geo g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = s.n[d];
    g.bc[d] = p.bc[d];
    g.hd[d] = s.hd[d];
  }
  g.h = p.h;
  g.ih = 1.0 / p.h;
  for (int d = 0; d < 3; ++d) g.w[d] = g.n[d] > 1 ? 1.0 / (g.hd[d] * g.hd[d]) : 0.0;
  g.sy = g.n[0];
  g.sz = (long long)g.n[0] * g.n[1];
  g.N = g.sz * g.n[2];
  return g;
}

const char* check_params(const fvm_params* p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "grid sizes must be >= 1";
  if ((long long)p->nx * p->ny * p->nz > 2147483647LL) return "more than 2^31-1 cells";
  if (!(p->h > 0.0)) return "h must be > 0";
  int ndir = 0;
  for (int d = 0; d < 3; ++d) {
    if (p->bc[d] != FVM_BC_PERIODIC && p->bc[d] != FVM_BC_WALL) return "bc must be 0 or 1";
    int n = d == 0 ? p->nx : (d == 1 ? p->ny : p->nz);
    if (p->bc[d] == FVM_BC_WALL && n < 4) return "a wall axis needs >= 4 cells";
    // red-black Gauss-Seidel colours cells by (i + j + k) mod 2, which is a
    // 2-colouring under wrap only for an even cell count
    if (p->bc[d] == FVM_BC_PERIODIC && n > 1 && n % 2)
      return "a periodic axis needs an even number of cells (or one)";
    bool dl = p->tbc[2 * d] == FVM_TBC_DIRICHLET, dh = p->tbc[2 * d + 1] == FVM_TBC_DIRICHLET;
    if ((dl || dh) && p->bc[d] != FVM_BC_WALL) return "Dirichlet temperature needs a wall axis";
    if (dl || dh) ++ndir;
  }
  if (ndir > 1) return "Dirichlet temperature on more than one axis is not supported";
  for (int q = 0; q < 2; ++q) {
    if (!(p->rho[q] > 0.0) || !(p->cp[q] > 0.0) || !(p->lambda[q] > 0.0) || !(p->mu[q] >= 0.0))
      return "rho, cp, lambda must be > 0 and mu >= 0";
  }
  if (p->precision != FVM_F64 && p->precision != FVM_MIXED) return "precision must be 0 or 1";
  if (p->smooth_passes < 0 || p->mg_levels < 1 || p->mg_pre < 0 || p->mg_post < 0 ||
      p->mg_max_cycles < 1 || p->mg_fixed_cycles < 0 || p->coarse_maxit < 1 ||
      p->mx_inner_cycles < 1)
    return "multigrid counts out of range";
  if (!(p->mg_rtol > 0.0) || !(p->coarse_rtol > 0.0)) return "tolerances must be > 0";
  if (!(p->weno_eps > 0.0)) return "weno_eps must be > 0";
  if (p->smooth_passes > 2) return "smooth_passes above 2 is not supported";
  if (p->q_power != 0.0 && !(p->q_radius > 0.0)) return "q_radius must be > 0";
  if (p->adjoint != 0 && p->adjoint != 1) return "adjoint must be 0 or 1";
  if (p->adjoint && p->precision != FVM_F64) return "the adjoint needs precision F64";
  if (p->concentration != 0 && p->concentration != 1) return "concentration must be 0 or 1";
  if (p->alpha_scheme != 0 && p->alpha_scheme != 1) return "alpha_scheme must be 0 or 1";
  if (p->mg_coarse_sweeps < 0) return "mg_coarse_sweeps must be >= 0";
  if (p->alpha_scheme == 1 && p->adjoint) return "the adjoint does not support the bounded scheme";
  if (p->concentration) {
    if (!(p->diff_c[0] >= 0.0) || !(p->diff_c[1] >= 0.0)) return "diff_c must be >= 0";
    if (!(p->weno_scale_c != 0.0)) return "weno_scale_c must be nonzero";
    if (p->adjoint) return "the adjoint does not support a concentration";
  }
  return nullptr;
}

}  // namespace

struct fvm_ctx {
  fvm_params prm;
  Geo g;
  Phys ph;
  TBC tb;
  cudaStream_t stream;
  bool mixed;
  size_t rsz;            // bytes of the working precision
  char* ws;
  size_t ws_bytes;
  // stage buffers (working precision)
  void* A[6];            // stage copies: u, v, w, alpha, T and the concentration
  void* B[6];            // (null without one)
  void* fct[2];          // limiter ratios R+, R- of the bounded alpha transport
  void* as;
  void* tmp;
  void* kappa;
  void* M[3];
  void* us[3];
  double* b;             // projection right-hand side
  void* beta0[3];        // fine beta (double in F64, float in MIXED)
  float* e32;            // MIXED: inner correction
  float* r32;            // MIXED: inner right-hand side
  // hierarchy
  int nlev;
  LevelShape shp[kMaxLevels];
  void* lx[kMaxLevels];
  void* lb[kMaxLevels];
  void* lbeta[kMaxLevels][3];
  void* cg[3];
  // reduction scratch
  double* partial;
  double* scal;          // 16 doubles
  unsigned long long* maxbits;
  int* flags;
  double* dt_dev;
  int* lim_dev;
  // reverse mode (prm.adjoint = 1), double fields of N cells
  double* aL[5];         // adjoint of the input of the stage after the current one
  double* aE[5];         // adjoint of the current stage's E (u, v, w, alpha, T)
  double* ap;            // pressure of the adjoint projection
  double* apf;           // pressure warm start of the recomputed forward stages
  double* akap;          // adjoint of the curvature
  double* aM[3];         // adjoint of the Marangoni vector
  double* aat;           // adjoint of the smoothed alpha
  double* atmp;          // between the two smoothing transposes
  double* aK;            // kAdjSlots coefficient slots of the two-pass transposes
  double* apst[3];       // forward pressure of each stage (the density term)
  double adj_dt;         // dt of the step being adjoined
  // kernel timing with CUDA events (measurement aid, off by default)
  int prof;
  int prof_n;
  cudaEvent_t* prof_ev;      // 2 * kProfSlots events
  int* prof_cls;
  long nlaunch;              // kernels launched since the last count reset
  // CUDA graphs of the whole pressure solve with its stopping test on the
  // device (a conditional WHILE node), keyed by the solution pointer p
  int graphs_ok;             // 1: try stream capture; 0: eager launches only
  struct GEntry { const void* p; cudaGraphExec_t exec; long nk; } gcache[8];
  int gnext;
  long nk_body;              // kernels of one cycle (refinement) of a graph's loop
  SolveCtl* ctl;             // device: controller of the solve in flight
  SolveCtl* rec;             // device: kRecords records (stages 0..2, lone solve 3)
  int* sticky;               // device: worst status of graph solves since fvm_sync
  unsigned long long* runs;  // device: loop cycles run by graph solves
  unsigned long long runs_base;  // value of *runs at the last launch-count reset
  long prof_launches[FVM_KCLASS_COUNT];
  double prof_ms[FVM_KCLASS_COUNT];
  char err[512];
};

namespace {

constexpr int kProfSlots = 4096;
constexpr int kRecords = 4;   // solve records: the three stages of a step, a lone solve

void prof_fold(fvm_ctx* c) {
  if (!c->prof_n) return;
  cudaStreamSynchronize(c->stream);
  for (int q = 0; q < c->prof_n; ++q) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[2 * q], c->prof_ev[2 * q + 1]) == cudaSuccess) {
      c->prof_ms[c->prof_cls[q]] += ms;
      c->prof_launches[c->prof_cls[q]] += 1;
    }
  }
  c->prof_n = 0;
}

struct ProfScope {
  fvm_ctx* c;
  int slot;
  ProfScope(fvm_ctx* ctx, int cls) : c(ctx), slot(-1) {
    if (!c->prof) return;
    if (c->prof_n == kProfSlots) prof_fold(c);
    slot = c->prof_n++;
    c->prof_cls[slot] = cls;
    cudaEventRecord(c->prof_ev[2 * slot], c->stream);
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], c->stream);
  }
};

// every kernel launch of the library goes through TIMED(ctx, class, kernels, call):
// it counts the kernels and, while profiling is on, brackets them with events
#define TIMED(ctx, cls, nk, ...) \
  do {                           \
    (ctx)->nlaunch += (nk);      \
    ProfScope _ps(ctx, cls);     \
    __VA_ARGS__;                 \
  } while (0)

size_t plan_workspace(const fvm_params& p, fvm_ctx* c) {
  Plan pl;
  LevelShape lv[kMaxLevels];
  int nl = build_levels(p, lv);
  long long N = (long long)p.nx * p.ny * p.nz;
  bool mixed = p.precision == FVM_MIXED;
  size_t rs = mixed ? sizeof(float) : sizeof(double);
  size_t ms = rs;   // multigrid precision: double in F64, float (inner) in MIXED
  size_t o_A[6], o_B[6], o_as, o_tmp, o_k, o_M[3], o_us[3], o_b, o_beta[3], o_e = 0, o_r = 0;
  const int nstage = p.concentration ? 6 : 5;
  for (int q = 0; q < nstage; ++q) o_A[q] = pl.take(N * rs);
  for (int q = 0; q < nstage; ++q) o_B[q] = pl.take(N * rs);
  size_t o_fct[2] = {0, 0};
  if (p.alpha_scheme == 1)
    for (int q = 0; q < 2; ++q) o_fct[q] = pl.take(N * rs);
  o_as = pl.take(N * rs);
  o_tmp = pl.take(N * rs);
  o_k = pl.take(N * rs);
  for (int q = 0; q < 3; ++q) o_M[q] = pl.take(N * rs);
  for (int q = 0; q < 3; ++q) o_us[q] = pl.take(N * rs);
  o_b = pl.take(N * sizeof(double));
  for (int q = 0; q < 3; ++q) o_beta[q] = pl.take(N * ms);
  if (mixed) {
    o_e = pl.take(N * sizeof(float));
    o_r = pl.take(N * sizeof(float));
  }
  size_t o_lx[kMaxLevels], o_lb[kMaxLevels], o_lbeta[kMaxLevels][3];
  for (int l = 1; l < nl; ++l) {
    long long n = (long long)lv[l].n[0] * lv[l].n[1] * lv[l].n[2];
    o_lx[l] = pl.take(n * ms);
    o_lb[l] = pl.take(n * ms);
    for (int q = 0; q < 3; ++q) o_lbeta[l][q] = pl.take(n * ms);
  }
  long long nc = (long long)lv[nl - 1].n[0] * lv[nl - 1].n[1] * lv[nl - 1].n[2];
  size_t o_cg[3];   // r, d and (Ad, x) in double
  for (int q = 0; q < 3; ++q) o_cg[q] = pl.take((q == 2 ? 2 : 1) * nc * sizeof(double));
  size_t o_part = pl.take(2 * kRedBlocks * sizeof(double));
  size_t o_scal = pl.take(16 * sizeof(double));
  size_t o_max = pl.take(8 * sizeof(unsigned long long));
  size_t o_flags = pl.take(8 * sizeof(int));
  size_t o_dt = pl.take(2 * sizeof(double));   // dt and 1/dt
  size_t o_lim = pl.take(sizeof(int));
  size_t o_ctl = pl.take((1 + kRecords) * sizeof(SolveCtl) + sizeof(int) + sizeof(unsigned long long));
  constexpr int kAdjFields = 21;
  size_t o_adj[kAdjFields];
  size_t o_K = 0;
  if (p.adjoint) {
    for (int q = 0; q < kAdjFields; ++q) o_adj[q] = pl.take(N * sizeof(double));
    o_K = pl.take((size_t)kAdjSlots * N * sizeof(double));
  }
  if (c) {
    char* w = c->ws;
    for (int q = 0; q < 6; ++q) {
      c->A[q] = q < nstage ? w + o_A[q] : nullptr;
      c->B[q] = q < nstage ? w + o_B[q] : nullptr;
    }
    for (int q = 0; q < 2; ++q) c->fct[q] = p.alpha_scheme == 1 ? w + o_fct[q] : nullptr;
    c->as = w + o_as;
    c->tmp = w + o_tmp;
    c->kappa = w + o_k;
    for (int q = 0; q < 3; ++q) {
      c->M[q] = w + o_M[q];
      c->us[q] = w + o_us[q];
      c->beta0[q] = w + o_beta[q];
    }
    c->b = (double*)(w + o_b);
    c->e32 = mixed ? (float*)(w + o_e) : nullptr;
    c->r32 = mixed ? (float*)(w + o_r) : nullptr;
    c->nlev = nl;
    for (int l = 0; l < nl; ++l) c->shp[l] = lv[l];
    for (int l = 1; l < nl; ++l) {
      c->lx[l] = w + o_lx[l];
      c->lb[l] = w + o_lb[l];
      for (int q = 0; q < 3; ++q) c->lbeta[l][q] = w + o_lbeta[l][q];
    }
    for (int q = 0; q < 3; ++q) c->cg[q] = w + o_cg[q];
    c->partial = (double*)(w + o_part);
    c->scal = (double*)(w + o_scal);
    c->maxbits = (unsigned long long*)(w + o_max);
    c->flags = (int*)(w + o_flags);
    c->dt_dev = (double*)(w + o_dt);
    c->lim_dev = (int*)(w + o_lim);
    c->ctl = (SolveCtl*)(w + o_ctl);
    c->rec = c->ctl + 1;
    c->runs = (unsigned long long*)(c->rec + kRecords);
    c->sticky = (int*)(c->runs + 1);
    if (p.adjoint) {
      double* a[kAdjFields];
      for (int q = 0; q < kAdjFields; ++q) a[q] = (double*)(w + o_adj[q]);
      for (int q = 0; q < 5; ++q) { c->aL[q] = a[q]; c->aE[q] = a[5 + q]; }
      c->ap = a[10];
      c->apf = a[11];
      c->akap = a[12];
      for (int q = 0; q < 3; ++q) c->aM[q] = a[13 + q];
      c->aat = a[16];
      c->atmp = a[17];
      for (int q = 0; q < 3; ++q) c->apst[q] = a[18 + q];
      c->aK = (double*)(w + o_K);
    } else {
      c->aK = nullptr;
      for (int q = 0; q < 5; ++q) { c->aL[q] = nullptr; c->aE[q] = nullptr; }
      c->ap = c->apf = c->akap = c->aat = c->atmp = nullptr;
      for (int q = 0; q < 3; ++q) c->apst[q] = nullptr;
      for (int q = 0; q < 3; ++q) c->aM[q] = nullptr;
    }
  }
  return pl.off;
}

fvm_status set_err(fvm_ctx* c, fvm_status s, const char* msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  return s;
}

fvm_status cuda_check(fvm_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
    return FVM_ECUDA;
  }
  return FVM_OK;
}

fvm_status read_scalar(fvm_ctx* c, const double* dsrc, double* host) {
  cudaError_t e = cudaMemcpyAsync(host, dsrc, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "device read: %s", cudaGetErrorString(e));
    return FVM_ECUDA;
  }
  return FVM_OK;
}

template <typename T>
MGLevel<T> mg_level(fvm_ctx* c, int l, T* x, T* b, T* const* beta) {
  MGLevel<T> L;
  L.geo = make_geo(c->prm, c->shp[l]);
  L.x = x;
  L.b = b;
  for (int q = 0; q < 3; ++q) {
    L.beta[q] = beta[q];
    L.w[q] = (T)L.geo.w[q];
  }
  for (int d = 0; d < 3; ++d) L.f[d] = c->shp[l].f[d];
  return L;
}

// hierarchy in precision T with level 0 given by (x0, b0, beta0)
template <typename T>
void hierarchy(fvm_ctx* c, T* x0, T* b0, T* const* beta0, MGLevel<T>* Ls) {
  Ls[0] = mg_level<T>(c, 0, x0, b0, beta0);
  for (int l = 1; l < c->nlev; ++l) {
    T* be[3] = {(T*)c->lbeta[l][0], (T*)c->lbeta[l][1], (T*)c->lbeta[l][2]};
    Ls[l] = mg_level<T>(c, l, (T*)c->lx[l], (T*)c->lb[l], be);
  }
}

template <typename T>
void coarsen_betas(fvm_ctx* c, MGLevel<T>* Ls) {
  for (int l = 0; l + 1 < c->nlev; ++l)
    TIMED(c, FVM_K_BETA, 1, launch_beta_coarsen<T>(Ls[l], Ls[l + 1], c->stream));
}

// what the sweeps of one smoothing step fold in
template <typename T>
struct SweepFold {
  const MGLevel<T>* corr = nullptr;   // first sweep: the coarse correction of this level (prolongation)
  bool zero = false;                  // first sweep: x starts at 0 (zeroes the other colour)
  bool skip_first = false;            // first sweep: already taken (by k_residual64)
  const int* gate = nullptr;          // first sweep: skipped on the device once *gate >= gate_min
  int gate_min = 0;
  double* addp = nullptr;             // last sweep: p += x (the mixed form's float level 0)
};

inline void addp_sweep(fvm_ctx* c, int kg, const MGLevel<float>& L, int colour, double* p) {
  TIMED(c, kg, 1, launch_gs_addp(L, colour, p, c->stream));
}
inline void addp_sweep(fvm_ctx*, int, const MGLevel<double>&, int, double*) {}

// `iters` Gauss-Seidel iterations on level l: a sweep of colour `first`,
// then one of the other colour.  The first sweep can apply the coarse
// correction (k_gs_prolong) or start from x = 0 (k_gs_zero), the last one can
// add x to p (k_gs_addp): each replaces a pass of its own over x, with the
// same numbers.
template <typename T>
void smooth(fvm_ctx* c, MGLevel<T>& L, int l, int iters, int first,
            const SweepFold<T>& f = SweepFold<T>()) {
  const int kg = l == 0 ? FVM_K_GS_FINE : FVM_K_GS_COARSE;
  const int last = 2 * iters - 1;
  for (int t = 0; t <= last; ++t) {
    const int colour = (t & 1) == 0 ? first : 1 - first;
    if (t == 0 && f.skip_first) continue;
    if (t == 0 && f.corr)
      TIMED(c, kg, 1, launch_gs_prolong<T>(L, *f.corr, colour, c->stream));
    else if (t == 0 && f.zero)
      TIMED(c, kg, 1, launch_gs_zero<T>(L, colour, c->stream));
    else if (t == last && f.addp)
      addp_sweep(c, kg, L, colour, f.addp);
    else if (t == 0 && f.gate)
      TIMED(c, kg, 1, launch_gs<T>(L, colour, c->stream, f.gate, f.gate_min));
    else
      TIMED(c, kg, 1, launch_gs<T>(L, colour, c->stream));
  }
}

// sweeps on the levels below the finest
int coarse_pre(const fvm_ctx* c) {
  return c->prm.mg_coarse_sweeps > 0 ? c->prm.mg_coarse_sweeps : c->prm.mg_pre;
}
int coarse_post(const fvm_ctx* c) {
  return c->prm.mg_coarse_sweeps > 0 ? c->prm.mg_coarse_sweeps : c->prm.mg_post;
}

// first level of the one-CTA coarse tail (at most kTailCells cells, not the
// finest, at least one level above the coarsest), or -1
int tail_start(const fvm_ctx* c) {
  for (int l = 1; l < c->nlev - 1; ++l) {
    const LevelShape& q = c->shp[l];
    if ((long long)q.n[0] * q.n[1] * q.n[2] <= kTailCells)
      return c->nlev - l <= kTailLevels ? l : -1;
  }
  return -1;
}

// V(pre, post) cycle: red-black sweeps before the coarse correction,
// black-red after, CG on the coarsest level; the levels from tail_start()
// down run in one kernel
// How the finest level's x starts: as it is, at 0 (not yet zeroed), with the
// first sweep already taken (by k_residual64 in the mixed form, or skipped
// because it would repeat the previous cycle's last sweep), or with that skip
// decided on the device (FP64 solve graph: from the second cycle on).
enum { kStartAsIs = 0, kStartZero = 1, kStartFirstSwept = 2, kStartGated = 3 };

// a cycle's first finest-level sweep repeats the previous cycle's last one
// (same colour, same right-hand side, the other colour unchanged) when both
// smoothing steps sweep on a finest level of its own
bool first_sweep_repeats(const fvm_ctx* c) {
  return c->prm.mg_pre > 0 && c->prm.mg_post > 0 && c->nlev > 1;
}

// the mixed form's residual kernel takes the first sweep of each inner solve
// when that solve begins with a sweep on a finest level of its own
bool residual_takes_first_sweep(const fvm_ctx* c) {
  return c->prm.mg_pre > 0 && c->nlev > 1 && c->prm.mx_inner_cycles > 0;
}

// the residual r = b - L p (double, stored as float) of the mixed form, with
// the next inner solve's first sweep when residual_takes_first_sweep()
void mixed_residual(fvm_ctx* c, double* p, const double* b, float* const* be) {
  const bool f = residual_takes_first_sweep(c);
  const float w32[3] = {(float)c->g.w[0], (float)c->g.w[1], (float)c->g.w[2]};
  TIMED(c, FVM_K_RESIDUAL64, 2,
        launch_residual64(c->g, p, b, be, c->r32, c->partial, c->scal + 1, c->stream,
                          f ? c->e32 : nullptr, w32));
}

// start: how level l's x starts (kStart*); addp: add level 0's x to p at the
// end (float only)
template <typename T>
void vcycle(fvm_ctx* c, MGLevel<T>* Ls, int l, double coarse_rtol, int start = kStartAsIs,
            double* addp = nullptr) {
  cudaStream_t s = c->stream;
  const int pre = l == 0 ? c->prm.mg_pre : coarse_pre(c);
  const int post = l == 0 ? c->prm.mg_post : coarse_post(c);
  const bool whole = l == tail_start(c) || l == c->nlev - 1;   // no sweeps of its own here
  const bool zero = start == kStartZero;
  if (zero && (whole || pre == 0))
    TIMED(c, FVM_K_MISC, 1, launch_zero<T>(Ls[l].x, Ls[l].geo.N, s));
  const bool fold_zero = zero && !whole && pre > 0;
  const bool fold_add = addp && !whole && post > 0;
  if (l == tail_start(c)) {
    TailArgs<T> A;
    A.nl = c->nlev - l;
    for (int q = 0; q < A.nl; ++q) A.L[q] = Ls[l + q];
    A.r = (double*)c->cg[0];
    A.d = (double*)c->cg[1];
    A.Ad = (double*)c->cg[2];
    A.rtol = coarse_rtol;
    A.maxit = c->prm.coarse_maxit;
    A.pre = coarse_pre(c);
    A.post = coarse_post(c);
    TIMED(c, FVM_K_COARSE_TAIL, 1, launch_coarse_tail<T>(A, s));
  } else if (l == c->nlev - 1) {
    TIMED(c, FVM_K_COARSE_CG, 1, launch_coarse_cg<T>(Ls[l], (double*)c->cg[0], (double*)c->cg[1], (double*)c->cg[2],
                                                   coarse_rtol, c->prm.coarse_maxit, s));
  } else {
    SweepFold<T> fpre;
    fpre.zero = fold_zero;
    fpre.skip_first = start == kStartFirstSwept;
    if (start == kStartGated) {
      // the controller counts the cycle being run: 1 in the first
      fpre.gate = &c->ctl->iters;
      fpre.gate_min = 2;
    }
    smooth<T>(c, Ls[l], l, pre, 0, fpre);
    // the next level's first sweep rides on the restriction when that level
    // sweeps on its own (not the tail, not the coarsest)
    const bool swept = l + 1 != tail_start(c) && l + 1 != c->nlev - 1 && coarse_pre(c) > 0;
    TIMED(c, l == 0 ? FVM_K_RESTRICT_FINE : FVM_K_RESTRICT_COARSE, 1,
          launch_residual_restrict<T>(Ls[l], Ls[l + 1], s, swept));
    vcycle<T>(c, Ls, l + 1, coarse_rtol, swept ? kStartFirstSwept : kStartAsIs);
    if (post > 0) {
      // the prolongation rides on the first post-smoothing sweep
      SweepFold<T> fpost;
      fpost.corr = &Ls[l + 1];
      fpost.addp = fold_add ? addp : nullptr;
      smooth<T>(c, Ls[l], l, post, 1, fpost);
    } else {
      TIMED(c, l == 0 ? FVM_K_PROLONG_FINE : FVM_K_PROLONG_COARSE, 1,
            launch_prolong<T>(Ls[l], Ls[l + 1], s));
    }
  }
  if (addp && !fold_add)
    TIMED(c, FVM_K_ADD_CORRECTION, 1, launch_add_correction(Ls[0].geo.N, addp, (const float*)Ls[0].x, s));
}

// F64: L p = b (b mean-free, double), beta0 already computed
fvm_status solve_f64(fvm_ctx* c, double* p, double* b, int* cycles_out, double* rel_out,
                     bool want_rel) {
  cudaStream_t s = c->stream;
  MGLevel<double> Ls[kMaxLevels];
  double* be[3] = {(double*)c->beta0[0], (double*)c->beta0[1], (double*)c->beta0[2]};
  hierarchy<double>(c, p, b, be, Ls);
  coarsen_betas<double>(c, Ls);
  const long long N = c->g.N;
  double bn2;
  TIMED(c, FVM_K_MISC, 2, launch_sum_field<double>(b, N, true, c->partial, c->scal + 0, s));
  fvm_status st = read_scalar(c, c->scal + 0, &bn2);
  if (st) return st;
  if (!isfinite(bn2)) return set_err(c, FVM_EUNSTABLE, "non-finite projection right-hand side");
  double bn = sqrt(bn2);
  int cycles = 0;
  double rel = 0.0;
  if (bn == 0.0) {
    TIMED(c, FVM_K_MISC, 1, launch_zero<double>(p, N, s));
    *cycles_out = 0;
    *rel_out = 0.0;
    return cuda_check(c, "poisson zero");
  }
  const int fixed = c->prm.mg_fixed_cycles;
  if (fixed > 0) {
    const int later = first_sweep_repeats(c) ? kStartFirstSwept : kStartAsIs;
    for (int q = 0; q < fixed; ++q)
      vcycle<double>(c, Ls, 0, c->prm.coarse_rtol, q == 0 ? kStartAsIs : later);
    cycles = fixed;
    if (want_rel) {
      double r2;
      TIMED(c, FVM_K_RESNORM, 2, launch_residual_norm2<double>(Ls[0], c->partial, c->scal + 1, s));
      st = read_scalar(c, c->scal + 1, &r2);
      if (st) return st;
      rel = sqrt(r2) / bn;
    }
  } else {
    for (;;) {
      double r2;
      TIMED(c, FVM_K_RESNORM, 2, launch_residual_norm2<double>(Ls[0], c->partial, c->scal + 1, s));
      st = read_scalar(c, c->scal + 1, &r2);
      if (st) return st;
      rel = sqrt(r2) / bn;
      if (!isfinite(rel)) return set_err(c, FVM_EUNSTABLE, "non-finite pressure residual");
      if (rel <= c->prm.mg_rtol || cycles >= c->prm.mg_max_cycles) break;
      vcycle<double>(c, Ls, 0, c->prm.coarse_rtol,
                     cycles > 0 && first_sweep_repeats(c) ? kStartFirstSwept : kStartAsIs);
      ++cycles;
    }
  }
  TIMED(c, FVM_K_MISC, 2, launch_sum_field<double>(p, N, false, c->partial, c->scal + 2, s));
  TIMED(c, FVM_K_MISC, 1, launch_sub_mean(p, N, c->scal + 2, s));
  *cycles_out = cycles;
  *rel_out = rel;
  st = cuda_check(c, "f64 pressure solve");
  if (st) return st;
  if (fixed == 0 && rel > c->prm.mg_rtol)
    return set_err(c, FVM_ENOCONV, "pressure solve reached mg_max_cycles above mg_rtol");
  return FVM_OK;
}

// MIXED: double defect correction around float V-cycles.  One refinement
// iteration is: e = 0; mx_inner_cycles float V-cycles on L e = r; p += e;
// r = b - L p in double (stored as float for the next iteration) and its
// norm.
void refine_once(fvm_ctx* c, MGLevel<float>* Ls, const float* alpha, double* p, double* b,
                 float* const* be, double crtol) {
  // e = 0, the inner cycles and p += e: the zeroing rides on the first sweep
  // of the first cycle (or that sweep was taken by the residual kernel), the
  // addition on the last sweep of the last one
  const int m = c->prm.mx_inner_cycles;
  const int start0 = residual_takes_first_sweep(c) ? kStartFirstSwept : kStartZero;
  // a cycle after the first begins with a colour-0 sweep right after the
  // previous cycle's last one, also of colour 0, on the same right-hand side
  // with the other colour unchanged: it would write the same values again,
  // so it is skipped (when both smoothing steps sweep on the finest level)
  const int startq = first_sweep_repeats(c) ? kStartFirstSwept : kStartAsIs;
  for (int q = 0; q < m; ++q)
    vcycle<float>(c, Ls, 0, crtol, q == 0 ? start0 : startq, q == m - 1 ? p : nullptr);
  mixed_residual(c, p, b, be);
}

fvm_status solve_mixed(fvm_ctx* c, const float* alpha, double* p, double* b, int* cycles_out,
                       double* rel_out, bool want_rel) {
  (void)want_rel;
  cudaStream_t s = c->stream;
  MGLevel<float> Ls[kMaxLevels];
  float* be[3] = {(float*)c->beta0[0], (float*)c->beta0[1], (float*)c->beta0[2]};
  hierarchy<float>(c, c->e32, c->r32, be, Ls);
  coarsen_betas<float>(c, Ls);
  const long long N = c->g.N;
  double bn2;
  TIMED(c, FVM_K_MISC, 2, launch_sum_field<double>(b, N, true, c->partial, c->scal + 0, s));
  fvm_status st = read_scalar(c, c->scal + 0, &bn2);
  if (st) return st;
  if (!isfinite(bn2)) return set_err(c, FVM_EUNSTABLE, "non-finite projection right-hand side");
  double bn = sqrt(bn2);
  if (bn == 0.0) {
    TIMED(c, FVM_K_MISC, 1, launch_zero<double>(p, N, s));
    *cycles_out = 0;
    *rel_out = 0.0;
    return cuda_check(c, "poisson zero");
  }
  const int fixed = c->prm.mg_fixed_cycles;
  const double crtol = c->prm.coarse_rtol > 1e-6 ? c->prm.coarse_rtol : 1e-6;
  int outer = 0;
  double rel = 0.0;
  mixed_residual(c, p, b, be);
  for (;;) {
    if (fixed > 0) {
      if (outer == fixed) {
        double r2;
        st = read_scalar(c, c->scal + 1, &r2);
        if (st) return st;
        rel = sqrt(r2) / bn;
        break;
      }
    } else {
      double r2;
      st = read_scalar(c, c->scal + 1, &r2);
      if (st) return st;
      rel = sqrt(r2) / bn;
      if (!isfinite(rel)) return set_err(c, FVM_EUNSTABLE, "non-finite pressure residual");
      if (rel <= c->prm.mg_rtol || outer >= c->prm.mg_max_cycles) break;
    }
    refine_once(c, Ls, alpha, p, b, be, crtol);
    ++outer;
  }
  TIMED(c, FVM_K_MISC, 2, launch_sum_field<double>(p, N, false, c->partial, c->scal + 2, s));
  TIMED(c, FVM_K_MISC, 1, launch_sub_mean(p, N, c->scal + 2, s));
  *cycles_out = outer;
  *rel_out = rel;
  st = cuda_check(c, "mixed pressure solve");
  if (st) return st;
  if (fixed == 0 && rel > c->prm.mg_rtol)
    return set_err(c, FVM_ENOCONV, "pressure solve reached mg_max_cycles above mg_rtol");
  return FVM_OK;
}

// ----- the pressure solve as one CUDA graph ----------------------------------
// prologue: coarse betas, controller reset, ||b||^2, the first residual norm
// and the first stopping test; loop (conditional WHILE node): one cycle (F64)
// or refinement (MIXED), its residual norm, the stopping test; epilogue: zero
// p for a zero right-hand side, remove the mean of p.  The same kernels in
// the same order as the host loops of solve_f64 / solve_mixed, so the
// results agree bit for bit; only the test is taken on the device.
void graph_prologue(fvm_ctx* c, double* p, cudaGraphConditionalHandle h) {
  cudaStream_t s = c->stream;
  const long long N = c->g.N;
  const int fixed = c->prm.mg_fixed_cycles;
  if (c->mixed) {
    MGLevel<float> Ls[kMaxLevels];
    float* be[3] = {(float*)c->beta0[0], (float*)c->beta0[1], (float*)c->beta0[2]};
    hierarchy<float>(c, c->e32, c->r32, be, Ls);
    coarsen_betas<float>(c, Ls);
    TIMED(c, FVM_K_MISC, 1, launch_ctl_reset(c->ctl, s));
    TIMED(c, FVM_K_MISC, 2, launch_sum_field<double>(c->b, N, true, c->partial, c->scal + 0, s));
    mixed_residual(c, p, c->b, be);
  } else {
    MGLevel<double> Ls[kMaxLevels];
    double* be[3] = {(double*)c->beta0[0], (double*)c->beta0[1], (double*)c->beta0[2]};
    hierarchy<double>(c, p, c->b, be, Ls);
    coarsen_betas<double>(c, Ls);
    TIMED(c, FVM_K_MISC, 1, launch_ctl_reset(c->ctl, s));
    TIMED(c, FVM_K_MISC, 2, launch_sum_field<double>(c->b, N, true, c->partial, c->scal + 0, s));
    TIMED(c, FVM_K_RESNORM, 2, launch_residual_norm2<double>(Ls[0], c->partial, c->scal + 1, s));
  }
  TIMED(c, FVM_K_MISC, 1,
        launch_ctl_step(h, c->ctl, c->scal + 0, c->scal + 1, c->prm.mg_rtol, c->prm.mg_max_cycles,
                        fixed, c->runs, s));
}

void graph_body(fvm_ctx* c, double* p, cudaGraphConditionalHandle h) {
  cudaStream_t s = c->stream;
  const int fixed = c->prm.mg_fixed_cycles;
  if (c->mixed) {
    MGLevel<float> Ls[kMaxLevels];
    float* be[3] = {(float*)c->beta0[0], (float*)c->beta0[1], (float*)c->beta0[2]};
    hierarchy<float>(c, c->e32, c->r32, be, Ls);
    const double crtol = c->prm.coarse_rtol > 1e-6 ? c->prm.coarse_rtol : 1e-6;
    refine_once(c, Ls, nullptr, p, c->b, be, crtol);
  } else {
    MGLevel<double> Ls[kMaxLevels];
    double* be[3] = {(double*)c->beta0[0], (double*)c->beta0[1], (double*)c->beta0[2]};
    hierarchy<double>(c, p, c->b, be, Ls);
    vcycle<double>(c, Ls, 0, c->prm.coarse_rtol,
                   first_sweep_repeats(c) ? kStartGated : kStartAsIs);
    TIMED(c, FVM_K_RESNORM, 2, launch_residual_norm2<double>(Ls[0], c->partial, c->scal + 1, s));
  }
  TIMED(c, FVM_K_MISC, 1,
        launch_ctl_step(h, c->ctl, c->scal + 0, c->scal + 1, c->prm.mg_rtol, c->prm.mg_max_cycles,
                        fixed, c->runs, s));
}

void graph_epilogue(fvm_ctx* c, double* p) {
  cudaStream_t s = c->stream;
  const long long N = c->g.N;
  TIMED(c, FVM_K_MISC, 1, launch_zero_if_rhs_zero(c->ctl, p, N, s));
  TIMED(c, FVM_K_MISC, 2, launch_sum_field<double>(p, N, false, c->partial, c->scal + 2, s));
  TIMED(c, FVM_K_MISC, 1, launch_sub_mean(p, N, c->scal + 2, s));
}

// the solve graph for solution pointer p (built on first use, cached); null
// when graphs are unavailable (the caller then runs the host loop)
cudaGraphExec_t solve_graph(fvm_ctx* c, double* p, long* nk_fixed) {
  for (int q = 0; q < 8; ++q)
    if (c->gcache[q].exec && c->gcache[q].p == p) {
      *nk_fixed = c->gcache[q].nk;
      return c->gcache[q].exec;
    }
  cudaStream_t s = c->stream;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t g = nullptr, tmp = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle h = 0;
  cudaGraphNode_t cond = nullptr;
  cudaGraphNode_t leaves[16];
  size_t nleaves = 0;
  const long n0 = c->nlaunch;
  long n_body = 0;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) == cudaSuccess &&
            cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, mode) == cudaSuccess;
  if (ok) {
    graph_prologue(c, p, h);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    ok = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess &&
         cs == cudaStreamCaptureStatusActive && nd >= 1 && nd <= 16;
    if (ok)
      for (size_t q = 0; q < nd; ++q) leaves[q] = deps[q];
    nleaves = nd;
    if (cudaStreamEndCapture(s, &tmp) != cudaSuccess) ok = false;
  }
  if (ok) {
    // zeroed storage: the parameter union has no default constructor
    alignas(cudaGraphNodeParams) unsigned char prm_raw[sizeof(cudaGraphNodeParams)];
    memset(prm_raw, 0, sizeof(prm_raw));
    cudaGraphNodeParams& prm = *reinterpret_cast<cudaGraphNodeParams*>(prm_raw);
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    ok = cudaGraphAddNode(&cond, g, leaves, nullptr, nleaves, &prm) == cudaSuccess;
    if (ok) {
      cudaGraph_t body = prm.conditional.phGraph_out[0];
      ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, mode) == cudaSuccess;
      if (ok) {
        const long nb0 = c->nlaunch;
        graph_body(c, p, h);
        n_body = c->nlaunch - nb0;
        if (cudaStreamEndCapture(s, &tmp) != cudaSuccess) ok = false;
      }
    }
  }
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(s, g, &cond, nullptr, 1, mode) == cudaSuccess;
    if (ok) {
      graph_epilogue(c, p);
      if (cudaStreamEndCapture(s, &tmp) != cudaSuccess) ok = false;
    }
  }
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  const long n_fixed = c->nlaunch - n0 - n_body;
  c->nlaunch = n0;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(s, &tmp);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();
    c->graphs_ok = 0;
    return nullptr;
  }
  auto& slot = c->gcache[c->gnext];
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot.p = p;
  slot.exec = exec;
  slot.nk = n_fixed;
  c->nk_body = n_body;
  c->gnext = (c->gnext + 1) % 8;
  *nk_fixed = n_fixed;
  return exec;
}

// The pressure solve of a stage (record slot 0..2) or of fvm_poisson_solve
// (slot 3), with beta0 already formed from alpha.  On the graph path the
// cycles, the residual and the status stay on the device (record `slot`
// and the sticky status) and *dev_side is set; otherwise the host loop
// fills cyc, rel and returns the status.
fvm_status solve(fvm_ctx* c, const void* alpha, double* p, int slot, int* cyc, double* rel,
                 bool want_rel, bool* dev_side) {
  *dev_side = false;
  if (c->graphs_ok && !c->prof) {
    long nk = 0;
    cudaGraphExec_t exec = solve_graph(c, p, &nk);
    if (exec) {
      if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) return cuda_check(c, "solve graph launch");
      c->nlaunch += nk;
      TIMED(c, FVM_K_MISC, 1, launch_ctl_store(c->ctl, c->rec + slot, c->sticky, c->stream));
      *dev_side = true;
      *cyc = 0;
      *rel = 0.0;
      return FVM_OK;
    }
  }
  if (c->mixed) return solve_mixed(c, (const float*)alpha, p, c->b, cyc, rel, want_rel);
  return solve_f64(c, p, c->b, cyc, rel, want_rel);
}

// status of a device-side record, as the host loop would have returned it
fvm_status record_status(fvm_ctx* c, const SolveCtl& r) {
  if (r.status == FVM_EUNSTABLE)
    return set_err(c, FVM_EUNSTABLE, "non-finite projection right-hand side or residual");
  if (r.status == FVM_ENOCONV)
    return set_err(c, FVM_ENOCONV, "pressure solve reached mg_max_cycles above mg_rtol");
  return FVM_OK;
}

template <typename R>
Fields<R> fields_of(void* const* a) {
  Fields<R> f;
  f.u[0] = (R*)a[0];
  f.u[1] = (R*)a[1];
  f.u[2] = (R*)a[2];
  f.alpha = (R*)a[3];
  f.T = (R*)a[4];
  f.c = (R*)a[5];
  return f;
}

// one forward-Euler stage E(X) and Y = a Sn + b E(X)
template <typename R>
fvm_status stage(fvm_ctx* c, Fields<R> X, Fields<R> Sn, Fields<R> Y, double* p, double ca,
                 double cb, double xc, int slot, int* cyc, double* rel, bool want_rel,
                 bool* dev_side) {
  cudaStream_t s = c->stream;
  const Geo& g = c->g;
  R* M[3] = {(R*)c->M[0], (R*)c->M[1], (R*)c->M[2]};
  R* us[3] = {(R*)c->us[0], (R*)c->us[1], (R*)c->us[2]};
  // smoothed alpha, normals, curvature and Marangoni vector in one kernel
  TIMED(c, FVM_K_INTERFACE, 1, launch_interface<R>(g, c->ph, c->tb, c->prm.smooth_passes, X.alpha,
                                                X.T, X.c, (R*)c->kappa, M[0], M[1], M[2], s));
  if (c->fct[0])
    TIMED(c, FVM_K_SCALARS, 1, launch_fct_ratios<R>(g, c->ph, X, c->dt_dev, (R*)c->fct[0], (R*)c->fct[1], s));
  TIMED(c, FVM_K_SCALARS, 1, launch_scalars<R>(g, c->ph, c->tb, X, Sn, Y, c->dt_dev, ca, cb, xc,
                                            (const R*)c->fct[0], (const R*)c->fct[1], s));
  if (X.c)
    TIMED(c, FVM_K_SCALARS, 1, launch_concentration<R>(g, c->ph, X, Sn, Y, c->dt_dev, ca, cb, s));
  TIMED(c, FVM_K_MOMENTUM, 1, launch_momentum<R>(g, c->ph, c->tb, X, (R*)c->kappa, M[0], M[1], M[2],
                                              us[0], us[1], us[2], c->dt_dev, s));
  TIMED(c, FVM_K_DIV_RHS, 1, launch_div_rhs<R>(g, us, c->dt_dev, c->b, c->partial, s));
  TIMED(c, FVM_K_MISC, 1, launch_sum_partials(c->partial, kRedBlocks, c->scal + 3, s));
  TIMED(c, FVM_K_MISC, 1, launch_sub_mean(c->b, g.N, c->scal + 3, s));
  fvm_status st;
  if (c->mixed) {
    float* be[3] = {(float*)c->beta0[0], (float*)c->beta0[1], (float*)c->beta0[2]};
    TIMED(c, FVM_K_BETA, 1, launch_beta<R, float>(g, c->ph, (const R*)X.alpha, be[0], be[1], be[2], s));
    st = solve(c, X.alpha, p, slot, cyc, rel, want_rel, dev_side);
    if (st && st != FVM_ENOCONV) return st;
    TIMED(c, FVM_K_CORRECT, 1, launch_correct<R, float>(g, Sn, Y, us, p, be, c->dt_dev, ca, cb, s));
  } else {
    double* be[3] = {(double*)c->beta0[0], (double*)c->beta0[1], (double*)c->beta0[2]};
    TIMED(c, FVM_K_BETA, 1, launch_beta<R, double>(g, c->ph, (const R*)X.alpha, be[0], be[1], be[2], s));
    st = solve(c, X.alpha, p, slot, cyc, rel, want_rel, dev_side);
    if (st && st != FVM_ENOCONV) return st;
    TIMED(c, FVM_K_CORRECT, 1, launch_correct<R, double>(g, Sn, Y, us, p, be, c->dt_dev, ca, cb, s));
  }
  fvm_status st2 = cuda_check(c, "stage");
  return st2 ? st2 : st;
}

template <typename R>
fvm_status step_impl(fvm_ctx* c, fvm_state* st, long step_index, double dt_in,
                     fvm_step_info* info) {
  cudaStream_t s = c->stream;
  void* sp[6] = {st->u, st->v, st->w, st->alpha, st->T, c->prm.concentration ? st->c : nullptr};
  Fields<R> Sn = fields_of<R>(sp);
  Fields<R> A = fields_of<R>(c->A);
  Fields<R> B = fields_of<R>(c->B);
  int limiter = -1;
  if (dt_in > 0.0) {
    TIMED(c, FVM_K_DT, 1, launch_set_scalar(c->dt_dev, dt_in, s));
  } else {
    TIMED(c, FVM_K_DT, 1, launch_dt_reduce<R>(c->g, c->ph, Sn, c->maxbits, c->flags, s));
    TIMED(c, FVM_K_DT, 1,
          launch_dt_final(c->g, c->ph, c->prm.cfl, c->prm.c_cap, c->prm.c_visc, c->prm.c_therm,
                          c->prm.dt_max, c->maxbits, c->dt_dev, c->lim_dev, s));
  }
  static const double RK[3][3] = {{0.0, 1.0, 0.0}, {0.75, 0.25, 1.0}, {1.0 / 3.0, 2.0 / 3.0, 0.5}};
  Fields<R> Xs[3] = {Sn, A, B};
  Fields<R> Ys[3] = {A, B, Sn};
  int cyc[3] = {0, 0, 0};
  double rel[3] = {0, 0, 0};
  bool dev[3] = {false, false, false};
  fvm_status worst = FVM_OK;
  const bool want_rel = info != nullptr;
  for (int q = 0; q < 3; ++q) {
    double xc = c->prm.q_x0 + c->prm.q_speed * c->prm.h * ((double)step_index + RK[q][2]);
    fvm_status r = stage<R>(c, Xs[q], Sn, Ys[q], st->p, RK[q][0], RK[q][1], xc, q, &cyc[q],
                            &rel[q], want_rel, &dev[q]);
    if (r == FVM_ENOCONV) worst = r;
    else if (r) return r;
  }
  if (info) {
    TIMED(c, FVM_K_DIAGNOSTICS, 1,
          launch_diagnostics<R>(c->g, c->ph, Sn, st->p, c->dt_dev, c->partial, c->maxbits, c->flags, s));
    TIMED(c, FVM_K_DIAGNOSTICS, 1, launch_sum_partials(c->partial, kRedBlocks, c->scal + 4, s));
    TIMED(c, FVM_K_DIAGNOSTICS, 1,
          launch_sum_partials(c->partial + kRedBlocks, kRedBlocks, c->scal + 5, s));
    double hs[2], dt;
    unsigned long long mb;
    int flag, lim;
    cudaError_t e = cudaMemcpyAsync(hs, c->scal + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&mb, c->maxbits, sizeof(mb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, c->flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dt, c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lim, c->lim_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
    SolveCtl recs[3];
    const bool any_dev = dev[0] || dev[1] || dev[2];
    if (e == cudaSuccess && any_dev)
      e = cudaMemcpyAsync(recs, c->rec, sizeof(recs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_err(c, FVM_ECUDA, cudaGetErrorString(e));
    for (int q = 0; q < 3; ++q) {
      if (!dev[q]) continue;
      cyc[q] = recs[q].iters;
      rel[q] = recs[q].rel;
      fvm_status r = record_status(c, recs[q]);
      if (r == FVM_EUNSTABLE) return r;
      if (r == FVM_ENOCONV) worst = r;
    }
    double mdiv;
    memcpy(&mdiv, &mb, sizeof(double));
    double h3 = c->prm.h * c->prm.h * c->prm.h;
    info->dt = dt;
    info->dt_limiter = dt_in > 0.0 ? -1 : lim;
    for (int q = 0; q < 3; ++q) {
      info->vcycles[q] = cyc[q];
      info->rel_residual[q] = rel[q];
    }
    info->max_div_dt = mdiv * dt;
    info->vol_sum = hs[0] * h3;
    info->mass_sum = hs[1] * h3;
    info->nan_flag = flag;
    if (flag) return set_err(c, FVM_EUNSTABLE, "NaN or Inf in the new state");
  }
  (void)limiter;
  fvm_status e2 = cuda_check(c, "step");
  return e2 ? e2 : worst;
}

}  // namespace

extern "C" {

fvm_status fvm_workspace_size(const fvm_params* prm, size_t* bytes) {
  if (!bytes) return FVM_EINVAL;
  if (check_params(prm)) return FVM_EINVAL;
  *bytes = plan_workspace(*prm, nullptr);
  return FVM_OK;
}

fvm_status fvm_create(const fvm_params* prm, void* workspace, size_t bytes, void* cuda_stream,
                      fvm_ctx** out) {
  if (!out) return FVM_EINVAL;
  *out = nullptr;
  if (check_params(prm)) return FVM_EINVAL;
  size_t need = plan_workspace(*prm, nullptr);
  if (!workspace) return FVM_EINVAL;
  if (((uintptr_t)workspace) % kAlign) return FVM_EINVAL;
  if (bytes < need) return FVM_ENOMEM;
  fvm_ctx* c = new (std::nothrow) fvm_ctx;
  if (!c) return FVM_ENOMEM;
  memset(c, 0, sizeof(*c));
  c->prm = *prm;
  c->stream = (cudaStream_t)cuda_stream;
  c->mixed = prm->precision == FVM_MIXED;
  c->rsz = c->mixed ? sizeof(float) : sizeof(double);
  c->ws = (char*)workspace;
  c->ws_bytes = bytes;
  plan_workspace(*prm, c);
  c->g = make_geo(*prm, c->shp[0]);
  Phys& ph = c->ph;
  for (int q = 0; q < 2; ++q) {
    ph.rho[q] = prm->rho[q];
    ph.mu[q] = prm->mu[q];
    ph.lam[q] = prm->lambda[q];
    ph.rcp[q] = prm->rho[q] * prm->cp[q];
  }
  ph.sigma0 = prm->sigma0;
  ph.dsdT = prm->dsigma_dT;
  ph.T0 = prm->T0;
  for (int d = 0; d < 3; ++d) ph.g[d] = prm->g[d];
  ph.q_power = prm->q_power;
  ph.q_radius = prm->q_radius;
  ph.q_x0 = prm->q_x0;
  ph.q_y0 = prm->q_y0;
  ph.q_speed = prm->q_speed;
  ph.eps_a = prm->weno_eps * prm->weno_scale[0] * prm->weno_scale[0];
  ph.eps_T = prm->weno_eps * prm->weno_scale[1] * prm->weno_scale[1];
  ph.eps_u = prm->weno_eps * prm->weno_scale[2] * prm->weno_scale[2];
  ph.eps_n = 1e-8 / prm->h;
  ph.L[0] = prm->nx * prm->h;
  ph.L[1] = prm->ny * prm->h;
  ph.L[2] = prm->nz * prm->h;
  ph.dsdc = prm->concentration ? prm->dsigma_dc : 0.0;
  ph.c0 = prm->c0;
  ph.diff_c[0] = prm->diff_c[0];
  ph.diff_c[1] = prm->diff_c[1];
  ph.eps_c = prm->weno_eps * prm->weno_scale_c * prm->weno_scale_c;
  TBC& tb = c->tb;
  tb.axis = -1;
  for (int d = 0; d < 3; ++d) {
    bool dl = prm->tbc[2 * d] == FVM_TBC_DIRICHLET, dh = prm->tbc[2 * d + 1] == FVM_TBC_DIRICHLET;
    if (dl || dh) {
      tb.axis = d;
      tb.dir[0] = dl;
      tb.dir[1] = dh;
      tb.T0[0] = prm->tbc_T0[2 * d];
      tb.T0[1] = prm->tbc_T0[2 * d + 1];
      tb.amp[0] = prm->tbc_dTamp[2 * d];
      tb.amp[1] = prm->tbc_dTamp[2 * d + 1];
      tb.s_axis = d == 0 ? 1 : 0;
      tb.Ls = ph.L[tb.s_axis];
    }
  }
  c->graphs_ok = 1;
  if (cudaMemsetAsync(c->ctl, 0, (1 + kRecords) * sizeof(SolveCtl) + sizeof(int) +
                                     sizeof(unsigned long long), c->stream) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return FVM_ECUDA;
  }
  snprintf(c->err, sizeof(c->err), "ok");
  *out = c;
  return FVM_OK;
}

fvm_status fvm_destroy(fvm_ctx* ctx) {
  if (!ctx) return FVM_EINVAL;
  for (int q = 0; q < 8; ++q)
    if (ctx->gcache[q].exec) cudaGraphExecDestroy(ctx->gcache[q].exec);
  if (ctx->prof_ev) {
    for (int q = 0; q < 2 * kProfSlots; ++q) cudaEventDestroy(ctx->prof_ev[q]);
    free(ctx->prof_ev);
    free(ctx->prof_cls);
  }
  delete ctx;
  return FVM_OK;
}

fvm_status fvm_profile(fvm_ctx* ctx, int on) {
  if (!ctx) return FVM_EINVAL;
  if (on && !ctx->prof_ev) {
    ctx->prof_ev = (cudaEvent_t*)calloc(2 * kProfSlots, sizeof(cudaEvent_t));
    ctx->prof_cls = (int*)calloc(kProfSlots, sizeof(int));
    if (!ctx->prof_ev || !ctx->prof_cls) return set_err(ctx, FVM_ENOMEM, "host allocation failed");
    for (int q = 0; q < 2 * kProfSlots; ++q)
      if (cudaEventCreate(&ctx->prof_ev[q]) != cudaSuccess)
        return set_err(ctx, FVM_ECUDA, "cudaEventCreate failed");
  }
  if (!on) prof_fold(ctx);
  if (on) {
    prof_fold(ctx);
    for (int q = 0; q < FVM_KCLASS_COUNT; ++q) {
      ctx->prof_launches[q] = 0;
      ctx->prof_ms[q] = 0.0;
    }
  }
  ctx->prof = on ? 1 : 0;
  return FVM_OK;
}

fvm_status fvm_launch_count(fvm_ctx* ctx, int reset, long* count) {
  if (!ctx || !count) return FVM_EINVAL;
  // kernels of the device-side solve loops: cycles run so far times the
  // kernels of one cycle (read after the stream has drained)
  unsigned long long runs = 0;
  cudaError_t e = cudaMemcpyAsync(&runs, ctx->runs, sizeof(runs), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, FVM_ECUDA, cudaGetErrorString(e));
  *count = ctx->nlaunch + (long)(runs - ctx->runs_base) * ctx->nk_body;
  if (reset) {
    ctx->nlaunch = 0;
    ctx->runs_base = runs;
  }
  return FVM_OK;
}

fvm_status fvm_sync(fvm_ctx* ctx) {
  if (!ctx) return FVM_EINVAL;
  int sticky = 0;
  cudaError_t e = cudaMemcpyAsync(&sticky, ctx->sticky, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->sticky, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, FVM_ECUDA, cudaGetErrorString(e));
  if (sticky == FVM_EUNSTABLE)
    return set_err(ctx, FVM_EUNSTABLE, "a pressure solve met a non-finite norm");
  if (sticky == FVM_ENOCONV)
    return set_err(ctx, FVM_ENOCONV, "a pressure solve reached mg_max_cycles above mg_rtol");
  return FVM_OK;
}

fvm_status fvm_profile_read(fvm_ctx* ctx, int kernel_class, long* launches, double* total_ms) {
  if (!ctx || kernel_class < 0 || kernel_class >= FVM_KCLASS_COUNT || !launches || !total_ms)
    return FVM_EINVAL;
  prof_fold(ctx);
  *launches = ctx->prof_launches[kernel_class];
  *total_ms = ctx->prof_ms[kernel_class];
  return FVM_OK;
}

fvm_status fvm_step(fvm_ctx* ctx, fvm_state* st, long step_index, double dt, fvm_step_info* info) {
  if (!ctx) return FVM_EINVAL;
  if (!st || !st->u || !st->v || !st->w || !st->alpha || !st->T || !st->p)
    return set_err(ctx, FVM_EINVAL, "null state pointer");
  if (ctx->prm.concentration && !st->c)
    return set_err(ctx, FVM_EINVAL, "null concentration with concentration = 1");
  if (!(dt == dt)) return set_err(ctx, FVM_EINVAL, "dt is NaN");
  cudaGetLastError();
  if (ctx->mixed) return step_impl<float>(ctx, st, step_index, dt, info);
  return step_impl<double>(ctx, st, step_index, dt, info);
}

fvm_status fvm_poisson_solve(fvm_ctx* ctx, const void* alpha, const double* rhs, double* p,
                             fvm_step_info* info) {
  if (!ctx) return FVM_EINVAL;
  if (!alpha || !rhs || !p) return set_err(ctx, FVM_EINVAL, "null pointer");
  cudaGetLastError();
  cudaStream_t s = ctx->stream;
  const Geo& g = ctx->g;
  cudaError_t e = cudaMemcpyAsync(ctx->b, rhs, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return set_err(ctx, FVM_ECUDA, cudaGetErrorString(e));
  TIMED(ctx, FVM_K_MISC, 2, launch_sum_field<double>(ctx->b, g.N, false, ctx->partial, ctx->scal + 3, s));
  TIMED(ctx, FVM_K_MISC, 1, launch_sub_mean(ctx->b, g.N, ctx->scal + 3, s));
  int cyc = 0;
  double rel = 0.0;
  fvm_status st;
  bool dev_side = false;
  if (ctx->mixed) {
    float* be[3] = {(float*)ctx->beta0[0], (float*)ctx->beta0[1], (float*)ctx->beta0[2]};
    TIMED(ctx, FVM_K_BETA, 1, launch_beta<float, float>(g, ctx->ph, (const float*)alpha, be[0], be[1], be[2], s));
  } else {
    double* be[3] = {(double*)ctx->beta0[0], (double*)ctx->beta0[1], (double*)ctx->beta0[2]};
    TIMED(ctx, FVM_K_BETA, 1, launch_beta<double, double>(g, ctx->ph, (const double*)alpha, be[0], be[1], be[2], s));
  }
  st = solve(ctx, alpha, p, 3, &cyc, &rel, info != nullptr, &dev_side);
  if (dev_side && info) {
    SolveCtl r;
    e = cudaMemcpyAsync(&r, ctx->rec + 3, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_err(ctx, FVM_ECUDA, cudaGetErrorString(e));
    cyc = r.iters;
    rel = r.rel;
    st = record_status(ctx, r);
  }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->vcycles[0] = cyc;
    info->rel_residual[0] = rel;
    info->dt_limiter = -1;
  }
  if (st) return st;
  return cuda_check(ctx, "poisson");
}

}  // extern "C"

namespace {
template <typename R>
fvm_status predict_impl(fvm_ctx* c, const fvm_state* X_, long step_index, double dt,
                        void* const* ustar, void* alpha_out, void* T_out) {
  cudaStream_t s = c->stream;
  const Geo& g = c->g;
  void* xp[6] = {X_->u, X_->v, X_->w, X_->alpha, X_->T, c->prm.concentration ? X_->c : nullptr};
  Fields<R> X = fields_of<R>(xp);
  Fields<R> Y = X;
  Y.alpha = (R*)alpha_out;
  Y.T = (R*)T_out;
  TIMED(c, FVM_K_DT, 1, launch_set_scalar(c->dt_dev, dt, s));
  const double xc = c->prm.q_x0 + c->prm.q_speed * c->prm.h * (double)step_index;
  R* M[3] = {(R*)c->M[0], (R*)c->M[1], (R*)c->M[2]};
  TIMED(c, FVM_K_INTERFACE, 1, launch_interface<R>(g, c->ph, c->tb, c->prm.smooth_passes, X.alpha,
                                                X.T, X.c, (R*)c->kappa, M[0], M[1], M[2], s));
  Y.c = nullptr;   // the concentration update is not part of the predictor's outputs
  if (c->fct[0])
    TIMED(c, FVM_K_SCALARS, 1, launch_fct_ratios<R>(g, c->ph, X, c->dt_dev, (R*)c->fct[0], (R*)c->fct[1], s));
  TIMED(c, FVM_K_SCALARS, 1, launch_scalars<R>(g, c->ph, c->tb, X, X, Y, c->dt_dev, 0.0, 1.0, xc,
                                            (const R*)c->fct[0], (const R*)c->fct[1], s));
  TIMED(c, FVM_K_MOMENTUM, 1, launch_momentum<R>(g, c->ph, c->tb, X, (R*)c->kappa, M[0], M[1], M[2],
                                              (R*)ustar[0], (R*)ustar[1], (R*)ustar[2], c->dt_dev, s));
  return cuda_check(c, "stage predictor");
}
}  // namespace

extern "C" fvm_status fvm_stage_predict(fvm_ctx* ctx, const fvm_state* X, long step_index,
                                        double dt, void* const ustar[3], void* alpha_out,
                                        void* T_out) {
  if (!ctx) return FVM_EINVAL;
  if (!X || !X->u || !X->v || !X->w || !X->alpha || !X->T || !ustar || !ustar[0] || !ustar[1] ||
      !ustar[2] || !alpha_out || !T_out)
    return set_err(ctx, FVM_EINVAL, "null pointer");
  if (!(dt > 0.0)) return set_err(ctx, FVM_EINVAL, "dt must be > 0");
  cudaGetLastError();
  if (ctx->mixed) return predict_impl<float>(ctx, X, step_index, dt, ustar, alpha_out, T_out);
  return predict_impl<double>(ctx, X, step_index, dt, ustar, alpha_out, T_out);
}

// ----- reverse mode of one FP64 step ------------------------------------------
namespace {

const double kRK[3][3] = {{0.0, 1.0, 0.0}, {0.75, 0.25, 1.0}, {1.0 / 3.0, 2.0 / 3.0, 0.5}};

double source_x(const fvm_ctx* c, long step_index, int q) {
  return c->prm.q_x0 + c->prm.q_speed * c->prm.h * ((double)step_index + kRK[q][2]);
}

// Adjoint of one stage E(X) = (P u*(X), alpha + dt R_alpha(X), T + dt R_T(X)):
// given aE = dJ/dE, adds (dE/dX)^T aE to lu and dJ/dtheta to scal[8..9].
// X is the stage input.  kappa, as, tmp, us, b, beta0 and the adjoint
// buffers serve as scratch; aE is overwritten.
fvm_status adjoint_stage(fvm_ctx* c, const double* const* X, double xc, double* const* lu,
                         const double* pfw, int* cyc, double* rel) {
  cudaStream_t s = c->stream;
  const Geo& g = c->g;
  const long long N = g.N;
  const bool density = c->ph.rho[0] != c->ph.rho[1];
  // 0. forward quantities of the stage input: face coefficients, curvature,
  //    Marangoni vector, smoothed alpha and, with unequal densities, the
  //    momentum predictor's force sum Phi = V + f_n + f_M per face
  double* be[3] = {(double*)c->beta0[0], (double*)c->beta0[1], (double*)c->beta0[2]};
  TIMED(c, FVM_K_BETA, 1, launch_beta<double, double>(g, c->ph, X[3], be[0], be[1], be[2], s));
  double* M[3] = {(double*)c->M[0], (double*)c->M[1], (double*)c->M[2]};
  const int passes = c->prm.smooth_passes;
  TIMED(c, FVM_K_INTERFACE, 1, launch_interface<double>(g, c->ph, c->tb, passes, X[3], X[4], nullptr,
                                                     (double*)c->kappa, M[0], M[1], M[2], s));
  const double* at = X[3];
  if (passes == 1) {
    TIMED(c, FVM_K_SMOOTH, 1, launch_smooth<double>(g, X[3], (double*)c->as, s));
    at = (const double*)c->as;
  } else if (passes == 2) {
    TIMED(c, FVM_K_SMOOTH, 1, launch_smooth<double>(g, X[3], (double*)c->tmp, s));
    TIMED(c, FVM_K_SMOOTH, 1, launch_smooth<double>(g, (const double*)c->tmp, (double*)c->as, s));
    at = (const double*)c->as;
  }
  // scratch from the coefficient slots (free until the transposes below)
  double* phi[3] = {c->aK, c->aK + N, c->aK + 2 * N};
  double* ustar[3] = {c->aK + 3 * N, c->aK + 4 * N, c->aK + 5 * N};
  double* wbeta[3] = {c->aK + 6 * N, c->aK + 7 * N, c->aK + 8 * N};
  if (density) {
    const double* Xc[5] = {X[0], X[1], X[2], X[3], X[4]};
    Fields<double> Xf;
    for (int d = 0; d < 3; ++d) Xf.u[d] = (double*)Xc[d];
    Xf.alpha = (double*)Xc[3];
    Xf.T = (double*)Xc[4];
    Xf.c = nullptr;
    TIMED(c, FVM_K_MOMENTUM, 1,
          launch_momentum<double>(g, c->ph, c->tb, Xf, (double*)c->kappa, M[0], M[1], M[2],
                                  ustar[0], ustar[1], ustar[2], c->dt_dev, s, phi));
  }
  // 1. projection: u = P u* with P = I + beta G L^+ D, so the adjoint of u*
  //    is P^T aE_u = aE_u + G L^+ D (beta aE_u): the same solve on the
  //    divergence of beta aE_u, then the plain gradient (wall faces zeroed on
  //    both sides, as the forward zeroes them)
  double* aEu[3] = {c->aE[0], c->aE[1], c->aE[2]};
  double* lus[3] = {(double*)c->us[0], (double*)c->us[1], (double*)c->us[2]};
  TIMED(c, FVM_K_ADJOINT, 1, launch_zero_wall_faces(g, aEu, s));
  TIMED(c, FVM_K_ADJOINT, 1, launch_face_mul(g, be, aEu, wbeta, s));
  TIMED(c, FVM_K_DIV_RHS, 1, launch_div_rhs<double>(g, wbeta, c->dt_dev, c->b, c->partial, s));
  TIMED(c, FVM_K_MISC, 1, launch_sum_partials(c->partial, kRedBlocks, c->scal + 3, s));
  TIMED(c, FVM_K_MISC, 1, launch_sub_mean(c->b, N, c->scal + 3, s));
  TIMED(c, FVM_K_MISC, 1, launch_zero<double>(c->ap, N, s));
  fvm_status st = solve_f64(c, c->ap, c->b, cyc, rel, true);
  if (st && st != FVM_ENOCONV) return st;
  fvm_status worst = st;
  TIMED(c, FVM_K_CORRECT, 1, launch_sub_grad(g, aEu, c->ap, c->dt_dev, lus, s));
  TIMED(c, FVM_K_MISC, 1, launch_zero<double>(c->akap, N, s));
  for (int d = 0; d < 3; ++d) TIMED(c, FVM_K_MISC, 1, launch_zero<double>(c->aM[d], N, s));
  TIMED(c, FVM_K_MISC, 1, launch_zero<double>(c->aat, N, s));
  // 3. transposes of the scalar update, the momentum predictor and the
  //    interface geometry, then of the smoothing passes
  AdjArgs A;
  A.g = g;
  A.tb = c->tb;
  for (int q = 0; q < 5; ++q) A.X[q] = X[q];
  A.kappa = (const double*)c->kappa;
  A.at = at;
  for (int d = 0; d < 3; ++d) A.lus[d] = lus[d];
  A.laE = c->aE[3];
  A.lTE = c->aE[4];
  for (int q = 0; q < 5; ++q) A.lu[q] = lu[q];
  A.lkap = c->akap;
  for (int d = 0; d < 3; ++d) A.lM[d] = c->aM[d];
  A.lat = c->aat;
  A.dth = c->scal + 8;
  A.K = c->aK;
  A.dt = c->adj_dt;
  const Phys& ph = c->ph;
  A.eps_a = ph.eps_a;
  A.eps_T = ph.eps_T;
  A.eps_u = ph.eps_u;
  A.eps_n = ph.eps_n;
  for (int q = 0; q < 2; ++q) {
    A.rho[q] = ph.rho[q];
    A.mu[q] = ph.mu[q];
    A.lam[q] = ph.lam[q];
    A.rcp[q] = ph.rcp[q];
  }
  for (int d = 0; d < 3; ++d) {
    A.beta[d] = be[d];
    A.phi[d] = phi[d];
  }
  A.pfw = pfw;
  A.sigma0 = ph.sigma0;
  A.dsdT = ph.dsdT;
  A.T0 = ph.T0;
  const double r2 = ph.q_radius * ph.q_radius;
  A.qunit = r2 > 0.0 ? 2.0 / (M_PI * r2) : 0.0;
  A.ir2 = r2 > 0.0 ? 1.0 / r2 : 0.0;
  A.xc = xc;
  A.yc = ph.q_y0;
  A.qpower = ph.q_power;
  for (int d = 0; d < 3; ++d) A.L[d] = ph.L[d];
  if (density) TIMED(c, FVM_K_ADJOINT, 1, launch_adj_density(A, s));
  TIMED(c, FVM_K_ADJOINT, 8, launch_adj_scalars(A, s));
  TIMED(c, FVM_K_ADJOINT, 7, launch_adj_momentum(A, s));
  TIMED(c, FVM_K_ADJOINT, 8, launch_adj_interface(A, s));
  // the smoothing pass is a symmetric matrix: its transpose is itself
  const double* lsm = c->aat;
  if (passes == 1) {
    TIMED(c, FVM_K_SMOOTH, 1, launch_smooth<double>(g, c->aat, c->atmp, s));
    lsm = c->atmp;
  } else if (passes == 2) {
    TIMED(c, FVM_K_SMOOTH, 1, launch_smooth<double>(g, c->aat, c->atmp, s));
    TIMED(c, FVM_K_SMOOTH, 1, launch_smooth<double>(g, (const double*)c->atmp, c->aat, s));
  }
  TIMED(c, FVM_K_ADJOINT, 1, launch_axpby(N, 1.0, lsm, 1.0, lu[3], s));
  fvm_status e = cuda_check(c, "adjoint stage");
  return e ? e : worst;
}

fvm_status step_adjoint_impl(fvm_ctx* c, const fvm_state* st_n, long step_index, double dt,
                             const fvm_state* lam_np1, fvm_state* lam_n, double* dtheta) {
  cudaStream_t s = c->stream;
  const long long N = c->g.N;
  c->adj_dt = dt;
  TIMED(c, FVM_K_DT, 1, launch_set_scalar(c->dt_dev, dt, s));
  // recompute the inputs of stages 2 and 3 (A, B) from st_n
  cudaError_t ce =
      cudaMemcpyAsync(c->apf, st_n->p, N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (ce != cudaSuccess) return set_err(c, FVM_ECUDA, cudaGetErrorString(ce));
  void* sp[6] = {st_n->u, st_n->v, st_n->w, st_n->alpha, st_n->T, nullptr};
  Fields<double> Sn = fields_of<double>(sp);
  Fields<double> A = fields_of<double>(c->A);
  Fields<double> B = fields_of<double>(c->B);
  int cyc = 0;
  double rel = 0.0;
  fvm_status worst = FVM_OK;
  bool recomputed_on_device = false;
  // with unequal densities the third stage is recomputed as well (into the
  // free adjoint buffers): every stage's forward pressure enters the adjoint
  const bool density = c->ph.rho[0] != c->ph.rho[1];
  Fields<double> Y2 = fields_of<double>(c->A);
  for (int f = 0; f < 5; ++f) {
    double* t = c->aL[f];
    if (f < 3) Y2.u[f] = t;
    else if (f == 3) Y2.alpha = t;
    else Y2.T = t;
  }
  for (int q = 0; q < (density ? 3 : 2); ++q) {
    bool dev_side = false;
    Fields<double> Xs = q == 0 ? Sn : (q == 1 ? A : B);
    Fields<double> Ys = q == 0 ? A : (q == 1 ? B : Y2);
    fvm_status r = stage<double>(c, Xs, Sn, Ys, c->apf, kRK[q][0], kRK[q][1],
                                 source_x(c, step_index, q), q, &cyc, &rel, false, &dev_side);
    recomputed_on_device = recomputed_on_device || dev_side;
    if (r == FVM_ENOCONV) worst = r;
    else if (r) return r;
    if (density) {
      ce = cudaMemcpyAsync(c->apst[q], c->apf, N * sizeof(double), cudaMemcpyDeviceToDevice, s);
      if (ce != cudaSuccess) return set_err(c, FVM_ECUDA, cudaGetErrorString(ce));
    }
  }
  const double* Xq[3][5] = {
      {(const double*)st_n->u, (const double*)st_n->v, (const double*)st_n->w,
       (const double*)st_n->alpha, (const double*)st_n->T},
      {(const double*)c->A[0], (const double*)c->A[1], (const double*)c->A[2],
       (const double*)c->A[3], (const double*)c->A[4]},
      {(const double*)c->B[0], (const double*)c->B[1], (const double*)c->B[2],
       (const double*)c->B[3], (const double*)c->B[4]}};
  double* out[5] = {(double*)lam_n->u, (double*)lam_n->v, (double*)lam_n->w,
                    (double*)lam_n->alpha, (double*)lam_n->T};
  const double* lamY[5] = {(const double*)lam_np1->u, (const double*)lam_np1->v,
                           (const double*)lam_np1->w, (const double*)lam_np1->alpha,
                           (const double*)lam_np1->T};
  TIMED(c, FVM_K_MISC, 1, launch_zero<double>(c->scal + 8, 2, s));
  // reverse sweep over Y_q = a_q S_n + b_q E(X_q), X_0 = S_n, X_{q+1} = Y_q:
  // out accumulates the a_q terms and, last, the stage-1 transpose
  for (int q = 2; q >= 0; --q) {
    for (int f = 0; f < 5; ++f) {
      if (q == 2) {
        TIMED(c, FVM_K_ADJOINT, 1, launch_axpby(N, kRK[q][0], lamY[f], 0.0, out[f], s));
      } else if (kRK[q][0] != 0.0) {
        TIMED(c, FVM_K_ADJOINT, 1, launch_axpby(N, kRK[q][0], lamY[f], 1.0, out[f], s));
      }
      TIMED(c, FVM_K_ADJOINT, 1, launch_axpby(N, kRK[q][1], lamY[f], 0.0, c->aE[f], s));
    }
    double* const* lu = out;
    if (q > 0) {
      for (int f = 0; f < 5; ++f) TIMED(c, FVM_K_MISC, 1, launch_zero<double>(c->aL[f], N, s));
      lu = c->aL;
    }
    fvm_status r = adjoint_stage(c, Xq[q], source_x(c, step_index, q), lu,
                                 density ? c->apst[q] : nullptr, &cyc, &rel);
    if (r == FVM_ENOCONV) worst = r;
    else if (r) return r;
    for (int f = 0; f < 5; ++f) lamY[f] = c->aL[f];
  }
  TIMED(c, FVM_K_ADJOINT, 1, launch_zero_wall_faces(c->g, out, s));
  double th[2];
  SolveCtl recs[3];
  ce = cudaMemcpyAsync(th, c->scal + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess && recomputed_on_device)
    ce = cudaMemcpyAsync(recs, c->rec, sizeof(recs), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return set_err(c, FVM_ECUDA, cudaGetErrorString(ce));
  if (recomputed_on_device)
    for (int q = 0; q < (density ? 3 : 2); ++q) {
      fvm_status r = record_status(c, recs[q]);
      if (r == FVM_EUNSTABLE) return r;
      if (r == FVM_ENOCONV) worst = r;
    }
  dtheta[0] += th[0];
  dtheta[1] += th[1];
  fvm_status e = cuda_check(c, "step adjoint");
  return e ? e : worst;
}

}  // namespace

extern "C" fvm_status fvm_step_adjoint(fvm_ctx* ctx, const fvm_state* st_n, long step_index,
                                       double dt, const fvm_state* lam_np1, fvm_state* lam_n,
                                       double dtheta[2]) {
  if (!ctx) return FVM_EINVAL;
  if (!st_n || !st_n->u || !st_n->v || !st_n->w || !st_n->alpha || !st_n->T || !st_n->p ||
      !lam_np1 || !lam_np1->u || !lam_np1->v || !lam_np1->w || !lam_np1->alpha || !lam_np1->T ||
      !lam_n || !lam_n->u || !lam_n->v || !lam_n->w || !lam_n->alpha || !lam_n->T || !dtheta)
    return set_err(ctx, FVM_EINVAL, "null pointer");
  if (!ctx->prm.adjoint) return set_err(ctx, FVM_EINVAL, "context created without adjoint = 1");
  if (ctx->mixed) return set_err(ctx, FVM_EUNSUPPORTED, "the adjoint is FP64 only");
  const fvm_params& p = ctx->prm;
  if (p.mu[0] != p.mu[1] || p.lambda[0] != p.lambda[1] ||
      p.rho[0] * p.cp[0] != p.rho[1] * p.cp[1])
    return set_err(ctx, FVM_EUNSUPPORTED,
                   "the adjoint needs equal viscosity, conductivity and rho c_p in both phases");
  if (!(dt > 0.0)) return set_err(ctx, FVM_EINVAL, "dt must be > 0");
  const void* a[5] = {lam_np1->u, lam_np1->v, lam_np1->w, lam_np1->alpha, lam_np1->T};
  const void* b[5] = {lam_n->u, lam_n->v, lam_n->w, lam_n->alpha, lam_n->T};
  for (int q = 0; q < 5; ++q)
    for (int r = 0; r < 5; ++r)
      if (a[q] == b[r]) return set_err(ctx, FVM_EINVAL, "lam_n aliases lam_np1");
  cudaGetLastError();
  return step_adjoint_impl(ctx, st_n, step_index, dt, lam_np1, lam_n, dtheta);
}

extern "C" {

const char* fvm_status_string(fvm_status s) {
  switch (s) {
    case FVM_OK: return "ok";
    case FVM_EINVAL: return "invalid argument";
    case FVM_ENOMEM: return "workspace too small";
    case FVM_ECUDA: return "CUDA error";
    case FVM_ENOCONV: return "pressure solve did not converge";
    case FVM_EUNSTABLE: return "non-finite values";
    case FVM_ETIMEOUT: return "device wait timed out";
    case FVM_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* fvm_last_error(const fvm_ctx* ctx) { return ctx ? ctx->err : "no context"; }

const char* fvm_version(void) { return "fvm-gb300 0.1"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free pressure solve.
//
// Some callers cannot call cudaMalloc: a plugin running inside a host
// application that owns the whole device memory pool and hands the library
// only its own field pointers, or real-time loops where any allocation is
// forbidden once running.  fvm_poisson_solve_noalloc() serves them: it keeps
// its scratch in the file-scope device array below, so neither it nor the
// caller allocates anything.  The array is sized for grids of up to 64^3
// cells and is held by every GPU that loads the library, until exit.
//
// In host code the array's name is only a host-side stand-in, never a device
// address.  The first call on each device therefore looks up the real
// address with cudaGetSymbolAddress() while that device is current and keeps
// it for the device; make that first call before any stream capture.  All
// calls share the one array and it keeps the previous call's contents: the
// solve initialises every scratch value it reads (the right-hand side copy,
// the face coefficients, each level's correction, the reduction slots), and
// calls that overlap on the GPU (other streams, other host threads) race on
// the array.
static constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kNoAllocMaxDevices = 64;

void* g_noalloc_ptr[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// device address of the scratch array on the current device (looked up once
// per device, under a lock, so that host threads may make first calls
// concurrently; the address stays valid until cudaDeviceReset on the device)
fvm_status noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return FVM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return FVM_ECUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return FVM_OK;
}

// layout of the pressure solve's scratch only (no stage buffers)
size_t plan_noalloc(const fvm_params& p, fvm_ctx* c, char* base) {
  Plan pl;
  LevelShape lv[kMaxLevels];
  const int nl = build_levels(p, lv);
  const long long N = (long long)p.nx * p.ny * p.nz;
  const bool mixed = p.precision == FVM_MIXED;
  const size_t ms = mixed ? sizeof(float) : sizeof(double);
  size_t o_b = pl.take(N * sizeof(double));
  size_t o_beta[3];
  for (int q = 0; q < 3; ++q) o_beta[q] = pl.take(N * ms);
  size_t o_e = 0, o_r = 0;
  if (mixed) {
    o_e = pl.take(N * sizeof(float));
    o_r = pl.take(N * sizeof(float));
  }
  size_t o_lx[kMaxLevels], o_lb[kMaxLevels], o_lbeta[kMaxLevels][3];
  for (int l = 1; l < nl; ++l) {
    const long long n = (long long)lv[l].n[0] * lv[l].n[1] * lv[l].n[2];
    o_lx[l] = pl.take(n * ms);
    o_lb[l] = pl.take(n * ms);
    for (int q = 0; q < 3; ++q) o_lbeta[l][q] = pl.take(n * ms);
  }
  const long long nc = (long long)lv[nl - 1].n[0] * lv[nl - 1].n[1] * lv[nl - 1].n[2];
  size_t o_cg[3];
  for (int q = 0; q < 3; ++q) o_cg[q] = pl.take((q == 2 ? 2 : 1) * nc * sizeof(double));
  size_t o_part = pl.take(2 * kRedBlocks * sizeof(double));
  size_t o_scal = pl.take(16 * sizeof(double));
  if (c) {
    c->b = (double*)(base + o_b);
    for (int q = 0; q < 3; ++q) c->beta0[q] = base + o_beta[q];
    c->e32 = mixed ? (float*)(base + o_e) : nullptr;
    c->r32 = mixed ? (float*)(base + o_r) : nullptr;
    c->nlev = nl;
    for (int l = 0; l < nl; ++l) c->shp[l] = lv[l];
    for (int l = 1; l < nl; ++l) {
      c->lx[l] = base + o_lx[l];
      c->lb[l] = base + o_lb[l];
      for (int q = 0; q < 3; ++q) c->lbeta[l][q] = base + o_lbeta[l][q];
    }
    for (int q = 0; q < 3; ++q) c->cg[q] = base + o_cg[q];
    c->partial = (double*)(base + o_part);
    c->scal = (double*)(base + o_scal);
  }
  return pl.off;
}

// material constants of the solve, as fvm_create() sets them
void noalloc_physics(const fvm_params* prm, fvm_ctx* c) {
  for (int q = 0; q < 2; ++q) {
    c->ph.rho[q] = prm->rho[q];
    c->ph.mu[q] = prm->mu[q];
    c->ph.lam[q] = prm->lambda[q];
    c->ph.rcp[q] = prm->rho[q] * prm->cp[q];
  }
  c->ph.eps_n = 1e-8 / prm->h;
  c->ph.L[0] = prm->nx * prm->h;
  c->ph.L[1] = prm->ny * prm->h;
  c->ph.L[2] = prm->nz * prm->h;
  c->tb.axis = -1;
}

}  // namespace

extern "C" fvm_status fvm_poisson_solve_noalloc(const fvm_params* prm, const void* alpha,
                                                const double* rhs, double* p, void* cuda_stream,
                                                fvm_step_info* info) {
  if (check_params(prm) || !alpha || !rhs || !p) return FVM_EINVAL;
  if (plan_noalloc(*prm, nullptr, nullptr) > kNoAllocScratchBytes) return FVM_ENOMEM;
  void* base = nullptr;
  fvm_status st = noalloc_scratch(&base);
  if (st) return st;
  cudaGetLastError();
  fvm_ctx c;                       // host stack only: nothing is allocated
  memset(&c, 0, sizeof(c));
  c.prm = *prm;
  c.stream = (cudaStream_t)cuda_stream;
  c.mixed = prm->precision == FVM_MIXED;
  c.rsz = c.mixed ? sizeof(float) : sizeof(double);
  c.ws = (char*)base;
  c.ws_bytes = kNoAllocScratchBytes;
  plan_noalloc(*prm, &c, (char*)base);
  c.g = make_geo(*prm, c.shp[0]);
  noalloc_physics(prm, &c);
  cudaStream_t s = c.stream;
  const Geo& g = c.g;
  cudaError_t e = cudaMemcpyAsync(c.b, rhs, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FVM_ECUDA;
  }
  TIMED(&c, FVM_K_MISC, 2, launch_sum_field<double>(c.b, g.N, false, c.partial, c.scal + 3, s));
  TIMED(&c, FVM_K_MISC, 1, launch_sub_mean(c.b, g.N, c.scal + 3, s));
  int cyc = 0;
  double rel = 0.0;
  if (c.mixed) {
    float* be[3] = {(float*)c.beta0[0], (float*)c.beta0[1], (float*)c.beta0[2]};
    TIMED(&c, FVM_K_BETA, 1, launch_beta<float, float>(g, c.ph, (const float*)alpha, be[0], be[1], be[2], s));
    st = solve_mixed(&c, (const float*)alpha, p, c.b, &cyc, &rel, info != nullptr);
  } else {
    double* be[3] = {(double*)c.beta0[0], (double*)c.beta0[1], (double*)c.beta0[2]};
    TIMED(&c, FVM_K_BETA, 1, launch_beta<double, double>(g, c.ph, (const double*)alpha, be[0], be[1], be[2], s));
    st = solve_f64(&c, p, c.b, &cyc, &rel, info != nullptr);
  }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->vcycles[0] = cyc;
    info->rel_residual[0] = rel;
    info->dt_limiter = -1;
  }
  if (st) return st;
  return cuda_check(&c, "poisson (no allocation)");
}
