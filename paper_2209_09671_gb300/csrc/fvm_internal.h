// Internal declarations shared by the translation units of libfvm.
// Host-side launchers are declared here; kernels live in fvm_stage.cu
// (one forward-Euler stage: smoothing, interface geometry, scalar transport,
// momentum predictor, projection right-hand side, correction) and fvm_mg.cu
// (geometric multigrid, reductions); the reverse-mode kernels are declared in
// fvm_adjoint.h.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/fvm.h"

namespace fvm {

enum { PER = 0, WALL = 1 };

// Geometry of one grid level.
struct Geo {
  int n[3];          // cells per axis x, y, z
  int bc[3];         // PER or WALL per axis
  double h;          // cell edge of the finest level (fine kernels)
  double ih;         // 1 / h
  double hd[3];      // cell edge per axis on this level (multigrid)
  double w[3];       // 1 / hd^2 (0 for an axis of one cell: no coupling)
  long long sy, sz;  // strides of y and z
  long long N;       // cell count (< 2^31, checked at create)
};

// Dirichlet temperature walls (at most one axis carries them).
struct TBC {
  int axis;           // -1: no Dirichlet side
  int dir[2];         // 1 if the low / high side of `axis` is Dirichlet
  double T0[2], amp[2];
  int s_axis;         // tangential coordinate of the cosine
  double Ls;          // domain length along s_axis
};

// Material and source parameters (in the form the kernels use).
struct Phys {
  double rho[2], mu[2], lam[2], rcp[2];   // rcp = rho * cp per phase
  double sigma0, dsdT, T0;
  double g[3];
  double q_power, q_radius, q_x0, q_y0, q_speed;
  double eps_a, eps_T, eps_u;             // WENO eps per field
  double eps_n;                           // normal regulariser 1e-8 / h
  double L[3];                            // domain lengths
  double dsdc, c0;                        // sigma += dsdc (c - c0) with a concentration
  double diff_c[2];                       // diffusivity of c per phase
  double eps_c;                           // WENO eps of c
};

// Pointers of one state (u, v, w, alpha, T and the concentration c, null
// when there is none) in the working precision R.
template <typename R>
struct Fields {
  R* u[3];
  R* alpha;
  R* T;
  R* c;
};

// One multigrid level in precision T.
template <typename T>
struct MGLevel {
  Geo geo;
  T* x;
  T* b;
  T* beta[3];
  T w[3];            // 1 / hd^2 in the level's precision (0: no coupling)
  int f[3];          // coarsening factor to the next level
};

constexpr int kMaxLevels = 24;
// thread-block tile of the stage kernels (x fastest)
constexpr int kBX = 32, kBY = 4, kBZ = 4;
constexpr int kRedBlocks = 1024;   // partial-sum slots of the two-pass reductions

// ----- stage launchers (fvm_stage.cu) --------------------------------------
template <typename R>
void launch_smooth(const Geo& g, const R* in, R* out, cudaStream_t s);
// smoothing (passes 0..2), face normals, curvature and Marangoni vector
template <typename R>
void launch_interface(const Geo& g, const Phys& ph, const TBC& tb, int passes, const R* alpha,
                      const R* T, const R* c, R* kappa, R* M0, R* M1, R* M2, cudaStream_t s);
// fct_p / fct_m: limiter ratios of the bounded alpha transport (null: WENO5)
template <typename R>
void launch_scalars(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, Fields<R> Sn,
                    Fields<R> Y, const double* dt, double a, double b, double xc_shift,
                    const R* fct_p, const R* fct_m, cudaStream_t s);
// limiter ratios R+, R- of the bounded alpha transport (flux-corrected
// blend of upwind and WENO5 fluxes with the bounds 0 and 1)
template <typename R>
void launch_fct_ratios(const Geo& g, const Phys& ph, Fields<R> X, const double* dt, R* Rp, R* Rm,
                       cudaStream_t s);
// transport of the concentration c (WENO5 advection, diffusion) and its stage
// update Y.c = a Sn.c + b (X.c + dt R_c)
template <typename R>
void launch_concentration(const Geo& g, const Phys& ph, Fields<R> X, Fields<R> Sn, Fields<R> Y,
                          const double* dt, double a, double b, cudaStream_t s);
// phi (optional): the force sum V + f_n + f_M of every face before 1/rho_f
template <typename R>
void launch_momentum(const Geo& g, const Phys& ph, const TBC& tb, Fields<R> X, const R* kappa,
                     const R* M0, const R* M1, const R* M2, R* us0, R* us1, R* us2,
                     const double* dt, cudaStream_t s, R* const* phi = nullptr);
template <typename R>
void launch_div_rhs(const Geo& g, R* const* us, const double* dt, double* b, double* partial,
                    cudaStream_t s);
template <typename R, typename B>
void launch_beta(const Geo& g, const Phys& ph, const R* alpha, B* b0, B* b1, B* b2,
                 cudaStream_t s);
template <typename R, typename B>
void launch_correct(const Geo& g, Fields<R> Sn, Fields<R> Y, R* const* us, const double* p,
                    B* const* beta, const double* dt, double a, double b, cudaStream_t s);
template <typename R>
void launch_dt_reduce(const Geo& g, const Phys& ph, Fields<R> X, unsigned long long* maxbits,
                      int* nanflag, cudaStream_t s);
void launch_dt_final(const Geo& g, const Phys& ph, double cfl, double c_cap, double c_visc,
                     double c_therm, double dt_max, const unsigned long long* maxbits,
                     double* dt, int* limiter, cudaStream_t s);
void launch_set_scalar(double* dst, double v, cudaStream_t s);
template <typename R>
void launch_diagnostics(const Geo& g, const Phys& ph, Fields<R> X, const double* p,
                        const double* dt, double* partial, unsigned long long* maxbits,
                        int* nanflag, cudaStream_t s);

// ----- reductions and multigrid (fvm_mg.cu) ----------------------------------
// Deterministic two-pass sums: per-block partial sums in `partial`, then one
// block adds them in a fixed order into *out.
void launch_sum_partials(const double* partial, int nparts, double* out, cudaStream_t s);
template <typename T>
void launch_sum_field(const T* a, long long n, bool squares, double* partial, double* out,
                      cudaStream_t s);
void launch_sub_mean(double* a, long long n, const double* sum, cudaStream_t s);
template <typename T>
void launch_zero(T* a, long long n, cudaStream_t s);

// gate (optional): the sweep does nothing once *gate >= gate_min
template <typename T>
void launch_gs(const MGLevel<T>& L, int colour, cudaStream_t s, const int* gate = nullptr,
               int gate_min = 0);


template <typename T>
void launch_residual_restrict(const MGLevel<T>& F, const MGLevel<T>& C, cudaStream_t s,
                              bool sweep = false);
template <typename T>
void launch_prolong(const MGLevel<T>& F, const MGLevel<T>& C, cudaStream_t s);
// a sweep of `colour` on F reading the other colour plus the coarse
// correction C.x of its parent cells (the prolongation folded into the sweep)
template <typename T>
void launch_gs_prolong(const MGLevel<T>& F, const MGLevel<T>& C, int colour, cudaStream_t s);
// a sweep of `colour` from x = 0 that also zeroes the other colour
template <typename T>
void launch_gs_zero(const MGLevel<T>& L, int colour, cudaStream_t s);
// a float sweep of `colour` that adds the new values of its cells and the
// values of the other colour to the double p (p += x after the sweep)
void launch_gs_addp(const MGLevel<float>& L, int colour, double* p, cudaStream_t s);
template <typename T>
void launch_beta_coarsen(const MGLevel<T>& F, const MGLevel<T>& C, cudaStream_t s);
// The coarse tail of a V-cycle (levels of at most kTailCells cells, the
// coarsest solved by CG) in one CTA
constexpr int kTailCells = 4096;
constexpr int kTailLevels = 8;
template <typename T>
struct TailArgs {
  int nl;                      // levels in the tail, the last one the coarsest
  MGLevel<T> L[kTailLevels];
  double *r, *d, *Ad;          // CG vectors (as launch_coarse_cg)
  double rtol;
  int maxit, pre, post;
};
template <typename T>
void launch_coarse_tail(const TailArgs<T>& A, cudaStream_t s);
// CG vectors are double in both precisions (the coarsest level is small)
template <typename T>
void launch_coarse_cg(const MGLevel<T>& L, double* r, double* d, double* Ad, double rtol,
                      int maxit, cudaStream_t s);
// ||b - L x||^2 into *out (double), x, b, beta in precision T
template <typename T>
void launch_residual_norm2(const MGLevel<T>& L, double* partial, double* out, cudaStream_t s);
// Mixed form: r = b - L p in double with float beta; writes r32 and ||r||^2
void launch_residual64(const Geo& g, const double* p, const double* b, float* const* beta,
                       float* r32, double* partial, double* out, cudaStream_t s,
                       float* e32 = nullptr, const float* w32 = nullptr);
void launch_add_correction(long long n, double* p, const float* e, cudaStream_t s);

// ----- device-side control of the pressure solve (fvm_mg.cu) -----------------
// The stopping test of a solve runs on the device, inside a CUDA graph with
// a conditional WHILE node: after every cycle (refinement) the controller
// kernel forms ||b - L p|| / ||b|| from the two reduction slots and sets the
// node's condition, so the host never waits for a residual.
struct SolveCtl {
  int iters;      // cycles (F64) or refinements (MIXED) done
  int status;     // 0, FVM_ENOCONV or FVM_EUNSTABLE
  int zero;       // 1: ||b|| = 0, the solution is set to 0
  int pad;
  double rel;     // last relative residual
};
void launch_ctl_reset(SolveCtl* ctl, cudaStream_t s);
// bn2 = ||b||^2 and r2 = ||b - L p||^2 (device); fixed > 0: exactly `fixed`
// cycles; runs_total counts the cycles of every solve (launch bookkeeping)
void launch_ctl_step(cudaGraphConditionalHandle h, SolveCtl* ctl, const double* bn2,
                     const double* r2, double rtol, int maxit, int fixed,
                     unsigned long long* runs_total, cudaStream_t s);
void launch_zero_if_rhs_zero(const SolveCtl* ctl, double* p, long long n, cudaStream_t s);
// copy the controller into a per-stage record and raise the sticky status
void launch_ctl_store(const SolveCtl* ctl, SolveCtl* rec, int* sticky, cudaStream_t s);

}  // namespace fvm
