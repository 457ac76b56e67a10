/*
 * fvm.h -- C ABI of the GB300 library for one explicit time step of the
 * thermocapillary two-phase finite-volume method of Zimbrod, Schreter &
 * Schilp (2022): conservative phase-fraction transport (Sec. III, Eq. 1),
 * capillary stress split into a normal CSF force and a tangential Marangoni
 * force (Sec. III, Eq. 2-4), surface tension evaluated as a cell field and
 * differentiated directly (Sec. III, Eq. 5; Sec. IV), high-order WENO face
 * values (Sec. IV) and the incompressible Navier-Stokes / energy equations
 * that Sec. III names, closed by a density-weighted pressure projection.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Grid      nx x ny x nz cubic cells of edge h.  Every field is a dense
 *            array of nx*ny*nz elements in C order [k][j][i] (x fastest).
 *  Faces     velocities live on cell faces (MAC layout) in "low face" form:
 *            u[k][j][i] is the x-velocity on the face between cells i-1 and
 *            i; likewise v on y-faces and w on z-faces.  The face at index n
 *            is implied: 0 on a wall axis, equal to face 0 on a periodic
 *            axis.  On a wall axis the stored face 0 is the wall; it is
 *            ignored on input and written as 0.
 *  Phases    alpha = 1 is the phase with index [1] of the property pairs.
 *  Memory    all field pointers are DEVICE pointers owned by the caller.
 *            The library never allocates device memory: the caller passes a
 *            workspace of fvm_workspace_size() bytes to fvm_create() and
 *            keeps it alive until fvm_destroy().  The library never frees
 *            caller memory.
 *  Streams   work is enqueued on the stream given to fvm_create().
 *            fvm_step and fvm_poisson_solve with info == NULL return without
 *            waiting for the device: each pressure solve runs as one CUDA
 *            graph whose stopping test (||b - L p|| <= mg_rtol ||b||, or
 *            mg_fixed_cycles cycles) is taken on the device by a conditional
 *            loop node, so the host never reads a residual.  A solve that
 *            stops at mg_max_cycles above mg_rtol or meets a non-finite norm
 *            is then recorded on the device and reported by fvm_sync().  With
 *            info != NULL the call waits once, at its end, and returns that
 *            status itself.  The first solve with a given p pointer builds
 *            its graph (stream capture on the context's stream, so that
 *            stream must not be capturing then); while profiling is on
 *            (fvm_profile) the solves run as eager launches with a host
 *            loop instead.
 *  Errors    functions return an fvm_status; no C++ exception, abort or
 *            device trap crosses the ABI.  fvm_last_error() gives a message.
 *  Precision FVM_F64: u, v, w, alpha, T are double.  FVM_MIXED: they are
 *            float; the pressure p, the projection right-hand side, the
 *            outer residual of the pressure solve, the divergence check and
 *            the diagnostic sums stay double.
 */
#ifndef FVM_H
#define FVM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FVM_OK = 0,
  FVM_EINVAL = 1,        /* bad argument or parameter                         */
  FVM_ENOMEM = 2,        /* workspace too small                               */
  FVM_ECUDA = 3,         /* a CUDA runtime call failed                        */
  FVM_ENOCONV = 4,       /* pressure solve hit mg_max_cycles above mg_rtol    */
  FVM_EUNSTABLE = 5,     /* NaN or Inf in the state or a residual             */
  FVM_ETIMEOUT = 6,      /* reserved: a bounded device wait ran out           */
  FVM_EUNSUPPORTED = 7   /* valid but not implemented (see fvm_last_error)    */
} fvm_status;

typedef enum { FVM_F64 = 0, FVM_MIXED = 1 } fvm_precision;
typedef enum { FVM_BC_PERIODIC = 0, FVM_BC_WALL = 1 } fvm_bc_kind;
typedef enum { FVM_TBC_NEUMANN = 0, FVM_TBC_DIRICHLET = 1 } fvm_tbc_kind;

/* Parameters of the discrete method.  Sides are ordered -x,+x,-y,+y,-z,+z. */
typedef struct {
  int nx, ny, nz;            /* cells; a wall axis needs >= 4 cells, a periodic */
                             /* axis an even count or 1 (red-black colouring)   */
  double h;                  /* cell edge [m]                                   */
  int bc[3];                 /* fvm_bc_kind per axis x, y, z (no-slip walls)     */
  int tbc[6];                /* fvm_tbc_kind per side; Dirichlet on one axis max */
  double tbc_T0[6];          /* Dirichlet wall temperature                       */
  double tbc_dTamp[6];       /*   T_w = T0 + dTamp cos(2 pi s / L_s), s = x on   */
                             /*   y- and z-walls, s = y on x-walls               */
  double rho[2], mu[2], cp[2], lambda[2];  /* [0]: alpha = 0 phase, [1]: alpha = 1 */
  double sigma0, dsigma_dT, T0;            /* sigma(T) = sigma0 + dsigma_dT (T - T0) */
  double g[3];                             /* gravity [m/s^2]                    */
  double q_power, q_radius, q_x0, q_y0;    /* Gaussian surface heat flux          */
  double q_speed;                          /* centre moves q_speed*h per step in +x */
  double cfl, c_cap, c_visc, c_therm, dt_max; /* time-step limit constants       */
  double weno_eps, weno_scale[3];          /* WENO5 eps = weno_eps*scale^2 for    */
                                           /* alpha, T, velocity                 */
  int smooth_passes;                       /* [1,2,1]/4 passes for curvature      */
  int mg_levels, mg_pre, mg_post;          /* hierarchy depth cap, V(pre,post)    */
  int mg_max_cycles, mg_fixed_cycles;      /* fixed > 0: exactly that many cycles */
  double mg_rtol;                          /* ||b - L p|| <= rtol ||b||           */
  double coarse_rtol; int coarse_maxit;    /* CG on the coarsest level            */
  int precision;                           /* fvm_precision                       */
  int mx_inner_cycles;                     /* float V-cycles per double refinement */
  int adjoint;                             /* 1: also reserve the buffers of      */
                                           /* fvm_step_adjoint (F64 only)        */
  /* solutal Marangoni (Eq. 5, second term): a transported concentration c,
   * advected by WENO5 like T and diffused with the harmonic face mean of the
   * mixture diffusivity (no flux through walls); sigma(c, T) = sigma0 +
   * dsigma_dT (T - T0) + dsigma_dc (c - c0) is formed per cell and
   * differentiated as a field (Sec. IV).  concentration = 0 leaves c out. */
  int concentration;                       /* 1: fvm_state.c is transported      */
  double dsigma_dc, c0;
  double diff_c[2];                        /* diffusivity of c per phase (>= 0)  */
  double weno_scale_c;                     /* WENO5 eps = weno_eps*scale_c^2     */
  /* phase-fraction fluxes (Eq. 1): 0 WENO5; 1 bounded, the flux-corrected
   * blend (Zalesak 1979) of the first-order upwind and the WENO5 flux that
   * keeps every stage's alpha within [0, 1] (the paper's Sec. V-A mixes
   * first-order bounded and high-order WENO schemes); not with adjoint = 1 */
  int alpha_scheme;
  /* red-black sweeps before and after the coarse correction on every level
   * below the finest (0: mg_pre and mg_post there too); the coarse levels are
   * small and cache-resident, and three sweeps there halve the V-cycle's
   * convergence factor on the melt-pool operator (0.15 -> 0.08) */
  int mg_coarse_sweeps;
} fvm_params;

/* Caller-owned device fields of one state. u, v, w, alpha, T (and c): double
 * (F64) or float (MIXED); p: double in both forms.  c is the concentration
 * when fvm_params.concentration = 1 (required then, ignored otherwise). */
typedef struct {
  void *u, *v, *w, *alpha, *T;
  double *p;
  void *c;
} fvm_state;

typedef struct {
  double dt;              /* step used                                          */
  int dt_limiter;         /* 0 CFL, 1 capillary, 2 viscous, 3 thermal, 4 dt_max,  */
                          /* -1 when the caller gave dt                         */
  int vcycles[3];         /* pressure V-cycles (F64) or refinements (MIXED) per stage */
  double rel_residual[3]; /* final ||b - L p|| / ||b|| per stage                  */
  double max_div_dt;      /* max |D u| dt of the new velocity                   */
  double vol_sum;         /* sum alpha h^3                                      */
  double mass_sum;        /* sum rho(alpha) h^3                                 */
  int nan_flag;           /* 1 if the new state holds NaN/Inf                   */
} fvm_step_info;

typedef struct fvm_ctx fvm_ctx;

/* Bytes of device workspace the parameters need (host only, no CUDA call).
 * Returns FVM_EINVAL for invalid parameters. */
fvm_status fvm_workspace_size(const fvm_params* prm, size_t* bytes);

/* Bind parameters, a caller-owned device workspace of at least
 * fvm_workspace_size() bytes (256-byte aligned) and a cudaStream_t (NULL =
 * legacy default stream) into a context.  The context (host memory) is owned
 * by the library until fvm_destroy().  No device memory is allocated. */
fvm_status fvm_create(const fvm_params* prm, void* workspace, size_t bytes,
                      void* cuda_stream, fvm_ctx** out);

fvm_status fvm_destroy(fvm_ctx* ctx);

/* One SSP-RK3 step with a projection per stage (the paper's Sec. III system,
 * time integrator and coupling as the design notes read them), in place on
 * *st.  step_index places the moving heat source; dt <= 0 selects the
 * minimum of the CFL, capillary, viscous and thermal limits and dt_max.
 * info may be NULL.  Returns FVM_ENOCONV / FVM_EUNSTABLE as documented. */
fvm_status fvm_step(fvm_ctx* ctx, fvm_state* st, long step_index, double dt,
                    fvm_step_info* info);

/* Wait for the context's stream and return the worst status recorded by
 * the device-side pressure solves since the previous fvm_sync (FVM_ENOCONV
 * or FVM_EUNSTABLE; FVM_OK if none), clearing it. */
fvm_status fvm_sync(fvm_ctx* ctx);

/* The density-weighted pressure solve alone: L p = rhs with
 * (L p)_c = sum_faces beta_f (p_c - p_nb)/h^2, beta_f = 2/(rho_L + rho_R) from
 * alpha (0 on wall faces).  rhs (double, device) is made mean-free on a
 * device copy; p (double, device) is the initial guess on entry and the
 * mean-free solution on exit.  alpha is double (F64) or float (MIXED); in
 * MIXED form the solve is the float multigrid inside double defect
 * correction.  info->vcycles[0] and rel_residual[0] report the solve. */
fvm_status fvm_poisson_solve(fvm_ctx* ctx, const void* alpha, const double* rhs,
                             double* p, fvm_step_info* info);

/* Allocation-free variant of fvm_poisson_solve (the paper has no
 * counterpart: this serves callers that cannot allocate device memory, such
 * as a plugin inside a host application that owns the whole device memory
 * pool, or a real-time loop that must not allocate once running).
 * No context and no workspace: the solve's scratch lives in a static device
 * array of 16 MiB inside the library (held by every GPU that loads it until
 * exit), so nothing is allocated by the caller or by this call.
 *   prm      parameters as for fvm_create(); only the grid, boundary kinds,
 *            rho, the multigrid fields and precision are used.  Grids whose
 *            solve needs more than the 16 MiB (64^3 cells fit in both
 *            precisions) return FVM_ENOMEM before any device work.
 *   alpha    device, nx*ny*nz double (FVM_F64) or float (FVM_MIXED)
 *   rhs      device, nx*ny*nz double; read only (made mean-free on a copy)
 *   p        device, nx*ny*nz double: initial guess in, mean-free solution out
 *   cuda_stream  cudaStream_t for all work (NULL = legacy default stream)
 *   info     may be NULL; vcycles[0] and rel_residual[0] report the solve
 * Same arithmetic and status codes as fvm_poisson_solve (no fvm_last_error
 * message: there is no context).  The first call on a device looks up the
 * array's device address with cudaGetSymbolAddress, so make it before any
 * stream capture on that device; the address is kept until the process
 * exits and is not valid after a cudaDeviceReset of that device.  Every call
 * shares the array; calls that overlap on the GPU (several streams or host
 * threads at once) race. */
fvm_status fvm_poisson_solve_noalloc(const fvm_params* prm, const void* alpha,
                                     const double* rhs, double* p, void* cuda_stream,
                                     fvm_step_info* info);

/* The first forward-Euler stage without its projection, for testing the
 * stage-local operators at full size: smoothing, normals, curvature and
 * Marangoni vector (Sec. III, Eq. 2-5), WENO5 transport of alpha (Eq. 1) and
 * T with conduction and the surface heat flux, and the momentum predictor.
 * X: device state (p unused); dt > 0; heat-source centre at step_index.
 * ustar[3]: device outputs u*, v*, w* (working precision); alpha_out, T_out:
 * device outputs alpha + dt R_alpha and T + dt R_T.  Outputs must not alias
 * the inputs.  Uses the context's workspace. */
fvm_status fvm_stage_predict(fvm_ctx* ctx, const fvm_state* X, long step_index, double dt,
                             void* const ustar[3], void* alpha_out, void* T_out);

/* Reverse mode of one FP64 step at a given dt (the discrete adjoint that a
 * gradient-based calibration of the Sec. III model needs; the paper itself
 * differentiates nothing, so the entry point extends it).  With
 * S_{n+1} = Step(S_n; theta), theta = (dsigma_dT, q_power), it returns
 *   lam_n     = (dS_{n+1}/dS_n)^T lam_np1           (u, v, w, alpha, T)
 *   dtheta[q] = (dS_{n+1}/dtheta_q)^T lam_np1       (added to dtheta)
 * st_n: the state before the step (device, double; read only, p is the
 * warm start of the recomputed projections); lam_np1 (read only) and lam_n
 * (written, must not alias lam_np1): device double fields, layout as the
 * state; their p members are ignored.  dtheta: host, 2 doubles, ACCUMULATED
 * into (the caller zeroes them).  The stages are recomputed from st_n; the
 * three projections are adjoined by the same multigrid solve: with
 * u = P u*, P = I + beta G L^+ D, the adjoint of u* is P^T = I + G L^+ D beta
 * (L = -D beta G is symmetric); with unequal densities beta = 1/rho_f
 * depends on alpha, and the derivative of both 1/rho_f factors (momentum
 * predictor and projection) adds to the adjoint of alpha, using each
 * stage's recomputed forward pressure.  Requirements, else an error and no
 * write: a context created with adjoint = 1 (EINVAL; fvm_create accepts
 * adjoint = 1 only with precision F64, no concentration and alpha_scheme 0,
 * and the workspace then holds 43 more double fields of N cells), equal mu,
 * lambda and rho*cp in both phases (EUNSUPPORTED: the transport
 * coefficients are then constant; the densities may differ), dt > 0
 * (EINVAL).  A projection that stops at
 * mg_max_cycles above mg_rtol returns FVM_ENOCONV after completing the
 * sweep.  The derivative of |g| at g = 0 is taken as 0.  Entries of lam_n on
 * wall faces are 0.  Synchronises the context's stream. */
fvm_status fvm_step_adjoint(fvm_ctx* ctx, const fvm_state* st_n, long step_index,
                            double dt, const fvm_state* lam_np1, fvm_state* lam_n,
                            double dtheta[2]);

/* ---- measurement aid (no counterpart in the paper) ----------------------
 * Kernel classes timed with CUDA events on the context's stream while
 * profiling is on.  fvm_profile(ctx, 1) creates the events on first use
 * (driver objects, no device memory from the workspace) and zeroes the
 * totals; fvm_profile(ctx, 0) stops recording.  fvm_profile_read()
 * synchronises the stream and returns the launches and total milliseconds of
 * one class since the last fvm_profile(ctx, 1).  Timing adds two event
 * records per launch. */
typedef enum {
  FVM_K_SMOOTH = 0, FVM_K_INTERFACE, FVM_K_SCALARS, FVM_K_MOMENTUM, FVM_K_DIV_RHS,
  FVM_K_BETA, FVM_K_GS_FINE, FVM_K_GS_COARSE, FVM_K_RESTRICT_FINE, FVM_K_RESTRICT_COARSE,
  FVM_K_PROLONG_FINE, FVM_K_PROLONG_COARSE, FVM_K_COARSE_CG, FVM_K_RESNORM,
  FVM_K_RESIDUAL64, FVM_K_ADD_CORRECTION, FVM_K_CORRECT, FVM_K_DT, FVM_K_DIAGNOSTICS,
  FVM_K_MISC, FVM_K_ADJOINT, FVM_K_COARSE_TAIL, FVM_KCLASS_COUNT
} fvm_kernel_class;

fvm_status fvm_profile(fvm_ctx* ctx, int on);
fvm_status fvm_profile_read(fvm_ctx* ctx, int kernel_class, long* launches, double* total_ms);

/* Fused multiply-add throughput of the current device (no counterpart in
 * the paper; the peak against which kernels bound by arithmetic are
 * reported).  precision FVM_F64 times double FMAs, FVM_MIXED float FMAs:
 * eight independent register chains per thread over 8 blocks of 256 threads
 * per SM, best of three timed launches after one warm-up launch, timed with
 * CUDA events on cuda_stream (NULL = legacy default stream); synchronises the
 * stream.  tflops: 2 flops per FMA / time; ms: the best launch time.  No
 * device memory is allocated (the chains keep their result in registers). */
fvm_status fvm_fma_peak(int precision, void* cuda_stream, double* tflops, double* ms);

/* Number of CUDA kernels the context has launched (counted always, host
 * side); reset != 0 zeroes the counter after reading it. */
fvm_status fvm_launch_count(fvm_ctx* ctx, int reset, long* count);

const char* fvm_status_string(fvm_status s);
const char* fvm_last_error(const fvm_ctx* ctx);

/* Library version string. */
const char* fvm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FVM_H */
