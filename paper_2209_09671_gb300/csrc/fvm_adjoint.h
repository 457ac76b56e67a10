// Reverse-mode kernels of one FP64 stage (fvm_adjoint.cu) and their
// argument block.
#pragma once

#include "fvm_internal.h"

namespace fvm {

// Arguments of the reverse-mode kernels of one FP64 stage.
struct AdjArgs {
  Geo g;
  TBC tb;
  const double* X[5];      // stage input u, v, w, alpha, T
  const double* kappa;     // curvature of the stage input
  const double* at;        // smoothed alpha of the stage input
  const double* lus[3];    // adjoint of u*, v*, w*
  const double* laE;       // adjoint of alpha + dt R_alpha
  const double* lTE;       // adjoint of T + dt R_T
  double* lu[5];           // accumulated adjoint of the stage input
  double* lkap;            // adjoint of kappa
  double* lM[3];           // adjoint of the Marangoni vector
  double* lat;             // adjoint of the smoothed alpha
  double* dth;             // [2]: d/d(dsigma/dT), d/d(q_power)
  double* K;               // kAdjSlots coefficient slots of N doubles each
  double dt, eps_a, eps_T, eps_u, eps_n;
  double rho[2], mu[2], lam[2], rcp[2];
  const double* beta[3];   // 1 / rho_f on the faces of the stage input (low-face form)
  const double* pfw;       // the stage's forward pressure (density term)
  const double* phi[3];    // the stage's forward V + f_n + f_M per face (density term)
  double sigma0, dsdT, T0;
  double qunit, ir2, xc, yc, qpower;   // qunit: peak flux per watt, 2/(pi r^2)
  double L[3];
};
constexpr int kAdjSlots = 22;
// each returns the number of kernels it launched
int launch_adj_momentum(const AdjArgs& A, cudaStream_t s);    // needs lus; adds lkap, lM
int launch_adj_scalars(const AdjArgs& A, cudaStream_t s);     // needs laE, lTE
int launch_adj_interface(const AdjArgs& A, cudaStream_t s);   // needs lkap, lM; adds lat
// d/d alpha of the stage's two 1/rho_f factors (the momentum predictor's and
// the projection's, with the adjoint of u* in lus): adds to lu[3]
int launch_adj_density(const AdjArgs& A, cudaStream_t s);
// out_d = u_d - dt (p_c - p_{c - e_d}) / h on every face, 0 on wall faces
void launch_sub_grad(const Geo& g, double* const* u, const double* p, const double* dt,
                     double* const* out, cudaStream_t s);
// out_d = beta_d u_d (face-wise products)
void launch_face_mul(const Geo& g, double* const* beta, double* const* u, double* const* out,
                     cudaStream_t s);
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s);
void launch_zero_wall_faces(const Geo& g, double* const* u, cudaStream_t s);

}  // namespace fvm
