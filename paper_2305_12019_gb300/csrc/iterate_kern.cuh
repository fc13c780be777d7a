// Arguments and launcher of the kernelized n-space iteration (iterate_kern.cu):
// Algorithm 1 run on K = Z~^T Z~ alone, with no pass over Z inside the loop.
#pragma once

#include "solver.cuh"

namespace gdwd {

struct KernArgs {
  const float2* P;       // n x ldP, G^{-1} as double-float
  const float2* Kd;      // n x ldP, K = Z~^T Z~ = mu (G - I) as double-float
  int ldP;
  const float2* pdf;     // p = G^{-1} y as double-float, padded to ldP
  const double* p;
  const double* y;
  const double* e;
  const double* omega;   // q wt_i^q
  const double* wt;
  int64_t n;
  double inv_s, q, C, mu, tau, R, tol, kappa;
  int max_iter;
  int stop_rule;
  int grid;
  int refresh;           // 1: U_u = K a_u, U_rho = K a_rho at launch start (a stored iterate)
  uint64_t timeout_ns;
  // n-space state
  double *r, *xi, *alpha, *b;
  float2 *rhsA, *rhsB;
  double *Uu, *Ur;       // K a_u, K a_rho
  double *au, *ar, *ag;  // coefficients of u, rho and g in the columns of Z~
  double *KG, *KR;       // K a_g and K a_rho of the last iteration (its deferred update)
  float2* vdf;           // 3 x ldP: alpha, a_g, a_rho as double-float (GEMV right-hand sides)
  double* scal;          // grid x S_COUNT partial sums
  unsigned* bar;
  int* err;
  Ctrl* ctrl;
};

// Largest n the kernelized iteration accepts on `grid` CTAs (one row per thread).
int64_t kern_max_n(int grid, int smem_limit);
cudaError_t run_iterate_kern(const KernArgs& a, int smem_limit, cudaStream_t st);
// Kd = mu (G - I) as double-float, rows padded to ldP with zeros.
cudaError_t run_kern_matrix(const double* G, int64_t n, int ldP, double mu, float2* Kd, cudaStream_t st);
// x_i = (a_g,i + a_rho,i / (sigma_prev sqrt(mu))) / zscale, the coefficients of
// the Step-1c w of the last iterate; sigma_prev from the control block.
cudaError_t run_kern_wcoef(const double* ag, const double* ar, const Ctrl* ctrl, double sqmu, double zscale, int64_t n,
                           double* x, cudaStream_t st);

}  // namespace gdwd
