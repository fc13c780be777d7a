// The inexact solver of eq-linsys for d and n both large (solver = 2): Algorithm
// 1 with Steps 1a and 1c solved by preconditioned conjugate gradients on the
// matrix-free (d+1) x (d+1) operator A = U U^T + diag(mu I, 0), U = [Z~; y^T]
// (Sec. 3.3.3 with T = 0), to the accuracy eq-linsys-tol with the summable
// tolerances eps_k = c / (k+1)^1.5, and Step 1c's solve skipped when Step 1a's
// solution already meets 5 eps_k for the new right-hand side.  No n x n or
// d x d matrix is formed; every product with A is two passes over the stored Z.
#pragma once

#include "solver.cuh"

namespace gdwd {

constexpr int kIxBlocks = 256;   // blocks of the reducing kernels (their partial sums)
constexpr int kIxSlots = 12;     // partial sums per block at most

struct IxArgs {
  int64_t d, n;
  const double* y;
  const double* e;
  const double* omega;      // q wt^q
  const double* wt;
  const double* mw;         // d: the Jacobi preconditioner of the w block, diag(Z~ Z~^T) + mu
  double q, C, mu, tau, R, tol, kappa, eps_c;
  int max_iter;
  int stop_rule;
  // state
  double *r, *xi, *alpha, *ztw;   // n (ztw = Z~^T w)
  double *w, *u, *rho;            // d
  double beta;
  // work
  double *v, *tn, *zp, *dr;       // n
  double *hw, *cr, *cz, *cp, *cap, *td;   // d
  double* part;                   // kIxSlots x kIxBlocks block partials (device)
  double* hpart;                  // the same on the host (pinned)
};

// Products with the stored data: trans != 0 gives out = Z~^T x (n from d),
// trans == 0 gives out = Z~ x (d from n).
struct IxPasses {
  cudaError_t (*apply)(int trans, const double* x, double* out, void* ctx);
  void* ctx;
};

struct IxResult {
  double beta, pobj, dobj, kkt, sigma;
  double eta_p1, eta_p2, eta_p3, eta_d1, eta_d2, eta_d3, eta_c1, eta_c2, eta_c3, eta_gap;
  int iters, status;
  int64_t cg_steps, step1c_solves;
};

// The set-up of the preconditioner: mw_j = sum_i (sc_i Zq_ji)^2 + mu over the
// slab layout (F32 or F64 storage).
cudaError_t run_row_sumsq(int store, const Layout& L, const double* sc, double mu, double* mw, cudaStream_t st);

// Algorithm 1 from the initial iterate to the stop rule (or max_iter), with
// sigma0 the first sigma.  All vectors of a are device memory; the loop is driven
// from the host (a few scalars read back per conjugate-gradient step).
cudaError_t run_inexact(IxArgs& a, const IxPasses& ps, double sigma0, cudaStream_t st, IxResult* res);

}  // namespace gdwd
