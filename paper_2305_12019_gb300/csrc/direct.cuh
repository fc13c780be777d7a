// The direct (d-space) solver of eq-linsys (Sec. 3.3.1): arguments and launchers.
#pragma once

#include "solver.cuh"

namespace gdwd {

constexpr int kDirMaxBlocks = 1024;   // blocks of the per-sample kernels (their partial sums)

// slots of the per-block partial sums of the per-sample kernels: the n-space
// KKT sums (Scal slots S_RES2 .. S_DUAL_A), then y^T (xi - r) and y^T alpha
enum DirScal { DS_YXR = S_COUNT, DS_YA, DS_COUNT };
constexpr int DS_SLOTS = DS_COUNT;

struct DirArgs {
  int64_t d, n;
  const float2* P;       // d x ldP: G'^{-1}, G' = I + Z~ Z~^T / mu, double-float
  int ldP;
  const float2* pdf;     // p = G'^{-1} b^, b^ = Z~ y (double-float, padded to ldP)
  const double* p;       // p in FP64
  double s;              // b^T p
  const double* y;
  const double* e;
  const double* omega;
  const double* wt;
  double q, C, mu, tau, R, tol, kappa;
  int max_iter, stop_rule;
  // n-space
  double *r, *xi, *alpha, *t;   // t: Z~^T w of the last pass
  double *dv, *dv2;             // per-sample coefficients of the next pass(es)
  // d-space
  double *u, *rho, *w, *g, *x;  // x: d + 1 (G'^{-1} h_w and p^T h_w)
  float2* hw;                   // h_w as double-float, ldP
  double *Zxr, *Za, *Zdr;       // Z~ (xi - r), Z~ alpha, Z~ (r+ - r)
  double* scal;                 // DS_COUNT x nblk block partial sums
  double* dscal;                // nblk: y^T (r+ - r)
  int nblk;
  Ctrl* ctrl;
};

// The streaming passes of one iteration over the stored Z^T: trans = 0 gives
// out = Z~^T x (n-vector from a d-vector), trans = 1 gives out = Z~ x.
struct DirPasses {
  cudaError_t (*apply)(int trans, const double* x, double* out, void* ctx);
  // out = Z~ x and out2 = Z~ x2 in one read of the stored data
  cudaError_t (*apply2)(const double* x, const double* x2, double* out, double* out2, void* ctx);
  void* ctx;
};

int dir_blocks(int64_t n);
// The products with the stored Z^T (F32 / F64 storage; double-float or FP64
// sums): trans = 0 gives out = Z~^T x (n), trans = 1 gives out = Z~ x (d) through
// part (d x NB per-slab partials).
cudaError_t run_dir_product(const Layout& L, int store, int trans, const double* x, const double* sc, double* out,
                            double* part, cudaStream_t st);
// out = Z~ x and out2 = Z~ x2 (one read of the slabs for FP32 storage)
cudaError_t run_dir_product2(const Layout& L, int store, const double* x, const double* x2, const double* sc,
                             double* out, double* out2, double* part, double* part2, cudaStream_t st);
cudaError_t run_transpose(const void* Z, int zdt, int64_t d, int64_t n, int64_t ld, void* out, cudaStream_t st);
// one iteration of Algorithm 1 (all its kernels; a no-op once ctrl->done is set)
cudaError_t run_dir_iteration(const DirArgs& a, const DirPasses& ps, cudaStream_t st);
cudaError_t run_dir_finish(const double* w, double zscale, int64_t d, double* out, cudaStream_t st);

}  // namespace gdwd
