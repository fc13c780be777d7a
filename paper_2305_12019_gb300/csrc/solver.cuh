// Device data structures of libgdwd shared by the set-up and iteration kernels.
#pragma once

#include "common.cuh"

namespace gdwd {

// Slab layout of the stored Z in HBM.  The d rows are cut into NB slabs of TB
// rows (the last one zero-padded); slab s is one contiguous block of n columns
// of TB elements (column-major inside the slab).  One CTA streams a whole slab
// as a sequence of contiguous chunks of CW columns with 1-D bulk copies, so
// both products of an iteration -- Z~^T g' (dots down each column) and Z~ c
// (axpys across columns) -- read Z once, linearly, with no cross-CTA traffic
// except the n-vector of per-slab partial dots.
struct Layout {
  const void* Z;
  int64_t d, n;
  int TB;          // rows per slab (TB * esize % 16 == 0)
  int NB;          // slabs
  int CW;          // columns per streamed chunk
  int esize;       // bytes per stored element
};

__host__ __device__ inline int64_t slab_elems(const Layout& L) { return (int64_t)L.TB * L.n; }

// Number of scalar partial sums each CTA contributes per iteration.
enum Scal {
  S_RES2 = 0,   // ||Z~^T w + beta y + xi - r||^2
  S_YA,         // y^T alpha
  S_XICA,       // xi^T (C e - alpha)
  S_AMS2,       // ||alpha - s||^2, s_i = omega_i / r_i^(q+1)
  S_AMIN2,      // ||min(0, alpha)||^2
  S_AMAX2,      // ||max(0, alpha - C e)||^2
  S_PRIM_R,     // sum wt_i^q r_i^-q
  S_PRIM_XI,    // sum e_i xi_i
  S_DUAL_A,     // sum (wt_i alpha_i)^(q/(q+1))
  S_G2,         // ||g||^2
  S_GRHO,       // <g, rho> (the iteration kernel: <y, g>, y = (1 - theta_prev) g + rho / (sigma sqrt(mu)))
  S_RHO2,       // ||rho||^2 (the iteration kernel: ||y||^2)
  S_A2,         // ||a||^2, a = Z~ alpha + sqrt(mu)(1 - tau) rho (the iteration kernel: ||v||^2, v = a - khat g)
  S_AG,         // <a, g> (the iteration kernel: <v, g>)
  S_TA2,        // ||Z~ alpha||^2
  S_COUNT = 16
};

// Phases of one iteration, each followed by its grid-barrier wait:
// 0 A, 1 wait, 2 R, 3 wait, 4 N1, 5 wait, 6 N2, 7 wait, 8 B, 9 wait, 10 S;
// sub-phases: 11 N2 rhs load + beta, 12 N2 rows of G^{-1}, 13 S partial-sum
// reduction, 14 N1 rhs load + beta-bar, 15 N1 rows of G^{-1}, 16 B prologue
// (coefficients, deferred d-update), 17 B stream, 18 N1 prox of the first row,
// 19 spare (the slot of a phase then holds only its remainder).
constexpr int kPhaseSlots = 20;
// n-space rows owned by one CTA of the iteration kernel (ceil(n / grid) <= this)
constexpr int kMaxRowsPerCta = 256;

// Iteration control block (device memory, read back by the host).
struct Ctrl {
  double sigma;        // sigma for the next iteration
  double sigma_prev;   // sigma the current (u, rho) update must use
  double theta;        // ball-projection factor of the pending u update
  double beta;         // beta of the last iterate
  double pobj, dobj, kkt;
  double eta_p1, eta_p2, eta_p3, eta_d1, eta_d2, eta_d3, eta_c1, eta_c2, eta_c3, eta_gap;
  double wnorm;
  int32_t it;          // iterations completed
  int32_t status;      // gdwd_status of the solve
  int32_t done;        // 1 once converged / failed
  int32_t pending;     // 1: u, rho still hold the iterate before the deferred update
  double phase_ns[kPhaseSlots];   // CTA 0's time per phase (compute, then barrier wait), summed
};

// Everything the persistent iteration kernel reads and writes.
template <typename CT>
struct IterArgs {
  Layout L;
  const double* sc;      // n: Z~_ji = sc_i * Zq_ji
  const float2* P;       // n x ldP, G^{-1} as double-float (hi, lo) pairs
  int ldP;
  const float2* pdf;     // n: p = G^{-1} y as double-float
  const double* p;       // n: p in FP64
  const double* y;       // n labels
  const double* e;       // n: penalty weights e_i
  const double* omega;   // n: q * wt_i^q
  const double* wt;      // n: wt_i
  double inv_s;          // 1 / (y^T p)
  double q, C, mu, tau, R, tol, kappa;
  int max_iter;
  int stop_rule;         // 0: kkt <= tol; 1: the rule of Sec. 4.3
  int grid;
  uint64_t timeout_ns;
  // n-space state
  double* r;
  double* xi;
  double* alpha;
  double* b;
  float2* rhsA;
  float2* rhsB;
  CT* cq;                // n: sc_i c_i   (pass B right-hand side 1)
  CT* aq;                // n: sc_i alpha_i (pass B right-hand side 2)
  double* Uu;            // n: Z~^T u of the starting iterate (rows of the owning CTA)
  double* Ur;            // n: Z~^T rho (rows of the owning CTA)
  double* kc;            // n: (G - I) c of the last iteration
  int refresh;           // 1: U_u, U_rho from u, rho by two passes over Z at launch start
  int dots_every;        // >= 1: pass B takes the column dots Z~^T u every dots_every iterations
  int stall_first_barrier;   // test hook: 1 makes the launch's first grid barrier wait for an
                             // arrival that never comes, so it runs out after timeout_ns
  int fuse;              // 1: Step 1a's solve of the next iteration is taken from three
                         // G^{-1} products made during the pass over Z (iterate.cu)
  float2* vrhs;          // [3][ldP] double-float right-hand sides of those products
  // d-space state, NB*TB long (padding rows stay 0)
  double* u;
  double* rho;
  double* g;
  CT* partial;           // n x NB per-slab partial dots (Z~^T u of pass B; start-up passes)
  double* scal;          // grid x S_COUNT
  unsigned* bar;
  int* err;
  Ctrl* ctrl;
};

// Joint C-grid iteration (iterate_multi.cu): K <= 4 instances in lock-step.
template <typename CT>
struct MultiArgs {
  Layout L;
  const double* sc;
  const float2* P;
  int ldP;
  const float2* pdf;
  const double* p;
  const double* y;
  const double* e;
  const double* omega;
  const double* wt;
  double inv_s, q, mu, tau, R, tol, kappa;
  double C[4];
  int K;                // instances in use (the rest start frozen)
  int max_iter, grid;
  int stop_rule;        // as in IterArgs
  uint64_t timeout_ns;
  int64_t dpad;
  double *r, *xi, *alpha, *b;   // [K][n]
  float2 *rhsA, *rhsB;          // [K][n]
  double *Uu, *Ur, *kc;         // [K][n]: Z~^T u_j, Z~^T rho_j (rows of the owning CTA), (G - I) c_j
  int dots_every;               // as in IterArgs
  int min_active;               // stop when fewer instances than this are still iterating
  CT* partial;                  // [K][n][NB]: column dots Z~^T u_j of pass B
  CT* coef;                     // [n][2K]: sc_i c_ij (j < K), then sc_i alpha_ij
  double *u, *rho, *g;          // [K][dpad]
  double* scal;                 // [K][S_COUNT][grid]
  unsigned* bar;
  int* err;
  Ctrl* ctrl;                   // [K]
};
int multi_max_k(int store, const Layout& L, int grid, int smem_limit);
cudaError_t run_multi_f64(int K, const MultiArgs<double>& a, int smem_limit, cudaStream_t st);
cudaError_t run_multi_f32(int store, int K, const MultiArgs<float>& a, int smem_limit, cudaStream_t st);

// Host-side launchers (defined in the .cu files).
int choose_chunk_cols(int store, const Layout& L, int grid, int smem_limit, bool wide = false);
cudaError_t run_iterate_f64(const IterArgs<double>& a, int smem_limit, cudaStream_t st);
cudaError_t run_iterate_f32(int store, const IterArgs<float>& a, int smem_limit, cudaStream_t st);
// wide = true reads FP32 storage into FP64 arithmetic (partial then holds n x NB
// doubles); other storage ignores it.
cudaError_t run_apply(int store, const Layout& L, int trans, const double* x, const double* sc, double* out,
                      void* partial, int grid, int smem_limit, int* err, uint64_t tmo, cudaStream_t st,
                      bool wide = false);

// set-up (setup.cu)
struct FactorArgs {
  const double* G;    // n x n FP64 G (row-major)
  float2* A;          // n x n double-float work: G, then L in the lower triangle
  float2* X;          // n x n double-float work: L^{-1}
  float2* P;          // n x ldP double-float G^{-1} (padding zero)
  int ldP;
  const double* y;
  double* p;          // n: p = G^{-1} y
  float2* pdf;        // n: p as double-float
  double* s_out;      // y^T p
  int64_t n;
  int grid;
  unsigned* bar;
  int* err;
  uint64_t timeout_ns;
};
cudaError_t run_ingest(const void* Z, int zdt, int64_t ldz, const Layout& L, void* out, int store, double* part,
                       int nparts, double* sumsq, int* nonfinite, double* sc, double* zscale, double* amax,
                       double* colscale, cudaStream_t st);
// Gram: tensor-core path (gram_tc.cu) for BF16 / FP16 / E4M3 storage, and for
// FP32 storage through its three-term BF16 split (which needs
// gram_tc_scratch_bytes() of device scratch), when gram_tc_supported(); SIMT
// double-float path (setup.cu) otherwise.
bool gram_tc_supported(int store, const Layout& L);
size_t gram_tc_scratch_bytes(int store, const Layout& L);
int gram_tc_ksplit(int store, const Layout& L, int sms);
cudaError_t run_gram_tc(int store, const Layout& L, int ksplit, double* Kpart, void* scratch, int* err,
                        uint64_t timeout_ns, cudaStream_t st);
int gram_ksplit(const Layout& L, int sms);
cudaError_t run_gram(int store, const Layout& L, int ksplit, double* Kpart, const double* sc, double mu, double* G,
                     bool tensor_cores, void* scratch, int* err, uint64_t timeout_ns, cudaStream_t st);
cudaError_t run_factor(const FactorArgs& a, cudaStream_t st);

cudaError_t launch_prox(const double* a, const double* r0, const double* omega, double sigma, double q,
                        int64_t n, double* out, cudaStream_t st);

}  // namespace gdwd
