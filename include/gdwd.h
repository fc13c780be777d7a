/*
 * gdwd.h -- C-ABI of libgdwd, a GB300 (sm_103a) solver for the generalized
 * Distance Weighted Discrimination model
 *
 *     min  sum_i theta_q(r_i) + C <e, xi>
 *     s.t. Z^T w + beta y + xi - r = 0,  ||w|| <= 1,  xi >= 0,
 *
 * theta_q(t) = t^-q for t > 0 (generalized DWD, Sec. 2, eq-primal of arXiv
 * 2305.12019), by the inexact sGS-ADMM of Algorithm 1 (Sec. 3) on the scaled
 * model eq-gen-scale (Sec. 4.2), with the linear system eq-linsys solved through
 * the n x n Gram matrix and Sherman-Morrison-Woodbury (SMW2, Sec. 3.3.2), the
 * r-subproblem eq-varphi by Newton's method (Sec. 3.2), the KKT residuals of
 * Sec. 4.3 and the sigma rule of Sec. 4.4.
 *
 * Conventions for every entry point:
 *   - it returns a gdwd_status and never aborts the process;
 *   - invalid arguments give GDWD_EINVAL and leave outputs untouched;
 *   - "device" pointers are CUDA global-memory pointers of the current device,
 *     "host" pointers are ordinary (pageable or pinned) host memory;
 *   - the caller keeps ownership of every buffer it passes; the library copies
 *     what it needs and owns only what it allocates inside a handle;
 *   - a handle is not thread-safe: one host thread at a time per handle;
 *   - all work is issued on the stream given in gdwd_options (0 = legacy default
 *     stream) and every call that returns results synchronizes that stream;
 *   - every device-side wait (grid barriers, bulk copies) is bounded by
 *     gdwd_options.timeout_s: when one runs out the kernel waits (bounded) for
 *     its own copies still in flight, records GDWD_ETIMEOUT and returns, and the
 *     context stays usable.
 * Fault injection for tests (environment variables, no effect while unset):
 *   GDWD_INJECT_ALLOC_FAIL=k  the k-th device allocation of a handle fails as if
 *                             the device were out of memory (gdwd_create then
 *                             returns GDWD_ENOMEM and no handle);
 *   GDWD_INJECT_STALL=1       the Z-streaming iteration kernel waits at its first
 *                             grid barrier for an arrival that never comes, so the
 *                             solve returns GDWD_ETIMEOUT after timeout_s.
 */
#ifndef GDWD_H
#define GDWD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GDWD_OK = 0,
  GDWD_EINVAL = 1,     /* bad argument (sizes, labels, q, C, non-finite data)          */
  GDWD_ENOMEM = 2,     /* device allocation failed                                     */
  GDWD_ENOTPD = 3,     /* Cholesky of I + Z~^T Z~ / mu met a pivot <= 0                 */
  GDWD_EMAXITER = 4,   /* max_iter reached before kkt <= tol; results are the last iterate */
  GDWD_ENUMERIC = 5,   /* NaN/Inf appeared in the iteration                             */
  GDWD_ETIMEOUT = 6,   /* a bounded device-side wait ran out; the kernel returned       */
  GDWD_ECUDA = 7,      /* a CUDA runtime call failed (message in gdwd_last_error)       */
  GDWD_EUNSUPPORTED = 8, /* valid request this build does not implement                 */
  GDWD_EAGAIN = 9        /* server: the request is still queued or running               */
} gdwd_status;

/* Element types, for the caller's Z and for the copy the handle stores. */
typedef enum {
  GDWD_F64 = 0,
  GDWD_F32 = 1,
  GDWD_BF16 = 2,
  GDWD_F16 = 3,
  GDWD_E4M3 = 4
} gdwd_dtype;

/* Solver options.  Fill with gdwd_default_options() and override fields. */
typedef struct {
  double mu;          /* D^2 = mu I in the split u = w (Sec. 3, eq-gen; D is "a positive
                         multiple of I").  Default 1.                                   */
  double tau;         /* dual step length of Step 3, in (0, (1+sqrt5)/2).  Default 1.618 */
  double tol;         /* stop when kkt = max(eta_P, eta_D, eta_C, eta_gap) <= tol
                         (Sec. 4.3 residuals, all relative).  Default 1e-6.             */
  double sigma0;      /* initial sigma; <= 0 selects min(10C, n)^q (Sec. 4.4).          */
  double timeout_s;   /* limit of every device-side wait (grid barrier, copies). Default 2 */
  int32_t max_iter;   /* iteration limit.  Default 20000.                              */
  int32_t store;      /* gdwd_dtype of the copy of Z kept on the device.  GDWD_F64 and
                         GDWD_F32 keep the values; GDWD_BF16, GDWD_F16 and GDWD_E4M3
                         keep Z_ji / s_i rounded to the format with a per-column FP64
                         scale s_i (see gdwd_get_stored), and the solve is then of the
                         stored (quantized) problem.  Default GDWD_F32.                 */
  int32_t grid;       /* CTAs of the persistent iteration kernel; 0 = one per SM.      */
  int32_t block_rows; /* rows of Z per slab of the device layout; 0 = automatic.        */
  void* stream;       /* cudaStream_t for all work of the handle; NULL = default stream */
  int32_t refine;     /* BF16/F16/E4M3 storage only: 1 keeps an FP32 master copy of Z
                         (with its own Gram factor) and follows each quantized solve by
                         a warm-started solve on the master data, so that kkt <= tol
                         holds for the original data.  Default 0.                       */
  int32_t cgrid_sequential; /* 0 (default): gdwd_solve with several C iterates up to
                         four of them in lock-step in one persistent launch, so each
                         pass over Z serves all of them; 1: one C at a time.         */
  int32_t gram_path;  /* 0 (default): the Gram of BF16, F16 and E4M3 storage runs on
                         the tensor cores (tcgen05.mma; exact products, FP32 sums of at
                         most 256 rows folded into double-float); F32 storage too,
                         through a three-term BF16 split of each value (six exact
                         products per pair, the dropped terms below 2^-23 of the
                         product; a temporary 6 d n bytes during gdwd_create), when
                         the contraction has at most 65536 rows (d for this solver,
                         n for the direct one); F64 on the SIMT FP64 kernel; 1: the
                         SIMT kernel for every storage.  */
  int32_t stop_rule;  /* 0 (default): stop when kkt = max(eta_P, eta_D, eta_C, eta_gap)
                         <= tol; 1: the rule of Sec. 4.3: max(eta_P, eta_D) < tol,
                         min(eta_C, eta_gap) < sqrt(tol) and max(eta_C, eta_gap) < 0.05
                         (the paper uses tol = 1e-5 with max_iter = 2000).          */
  int32_t dots_every; /* b = Z~^T g' is carried in n-space from Z~^T u, Z~^T rho and
                         (G - I) c; every dots_every-th iteration Z~^T u is taken
                         directly from the pass over Z, bounding the number of
                         iterations over which the Gram's rounding can accumulate.
                         0 (default): 16 for FP64 / FP32 storage, 4 for BF16 / FP16 /
                         E4M3 storage (tensor-core Gram); 1: every iteration.     */
  int32_t kernelized; /* 0 (default): every iteration streams the stored Z once;
                         1: the kernelized n-space iteration.  From the initial
                         iterate w = u = rho = 0 every d-space iterate lies in the
                         range of Z~, so the loop runs on K = Z~^T Z~ alone: two
                         G^{-1} products and one K product with three columns per
                         iteration, O(n^2) and independent of d, and
                         w = Z~ (a_g + a_rho / (sigma sqrt(mu))) is formed once after
                         the loop by one pass over Z.  Keeps K as double-float
                         (8 n^2 bytes more).  Several C values are then solved one
                         after the other.  A solve starts only from the iterate of
                         a kernelized handle (the refinement sweep's master is one).
                         -1: chosen per problem: the kernelized loop wherever n fits
                         it, else the streaming loop (solver = 0; the other solvers
                         stream).  */
  int32_t solver;     /* solver of eq-linsys.  0 (default): SMW2 through the n x n
                         Gram matrix (Sec. 3.3.2), for n << d.  1: the direct solver
                         of Sec. 3.3.1 for d << n: the (d+1) x (d+1) system through
                         the d x d matrix I + Z~ Z~^T / mu (factored once, FP64
                         diagonal tiles, double-float inverse) with its border
                         eliminated in closed form; Z^T is stored with samples as
                         rows, and each iteration reads it four times (five products
                         with Z~) around the per-sample Steps 1b, 2 and 3.  Every
                         solve starts from the initial iterate.  With
                         solver = 1: F32 or F64 storage, refine = 0 and kernelized =
                         0 (else EUNSUPPORTED); gdwd_apply,
                         gdwd_get_stored and gdwd_suggest_C return EUNSUPPORTED and
                         gdwd_gram returns the d x d matrix I + Z~ Z~^T / mu.
                         2: the inexact solver for d and n both large (Sec. 3.3.3
                         with T = 0): no n x n or d x d matrix is formed; Steps 1a
                         and 1c solve eq-linsys by Jacobi-preconditioned conjugate
                         gradients on the matrix-free (d+1) x (d+1) operator (two
                         passes over the stored Z per step) to the accuracy
                         eq-linsys-tol with eps_k = c / (k+1)^1.5, c = 1 / ||Z~||_F
                         (Algorithm 1), and Step 1c reuses Step 1a's solution when it
                         already meets 5 eps_k for the new right-hand side.  F32 or
                         F64 storage, refine = 0, kernelized = 0 (else
                         EUNSUPPORTED); gdwd_gram and gdwd_suggest_C return
                         EUNSUPPORTED; gdwd_result.reserved[1] holds the CG steps
                         and reserved[2] the iterations in which Step 1c solved. */
  int32_t reserved_i32;
  int64_t reserved[4];
} gdwd_options;

/* Outcome of one solve (one value of C). */
typedef struct {
  double beta;        /* intercept of the hyperplane w^T x + beta = 0                  */
  double primal_obj;  /* sum r_i^-q + C <e, xi> at the final iterate (Sec. 4.3)         */
  double dual_obj;    /* kappa sum alpha_i^(q/(q+1)) - ||Z alpha|| (Sec. 4.3)           */
  double kkt;         /* max of all relative residuals below                            */
  double eta_p;       /* max(eta_P1, eta_P2, eta_P3)                                    */
  double eta_d;       /* max(eta_D1, eta_D2, eta_D3), eta_D3 = ||Z~ alpha + D rho||/(1+C) */
  double eta_c;       /* max(eta_C1, eta_C2, eta_C3)                                    */
  double eta_gap;     /* |primal - dual| / (1 + |primal| + |dual|)                      */
  double sigma;       /* final sigma                                                    */
  double zscale;      /* Z_scale = sqrt(||Z||_F) (Sec. 4.2)                              */
  double t_setup_ms;  /* device time of gdwd_create's work (ingest, Gram, factor)       */
  double t_solve_ms;  /* device time of the iterations of this solve                   */
  int32_t iters;      /* ADMM iterations performed                                      */
  int32_t status;     /* gdwd_status of this solve                                      */
  int64_t reserved[4];
} gdwd_result;

typedef struct gdwd_handle gdwd_handle;

/* Fills *o with the defaults listed above.  EINVAL if o is NULL. */
gdwd_status gdwd_default_options(gdwd_options* o);

/*
 * Creates a solver for one data set and does its set-up on the device:
 * copy/convert Z into the handle's slab layout, Z_scale = sqrt(||Z||_F) and the
 * scaled data Z~ = Z / Z_scale (Sec. 4.2), the Gram matrix K = Z~^T Z~ and the
 * SMW2 set-up of Sec. 3.3.2: G = I_n + K / mu = L L^T (Cholesky, FP64), its
 * inverse, p = G^{-1} y and s = y^T p.  None of this depends on sigma or C, so
 * one handle serves every solve and every C.
 *
 *   Z          d x n, column-major with leading dimension ldz >= d; column i is
 *              y_i x_i (Z = X diag(y), eq-r).  Element type zdt (GDWD_F64 or
 *              GDWD_F32).  Host memory if z_on_device == 0, else device memory.
 *   d, n       feature dimension and sample count; d >= 1, n >= 2.
 *   y          n labels in {-1, +1}, host memory; both classes must occur.
 *   q          exponent of theta_q, q > 0 (eq-primal).
 *   C          penalty, C > 0 (eq-primal); the default C of gdwd_solve.
 *   o          options (NULL = defaults).
 *   out        receives the handle; set to NULL on failure.
 * Errors: EINVAL (sizes, labels, q, C, non-finite Z), ENOMEM, ENOTPD, ECUDA.
 */
gdwd_status gdwd_create(const void* Z, int32_t zdt, int64_t d, int64_t n, int64_t ldz, int32_t z_on_device,
                        const double* y, double q, double C, const gdwd_options* o, gdwd_handle** out);

/*
 * Runs Algorithm 1 to kkt <= tol (or max_iter) for each of the nC penalties in
 * Cs (NULL or nC == 0: the C given to gdwd_create, one solve).
 *
 *   w          d x nC output, column j = the hyperplane normal for Cs[j] in the
 *              original (unscaled) units, w = w~ / Z_scale (Sec. 4.2).  Host
 *              memory if w_on_device == 0, else device memory.  May be NULL.
 *   alpha      n x nC output multipliers (host memory), or NULL.
 *   res        nC results, host memory; must not be NULL.
 * Returns the worst status over the nC solves (GDWD_OK if all converged).
 */
gdwd_status gdwd_solve(gdwd_handle* h, const double* Cs, int32_t nC, double* w, int32_t w_on_device,
                       double* alpha, gdwd_result* res);

/* Frees a handle and all device memory it owns.  NULL is a no-op. */
gdwd_status gdwd_free(gdwd_handle* h);

/* Message of the last error of h, or of the calling thread when h is NULL. */
const char* gdwd_last_error(const gdwd_handle* h);

/*
 * Element-wise r-subproblem of Step 1b (eq-1c / eq-varphi, Sec. 3.2): for each i,
 * out_i = argmin_{s > 0} (omega_i / q) s^-q + sigma/2 (s - a_i)^2, the unique
 * positive root of s^(q+1) (s - a_i) = omega_i / sigma, by safeguarded Newton
 * warm-started at r0_i.  All arrays are device memory of length n; omega may be
 * NULL (omega_i = q, the unweighted model) and r0 may be NULL (cold start).
 * stream: cudaStream_t or NULL.  Errors: EINVAL (n < 0, q <= 0, sigma <= 0), ECUDA.
 */
gdwd_status gdwd_prox(const double* a, const double* r0, const double* omega, double sigma, double q,
                      int64_t n, double* out, void* stream);

/*
 * Products with the handle's stored, scaled data Z~ = Z / Z_scale, by the same
 * streaming kernels the iteration uses: trans != 0 gives out = Z~^T x (x: d,
 * out: n), trans == 0 gives out = Z~ x (x: n, out: d).  x and out are device
 * memory (FP64).  Errors: EINVAL, ECUDA.
 */
gdwd_status gdwd_apply(gdwd_handle* h, int32_t trans, const double* x, double* out);

/*
 * Copies the FP64 Gram matrix G = I + Z~^T Z~ / mu built by gdwd_create (n x n,
 * row-major, symmetric) to G_out (host memory, n*n doubles).  Errors: EINVAL, ECUDA.
 */
gdwd_status gdwd_gram(gdwd_handle* h, double* G_out);

/*
 * Weighted DWD (Sec. 4.5): the r-term of eq-primal becomes sum_i wt_i^q / r_i^q
 * and the penalty C <e, xi>.  e and wt are host arrays of n positive finite
 * doubles (copied; NULL = all ones, the default after gdwd_create).  They hold
 * for every later gdwd_solve of h (and of its FP32 master copy when refine = 1).
 * Errors: EINVAL (NULL handle, a non-positive or non-finite entry), ECUDA.
 */
gdwd_status gdwd_set_weights(gdwd_handle* h, const double* e, const double* wt);

/*
 * The class-balancing weights of Sec. 4.5: with n_+ and n_- the class sizes,
 * K = n / log(n) and tau_+- = (n_+- / K)^(1/(1+q)), wt_i = tau_- / max(tau_+, tau_-)
 * for y_i = +1 and tau_+ / max(tau_+, tau_-) for y_i = -1.  Host-only: y (n
 * labels +-1) and wt (n doubles, written) are host arrays.
 * Errors: EINVAL (n < 2, q <= 0, a label not +-1, a class empty).
 */
gdwd_status gdwd_imbalance_weights(const double* y, int64_t n, double q, double* wt);

/*
 * The penalty parameter of Sec. 4.1 for the handle's data:
 * C = 10^(q+1) max{1, 10^(q-1) log(n) max(1000, d)^(1/3) / dist^(q+1)}, with dist
 * the median of the Euclidean distances ||x_i - x_j|| over pairs of opposite
 * labels (the mean of the two middle ones for an even count), taken from the
 * Gram matrix of the stored data (for BF16 / FP16 / E4M3 storage: of the
 * quantized data).  Writes *C_out (host).  Errors: EINVAL, ECUDA, ENOMEM.
 */
gdwd_status gdwd_suggest_C(gdwd_handle* h, double* C_out);

/* Sizes and layout chosen by gdwd_create (for diagnostics and benchmarks). */
typedef struct {
  int64_t d, n;
  int32_t store;         /* gdwd_dtype of the stored Z                       */
  int32_t block_rows;    /* rows per slab                                    */
  int32_t slabs;         /* number of slabs                                  */
  int32_t grid;          /* CTAs of the persistent iteration kernel          */
  int64_t z_bytes;       /* bytes of the stored Z (one pass reads them once) */
  int64_t device_bytes;  /* all device memory owned by the handle            */
  double zscale;         /* Z_scale                                          */
  double t_setup_ms;     /* device time of the set-up                        */
  double t_ingest_ms;    /* of which: copy / quantize into the slab layout   */
  double t_gram_ms;      /*           Gram matrix G                          */
  double t_factor_ms;    /*           Cholesky, inverse, p, s                */
  int32_t gram_tensor_cores; /* 1: the Gram ran on the tcgen05 tensor cores       */
  int32_t kernelized;        /* 1: solves use the kernelized n-space iteration      */
  int32_t solver;            /* 0: SMW2 (n x n Gram), 1: direct (d x d, d << n)   */
  int32_t reserved_;
} gdwd_info;

gdwd_status gdwd_get_info(const gdwd_handle* h, gdwd_info* info);

/*
 * Device-side time of the last solve of h split by phase of the persistent
 * iteration kernel, as seen by its first CTA (globaltimer, nanoseconds summed
 * over iterations): ns[2k] = time in phase k, ns[2k+1] = the grid-barrier wait
 * that follows it, for k = 0 (the two start-up passes over Z of a warm start),
 * 1 (R: U_g, b, rhs1), 2 (N1: first n-space solve and Step 1b), 3 (N2: second
 * solve, Steps 2-3), 4 (B: the pass over Z); ns[10] = the KKT / sigma phase;
 * sub-phases split out of those: ns[11] N2 right-hand side load, ns[12] N2
 * rows of G^{-1} and p^T rhs (beta), ns[13] reduction of the per-CTA partial
 * sums, ns[14] N1 right-hand side load, ns[15] N1 rows of G^{-1} and p^T rhs,
 * ns[16] B prologue (coefficients, deferred d-space update), ns[17] B stream
 * over Z, ns[18] the Step 1b prox of the CTA's first row, ns[19] unused.  When
 * the first solve of an iteration is fused into the previous pass over Z, ns[2]
 * holds its combination and ns[3], ns[14], ns[15] stay empty for that
 * iteration (the joint C-grid kernel fills ns[2..10] and ns[13]; the kernelized
 * iteration has no pass over Z and reports its K product in ns[8], ns[9] and
 * the start-up product of a stored iterate in ns[0], ns[1]).  count (<= 20)
 * entries are written to ns (host).  Diagnostics only; the paper has no
 * counterpart.  Errors: EINVAL.
 */
gdwd_status gdwd_get_phase_times(const gdwd_handle* h, double* ns, int32_t count);

/*
 * Copies the data the handle stores back to the host: Zq (d x n, column-major,
 * element type = the handle's store dtype, d*n*size bytes) and colscale (n
 * doubles) such that the stored problem's Z is Zq_ji * colscale_i (colscale = 1
 * for FP64 / FP32 storage; for BF16 / FP16 / E4M3, colscale_i = max_j |Z_ji|
 * divided by 1, 32768 or 448 respectively, and Zq_ji = Z_ji / colscale_i rounded
 * to nearest-even, saturating for E4M3).  Either pointer may be NULL.
 * Diagnostics; the paper has no counterpart.  Errors: EINVAL, ECUDA.
 */
gdwd_status gdwd_get_stored(const gdwd_handle* h, void* Zq, double* colscale);

/*
 * Gram matrix without any allocation: K = Z^T Z (n x n, row-major, both
 * triangles, FP64 result of FP32 products summed in double-float) for a
 * column-major FP32 matrix Z (d x n, leading dimension ldz >= d).  Z and K are
 * device memory owned by the caller; work is queued on `stream` (NULL = default
 * stream) and the call returns without waiting for it.
 *
 * For callers that cannot allocate device memory at the point where they need
 * the product (code running under an allocator that must not be re-entered, or
 * an embedder that owns all device memory and hands out none): the scratch for the split-K
 * partial products lives in a fixed 32 MiB array inside the library, which
 * every GPU that loads the library keeps until the process exits.  Limits and
 * rules:
 *   - n * n <= 4,194,304 (n <= 2048); larger n gives GDWD_EINVAL;
 *   - the first call on a device looks up the array's device address (with that
 *     device current) and caches it; make that first call before any stream
 *     capture;
 *   - all calls share the one array, so calls whose work overlaps on the GPU
 *     (different streams, or different host threads without ordering) race and
 *     give wrong results; order them on one stream;
 *   - no cudaMalloc, cudaFree or allocating library routine is called.
 * The paper has no counterpart.  Errors: EINVAL (including n > 2048), ECUDA
 * (also when an earlier asynchronous error is still pending on entry: it is
 * left in place for the caller, and nothing is launched).
 */
gdwd_status gdwd_gram_noalloc(const float* Z, int64_t d, int64_t n, int64_t ldz, double* K, void* stream);

/*
 * ---------------------------------------------------------------- serving
 * Many independent problems of different (d, n, q, C) on one GPU.  A server
 * owns `slots` CUDA streams; each slot runs one problem at a time (create,
 * solve, free) with its persistent kernels restricted to sms / slots CTAs, so
 * the slots' work overlaps on the device.  Requests are taken in arrival order
 * as a slot frees up (continuous batching) and admitted only while the sum of
 * the device footprints of the problems in flight stays within hbm_budget
 * bytes (a request larger than the budget runs alone).  The paper solves one
 * problem at a time (Sec. 4.5); this layer has no counterpart there.
 */
typedef struct {
  const void* Z;        /* d x n column-major, column i = y_i x_i (as gdwd_create)     */
  int32_t zdt;          /* GDWD_F64 or GDWD_F32                                        */
  int32_t z_on_device;  /* 0: host memory, 1: device memory                            */
  int64_t d, n, ldz;
  const double* y;      /* n labels, host                                              */
  double q, C;
  gdwd_options opts;    /* store, tol, ...; stream and grid are set by the server      */
  double* w;            /* host output, d doubles (original units), or NULL            */
  double* alpha;        /* host output, n doubles, or NULL                             */
} gdwd_request;

typedef struct gdwd_server gdwd_server;

/* slots >= 1; hbm_budget in bytes (0 = 80% of the device's free memory). */
gdwd_status gdwd_server_create(int32_t slots, uint64_t hbm_budget, gdwd_server** out);

/* Queues a request (the struct is copied; Z, y, w and alpha must stay valid
   until the request completes).  ticket receives its id.  Never blocks. */
gdwd_status gdwd_server_submit(gdwd_server* s, const gdwd_request* r, uint64_t* ticket);

/* Result of a ticket: GDWD_EAGAIN while it is queued or running (wait == 0),
   else the request's own status with *res filled and latency_ms = completion
   minus submission time (host steady clock).  wait != 0 blocks until done.
   A ticket is released once its result has been returned. */
gdwd_status gdwd_server_poll(gdwd_server* s, uint64_t ticket, int32_t wait, gdwd_result* res, double* latency_ms);

/* Waits for all submitted requests, stops the workers, frees the server. */
gdwd_status gdwd_server_destroy(gdwd_server* s);

/* An uneven batch of nreq independent problems through a temporary server
   with `slots` concurrent slots; res[i] and latency (may be NULL) per request. */
gdwd_status gdwd_solve_batch(const gdwd_request* reqs, int32_t nreq, int32_t slots, gdwd_result* res,
                             double* latency_ms);

#ifdef __cplusplus
}
#endif

#endif /* GDWD_H */
