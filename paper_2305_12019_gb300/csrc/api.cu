// C-ABI of libgdwd (include/gdwd.h): argument checks, handle memory, set-up
// and solve orchestration on the caller's stream.  No computation of the
// method happens on the host: every step runs in the kernels of setup.cu,
// gram_tc.cu, iterate.cu, iterate_multi.cu, iterate_kern.cu and direct.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "direct.cuh"
#include "inexact.cuh"
#include "iterate_kern.cuh"
#include "solver.cuh"

namespace gdwd {
// ------------------------------------------------------------------ small kernels
__global__ void fill_kernel(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// w_j = (g_j + rho_j / (sigma_prev sqrt(mu))) / Z_scale: the Step-1c w of the last
// iteration in original units (Sec. 4.2).
__global__ void finish_w_kernel(const double* g, const double* rho, const Ctrl* ctrl, double sqmu, double zscale,
                                int64_t d, double* w) {
  const double gs = 1.0 / (ctrl->sigma_prev * sqmu);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x)
    w[j] = (g[j] + rho[j] * gs) / zscale;
}
}  // namespace gdwd

using namespace gdwd;

struct gdwd_handle {
  int device = 0;
  int sms = 0;
  bool gram_tc = false;   // the Gram ran on the tensor cores
  int smem_optin = 0;
  cudaStream_t stream = nullptr;
  gdwd_options opt{};
  int64_t d = 0, n = 0;
  int store = GDWD_F32;
  double q = 1.0, C = 1.0;
  Layout L{};
  int grid = 0;
  int ldP = 0;
  double zscale = 0.0;
  double s = 0.0;
  double t_setup_ms = 0.0;
  double t_stage_ms[3] = {0.0, 0.0, 0.0};   // ingest, Gram, factor
  size_t bytes = 0;
  std::vector<void*> allocs;
  int alloc_calls = 0;   // device allocations requested so far (fault-injection hook)
  // device arrays
  void* Z = nullptr;
  double *sc = nullptr, *y = nullptr, *e = nullptr, *omega = nullptr, *wt = nullptr, *p = nullptr, *G = nullptr;
  float2 *P = nullptr, *pdf = nullptr;
  double *r = nullptr, *xi = nullptr, *alpha = nullptr, *b = nullptr;
  float2 *rhsA = nullptr, *rhsB = nullptr, *vrhs = nullptr;
  double *Uu = nullptr, *Ur = nullptr, *kc = nullptr;   // n-space images of u, rho; (G - I) c
  void *cq = nullptr, *aq = nullptr, *partial = nullptr;
  double *u = nullptr, *rho = nullptr, *g = nullptr, *scal = nullptr, *wtmp = nullptr;
  // kernelized iteration (opt.kernelized): K as double-float, the coefficient
  // vectors of u, rho, g, the last K products, the GEMV right-hand sides
  float2 *Kd = nullptr, *vdf = nullptr;
  double *au = nullptr, *ar = nullptr, *ag = nullptr, *KG = nullptr, *KR = nullptr, *wcoef = nullptr;
  // direct solver (opt.solver = 1): Z^T is the stored matrix (samples as rows);
  // G, P, p, pdf are d x d / d-long; the state of Algorithm 1 in d-space
  bool direct = false;
  // inexact solver (opt.solver = 2): no n x n or d x d matrix; eq-linsys by CG
  bool inexact = false;
  double *mw = nullptr, *ztw = nullptr, *ixw = nullptr;
  double *ixv = nullptr, *ixtn = nullptr, *ixzp = nullptr, *ixdr = nullptr;
  double *ixhw = nullptr, *ixcr = nullptr, *ixcz = nullptr, *ixcp = nullptr, *ixcap = nullptr, *ixtd = nullptr;
  double* ixpart = nullptr;
  std::vector<double> ixhpart;
  double *bhat = nullptr, *t = nullptr, *dv = nullptr, *dv2 = nullptr, *dw = nullptr, *dx = nullptr;
  double *Zxr = nullptr, *Za = nullptr, *Zdr = nullptr, *dscal = nullptr;
  float2* hw = nullptr;
  int nblk = 0;
  double* dscalars = nullptr;   // [0] sumsq [1] zscale [2] s
  double *amax = nullptr, *colscale = nullptr;   // per-column |max| and storage scale s_i
  unsigned* bar = nullptr;
  int* err = nullptr;
  Ctrl* ctrl = nullptr;
  gdwd_handle* master = nullptr;   // FP32 copy used by the refinement sweep (refine = 1)
  // state of the joint C-grid kernel (up to 4 instances), allocated on first use
  struct {
    bool ready = false;
    double *r, *xi, *alpha, *b, *u, *rho, *g, *scal, *Uu, *Ur, *kc;
    float2 *rhsA, *rhsB;
    void *coef, *partial;
    Ctrl* ctrl;
  } ms;
  double phase_ns[kPhaseSlots] = {};
  std::string last_error;
};

static thread_local std::string g_thread_error;

namespace gdwd {
// Lets the serving layer hand a worker thread's message to the polling thread.
void set_thread_error(const std::string& m) { g_thread_error = m; }
}  // namespace gdwd

static gdwd_status fail(gdwd_handle* h, gdwd_status st, const std::string& msg) {
  if (h) h->last_error = msg;
  g_thread_error = msg;
  return st;
}

static gdwd_status cuda_fail(gdwd_handle* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? GDWD_ENOMEM : GDWD_ECUDA, m);
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

// Fault-injection hooks for tests, read from the environment (no effect while
// the variables are unset):
//   GDWD_INJECT_ALLOC_FAIL=k  the k-th device allocation of a handle (kept or
//                             temporary) fails as if the device were out of memory;
//   GDWD_INJECT_STALL=1       every launch of the Z-streaming iteration kernel
//                             waits at its first grid barrier for an arrival that
//                             never comes, so its bounded wait runs out.
static long env_long(const char* name) {
  const char* v = std::getenv(name);
  return v ? std::strtol(v, nullptr, 10) : 0;
}

// Every device allocation of a handle (kept or temporary) goes through here.
static cudaError_t dev_alloc(gdwd_handle* h, void** p, size_t bytes) {
  ++h->alloc_calls;
  const long inject = env_long("GDWD_INJECT_ALLOC_FAIL");
  if (inject > 0 && (long)h->alloc_calls == inject) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, h->stream);
}

template <typename T>
static cudaError_t halloc(gdwd_handle* h, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = dev_alloc(h, &q, bytes);
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  h->bytes += bytes;
  *p = (T*)q;
  return cudaMemsetAsync(q, 0, bytes, h->stream);
}

static void release(gdwd_handle* h) {
  for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
  h->allocs.clear();
}

extern "C" gdwd_status gdwd_default_options(gdwd_options* o) {
  if (!o) return fail(nullptr, GDWD_EINVAL, "gdwd_default_options: NULL");
  std::memset(o, 0, sizeof(*o));
  o->mu = 1.0;
  o->tau = 1.618;
  o->tol = 1e-6;
  o->sigma0 = 0.0;
  o->timeout_s = 2.0;
  o->max_iter = 20000;
  o->store = GDWD_F32;
  o->grid = 0;
  o->block_rows = 0;
  o->stream = nullptr;
  return GDWD_OK;
}

static int esize_of(int dt) { return dt == GDWD_F64 ? 8 : dt == GDWD_F32 ? 4 : dt == GDWD_E4M3 ? 1 : 2; }

// Chooses slab height, slab count, chunk width and grid (see Layout).
// Slab layout of the stored matrix: `rows` rows (d; the samples n for the
// direct solver, which stores Z^T) and `cols` columns.
static void plan_layout(gdwd_handle* h, int64_t rows, int64_t cols) {
  const int es = esize_of(h->store);
  // slab heights are a multiple of the 16-byte vector and of 4 rows (the Gram
  // tile loader reads 4 consecutive rows of a column)
  const int vec = std::max(16 / es, 4);
  const int gp = h->opt.grid > 0 ? std::min(h->opt.grid, h->sms) : h->sms;
  const int64_t d = rows;
  int TB;
  if (h->opt.block_rows > 0) {
    TB = (h->opt.block_rows + vec - 1) / vec * vec;
  } else {
    const int64_t tbmax = 256LL * vec;
    const int64_t k = std::max<int64_t>(1, (d + gp * tbmax - 1) / (gp * tbmax));
    int64_t t = (d + k * gp - 1) / (k * gp);
    t = (t + vec - 1) / vec * vec;
    TB = (int)std::max<int64_t>(t, 8LL * vec);
  }
  TB = std::min(TB, 256 * vec);
  const int NB = (int)((d + TB - 1) / TB);
  h->L.d = d;
  h->L.n = cols;
  h->L.TB = TB;
  h->L.NB = NB;
  h->L.esize = es;
  h->grid = (int)std::min<int64_t>(gp, std::max<int64_t>(NB, (cols + kWarps - 1) / kWarps));
  h->grid = std::max(h->grid, 1);
  // the inexact solver streams FP32 storage into FP64 arithmetic (wider staging)
  h->L.CW = choose_chunk_cols(h->store, h->L, h->grid, h->smem_optin - 8192, h->inexact);
}

static cudaError_t dir_apply(int trans, const double* x, double* out, void* ctx);

// Set-up of the direct solver (Sec. 3.3.1): Z^T into the slab layout, its Gram
// G' = I + Z~ Z~^T / mu (d x d), b^ = Z~ y, and the factor of G' with p = G'^{-1} b^,
// s = b^T p.  h has its device, options and problem sizes set.
static gdwd_status create_direct(gdwd_handle* h, const void* Z, int zdt, int64_t ldz, int z_on_device,
                                 const double* y) {
  const int64_t d = h->d, n = h->n;
  h->direct = true;
  plan_layout(h, n, d);
  if ((d + h->grid - 1) / h->grid > kMaxRowsPerCta)
    return fail(h, GDWD_EUNSUPPORTED, "gdwd_create: d too large for the d x d factor of the direct solver");
  h->nblk = dir_blocks(n);
  cudaEvent_t e0, e1, evg, ef0;
  CK(cudaEventCreate(&e0), "cudaEventCreate");
  CK(cudaEventCreate(&e1), "cudaEventCreate");
  CK(cudaEventCreate(&evg), "cudaEventCreate");
  CK(cudaEventCreate(&ef0), "cudaEventCreate");
  CK(cudaEventRecord(e0, h->stream), "cudaEventRecord");
  const int64_t npad = (int64_t)h->L.NB * h->L.TB;
  const int es = h->L.esize;
  const int zes = esize_of(zdt);
  void* zbuf = nullptr;
  CK(dev_alloc(h, (void**)&zbuf, (size_t)npad * d * es), "cudaMalloc(Z)");
  h->allocs.push_back(zbuf);
  h->bytes += (size_t)npad * d * es;
  h->Z = zbuf;
  h->L.Z = zbuf;
  h->ldP = (int)((d + 1) / 2 * 2);
  CK(halloc(h, &h->sc, d), "alloc");
  CK(halloc(h, &h->amax, d), "alloc");
  CK(halloc(h, &h->colscale, d), "alloc");
  CK(halloc(h, &h->y, n), "alloc");
  CK(halloc(h, &h->e, n), "alloc");
  CK(halloc(h, &h->omega, n), "alloc");
  CK(halloc(h, &h->wt, n), "alloc");
  CK(halloc(h, &h->p, d), "alloc");
  CK(halloc(h, &h->G, (size_t)d * d), "alloc(G)");
  CK(halloc(h, &h->P, (size_t)d * h->ldP), "alloc(P)");
  CK(halloc(h, &h->pdf, h->ldP), "alloc");
  CK(halloc(h, &h->bhat, d), "alloc");
  CK(halloc(h, &h->r, n), "alloc");
  CK(halloc(h, &h->xi, n), "alloc");
  CK(halloc(h, &h->alpha, n), "alloc");
  CK(halloc(h, &h->t, n), "alloc");
  CK(halloc(h, &h->dv, n), "alloc");
  CK(halloc(h, &h->dv2, n), "alloc");
  CK(halloc(h, &h->u, d), "alloc");
  CK(halloc(h, &h->rho, d), "alloc");
  CK(halloc(h, &h->dw, d), "alloc");
  CK(halloc(h, &h->g, d), "alloc");
  CK(halloc(h, &h->dx, d + 1), "alloc");
  CK(halloc(h, &h->hw, h->ldP), "alloc");
  CK(halloc(h, &h->Zxr, d), "alloc");
  CK(halloc(h, &h->Za, d), "alloc");
  CK(halloc(h, &h->Zdr, d), "alloc");
  CK(halloc(h, &h->wtmp, d), "alloc");
  CK(halloc(h, &h->scal, (size_t)DS_SLOTS * h->nblk), "alloc");
  CK(halloc(h, &h->dscal, h->nblk), "alloc");
  CK(halloc(h, (uint8_t**)&h->partial, (size_t)2 * d * h->L.NB * sizeof(double)), "alloc");   // two products
  CK(halloc(h, &h->dscalars, 8), "alloc");
  CK(halloc(h, &h->bar, 4), "alloc");
  CK(halloc(h, &h->err, 4), "alloc");
  CK(halloc(h, (uint8_t**)&h->ctrl, sizeof(Ctrl)), "alloc");
  CK(cudaMemcpyAsync(h->y, y, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy y");
  const int fb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  fill_kernel<<<fb, 256, 0, h->stream>>>(h->e, n, 1.0);
  fill_kernel<<<fb, 256, 0, h->stream>>>(h->wt, n, 1.0);
  fill_kernel<<<fb, 256, 0, h->stream>>>(h->omega, n, h->q);
  // ingest: the caller's Z (d x n, column-major) transposed to n x d, then the
  // slab layout with samples as rows
  const void* zsrc = Z;
  void* staging = nullptr;
  int64_t ld = ldz;
  if (!z_on_device) {
    CK(dev_alloc(h, (void**)&staging, (size_t)d * n * zes), "cudaMalloc(staging)");
    cudaError_t ec = cudaMemcpy2DAsync(staging, (size_t)d * zes, Z, (size_t)ldz * zes, (size_t)d * zes, (size_t)n,
                                       cudaMemcpyHostToDevice, h->stream);
    if (ec != cudaSuccess) {
      cudaFreeAsync(staging, h->stream);
      return cuda_fail(h, ec, "copy Z");
    }
    zsrc = staging;
    ld = d;
  }
  void* zt = nullptr;
  cudaError_t ei = dev_alloc(h, (void**)&zt, (size_t)d * n * zes);
  if (ei == cudaSuccess) ei = run_transpose(zsrc, zdt, d, n, ld, zt, h->stream);
  const int nparts = 1024;
  double* part = nullptr;
  if (ei == cudaSuccess) ei = dev_alloc(h, (void**)&part, nparts * sizeof(double));
  if (ei == cudaSuccess)
    ei = run_ingest(zt, zdt, n, h->L, h->Z, h->store, part, nparts, h->dscalars, h->err, h->sc, h->dscalars + 1,
                    h->amax, h->colscale, h->stream);
  int nf = 0;
  if (ei == cudaSuccess) ei = cudaMemcpyAsync(&nf, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (ei == cudaSuccess) ei = cudaStreamSynchronize(h->stream);
  if (part) cudaFreeAsync(part, h->stream);
  if (zt) cudaFreeAsync(zt, h->stream);
  if (staging) cudaFreeAsync(staging, h->stream);
  if (ei != cudaSuccess) return cuda_fail(h, ei, "ingest");
  if (nf) return fail(h, GDWD_EINVAL, "gdwd_create: Z has non-finite entries");
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream), "memset");
  // G' = I + Z~ Z~^T / mu: the Gram of the stored Z^T
  CK(cudaEventRecord(evg, h->stream), "cudaEventRecord");
  const bool tc = h->opt.gram_path == 0 && gram_tc_supported(h->store, h->L);
  const int ks = tc ? gram_tc_ksplit(h->store, h->L, h->sms) : gram_ksplit(h->L, h->sms);
  double* Kpart = nullptr;
  CK(dev_alloc(h, (void**)&Kpart, (size_t)ks * d * d * sizeof(double)), "cudaMalloc(Kpart)");
  void* gscratch = nullptr;
  const size_t gsb = tc ? gram_tc_scratch_bytes(h->store, h->L) : 0;
  cudaError_t eg = gsb ? dev_alloc(h, &gscratch, gsb) : cudaSuccess;
  if (eg == cudaSuccess)
    eg = run_gram(h->store, h->L, ks, Kpart, h->sc, h->opt.mu, h->G, tc, gscratch, h->err,
                  (uint64_t)(h->opt.timeout_s * 1e9), h->stream);
  if (gscratch) cudaFreeAsync(gscratch, h->stream);
  if (eg == cudaSuccess) {
    CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream), "memset");
    eg = dir_apply(1, h->y, h->bhat, h);   // b^ = Z~ y
  }
  int gerr = 0;
  if (eg == cudaSuccess) eg = cudaMemcpyAsync(&gerr, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (eg == cudaSuccess) eg = cudaStreamSynchronize(h->stream);
  cudaFreeAsync(Kpart, h->stream);
  if (eg != cudaSuccess) return cuda_fail(h, eg, "gram");
  if (gerr) return fail(h, (gdwd_status)gerr, "gdwd_create: a set-up kernel timed out");
  h->gram_tc = tc;
  // factor of G', p = G'^{-1} b^, s = b^T p
  CK(cudaEventRecord(ef0, h->stream), "cudaEventRecord");
  float2 *A = nullptr, *X = nullptr;
  CK(dev_alloc(h, (void**)&A, (size_t)d * d * sizeof(float2)), "cudaMalloc(A)");
  cudaError_t ef = dev_alloc(h, (void**)&X, (size_t)d * d * sizeof(float2));
  if (ef == cudaSuccess) ef = cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->stream);
  if (ef == cudaSuccess) {
    FactorArgs fa{h->G, A, X, h->P, h->ldP, h->bhat, h->p, h->pdf, h->dscalars + 2, d, h->grid, h->bar, h->err,
                  (uint64_t)(h->opt.timeout_s * 1e9)};
    ef = run_factor(fa, h->stream);
  }
  int ferr = 0;
  if (ef == cudaSuccess) ef = cudaMemcpyAsync(&ferr, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  double hs[3] = {0, 0, 0};
  if (ef == cudaSuccess) ef = cudaMemcpyAsync(hs, h->dscalars, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (ef == cudaSuccess) ef = cudaEventRecord(e1, h->stream);
  if (ef == cudaSuccess) ef = cudaStreamSynchronize(h->stream);
  cudaFreeAsync(A, h->stream);
  cudaFreeAsync(X, h->stream);
  if (ef != cudaSuccess) return cuda_fail(h, ef, "factor");
  if (ferr == GDWD_ENOTPD) return fail(h, GDWD_ENOTPD, "gdwd_create: Cholesky met a non-positive pivot");
  if (ferr) return fail(h, (gdwd_status)ferr, "gdwd_create: factor kernel reported an error");
  h->zscale = hs[1];
  h->s = hs[2];
  float ms = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventElapsedTime(&m1, e0, evg);
  cudaEventElapsedTime(&m2, evg, ef0);
  cudaEventElapsedTime(&m3, ef0, e1);
  h->t_setup_ms = ms;
  h->t_stage_ms[0] = m1;
  h->t_stage_ms[1] = m2;
  h->t_stage_ms[2] = m3;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(evg);
  cudaEventDestroy(ef0);
  // the border's Schur complement n - s / mu is positive (A is positive definite)
  if (!((double)n - h->s / h->opt.mu > 0.0) || !std::isfinite(h->s))
    return fail(h, GDWD_ENUMERIC, "gdwd_create: the Schur complement of the direct solver is not positive");
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_create(const void* Z, int32_t zdt, int64_t d, int64_t n, int64_t ldz, int32_t z_on_device,
                                   const double* y, double q, double C, const gdwd_options* o, gdwd_handle** out) {
  if (!out) return fail(nullptr, GDWD_EINVAL, "gdwd_create: out is NULL");
  *out = nullptr;
  if (!Z || !y) return fail(nullptr, GDWD_EINVAL, "gdwd_create: Z or y is NULL");
  if (d < 1 || n < 2 || ldz < d) return fail(nullptr, GDWD_EINVAL, "gdwd_create: need d >= 1, n >= 2, ldz >= d");
  if (zdt != GDWD_F64 && zdt != GDWD_F32) return fail(nullptr, GDWD_EINVAL, "gdwd_create: Z must be F64 or F32");
  if (!(q > 0.0) || !std::isfinite(q)) return fail(nullptr, GDWD_EINVAL, "gdwd_create: q must be > 0");
  if (!(C > 0.0) || !std::isfinite(C)) return fail(nullptr, GDWD_EINVAL, "gdwd_create: C must be > 0");
  int npos = 0, nneg = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (y[i] == 1.0) ++npos;
    else if (y[i] == -1.0) ++nneg;
    else return fail(nullptr, GDWD_EINVAL, "gdwd_create: labels must be -1 or +1");
  }
  if (!npos || !nneg) return fail(nullptr, GDWD_EINVAL, "gdwd_create: both classes must occur");
  gdwd_options opt;
  gdwd_default_options(&opt);
  if (o) opt = *o;
  if (!(opt.mu > 0.0) || !(opt.tau > 0.0 && opt.tau < 1.6180339887498949) || !(opt.tol > 0.0) || opt.max_iter < 1 ||
      !(opt.timeout_s > 0.0))
    return fail(nullptr, GDWD_EINVAL, "gdwd_create: bad options (mu > 0, 0 < tau < golden ratio, tol > 0, max_iter >= 1)");
  if (opt.store < GDWD_F64 || opt.store > GDWD_E4M3) return fail(nullptr, GDWD_EINVAL, "gdwd_create: bad store dtype");
  if (opt.gram_path != 0 && opt.gram_path != 1) return fail(nullptr, GDWD_EINVAL, "gdwd_create: gram_path must be 0 or 1");
  if (opt.stop_rule != 0 && opt.stop_rule != 1) return fail(nullptr, GDWD_EINVAL, "gdwd_create: stop_rule must be 0 or 1");
  if (opt.dots_every < 0) return fail(nullptr, GDWD_EINVAL, "gdwd_create: dots_every must be >= 0");
  if (opt.kernelized < -1 || opt.kernelized > 1)
    return fail(nullptr, GDWD_EINVAL, "gdwd_create: kernelized must be -1, 0 or 1");
  if (opt.solver < 0 || opt.solver > 2) return fail(nullptr, GDWD_EINVAL, "gdwd_create: solver must be 0, 1 or 2");
  if (opt.solver == 2 && (opt.refine || opt.kernelized == 1 || (opt.store != GDWD_F32 && opt.store != GDWD_F64)))
    return fail(nullptr, GDWD_EUNSUPPORTED,
                "gdwd_create: the inexact solver runs with F32 or F64 storage, without refine and kernelized");
  if (opt.solver == 1 && (opt.refine || opt.kernelized == 1 || (opt.store != GDWD_F32 && opt.store != GDWD_F64)))
    return fail(nullptr, GDWD_EUNSUPPORTED,
                "gdwd_create: the direct solver runs with F32 or F64 storage, without refine and kernelized");

  gdwd_handle* h = new gdwd_handle();
  h->opt = opt;
  if (opt.solver != 0) h->opt.kernelized = 0;   // "auto" means the streaming products there
  h->stream = (cudaStream_t)opt.stream;
  h->d = d;
  h->n = n;
  h->store = opt.store;
  h->q = q;
  h->C = C;
  gdwd_status st = GDWD_OK;
  auto bail = [&](gdwd_status s2) {
    release(h);
    delete h;
    return s2;
  };
  {
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "cudaGetDevice"));
    // handle memory comes from the device's stream-ordered pool; keep freed blocks
    // cached in the pool so that creating the next handle does not go to the driver
    static bool pool_set[64] = {};
    static std::mutex pool_mu;
    std::lock_guard<std::mutex> pool_lock(pool_mu);
    if (h->device >= 0 && h->device < 64 && !pool_set[h->device]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      pool_set[h->device] = true;
    }
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (!coop) return bail(fail(nullptr, GDWD_ECUDA, "device does not support cooperative launch"));
  }
  if (opt.solver == 1) {
    st = create_direct(h, Z, zdt, ldz, z_on_device, y);
    if (st != GDWD_OK) return bail(st);
    *out = h;
    return GDWD_OK;
  }
  h->inexact = opt.solver == 2;
  plan_layout(h, d, n);
  if (h->opt.kernelized < 0) {
    // auto: the kernelized loop wherever K fits it.  It was the faster of the
    // two on every measured workload (no pass over Z between the n-space
    // phases), and with 16- or 8-bit storage the more robust: all its products
    // go through the one Gram, while the streaming loop mixes the Gram's
    // tensor-core rounding with direct products of the stored codes (on a
    // served FP16 stream 27 of 419 requests then missed kkt 1e-6).
    h->opt.kernelized = n <= kern_max_n(h->grid, h->smem_optin - 16384) ? 1 : 0;
  }
  if (!h->inexact && (n + h->grid - 1) / h->grid > kMaxRowsPerCta)
    return bail(fail(nullptr, GDWD_EUNSUPPORTED, "gdwd_create: n too large for the n x n factor path of this build"));
  if (h->opt.kernelized && n > kern_max_n(h->grid, h->smem_optin - 16384))
    return bail(fail(nullptr, GDWD_EUNSUPPORTED, "gdwd_create: n too large for the kernelized iteration"));
  st = [&]() -> gdwd_status {
    cudaEvent_t e0, e1, evg, ef0;
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    CK(cudaEventCreate(&e1), "cudaEventCreate");
    CK(cudaEventCreate(&evg), "cudaEventCreate");
    CK(cudaEventCreate(&ef0), "cudaEventCreate");
    CK(cudaEventRecord(e0, h->stream), "cudaEventRecord");
    const int64_t dpad = (int64_t)h->L.NB * h->L.TB;
    const int es = h->L.esize;
    const int zes = esize_of(zdt);
    // persistent arrays
    void* zbuf = nullptr;
    CK(dev_alloc(h, (void**)&zbuf, (size_t)dpad * n * es), "cudaMalloc(Z)");
    h->allocs.push_back(zbuf);
    h->bytes += (size_t)dpad * n * es;
    h->Z = zbuf;
    h->L.Z = zbuf;
    h->ldP = (int)((n + 1) / 2 * 2);
    CK(halloc(h, &h->sc, n), "alloc");
    CK(halloc(h, &h->amax, n), "alloc");
    CK(halloc(h, &h->colscale, n), "alloc");
    CK(halloc(h, &h->y, n), "alloc");
    CK(halloc(h, &h->e, n), "alloc");
    CK(halloc(h, &h->omega, n), "alloc");
    CK(halloc(h, &h->wt, n), "alloc");
    CK(halloc(h, &h->r, n), "alloc");
    CK(halloc(h, &h->xi, n), "alloc");
    CK(halloc(h, &h->alpha, n), "alloc");
    const size_t ct = (h->store == GDWD_F64 || h->inexact) ? 8 : 4;   // the inexact solver's products are FP64
    if (!h->inexact) {
      CK(halloc(h, &h->p, n), "alloc");
      CK(halloc(h, &h->G, (size_t)n * n), "alloc(G)");
      CK(halloc(h, &h->P, (size_t)n * h->ldP), "alloc(P)");
      CK(halloc(h, &h->pdf, h->ldP), "alloc");   // padded to ldP (a zero pair for odd n): read as a G^{-1} row
      CK(cudaMemsetAsync(h->pdf, 0, (size_t)h->ldP * sizeof(float2), h->stream), "memset");
      CK(halloc(h, &h->b, n), "alloc");
      CK(halloc(h, &h->rhsA, h->ldP), "alloc");   // padded to ldP (zero pair): read as pairs
      CK(halloc(h, &h->Uu, n), "alloc");
      CK(halloc(h, &h->Ur, n), "alloc");
      CK(halloc(h, &h->kc, n), "alloc");
      CK(halloc(h, &h->rhsB, h->ldP), "alloc");
      // right-hand sides of the fused first solve, [3][ldP], padding zero
      CK(halloc(h, &h->vrhs, (size_t)3 * h->ldP), "alloc");
      CK(halloc(h, (uint8_t**)&h->cq, (n * ct + 15) / 16 * 16), "alloc");   // copied in 16-byte pieces
      CK(halloc(h, (uint8_t**)&h->aq, (n * ct + 15) / 16 * 16), "alloc");
    } else {
      for (double** pp : {&h->ztw, &h->ixv, &h->ixtn, &h->ixzp, &h->ixdr}) CK(halloc(h, pp, n), "alloc");
      for (double** pp : {&h->mw, &h->ixw, &h->ixhw, &h->ixcr, &h->ixcz, &h->ixcp, &h->ixcap, &h->ixtd})
        CK(halloc(h, pp, dpad), "alloc");
      CK(halloc(h, &h->ixpart, (size_t)kIxSlots * kIxBlocks), "alloc");
      h->ixhpart.assign((size_t)kIxSlots * kIxBlocks, 0.0);
    }
    CK(halloc(h, (uint8_t**)&h->partial, (size_t)n * h->L.NB * ct), "alloc");
    CK(halloc(h, &h->u, dpad), "alloc");
    CK(halloc(h, &h->rho, dpad), "alloc");
    CK(halloc(h, &h->g, dpad), "alloc");
    CK(halloc(h, &h->wtmp, dpad), "alloc");
    CK(halloc(h, &h->scal, (size_t)h->sms * S_COUNT), "alloc");
    if (h->opt.kernelized) {
      CK(halloc(h, &h->Kd, (size_t)n * h->ldP), "alloc(K)");
      CK(halloc(h, &h->vdf, (size_t)3 * h->ldP), "alloc");
      CK(halloc(h, &h->au, n), "alloc");
      CK(halloc(h, &h->ar, n), "alloc");
      CK(halloc(h, &h->ag, n), "alloc");
      CK(halloc(h, &h->KG, n), "alloc");
      CK(halloc(h, &h->KR, n), "alloc");
      CK(halloc(h, &h->wcoef, n), "alloc");
    }
    CK(halloc(h, &h->dscalars, 8), "alloc");
    CK(halloc(h, &h->bar, 4), "alloc");
    CK(halloc(h, &h->err, 4), "alloc");
    CK(halloc(h, (uint8_t**)&h->ctrl, sizeof(Ctrl)), "alloc");
    // labels and unit weights (e = 1, wt = 1, omega = q)
    CK(cudaMemcpyAsync(h->y, y, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy y");
    const int fb = (int)std::min<int64_t>((n + 255) / 256, 1024);
    fill_kernel<<<fb, 256, 0, h->stream>>>(h->e, n, 1.0);
    fill_kernel<<<fb, 256, 0, h->stream>>>(h->wt, n, 1.0);
    fill_kernel<<<fb, 256, 0, h->stream>>>(h->omega, n, q);
    // ingest
    const void* zsrc = Z;
    void* staging = nullptr;
    int64_t ld = ldz;
    if (!z_on_device) {
      CK(dev_alloc(h, (void**)&staging, (size_t)d * n * zes), "cudaMalloc(staging)");
      cudaError_t ec = cudaMemcpy2DAsync(staging, (size_t)d * zes, Z, (size_t)ldz * zes, (size_t)d * zes, (size_t)n,
                                         cudaMemcpyHostToDevice, h->stream);
      if (ec != cudaSuccess) {
        cudaFreeAsync(staging, h->stream);
        return cuda_fail(h, ec, "copy Z");
      }
      zsrc = staging;
      ld = d;
    }
    // The set-up runs as one stream of kernels with a single synchronisation at
    // the end; the non-finite flag (err[1]) and the kernels' status (err[0]) are
    // read there.  Data with a non-finite entry still flows through the Gram and
    // the factor (whose bounded waits and pivot checks keep them finite in time)
    // and is refused at the end.
    const int nparts = 1024;
    double* part = nullptr;
    int* nonfinite = h->err + 1;
    CK(dev_alloc(h, (void**)&part, nparts * sizeof(double)), "cudaMalloc");
    cudaError_t ei = run_ingest(zsrc, zdt, ld, h->L, h->Z, h->store, part, nparts, h->dscalars, nonfinite, h->sc,
                                h->dscalars + 1, h->amax, h->colscale, h->stream);
    cudaFreeAsync(part, h->stream);
    if (staging) cudaFreeAsync(staging, h->stream);
    if (ei != cudaSuccess) return cuda_fail(h, ei, "ingest");
    if (h->inexact) {
      int nf = 0;
      CK(cudaMemcpyAsync(&nf, nonfinite, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "copy");
      CK(cudaStreamSynchronize(h->stream), "sync");
      if (nf) return fail(h, GDWD_EINVAL, "gdwd_create: Z has non-finite entries");
      // no Gram and no factor: the Jacobi preconditioner diag(Z~ Z~^T) + mu and Z_scale
      CK(cudaEventRecord(evg, h->stream), "cudaEventRecord");
      CK(run_row_sumsq(h->store, h->L, h->sc, h->opt.mu, h->mw, h->stream), "preconditioner");
      double hs[2] = {0, 0};
      CK(cudaMemcpyAsync(hs, h->dscalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy");
      CK(cudaEventRecord(e1, h->stream), "cudaEventRecord");
      CK(cudaStreamSynchronize(h->stream), "sync");
      h->zscale = hs[1];
      float ms = 0.f, m1 = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventElapsedTime(&m1, e0, evg);
      h->t_setup_ms = ms;
      h->t_stage_ms[0] = m1;
      h->t_stage_ms[1] = ms - m1;
      h->t_stage_ms[2] = 0.0;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      cudaEventDestroy(evg);
      cudaEventDestroy(ef0);
      if (!(h->zscale > 0.0) || !std::isfinite(h->zscale)) return fail(h, GDWD_EINVAL, "gdwd_create: Z is zero");
      return GDWD_OK;
    }
    // Gram and G = I + K / mu
    CK(cudaEventRecord(evg, h->stream), "cudaEventRecord");
    const bool tc = h->opt.gram_path == 0 && gram_tc_supported(h->store, h->L);
    const int ks = tc ? gram_tc_ksplit(h->store, h->L, h->sms) : gram_ksplit(h->L, h->sms);
    double* Kpart = nullptr;
    CK(dev_alloc(h, (void**)&Kpart, (size_t)ks * n * n * sizeof(double)), "cudaMalloc(Kpart)");
    void* gscratch = nullptr;     // the BF16 split of FP32 storage for the tensor-core Gram
    const size_t gsb = tc ? gram_tc_scratch_bytes(h->store, h->L) : 0;
    cudaError_t eg = gsb ? dev_alloc(h, &gscratch, gsb) : cudaSuccess;
    if (eg == cudaSuccess)
      eg = run_gram(h->store, h->L, ks, Kpart, h->sc, h->opt.mu, h->G, tc, gscratch, h->err,
                    (uint64_t)(h->opt.timeout_s * 1e9), h->stream);
    if (gscratch) cudaFreeAsync(gscratch, h->stream);
    cudaFreeAsync(Kpart, h->stream);
    if (eg != cudaSuccess) return cuda_fail(h, eg, "gram");
    h->gram_tc = tc;
    // Cholesky, inverse, p, s
    CK(cudaEventRecord(ef0, h->stream), "cudaEventRecord");
    float2 *A = nullptr, *X = nullptr;
    CK(dev_alloc(h, (void**)&A, (size_t)n * n * sizeof(float2)), "cudaMalloc(A)");
    cudaError_t ef = dev_alloc(h, (void**)&X, (size_t)n * n * sizeof(float2));
    if (ef == cudaSuccess) ef = cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->stream);
    const int fgrid = h->grid;   // the handle's SM share (all SMs unless restricted by opt.grid)
    if (ef == cudaSuccess) {
      FactorArgs fa{h->G, A, X, h->P, h->ldP, h->y, h->p, h->pdf, h->dscalars + 2, n, fgrid, h->bar, h->err,
                    (uint64_t)(h->opt.timeout_s * 1e9)};
      ef = run_factor(fa, h->stream);
    }
    if (ef == cudaSuccess && h->opt.kernelized) ef = run_kern_matrix(h->G, n, h->ldP, h->opt.mu, h->Kd, h->stream);
    int flags[2] = {0, 0};
    if (ef == cudaSuccess) ef = cudaMemcpyAsync(flags, h->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    double hs[3] = {0, 0, 0};
    if (ef == cudaSuccess) ef = cudaMemcpyAsync(hs, h->dscalars, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (ef == cudaSuccess) ef = cudaEventRecord(e1, h->stream);
    if (ef == cudaSuccess) ef = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(A, h->stream);
    cudaFreeAsync(X, h->stream);
    if (ef != cudaSuccess) return cuda_fail(h, ef, "factor");
    if (flags[1]) return fail(h, GDWD_EINVAL, "gdwd_create: Z has non-finite entries");
    if (flags[0] == GDWD_ENOTPD) return fail(h, GDWD_ENOTPD, "gdwd_create: Cholesky met a non-positive pivot");
    if (flags[0]) return fail(h, (gdwd_status)flags[0], "gdwd_create: the Gram or factor kernel reported an error");
    h->zscale = hs[1];
    h->s = hs[2];
    float ms = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventElapsedTime(&m1, e0, evg);
    cudaEventElapsedTime(&m2, evg, ef0);
    cudaEventElapsedTime(&m3, ef0, e1);
    h->t_setup_ms = ms;
    h->t_stage_ms[0] = m1;
    h->t_stage_ms[1] = m2;
    h->t_stage_ms[2] = m3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(evg);
    cudaEventDestroy(ef0);
    if (!(h->s > 0.0) || !std::isfinite(h->s)) return fail(h, GDWD_ENUMERIC, "gdwd_create: y^T G^{-1} y is not positive");
    return GDWD_OK;
  }();
  if (st != GDWD_OK) return bail(st);
  if (opt.refine && (opt.store == GDWD_BF16 || opt.store == GDWD_F16 || opt.store == GDWD_E4M3)) {
    gdwd_options om = opt;
    om.store = GDWD_F32;
    om.refine = 0;
    om.grid = h->grid;
    om.kernelized = h->opt.kernelized;   // the master continues the quantized solve's kind of iterate
    st = gdwd_create(Z, zdt, d, n, ldz, z_on_device, y, q, C, &om, &h->master);
    if (st != GDWD_OK) return bail(st);
  }
  *out = h;
  return GDWD_OK;
}

// iterations between direct Z~^T u column dots (0 = by storage: the Gram of
// FP64 / FP32 storage is within a few 1e-8, the tensor-core Gram within 5e-7)
static int dots_every_of(const gdwd_handle* h) {
  if (h->opt.dots_every > 0) return h->opt.dots_every;
  return (h->store == GDWD_F64 || h->store == GDWD_F32) ? 16 : 4;
}

template <typename CT>
static IterArgs<CT> make_args(gdwd_handle* h, double C, double sigma0, int refresh) {
  IterArgs<CT> a{};
  a.L = h->L;
  a.sc = h->sc;
  a.P = h->P;
  a.ldP = h->ldP;
  a.pdf = h->pdf;
  a.p = h->p;
  a.y = h->y;
  a.e = h->e;
  a.omega = h->omega;
  a.wt = h->wt;
  a.inv_s = 1.0 / h->s;
  a.q = h->q;
  a.C = C;
  a.mu = h->opt.mu;
  a.tau = h->opt.tau;
  a.R = h->zscale;
  a.tol = h->opt.tol;
  a.kappa = (h->q + 1.0) / h->q * std::pow(h->q, 1.0 / (h->q + 1.0));
  a.max_iter = h->opt.max_iter;
  a.stop_rule = h->opt.stop_rule;
  a.grid = h->grid;
  a.timeout_ns = (uint64_t)(h->opt.timeout_s * 1e9);
  a.r = h->r;
  a.xi = h->xi;
  a.alpha = h->alpha;
  a.b = h->b;
  a.rhsA = h->rhsA;
  a.Uu = h->Uu;
  a.Ur = h->Ur;
  a.kc = h->kc;
  a.refresh = refresh;
  a.dots_every = dots_every_of(h);
  a.stall_first_barrier = env_long("GDWD_INJECT_STALL") > 0 ? 1 : 0;
  a.fuse = 1;   // the fused first solve wherever its operands fit the ring (its products overlap barrier 8 and phase S)
  a.vrhs = h->vrhs;
  a.rhsB = h->rhsB;
  a.cq = (CT*)h->cq;
  a.aq = (CT*)h->aq;
  a.u = h->u;
  a.rho = h->rho;
  a.g = h->g;
  a.partial = (CT*)h->partial;
  a.scal = h->scal;
  a.bar = h->bar;
  a.err = h->err;
  a.ctrl = h->ctrl;
  return a;
}

static KernArgs make_kern_args(gdwd_handle* h, double C, int refresh) {
  KernArgs a{};
  a.P = h->P;
  a.Kd = h->Kd;
  a.ldP = h->ldP;
  a.pdf = h->pdf;
  a.p = h->p;
  a.y = h->y;
  a.e = h->e;
  a.omega = h->omega;
  a.wt = h->wt;
  a.n = h->n;
  a.inv_s = 1.0 / h->s;
  a.q = h->q;
  a.C = C;
  a.mu = h->opt.mu;
  a.tau = h->opt.tau;
  a.R = h->zscale;
  a.tol = h->opt.tol;
  a.kappa = (h->q + 1.0) / h->q * std::pow(h->q, 1.0 / (h->q + 1.0));
  a.max_iter = h->opt.max_iter;
  a.stop_rule = h->opt.stop_rule;
  a.grid = h->grid;
  a.refresh = refresh;
  a.timeout_ns = (uint64_t)(h->opt.timeout_s * 1e9);
  a.r = h->r;
  a.xi = h->xi;
  a.alpha = h->alpha;
  a.b = h->b;
  a.rhsA = h->rhsA;
  a.rhsB = h->rhsB;
  a.Uu = h->Uu;
  a.Ur = h->Ur;
  a.au = h->au;
  a.ar = h->ar;
  a.ag = h->ag;
  a.KG = h->KG;
  a.KR = h->KR;
  a.vdf = h->vdf;
  a.scal = h->scal;
  a.bar = h->bar;
  a.err = h->err;
  a.ctrl = h->ctrl;
  return a;
}

// The streaming passes of the direct solver over the stored Z^T: trans = 0 gives
// Z~^T x (per sample), trans = 1 gives Z~ x (per feature; partials per slab).
static cudaError_t dir_apply(int trans, const double* x, double* out, void* ctx) {
  gdwd_handle* h = static_cast<gdwd_handle*>(ctx);
  return run_dir_product(h->L, h->store, trans, x, h->sc, out, reinterpret_cast<double*>(h->partial), h->stream);
}

static cudaError_t dir_apply2(const double* x, const double* x2, double* out, double* out2, void* ctx) {
  gdwd_handle* h = static_cast<gdwd_handle*>(ctx);
  double* part = reinterpret_cast<double*>(h->partial);
  return run_dir_product2(h->L, h->store, x, x2, h->sc, out, out2, part, part + (size_t)h->d * h->L.NB, h->stream);
}

// One solve of the direct solver from the initial iterate of reading R3.  The
// host issues the iteration's kernels in batches of kDirBatch iterations (a
// captured CUDA graph after the first batch) and reads the control block
// between batches; kernels issued after convergence return at once (the
// streaming passes among them still run).
static gdwd_status solve_direct(gdwd_handle* h, double C, double* w, int w_on_device, double* alpha,
                                gdwd_result* res) {
  constexpr int kDirBatch = 8;
  const int64_t n = h->n, d = h->d;
  cudaStream_t st = h->stream;
  const double sigma0 = h->opt.sigma0 > 0 ? h->opt.sigma0 : std::pow(std::min(10.0 * C, (double)n), h->q);
  const int fb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  fill_kernel<<<fb, 256, 0, st>>>(h->r, n, 1.0);
  fill_kernel<<<fb, 256, 0, st>>>(h->xi, n, 1.0);
  CK(cudaMemsetAsync(h->alpha, 0, n * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->u, 0, d * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->rho, 0, d * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->Zxr, 0, d * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->Za, 0, d * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->scal, 0, (size_t)DS_SLOTS * h->nblk * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), st), "memset");
  Ctrl c0{};
  c0.sigma = sigma0;
  c0.sigma_prev = sigma0;
  c0.theta = 1.0;
  CK(cudaMemcpyAsync(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st), "copy ctrl");
  DirArgs a{};
  a.d = d;
  a.n = n;
  a.P = h->P;
  a.ldP = h->ldP;
  a.pdf = h->pdf;
  a.p = h->p;
  a.s = h->s;
  a.y = h->y;
  a.e = h->e;
  a.omega = h->omega;
  a.wt = h->wt;
  a.q = h->q;
  a.C = C;
  a.mu = h->opt.mu;
  a.tau = h->opt.tau;
  a.R = h->zscale;
  a.tol = h->opt.tol;
  a.kappa = (h->q + 1.0) / h->q * std::pow(h->q, 1.0 / (h->q + 1.0));
  a.max_iter = h->opt.max_iter;
  a.stop_rule = h->opt.stop_rule;
  a.r = h->r;
  a.xi = h->xi;
  a.alpha = h->alpha;
  a.t = h->t;
  a.dv = h->dv;
  a.dv2 = h->dv2;
  a.u = h->u;
  a.rho = h->rho;
  a.w = h->dw;
  a.g = h->g;
  a.x = h->dx;
  a.hw = h->hw;
  a.Zxr = h->Zxr;
  a.Za = h->Za;
  a.Zdr = h->Zdr;
  a.scal = h->scal;
  a.dscal = h->dscal;
  a.nblk = h->nblk;
  a.ctrl = h->ctrl;
  const DirPasses ps{dir_apply, dir_apply2, h};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(cudaEventRecord(e0, st), "event");
  Ctrl c{};
  int kerr = 0;
  // A batch is ~16 kernel launches per iteration.  The first batch runs
  // eagerly (it also sets the kernels' attributes); the later ones replay one
  // CUDA graph captured from the same calls, so the host issues one launch per
  // batch.  If capture is refused the batches stay eager.
  auto batch = [&]() -> cudaError_t {
    for (int b = 0; b < kDirBatch; ++b) {
      const cudaError_t e = run_dir_iteration(a, ps, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  struct GraphExec {
    cudaGraphExec_t x = nullptr;
    ~GraphExec() {
      if (x) cudaGraphExecDestroy(x);
    }
  } gx;
  bool use_graph = true;
  for (int it = 0; it < h->opt.max_iter; it += kDirBatch) {
    cudaError_t e = cudaSuccess;
    if (it > 0 && use_graph && !gx.x) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t eb = batch();
        e = cudaStreamEndCapture(st, &g);
        if (eb != cudaSuccess) e = eb;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&gx.x, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {   // nothing captured ran: run the batch eagerly from now on
        cudaGetLastError();
        gx.x = nullptr;
        use_graph = false;
      }
    }
    e = gx.x ? cudaGraphLaunch(gx.x, st) : batch();
    if (e != cudaSuccess) return cuda_fail(h, e, "direct solver iteration");
    CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "copy ctrl");
    CK(cudaMemcpyAsync(&kerr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy err");
    CK(cudaStreamSynchronize(st), "sync");
    if (c.done || kerr) break;
  }
  CK(cudaEventRecord(e1, st), "event");
  double* wdst = (w && w_on_device) ? w : h->wtmp;
  CK(run_dir_finish(h->dw, h->zscale, d, wdst, st), "finish");
  if (w && !w_on_device) CK(cudaMemcpyAsync(w, h->wtmp, d * sizeof(double), cudaMemcpyDeviceToHost, st), "copy w");
  if (alpha) CK(cudaMemcpyAsync(alpha, h->alpha, n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy alpha");
  CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "copy ctrl");
  CK(cudaStreamSynchronize(st), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::memset(h->phase_ns, 0, sizeof(h->phase_ns));
  std::memset(res, 0, sizeof(*res));
  res->beta = c.beta;
  res->primal_obj = c.pobj;
  res->dual_obj = c.dobj;
  res->kkt = c.kkt;
  res->eta_p = std::max(c.eta_p1, std::max(c.eta_p2, c.eta_p3));
  res->eta_d = std::max(c.eta_d1, std::max(c.eta_d2, c.eta_d3));
  res->eta_c = std::max(c.eta_c1, std::max(c.eta_c2, c.eta_c3));
  res->eta_gap = c.eta_gap;
  res->sigma = c.sigma;
  res->zscale = h->zscale;
  res->t_setup_ms = h->t_setup_ms;
  res->t_solve_ms = ms;
  res->iters = c.it;
  gdwd_status s = kerr ? (gdwd_status)kerr : (c.done ? (gdwd_status)c.status : GDWD_EMAXITER);
  res->status = s;
  if (kerr) return fail(h, s, "gdwd_solve: a device wait of the direct solver expired");
  return s;
}

// One solve for penalty C.  warm == NULL starts from the initial iterate of
// reading R3; otherwise the iterate (and sigma) of the last solve of `warm` (a
// handle of the same problem with another storage type) is the starting point.
// A state to start a solve from: another handle's last iterate (refinement sweep,
// iteration count restarts) or one instance of the joint C-grid kernel (it
// continues, counting on).
struct WarmSrc {
  const double *r, *xi, *alpha, *u, *rho, *g;
  const double *au, *ar, *ag;   // coefficient vectors of a kernelized handle (else NULL)
  const Ctrl* ctrl;           // device
  cudaStream_t stream;
  bool keep_count;
};

static WarmSrc warm_from(const gdwd_handle* o) {
  return WarmSrc{o->r, o->xi, o->alpha, o->u, o->rho, o->g, o->au, o->ar, o->ag, o->ctrl, o->stream, false};
}

static gdwd_status solve_one(gdwd_handle* h, double C, double* w, int w_on_device, double* alpha, gdwd_result* res,
                             const WarmSrc* warm = nullptr) {
  const int64_t n = h->n, d = h->d;
  const int64_t dpad = (int64_t)h->L.NB * h->L.TB;
  cudaStream_t st = h->stream;
  const double sigma0 = h->opt.sigma0 > 0 ? h->opt.sigma0 : std::pow(std::min(10.0 * C, (double)n), h->q);
  Ctrl c0{};
  if (!warm) {
    // initial iterate: r = xi = 1, w = u = 0, beta = 0, alpha = 0, rho = 0
    const int fb = (int)std::min<int64_t>((n + 255) / 256, 1024);
    fill_kernel<<<fb, 256, 0, st>>>(h->r, n, 1.0);
    fill_kernel<<<fb, 256, 0, st>>>(h->xi, n, 1.0);
    CK(cudaMemsetAsync(h->alpha, 0, n * sizeof(double), st), "memset");
    CK(cudaMemsetAsync(h->u, 0, dpad * sizeof(double), st), "memset");
    CK(cudaMemsetAsync(h->rho, 0, dpad * sizeof(double), st), "memset");
    CK(cudaMemsetAsync(h->g, 0, dpad * sizeof(double), st), "memset");
    c0.sigma = sigma0;
    c0.sigma_prev = sigma0;
    c0.theta = 1.0;
  } else {
    // warm start: copy the other handle's iterate (same scaled problem: both scale by
    // sqrt(||Z||_F) of the caller's data, so r, xi, alpha, u, rho, g carry over)
    CK(cudaStreamSynchronize(warm->stream), "sync");
    const size_t nb = n * sizeof(double), db = d * sizeof(double);
    CK(cudaMemcpyAsync(h->r, warm->r, nb, cudaMemcpyDeviceToDevice, st), "warm copy");
    CK(cudaMemcpyAsync(h->xi, warm->xi, nb, cudaMemcpyDeviceToDevice, st), "warm copy");
    CK(cudaMemcpyAsync(h->alpha, warm->alpha, nb, cudaMemcpyDeviceToDevice, st), "warm copy");
    if (h->opt.kernelized) {
      // the iterate is carried by its coefficient vectors; a handle without them
      // (a Z-streaming one) cannot hand over u and rho in this form
      if (!warm->au) return fail(h, GDWD_EUNSUPPORTED, "gdwd_solve: a kernelized solve starts only from a kernelized iterate");
      CK(cudaMemcpyAsync(h->au, warm->au, nb, cudaMemcpyDeviceToDevice, st), "warm copy");
      CK(cudaMemcpyAsync(h->ar, warm->ar, nb, cudaMemcpyDeviceToDevice, st), "warm copy");
      CK(cudaMemcpyAsync(h->ag, warm->ag, nb, cudaMemcpyDeviceToDevice, st), "warm copy");
    } else {
      if (!warm->u) return fail(h, GDWD_EUNSUPPORTED, "gdwd_solve: a Z-streaming solve starts only from a Z-streaming iterate");
      CK(cudaMemcpyAsync(h->u, warm->u, db, cudaMemcpyDeviceToDevice, st), "warm copy");
      CK(cudaMemcpyAsync(h->rho, warm->rho, db, cudaMemcpyDeviceToDevice, st), "warm copy");
      CK(cudaMemcpyAsync(h->g, warm->g, db, cudaMemcpyDeviceToDevice, st), "warm copy");
    }
    CK(cudaMemcpy(&c0, warm->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost), "warm ctrl");
    if (!warm->keep_count) c0.it = 0;
    c0.status = 0;
    c0.done = 0;
  }
  CK(cudaMemcpyAsync(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st), "copy ctrl");
  CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st), "memset");
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), st), "memset");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(cudaEventRecord(e0, st), "event");
  cudaError_t e;
  const int smem_limit = h->smem_optin - 8192;
  if (h->opt.kernelized)
    e = run_iterate_kern(make_kern_args(h, C, warm ? 1 : 0), smem_limit, st);
  else if (h->store == GDWD_F64)
    e = run_iterate_f64(make_args<double>(h, C, sigma0, warm ? 1 : 0), smem_limit, st);
  else
    e = run_iterate_f32(h->store, make_args<float>(h, C, sigma0, warm ? 1 : 0), smem_limit, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "iterate launch");
  CK(cudaEventRecord(e1, st), "event");
  Ctrl c{};
  int kerr = 0;
  CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "copy ctrl");
  CK(cudaMemcpyAsync(&kerr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy err");
  double* wdst = (w && w_on_device) ? w : h->wtmp;
  if (h->opt.kernelized) {
    // w = Z~ (a_g + a_rho / (sigma' sqrt(mu))) / Z_scale by one pass over the stored Z
    CK(run_kern_wcoef(h->ag, h->ar, h->ctrl, std::sqrt(h->opt.mu), h->zscale, n, h->wcoef, st), "finish");
    CK(run_apply(h->store, h->L, 0, h->wcoef, h->sc, wdst, h->partial, std::min(h->L.NB, 4096), smem_limit, h->err,
                 (uint64_t)(h->opt.timeout_s * 1e9), st),
       "finish");
  } else {
    const int wb = (int)std::min<int64_t>((d + 255) / 256, 2048);
    finish_w_kernel<<<wb, 256, 0, st>>>(h->g, h->rho, h->ctrl, std::sqrt(h->opt.mu), h->zscale, d, wdst);
    CK(cudaGetLastError(), "finish");
  }
  if (w && !w_on_device) CK(cudaMemcpyAsync(w, h->wtmp, d * sizeof(double), cudaMemcpyDeviceToHost, st), "copy w");
  if (alpha) CK(cudaMemcpyAsync(alpha, h->alpha, n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy alpha");
  int ferr = 0;
  if (h->opt.kernelized) CK(cudaMemcpyAsync(&ferr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy err");
  CK(cudaStreamSynchronize(st), "sync");
  if (!kerr) kerr = ferr;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::memcpy(h->phase_ns, c.phase_ns, sizeof(h->phase_ns));
  std::memset(res, 0, sizeof(*res));
  res->beta = c.beta;
  res->primal_obj = c.pobj;
  res->dual_obj = c.dobj;
  res->kkt = c.kkt;
  res->eta_p = std::max(c.eta_p1, std::max(c.eta_p2, c.eta_p3));
  res->eta_d = std::max(c.eta_d1, std::max(c.eta_d2, c.eta_d3));
  res->eta_c = std::max(c.eta_c1, std::max(c.eta_c2, c.eta_c3));
  res->eta_gap = c.eta_gap;
  res->sigma = c.sigma;
  res->zscale = h->zscale;
  res->t_setup_ms = h->t_setup_ms;
  res->t_solve_ms = ms;
  res->iters = c.it;
  gdwd_status s = kerr ? (gdwd_status)kerr : (gdwd_status)c.status;
  res->status = s;
  if (kerr) return fail(h, s, "gdwd_solve: iteration kernel stopped with a device error (bounded wait expired)");
  return s;
}

// The inexact solver (solver = 2): products with the stored data by the
// streaming kernels; trans != 0 gives Z~^T x, trans == 0 gives Z~ x.
static cudaError_t ix_apply(int trans, const double* x, double* out, void* ctx) {
  gdwd_handle* h = static_cast<gdwd_handle*>(ctx);
  return run_apply(h->store, h->L, trans, x, h->sc, out, h->partial, std::min(h->L.NB, 4096), h->smem_optin - 8192,
                   h->err, (uint64_t)(h->opt.timeout_s * 1e9), h->stream, true);
}

static gdwd_status solve_inexact(gdwd_handle* h, double C, double* w, int w_on_device, double* alpha,
                                 gdwd_result* res) {
  const int64_t n = h->n, d = h->d, dpad = (int64_t)h->L.NB * h->L.TB;
  cudaStream_t st = h->stream;
  const double sigma0 = h->opt.sigma0 > 0 ? h->opt.sigma0 : std::pow(std::min(10.0 * C, (double)n), h->q);
  // initial iterate: r = xi = 1, w = u = 0, beta = 0, alpha = 0, rho = 0
  const int fb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  fill_kernel<<<fb, 256, 0, st>>>(h->r, n, 1.0);
  fill_kernel<<<fb, 256, 0, st>>>(h->xi, n, 1.0);
  CK(cudaMemsetAsync(h->alpha, 0, n * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->ixw, 0, dpad * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->u, 0, dpad * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->rho, 0, dpad * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->ztw, 0, n * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), st), "memset");
  IxArgs a{};
  a.d = d;
  a.n = n;
  a.y = h->y;
  a.e = h->e;
  a.omega = h->omega;
  a.wt = h->wt;
  a.mw = h->mw;
  a.q = h->q;
  a.C = C;
  a.mu = h->opt.mu;
  a.tau = h->opt.tau;
  a.R = h->zscale;
  a.tol = h->opt.tol;
  a.kappa = (h->q + 1.0) / h->q * std::pow(h->q, 1.0 / (h->q + 1.0));
  a.eps_c = 1.0 / h->zscale;   // 1 / ||Z~||_F: ||Z~||_F = ||Z||_F / Z_scale = Z_scale
  a.max_iter = h->opt.max_iter;
  a.stop_rule = h->opt.stop_rule;
  a.r = h->r;
  a.xi = h->xi;
  a.alpha = h->alpha;
  a.ztw = h->ztw;
  a.w = h->ixw;
  a.u = h->u;
  a.rho = h->rho;
  a.beta = 0.0;
  a.v = h->ixv;
  a.tn = h->ixtn;
  a.zp = h->ixzp;
  a.dr = h->ixdr;
  a.hw = h->ixhw;
  a.cr = h->ixcr;
  a.cz = h->ixcz;
  a.cp = h->ixcp;
  a.cap = h->ixcap;
  a.td = h->ixtd;
  a.part = h->ixpart;
  a.hpart = h->ixhpart.data();
  const IxPasses ps{ix_apply, h};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(cudaEventRecord(e0, st), "event");
  IxResult r{};
  CK(run_inexact(a, ps, sigma0, st, &r), "inexact solver");
  CK(cudaEventRecord(e1, st), "event");
  int kerr = 0;
  CK(cudaMemcpyAsync(&kerr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy err");
  double* wdst = (w && w_on_device) ? w : h->wtmp;
  CK(run_dir_finish(h->ixw, h->zscale, d, wdst, st), "finish");
  if (w && !w_on_device) CK(cudaMemcpyAsync(w, h->wtmp, d * sizeof(double), cudaMemcpyDeviceToHost, st), "copy w");
  if (alpha) CK(cudaMemcpyAsync(alpha, h->alpha, n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy alpha");
  CK(cudaStreamSynchronize(st), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::memset(h->phase_ns, 0, sizeof(h->phase_ns));
  std::memset(res, 0, sizeof(*res));
  res->beta = r.beta;
  res->primal_obj = r.pobj;
  res->dual_obj = r.dobj;
  res->kkt = r.kkt;
  res->eta_p = std::max(r.eta_p1, std::max(r.eta_p2, r.eta_p3));
  res->eta_d = std::max(r.eta_d1, std::max(r.eta_d2, r.eta_d3));
  res->eta_c = std::max(r.eta_c1, std::max(r.eta_c2, r.eta_c3));
  res->eta_gap = r.eta_gap;
  res->sigma = r.sigma;
  res->zscale = h->zscale;
  res->t_setup_ms = h->t_setup_ms;
  res->t_solve_ms = ms;
  res->iters = r.iters;
  res->reserved[1] = r.cg_steps;        // conjugate-gradient steps of Steps 1a and 1c
  res->reserved[2] = r.step1c_solves;   // iterations in which Step 1c solved (the paper's "double")
  gdwd_status s = kerr ? (gdwd_status)kerr : (gdwd_status)r.status;
  res->status = s;
  if (kerr) return fail(h, s, "gdwd_solve: a device wait of the inexact solver expired");
  return s;
}

// Up to four values of C in lock-step in one launch of the joint kernel.
static gdwd_status solve_multi(gdwd_handle* h, const double* Cs, int K, int kker, double* w, int w_on_device,
                               double* alpha, gdwd_result* res) {
  const int64_t n = h->n, d = h->d;
  const int64_t dpad = (int64_t)h->L.NB * h->L.TB;
  cudaStream_t st = h->stream;
  const size_t ct = h->store == GDWD_F64 ? 8 : 4;
  auto& m = h->ms;
  if (!m.ready) {
    CK(halloc(h, &m.r, 4 * n), "alloc");
    CK(halloc(h, &m.xi, 4 * n), "alloc");
    CK(halloc(h, &m.alpha, 4 * n), "alloc");
    CK(halloc(h, &m.b, 4 * n), "alloc");
    CK(halloc(h, &m.rhsA, 4 * n), "alloc");
    CK(halloc(h, &m.rhsB, 4 * n), "alloc");
    CK(halloc(h, &m.Uu, 4 * n), "alloc");
    CK(halloc(h, &m.Ur, 4 * n), "alloc");
    CK(halloc(h, &m.kc, 4 * n), "alloc");
    CK(halloc(h, (uint8_t**)&m.coef, 8 * n * ct), "alloc");
    CK(halloc(h, (uint8_t**)&m.partial, 4 * (size_t)n * h->L.NB * ct), "alloc");
    CK(halloc(h, &m.u, 4 * dpad), "alloc");
    CK(halloc(h, &m.rho, 4 * dpad), "alloc");
    CK(halloc(h, &m.g, 4 * dpad), "alloc");
    CK(halloc(h, &m.scal, 4 * (size_t)S_COUNT * h->sms), "alloc");
    CK(halloc(h, (uint8_t**)&m.ctrl, 4 * sizeof(Ctrl)), "alloc");
    m.ready = true;
  }
  const int fb = (int)std::min<int64_t>((4 * n + 255) / 256, 1024);
  fill_kernel<<<fb, 256, 0, st>>>(m.r, 4 * n, 1.0);
  fill_kernel<<<fb, 256, 0, st>>>(m.xi, 4 * n, 1.0);
  CK(cudaMemsetAsync(m.alpha, 0, 4 * n * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(m.u, 0, 4 * dpad * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(m.rho, 0, 4 * dpad * sizeof(double), st), "memset");
  CK(cudaMemsetAsync(m.g, 0, 4 * dpad * sizeof(double), st), "memset");
  Ctrl c0[4] = {};
  for (int j = 0; j < 4; ++j) {
    const double Cj = Cs[j < K ? j : 0];
    const double s0 = h->opt.sigma0 > 0 ? h->opt.sigma0 : std::pow(std::min(10.0 * Cj, (double)n), h->q);
    c0[j].sigma = s0;
    c0[j].sigma_prev = s0;
    c0[j].theta = 1.0;
  }
  CK(cudaMemcpyAsync(m.ctrl, c0, sizeof(c0), cudaMemcpyHostToDevice, st), "copy ctrl");
  CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st), "memset");
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), st), "memset");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(cudaEventRecord(e0, st), "event");
  auto fill = [&](auto& a) {
    a.L = h->L;
    a.sc = h->sc;
    a.P = h->P;
    a.ldP = h->ldP;
    a.pdf = h->pdf;
    a.p = h->p;
    a.y = h->y;
    a.e = h->e;
    a.omega = h->omega;
    a.wt = h->wt;
    a.inv_s = 1.0 / h->s;
    a.q = h->q;
    a.mu = h->opt.mu;
    a.tau = h->opt.tau;
    a.R = h->zscale;
    a.tol = h->opt.tol;
    a.kappa = (h->q + 1.0) / h->q * std::pow(h->q, 1.0 / (h->q + 1.0));
    for (int j = 0; j < 4; ++j) a.C[j] = Cs[j < K ? j : 0];
    a.K = K;
    a.max_iter = h->opt.max_iter;
    a.stop_rule = h->opt.stop_rule;
    a.grid = h->grid;
    a.timeout_ns = (uint64_t)(h->opt.timeout_s * 1e9);
    a.dpad = dpad;
    a.r = m.r;
    a.xi = m.xi;
    a.alpha = m.alpha;
    a.b = m.b;
    a.rhsA = m.rhsA;
    a.rhsB = m.rhsB;
    a.Uu = m.Uu;
    a.Ur = m.Ur;
    a.kc = m.kc;
    a.dots_every = dots_every_of(h);
    a.min_active = K > 1 ? 2 : 1;   // a lone straggler continues in the single-instance kernel
    a.u = m.u;
    a.rho = m.rho;
    a.g = m.g;
    a.scal = m.scal;
    a.bar = h->bar;
    a.err = h->err;
    a.ctrl = m.ctrl;
  };
  const int smem_limit = h->smem_optin - 16384;
  cudaError_t e;
  if (h->store == GDWD_F64) {
    MultiArgs<double> a{};
    fill(a);
    a.coef = (double*)m.coef;
    a.partial = (double*)m.partial;
    e = run_multi_f64(kker, a, smem_limit, st);
  } else {
    MultiArgs<float> a{};
    fill(a);
    a.coef = (float*)m.coef;
    a.partial = (float*)m.partial;
    e = run_multi_f32(h->store, kker, a, smem_limit, st);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "joint C-grid launch");
  CK(cudaEventRecord(e1, st), "event");
  Ctrl c[4];
  int kerr = 0;
  CK(cudaMemcpyAsync(c, m.ctrl, sizeof(c), cudaMemcpyDeviceToHost, st), "copy ctrl");
  CK(cudaMemcpyAsync(&kerr, h->err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy err");
  const int wb = (int)std::min<int64_t>((d + 255) / 256, 2048);
  for (int j = 0; j < K; ++j) {
    double* wdst = (w && w_on_device) ? w + (size_t)j * d : h->wtmp;
    finish_w_kernel<<<wb, 256, 0, st>>>(m.g + (size_t)j * dpad, m.rho + (size_t)j * dpad, m.ctrl + j,
                                        std::sqrt(h->opt.mu), h->zscale, d, wdst);
    CK(cudaGetLastError(), "finish");
    if (w && !w_on_device)
      CK(cudaMemcpyAsync(w + (size_t)j * d, h->wtmp, d * sizeof(double), cudaMemcpyDeviceToHost, st), "copy w");
    if (alpha)
      CK(cudaMemcpyAsync(alpha + (size_t)j * n, m.alpha + (size_t)j * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                         st),
         "copy alpha");
    if (w && !w_on_device) CK(cudaStreamSynchronize(st), "sync");   // h->wtmp is reused per instance
  }
  CK(cudaStreamSynchronize(st), "sync");
  std::memcpy(h->phase_ns, c[0].phase_ns, sizeof(h->phase_ns));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  gdwd_status worst = GDWD_OK;
  for (int j = 0; j < K; ++j) {
    gdwd_result* r = res + j;
    std::memset(r, 0, sizeof(*r));
    r->beta = c[j].beta;
    r->primal_obj = c[j].pobj;
    r->dual_obj = c[j].dobj;
    r->kkt = c[j].kkt;
    r->eta_p = std::max(c[j].eta_p1, std::max(c[j].eta_p2, c[j].eta_p3));
    r->eta_d = std::max(c[j].eta_d1, std::max(c[j].eta_d2, c[j].eta_d3));
    r->eta_c = std::max(c[j].eta_c1, std::max(c[j].eta_c2, c[j].eta_c3));
    r->eta_gap = c[j].eta_gap;
    r->sigma = c[j].sigma;
    r->zscale = h->zscale;
    r->t_setup_ms = h->t_setup_ms;
    r->t_solve_ms = ms;   // the whole joint launch (shared by its instances)
    r->iters = c[j].it;
    r->status = kerr ? kerr : c[j].status;
    if (r->status != GDWD_OK && worst == GDWD_OK) worst = (gdwd_status)r->status;
  }
  if (kerr) return fail(h, (gdwd_status)kerr, "gdwd_solve: joint kernel stopped with a device error");
  // an instance still iterating when the others had stopped: continue it from its
  // state in the single-instance kernel (which does the work of one instance, where
  // the joint kernel would still pay for K)
  for (int j = 0; j < K; ++j) {
    if (c[j].status != GDWD_EMAXITER || c[j].it >= h->opt.max_iter) continue;
    const WarmSrc ws{m.r + (size_t)j * n, m.xi + (size_t)j * n, m.alpha + (size_t)j * n, m.u + (size_t)j * dpad,
                     m.rho + (size_t)j * dpad, m.g + (size_t)j * dpad, nullptr, nullptr, nullptr, m.ctrl + j, st,
                     true};
    const float joint_ms = ms;
    const gdwd_status sj = solve_one(h, Cs[j], w ? w + (size_t)j * d : nullptr, w_on_device,
                                     alpha ? alpha + (size_t)j * n : nullptr, res + j, &ws);
    res[j].t_solve_ms += joint_ms;
    if (sj != GDWD_OK && sj != GDWD_EMAXITER) return sj;
  }
  worst = GDWD_OK;
  for (int j = 0; j < K; ++j)
    if (res[j].status != GDWD_OK && worst == GDWD_OK) worst = (gdwd_status)res[j].status;
  return worst;
}

extern "C" gdwd_status gdwd_solve(gdwd_handle* h, const double* Cs, int32_t nC, double* w, int32_t w_on_device,
                                  double* alpha, gdwd_result* res) {
  if (!h || !res) return fail(h, GDWD_EINVAL, "gdwd_solve: NULL handle or result");
  if (nC < 0) return fail(h, GDWD_EINVAL, "gdwd_solve: nC < 0");
  const int count = (Cs && nC > 0) ? nC : 1;
  for (int k = 0; k < count; ++k) {
    const double C = (Cs && nC > 0) ? Cs[k] : h->C;
    if (!(C > 0.0) || !std::isfinite(C)) return fail(h, GDWD_EINVAL, "gdwd_solve: C must be > 0");
  }
  gdwd_status worst = GDWD_OK;
  // joint C-grid: groups of up to four C values per launch (one Z read per pass for all)
  const int kmax = (count >= 2 && !h->master && !h->opt.cgrid_sequential && !h->opt.kernelized && !h->direct &&
                    !h->inexact)
                       ? multi_max_k(h->store, h->L, h->grid, h->smem_optin - 16384)
                       : 1;
  int k0 = 0;
  while (kmax >= 2 && count - k0 >= 2) {
    const int K = std::min(kmax, count - k0);
    const int kker = K <= 2 ? 2 : 4;
    gdwd_status s = solve_multi(h, Cs + k0, K, kker, w ? w + (size_t)k0 * h->d : nullptr, w_on_device,
                                alpha ? alpha + (size_t)k0 * h->n : nullptr, res + k0);
    if (s != GDWD_OK && s != GDWD_EMAXITER) return s;
    if (s != GDWD_OK) worst = s;
    k0 += K;
  }
  for (int k = k0; k < count; ++k) {
    const double C = (Cs && nC > 0) ? Cs[k] : h->C;
    gdwd_status s;
    if (h->master) {
      // refinement sweep: the quantized solve, then the FP32 master warm-started from it
      gdwd_result rq;
      s = solve_one(h, C, nullptr, 0, nullptr, &rq);
      if (s != GDWD_OK && s != GDWD_EMAXITER) return s;
      const WarmSrc ws = warm_from(h);
      s = solve_one(h->master, C, w ? w + (size_t)k * h->d : nullptr, w_on_device,
                    alpha ? alpha + (size_t)k * h->n : nullptr, res + k, &ws);
      res[k].iters += rq.iters;
      res[k].t_solve_ms += rq.t_solve_ms;
      res[k].t_setup_ms = h->t_setup_ms + h->master->t_setup_ms;
      res[k].reserved[0] = rq.iters;   // iterations on the quantized data
      if (s != GDWD_OK && s != GDWD_EMAXITER) return fail(h, s, h->master->last_error);
    } else if (h->direct) {
      s = solve_direct(h, C, w ? w + (size_t)k * h->d : nullptr, w_on_device,
                       alpha ? alpha + (size_t)k * h->n : nullptr, res + k);
    } else if (h->inexact) {
      s = solve_inexact(h, C, w ? w + (size_t)k * h->d : nullptr, w_on_device,
                        alpha ? alpha + (size_t)k * h->n : nullptr, res + k);
    } else {
      s = solve_one(h, C, w ? w + (size_t)k * h->d : nullptr, w_on_device,
                    alpha ? alpha + (size_t)k * h->n : nullptr, res + k);
    }
    if (s != GDWD_OK && s != GDWD_EMAXITER) return s;
    if (s != GDWD_OK) worst = s;
  }
  return worst;
}

extern "C" gdwd_status gdwd_free(gdwd_handle* h) {
  if (!h) return GDWD_OK;
  if (h->master) gdwd_free(h->master);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  release(h);
  delete h;
  return GDWD_OK;
}

extern "C" const char* gdwd_last_error(const gdwd_handle* h) {
  return h ? h->last_error.c_str() : g_thread_error.c_str();
}

extern "C" gdwd_status gdwd_prox(const double* a, const double* r0, const double* omega, double sigma, double q,
                                 int64_t n, double* out, void* stream) {
  gdwd_handle* h = nullptr;
  if (n < 0 || !(q > 0.0) || !(sigma > 0.0)) return fail(nullptr, GDWD_EINVAL, "gdwd_prox: need n >= 0, q > 0, sigma > 0");
  if (n > 0 && (!a || !out)) return fail(nullptr, GDWD_EINVAL, "gdwd_prox: NULL array");
  CK(launch_prox(a, r0, omega, sigma, q, n, out, (cudaStream_t)stream), "gdwd_prox");
  CK(cudaStreamSynchronize((cudaStream_t)stream), "gdwd_prox sync");
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_apply(gdwd_handle* h, int32_t trans, const double* x, double* out) {
  if (!h || !x || !out) return fail(h, GDWD_EINVAL, "gdwd_apply: NULL argument");
  if (h->direct) return fail(h, GDWD_EUNSUPPORTED, "gdwd_apply: not on a handle of the direct solver");
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream), "memset");
  const int grid = h->L.NB;   // one CTA per slab
  CK(run_apply(h->store, h->L, trans, x, h->sc, out, h->partial, std::min(grid, 4096), h->smem_optin - 8192, h->err,
               (uint64_t)(h->opt.timeout_s * 1e9), h->stream),
     "gdwd_apply");
  int kerr = 0;
  CK(cudaMemcpyAsync(&kerr, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "copy err");
  CK(cudaStreamSynchronize(h->stream), "sync");
  if (kerr) return fail(h, (gdwd_status)kerr, "gdwd_apply: device wait expired");
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_gram(gdwd_handle* h, double* G_out) {
  if (!h || !G_out) return fail(h, GDWD_EINVAL, "gdwd_gram: NULL argument");
  if (h->inexact) return fail(h, GDWD_EUNSUPPORTED, "gdwd_gram: the inexact solver forms no Gram matrix");
  const size_t m = (size_t)(h->direct ? h->d : h->n);   // d x d for the direct solver
  CK(cudaMemcpyAsync(G_out, h->G, m * m * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy G");
  CK(cudaStreamSynchronize(h->stream), "sync");
  return GDWD_OK;
}

// ---------------------------------------------------------------- weights and C
// omega_i = q wt_i^q (the prox constant of the weighted r-term)
__global__ void omega_kernel(const double* wt, double q, int64_t n, double* omega) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    omega[i] = q * pow(wt[i], q);
}

static gdwd_status set_weights_one(gdwd_handle* h, const double* e, const double* wt) {
  const int64_t n = h->n;
  const int fb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  if (e) CK(cudaMemcpyAsync(h->e, e, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy e");
  else fill_kernel<<<fb, 256, 0, h->stream>>>(h->e, n, 1.0);
  if (wt) CK(cudaMemcpyAsync(h->wt, wt, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "copy wt");
  else fill_kernel<<<fb, 256, 0, h->stream>>>(h->wt, n, 1.0);
  omega_kernel<<<fb, 256, 0, h->stream>>>(h->wt, h->q, n, h->omega);
  CK(cudaGetLastError(), "omega");
  CK(cudaStreamSynchronize(h->stream), "sync");
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_set_weights(gdwd_handle* h, const double* e, const double* wt) {
  if (!h) return fail(nullptr, GDWD_EINVAL, "gdwd_set_weights: NULL handle");
  for (int64_t i = 0; i < h->n; ++i) {
    if (e && !(e[i] > 0.0 && std::isfinite(e[i])))
      return fail(h, GDWD_EINVAL, "gdwd_set_weights: e must be positive and finite");
    if (wt && !(wt[i] > 0.0 && std::isfinite(wt[i])))
      return fail(h, GDWD_EINVAL, "gdwd_set_weights: wt must be positive and finite");
  }
  gdwd_status st = set_weights_one(h, e, wt);
  if (st == GDWD_OK && h->master) st = set_weights_one(h->master, e, wt);
  return st;
}

extern "C" gdwd_status gdwd_imbalance_weights(const double* y, int64_t n, double q, double* wt) {
  if (!y || !wt || n < 2 || !(q > 0.0)) return fail(nullptr, GDWD_EINVAL, "gdwd_imbalance_weights: bad argument");
  int64_t np = 0, nm = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (y[i] == 1.0) ++np;
    else if (y[i] == -1.0) ++nm;
    else return fail(nullptr, GDWD_EINVAL, "gdwd_imbalance_weights: labels must be -1 or +1");
  }
  if (!np || !nm) return fail(nullptr, GDWD_EINVAL, "gdwd_imbalance_weights: both classes must occur");
  const double K = (double)n / std::log((double)n);
  const double tp = std::pow((double)np / K, 1.0 / (1.0 + q)), tm = std::pow((double)nm / K, 1.0 / (1.0 + q));
  const double mx = std::max(tp, tm);
  for (int64_t i = 0; i < n; ++i) wt[i] = (y[i] == 1.0 ? tm : tp) / mx;
  return GDWD_OK;
}

// ||x_i - x_j|| for every pair i in the +1 class, j in the -1 class, from the Gram of
// Z~: with x_i = y_i z_i, x_i - x_j = z_i + z_j, so the squared distance is
// K_ii + K_jj + 2 K_ij, K = mu Z_scale^2 (G - I).
__global__ void pair_dist_kernel(const double* G, int64_t n, const int* pos, int64_t np, const int* neg, int64_t nm,
                                 double kscale, double* out) {
  const int64_t total = np * nm;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = pos[idx / nm], j = neg[idx % nm];
    const double kii = G[i * n + i] - 1.0, kjj = G[j * n + j] - 1.0, kij = G[i * n + j];
    out[idx] = sqrt(fmax(0.0, kscale * (kii + kjj + 2.0 * kij)));
  }
}

extern "C" gdwd_status gdwd_suggest_C(gdwd_handle* h, double* C_out) {
  if (!h || !C_out) return fail(h, GDWD_EINVAL, "gdwd_suggest_C: NULL argument");
  if (h->direct || h->inexact)
    return fail(h, GDWD_EUNSUPPORTED, "gdwd_suggest_C: needs the n x n Gram (not on a direct or inexact handle)");
  const int64_t n = h->n;
  std::vector<double> y(n);
  CK(cudaMemcpyAsync(y.data(), h->y, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy y");
  CK(cudaStreamSynchronize(h->stream), "sync");
  std::vector<int> pos, neg;
  for (int64_t i = 0; i < n; ++i) (y[i] > 0 ? pos : neg).push_back((int)i);
  const int64_t np = (int64_t)pos.size(), nm = (int64_t)neg.size(), total = np * nm;
  int *dpos = nullptr, *dneg = nullptr;
  double* dd = nullptr;
  std::vector<double> dist(total);
  auto cleanup = [&]() {
    if (dpos) cudaFreeAsync(dpos, h->stream);
    if (dneg) cudaFreeAsync(dneg, h->stream);
    if (dd) cudaFreeAsync(dd, h->stream);
  };
  cudaError_t e = dev_alloc(h, (void**)&dpos, np * sizeof(int));
  if (e == cudaSuccess) e = dev_alloc(h, (void**)&dneg, nm * sizeof(int));
  if (e == cudaSuccess) e = dev_alloc(h, (void**)&dd, total * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dpos, pos.data(), np * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dneg, neg.data(), nm * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    const double kscale = h->opt.mu * h->zscale * h->zscale;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    pair_dist_kernel<<<blocks, 256, 0, h->stream>>>(h->G, n, dpos, np, dneg, nm, kscale, dd);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(dist.data(), dd, total * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(h, e, "gdwd_suggest_C");
  // median of the between-class distances (mean of the two middle ones for an even count)
  const int64_t mid = total / 2;
  std::nth_element(dist.begin(), dist.begin() + mid, dist.end());
  double med = dist[mid];
  if (total % 2 == 0) med = 0.5 * (med + *std::max_element(dist.begin(), dist.begin() + mid));
  // C = 10^(q+1) max{1, 10^(q-1) log(n) max(1000, d)^(1/3) / dist^(q+1)}  (Sec. 4.1)
  const double q = h->q;
  const double t = std::pow(10.0, q - 1.0) * std::log((double)n) * std::cbrt(std::max(1000.0, (double)h->d)) /
                   std::pow(med, q + 1.0);
  *C_out = std::pow(10.0, q + 1.0) * std::max(1.0, t);
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_get_info(const gdwd_handle* h, gdwd_info* info) {
  if (!h || !info) return fail(nullptr, GDWD_EINVAL, "gdwd_get_info: NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->d = h->d;
  info->n = h->n;
  info->store = h->store;
  info->block_rows = h->L.TB;
  info->slabs = h->L.NB;
  info->grid = h->grid;
  info->z_bytes = (int64_t)h->L.NB * h->L.TB * h->L.n * h->L.esize;
  info->device_bytes = (int64_t)h->bytes;
  info->zscale = h->zscale;
  info->t_setup_ms = h->t_setup_ms;
  info->t_ingest_ms = h->t_stage_ms[0];
  info->t_gram_ms = h->t_stage_ms[1];
  info->t_factor_ms = h->t_stage_ms[2];
  info->gram_tensor_cores = h->gram_tc ? 1 : 0;
  info->kernelized = h->opt.kernelized;
  info->solver = h->direct ? 1 : (h->inexact ? 2 : 0);
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_get_phase_times(const gdwd_handle* h, double* ns, int32_t count) {
  if (!h || !ns || count < 0 || count > kPhaseSlots) return fail(nullptr, GDWD_EINVAL, "gdwd_get_phase_times: bad argument");
  for (int k = 0; k < count; ++k) ns[k] = h->phase_ns[k];
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_get_stored(const gdwd_handle* h, void* Zq, double* colscale) {
  if (!h || (!Zq && !colscale)) return fail(nullptr, GDWD_EINVAL, "gdwd_get_stored: bad argument");
  if (h->direct) return fail(nullptr, GDWD_EUNSUPPORTED, "gdwd_get_stored: not on a direct-solver handle");
  gdwd_handle* hh = const_cast<gdwd_handle*>(h);
  const int es = h->L.esize;
  const int64_t d = h->d, n = h->n, TB = h->L.TB;
  if (Zq) {
    std::vector<uint8_t> buf((size_t)h->L.NB * TB * n * es);
    cudaError_t e = cudaMemcpyAsync(buf.data(), h->Z, buf.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(hh, e, "gdwd_get_stored");
    uint8_t* out = (uint8_t*)Zq;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < d; ++j) {
        const int64_t s = j / TB, jl = j - s * TB;
        std::memcpy(out + (i * d + j) * es, buf.data() + ((s * n + i) * TB + jl) * es, es);
      }
  }
  if (colscale) {
    if (h->store == GDWD_F64 || h->store == GDWD_F32) {
      for (int64_t i = 0; i < n; ++i) colscale[i] = 1.0;
    } else {
      cudaError_t e = cudaMemcpyAsync(colscale, h->colscale, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) return cuda_fail(hh, e, "gdwd_get_stored");
    }
  }
  return GDWD_OK;
}
