// Persistent iteration kernel of libgdwd: the whole inexact sGS-ADMM loop
// (Algorithm 1, Sec. 3) for one value of C runs in ONE cooperative launch with
// one CTA per SM and bounded grid barriers between its phases.
//
// The (d+1)x(d+1) system eq-linsys is solved in n-space.  With D^2 = mu I,
// G = I + Z~^T Z~ / mu, p = G^{-1} y, s = y^T p, g' = u + rho / (sigma sqrt(mu))
// and b = Z~^T g', the solution of eq-linsys for v = xi - r - alpha / sigma is
//     x = G^{-1}(b + v),  beta = -y^T x / s,  c = x + beta p,
//     Z~^T w = c - v - y beta,   w = g' - Z~ c / mu
// (Woodbury applied to the SMW2 form of Sec. 3.3.2; the CPU oracle uses the
// paper's d-space formulas eq-Ainv / eq-H instead, so the tests check this
// algebra).  The Step-1b prox input c^k of eq-1c is then c-bar + r^k, and Step 1c
// only changes x, beta, c.
//
// b = Z~^T g' needs no pass of its own.  With U_u = Z~^T u, U_rho = Z~^T rho and
// U_g = Z~^T g, the deferred Step 2/3 update u+ = theta g,
// rho+ = (1 - tau) rho - tau sigma sqrt(mu) (1 - theta) g maps to the same
// update of U_u, U_rho, and since g = u - Z~ c / mu,
//     U_g = Z~^T u - Z~^T Z~ c / mu = Z~^T u - (G - I) c,
//     (G - I) c = (G - I)(x + beta p) = rhs2 - x + beta (y - p)
// (G x = rhs2 and G p = y).  U_u follows u+ = theta g; every dots_every-th
// iteration Z~^T u is taken directly instead, as column dots on the chunks
// pass B streams anyway (u is known before the pass starts), so the Gram's
// rounding in (G - I) c accumulates over at most dots_every iterations; U_rho
// follows its recurrence, which contracts by |1 - tau| < 1.  One iteration
// therefore reads Z ONCE:
//
//   prologue             warm start: U_u, U_rho by two passes over Z (after the
//                        deferred update handed over); initial iterate: zero
//   phase R              U_g from the column dots and (G - I) c; the deferred
//                        n-space update; b; rhs1 = b + v-bar (rows of the CTA)
//   phase N1             x-bar = G^{-1} rhs1 (double-float GEMV), beta-bar,
//                        Step 1b prox (Newton, FP64), rhs2 = b + v
//   phase N2             x = G^{-1} rhs2, beta, c, Z~^T w; Step 2 xi and
//                        Step 3 alpha (n part); (G - I) c; n-space KKT sums
//   phase B  (Z pass)    deferred d-update of u, rho; t = Z~ c, ta = Z~ alpha;
//                        g = u - t / mu; d-space sums; (periodically) the
//                        column dots Z~^T u
//   phase S              all sums -> KKT residuals (Sec. 4.3), duality gap,
//                        sigma rule (Sec. 4.4), stop test; identical in every CTA
#include <algorithm>
#include <mutex>

#include "nspace.cuh"

namespace gdwd {

constexpr int kMaxStages = 8;

__global__ void prox_kernel(const double* a, const double* r0, const double* omega, double sigma, double q,
                            int64_t n, double* out) {
  const int qc = q_case(q);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double om = omega ? omega[i] : q;
    out[i] = prox_root(a[i], om / sigma, q, qc, r0 ? r0[i] : -1.0);
  }
}

cudaError_t launch_prox(const double* a, const double* r0, const double* omega, double sigma, double q,
                        int64_t n, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  prox_kernel<<<blocks, 256, 0, st>>>(a, r0, omega, sigma, q, n, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// pass-B row epilogue of the iteration: g = u - t / mu and the d-space sums
// ---------------------------------------------------------------------------
// eta_D3 needs ||kap g - a||^2 with kap = tau mu sigma (1 - theta), and eta_P2
// ||w - u+||^2 = ||(1 - theta) g + gs rho||^2, with theta = min(1, R / ||g||)
// known only after the pass.  Expanding them in sums of g, a and rho cancels
// catastrophically once the residuals are small, and the rounding then decides
// the sigma rule.  So the pass sums v = a - khat g and y = (1 - theta_prev) g +
// gs rho, with theta_prev the last iteration's theta and khat = tau mu sigma
// (1 - theta_prev); phase S expands both in the small theta_prev - theta (zero
// once theta settles).
struct IterEpi {
  const df* s_u;             // the CTA's slab rows of u, rho and g in shared memory (double-float)
  const df* s_rho;
  df* s_g;
  df inv_mu, a_coef;         // a = ta + a_coef * rho, a_coef = sqrt(mu)(1 - tau)
  df khat, omp, gs;          // v = a - khat g; y = omp g + gs rho, omp = 1 - theta_prev
  df sg2{0.f, 0.f}, syg{0.f, 0.f}, sy2{0.f, 0.f}, sv2{0.f, 0.f}, svg{0.f, 0.f}, sta2{0.f, 0.f};
  __device__ void row(int64_t, int m, df t, df ta) {
    const df gj = df_sum(s_u[m], df_neg(df_mul(t, inv_mu)));
    const df rj = s_rho[m];
    const df aj = df_sum(ta, df_mul(a_coef, rj));
    const df vj = df_sum(aj, df_neg(df_mul(khat, gj)));
    const df yj = df_sum(df_mul(omp, gj), df_mul(gs, rj));
    s_g[m] = gj;
    df_fma(sg2, gj, gj);
    df_fma(syg, yj, gj);
    df_fma(sy2, yj, yj);
    df_fma(sv2, vj, vj);
    df_fma(svg, vj, gj);
    df_fma(sta2, ta, ta);
  }
};

// sum over the NB slabs of one row's pass-A partials (lanes of a warp; df for FP32)
template <typename CT>
__device__ __forceinline__ double reduce_partials(const CT* pp, int NB, int lane) {
  if constexpr (sizeof(CT) == 8) {
    double acc = 0.0;
    for (int s2 = lane; s2 < NB; s2 += 32) acc += (double)pp[s2];
    return warp_sum(acc);
  } else {
    df acc{0.f, 0.f};
    for (int s2 = lane; s2 < NB; s2 += 32) df_add(acc, (float)pp[s2]);
    return df_to_double(df_warp_sum(acc));
  }
}

template <typename CT>
__device__ __forceinline__ void store_ct(CT* p, double v) { *p = (CT)v; }

// The CTA's n-space rows (at most kMaxRowsPerCta) live in shared memory for the
// whole launch: the iterate's row state and the per-row constants, one array
// of rpc doubles each, ahead of the phase-local region.  The row phases then
// touch global memory only for what other CTAs read.
enum RowSlot { RS_R, RS_XI, RS_AL, RS_B, RS_KC, RS_UU, RS_UR, RS_Y, RS_P, RS_CE, RS_E, RS_OM, RS_WT, RS_SC,
               RS_X1, RS_X2, RS_X3, RS_RES, RS_COUNT };

__host__ __device__ inline size_t row_state_bytes(int64_t rpc) {
  return ((size_t)RS_COUNT * (size_t)rpc * sizeof(double) + 127) & ~(size_t)127;
}

// The CTA's slab rows of u, rho, g (FP64) and of u in the compute type (the
// column dots' right-hand side) stay in shared memory for the whole launch, so
// the d-space update and the pass-B epilogue read no global memory; the global
// copies are written through.
__host__ __device__ inline size_t slab_state_bytes(int nslab_rows, int ct_size) {
  return ((size_t)nslab_rows * (3 * sizeof(double) + (size_t)ct_size) + 127) & ~(size_t)127;
}

// ---------------------------------------------------------------------------
// Step 1a of the next iteration without a solve of its own.  Its right-hand
// side rhs1 = b+ + xi - r - alpha / sigma' is linear in three n-vectors known at
// the end of phase N2,
//     V1 = U_g,  V2 = (1 - tau) U_rho / sqrt(mu) - alpha,  V3 = xi - r,
//     rhs1 = a1 V1 + V2 / sigma' + V3,  a1 = theta - tau (sigma / sigma') (1 - theta),
// whose coefficients wait only for phase S (theta, sigma').  When the sigma rule
// keeps sigma' = sigma (every iteration but a few) this is
//     rhs1 = a1 V1 + W,  W = V2 / sigma + V3,  a1 = theta - tau (1 - theta),
// so x-bar = G^{-1} rhs1 = a1 X1 + XW with X1 = G^{-1} V1, XW = G^{-1} W, and
// p^T rhs1 likewise.  The two products of this CTA's rows (and of the row p^T)
// are formed while phase S runs: the rows of G^{-1}, the row p^T, V1 and W (all
// double-float, ldP long) are copied into the idle ring during the wait at
// barrier 8, and warps 4-7 multiply them while warps 0-3 run phase S.  If sigma
// changes, phase R takes Step 1a the ordinary way (barrier, then one product).
// ---------------------------------------------------------------------------
constexpr int kFuseRowsPerWarp = 2;

struct FusedGemv {
  const float2* P;
  int ldP;
  const float2* pdf;
  const float2* vrhs;     // [2][ldP]: V1, W
  int64_t r0;
  int nrows;
  int W;                  // columns per extra chunk (even)
  int nx;                 // extra chunks: ceil(ldP / W)
  double* s_acc;          // shared, (nrows + 1) x 3 sums of the slices
  __device__ int count() const { return nx; }
  __device__ void issue(int e, uint8_t* dst, uint64_t* bar) const {
    // V1..V3 were written by other CTAs' generic stores before the grid barrier;
    // order them before this thread's bulk (async-proxy) reads
    asm volatile("fence.proxy.async;" ::: "memory");
    const int j0 = e * W;
    const int w = min(W, ldP - j0);
    const uint32_t bytes = (uint32_t)w * (uint32_t)sizeof(float2);
    mbar_expect_tx(bar, bytes * (uint32_t)(nrows + 3));
    const size_t slice = (size_t)W * sizeof(float2);
    for (int t = 0; t < nrows; ++t) bulk_g2s(dst + t * slice, P + (size_t)(r0 + t) * ldP + j0, bytes, bar);
    bulk_g2s(dst + nrows * slice, pdf + j0, bytes, bar);
    for (int k = 0; k < 2; ++k) bulk_g2s(dst + (nrows + 1 + k) * slice, vrhs + (size_t)k * ldP + j0, bytes, bar);
  }
  // the rows (and p^T, row nrows) on warps w0 .. w0 + nw - 1, one warp per row
  __device__ void consume(int e, const uint8_t* buf, int w0 = 0, int nw = kWarps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = min(W, ldP - e * W);
    const int npair = w / 2;
    const size_t slice = (size_t)W * sizeof(float2);
    const float4* V1 = reinterpret_cast<const float4*>(buf + (nrows + 1) * slice);
    const float4* V2 = reinterpret_cast<const float4*>(buf + (nrows + 2) * slice);
    // two rows per pass: each load of V1 and W serves both
    for (int t = warp - w0; t <= nrows; t += 2 * nw) {
      const int tb = t + nw;
      const bool two = tb <= nrows;
      const float4* Pa = reinterpret_cast<const float4*>(buf + t * slice);
      const float4* Pb = reinterpret_cast<const float4*>(buf + (two ? tb : t) * slice);
      df a1{0.f, 0.f}, a2{0.f, 0.f}, b1{0.f, 0.f}, b2{0.f, 0.f};
      df c1{0.f, 0.f}, c2{0.f, 0.f}, d1{0.f, 0.f}, d2{0.f, 0.f};
      for (int j = lane; j < npair; j += 32) {
        const float4 pa = Pa[j], pb = Pb[j], x1 = V1[j], x2 = V2[j];
        const df x1a{x1.x, x1.y}, x1b{x1.z, x1.w}, x2a{x2.x, x2.y}, x2b{x2.z, x2.w};
        df_fma(a1, df{pa.x, pa.y}, x1a);
        df_fma(a2, df{pa.x, pa.y}, x2a);
        df_fma(b1, df{pa.z, pa.w}, x1b);
        df_fma(b2, df{pa.z, pa.w}, x2b);
        df_fma(c1, df{pb.x, pb.y}, x1a);
        df_fma(c2, df{pb.x, pb.y}, x2a);
        df_fma(d1, df{pb.z, pb.w}, x1b);
        df_fma(d2, df{pb.z, pb.w}, x2b);
      }
      df_add(a1, b1);
      df_add(a2, b2);
      df_add(c1, d1);
      df_add(c2, d2);
      a1 = df_warp_sum(a1);
      a2 = df_warp_sum(a2);
      c1 = df_warp_sum(c1);
      c2 = df_warp_sum(c2);
      if (lane == 0) {
        const double v[4] = {df_to_double(a1), df_to_double(a2), df_to_double(c1), df_to_double(c2)};
        for (int r = 0; r < (two ? 2 : 1); ++r) {
          double* acc = s_acc + (r ? tb : t) * 2;
          if (e == 0) {
            acc[0] = v[2 * r];
            acc[1] = v[2 * r + 1];
          } else {
            acc[0] += v[2 * r];
            acc[1] += v[2 * r + 1];
          }
        }
      }
    }
  }
};

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) iterate_kernel(IterArgs<typename ElemTraits<T>::compute_t> a,
                                                              int stages, int stage_bytes) {
  using CT = typename ElemTraits<T>::compute_t;
  constexpr int VEC = ElemTraits<T>::kVec;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t s_bars[kMaxStages];
  __shared__ int s_flag, s_abort;
  __shared__ double s_tot[S_COUNT];
  __shared__ double s_ctl[15];
  __shared__ double s_pd[4];     // pobj, dobj, theta, ||w||
  __shared__ float s_etaf[11];   // gap, the nine residuals, kkt
  __shared__ int s_ictl[2];      // done, status

  const Layout& L = a.L;
  const int cta = blockIdx.x, grid = a.grid;
  const int64_t n = L.n, d = L.d;
  const int TB = L.TB, NB = L.NB;
  const int Q = TB / VEC;
  const int H = kThreads / L.CW;
  const int G = Q <= kThreads ? kThreads / Q : 1;
  const int nmy = (NB > cta) ? (NB - cta + grid - 1) / grid : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // contiguous block of G^{-1} rows (and n-space entries) owned by this CTA
  const int64_t rpc = (n + grid - 1) / grid;
  const int64_t r0 = ((int64_t)cta * rpc < n) ? (int64_t)cta * rpc : n;
  const int nrows = (int)(((r0 + rpc < n) ? r0 + rpc : n) - r0);
  __shared__ float s_xh[kMaxRowsPerCta + 1], s_xl[kMaxRowsPerCta + 1];   // + the p^T rhs row
  __shared__ double s_ug[kMaxRowsPerCta];                                 // Z~^T u from the column dots
  __shared__ float2 s_rb[kMaxRowsPerCta];                                 // rhs2 of the CTA's rows
  __shared__ double s_gx[kFuseRowsPerWarp * kWarps * 2];                  // fused products: rows, then p^T
  // the iteration's double-float constants theta, -tau sigma_prev sqrt(mu)
  // (1 - theta), khat = tau mu sigma (1 - theta), 1 - theta and gs = 1 / (sigma
  // sqrt(mu)), formed once per CTA by five lanes during the wait at barrier 4
  // (a warp-level FP64 instruction occupies the SM's FP64 unit ~19 cycles, so
  // the same products formed by every warp cost about a microsecond)
  __shared__ df s_itdf[5];
  const int qcase = q_case(a.q);
  const double sqmu = sqrt(a.mu), inv_mu = 1.0 / a.mu, inv_sqmu = 1.0 / sqmu;
  const df inv_mu_df = df_from(inv_mu), acoef_df = df_from(sqmu * (1.0 - a.tau)), omtau = df_from(1.0 - a.tau);
  const double den = 1.0 + a.C;
  const double inv_q = 1.0 / a.q;
  const float inv_den = (float)(1.0 / den);
  const double sqrt_tol = sqrt(a.tol);
  const SPhaseArgs sq{a.C, a.kappa, a.R, a.mu, a.tau, sqmu, a.tol, sqrt_tol, inv_den, a.stop_rule, float_at_most(a.tol)};

  Ring rg;
  rg.buf = smem;
  rg.bars = s_bars;
  rg.stages = stages;
  rg.stage_bytes = stage_bytes;
  double* rs = reinterpret_cast<double*>(smem + (size_t)stages * stage_bytes);   // row state
  const int rld = (int)rpc;
#define RS(slot, t) rs[(slot) * rld + (t)]
  const int nslab_max = (NB + grid - 1) / grid * TB;                              // slab rows, any CTA
  uint8_t* sst = smem + (size_t)stages * stage_bytes + row_state_bytes(rpc);      // slab state
  df* s_u = reinterpret_cast<df*>(sst);
  df* s_rho = s_u + nslab_max;
  df* s_g = s_rho + nslab_max;
  CT* s_up = reinterpret_cast<CT*>(s_g + nslab_max);
  uint8_t* uni = sst + slab_state_bytes(nslab_max, (int)sizeof(CT));              // phase-local region
  if (threadIdx.x == 0) s_abort = 0;
  ring_init(rg);
  // the fused first solve needs every row of the CTA (and p^T) on at most
  // kFuseRowsPerWarp rows per warp, and the ring's stages to hold slices of all
  // of them and of the three right-hand sides at once (their copies are issued
  // when pass B ends and land during barrier 8 and phase S)
  const int fuse_w = (int)((size_t)stage_bytes / ((size_t)(rpc + 3) * sizeof(float2))) & ~1;
  const int fuse_nx = fuse_w >= 16 ? (a.ldP + fuse_w - 1) / fuse_w : 0;
  const bool can_fuse =
      a.fuse && a.vrhs && rpc + 1 <= kFuseRowsPerWarp * (kWarps / 2) && fuse_w >= 16 && fuse_nx <= stages;
  FusedGemv fx{a.P, a.ldP, a.pdf, a.vrhs, r0, nrows, fuse_w, can_fuse ? fuse_nx : 0, s_gx};

  unsigned gen = 0;
  // per-phase timing by CTA 0, thread 0 (globaltimer, a few instructions per phase)
  __shared__ unsigned long long s_tacc[kPhaseSlots], s_tprev;
  const bool timing = (cta == 0 && threadIdx.x == 0);
  if (timing) {
    for (int k = 0; k < kPhaseSlots; ++k) s_tacc[k] = 0;
    s_tprev = globaltimer();
  }
  double sig = a.ctrl->sigma, sig_prev = a.ctrl->sigma_prev, theta = a.ctrl->theta;
  int pending = a.ctrl->pending;
  int it0 = a.ctrl->it;
  int status = GDWD_EMAXITER;
  double beta = 0.0;

#define GDWD_MARK(k)                       \
  do {                                     \
    if (timing) {                          \
      const uint64_t t_ = globaltimer();   \
      s_tacc[k] += t_ - s_tprev;           \
      s_tprev = t_;                        \
    }                                      \
  } while (0)
#define GDWD_BARRIER_SIDE(k, ...)                                                                    \
  do {                                                                                               \
    GDWD_MARK(k);                                                                                    \
    if (!grid_barrier_side(a.bar, (unsigned)grid, gen, a.err, a.timeout_ns, &s_flag,                 \
                           (a.stall_first_barrier && gen == 0) ? 1u : 0u, __VA_ARGS__)) {            \
      ring_drain_prefetched(rg, a.err, a.timeout_ns);                                                \
      return;                                                                                        \
    }                                                                                                \
    GDWD_MARK(k + 1);                                                                                \
  } while (0)
#define GDWD_BARRIER(k)                                                                              \
  do {                                                                                               \
    GDWD_MARK(k);                                                                                    \
    if (!grid_barrier(a.bar, (unsigned)grid, gen, a.err, a.timeout_ns, &s_flag,                      \
                      (a.stall_first_barrier && gen == 0) ? 1u : 0u)) {                              \
      ring_drain_prefetched(rg, a.err, a.timeout_ns);                                                \
      return;                                                                                        \
    }                                                                                                \
    GDWD_MARK(k + 1);                                                                                \
  } while (0)

  const int npair = (int)((n + 1) / 2);

  // ---------------- prologue: U_u = Z~^T u and U_rho = Z~^T rho of the starting
  // iterate for this CTA's rows.  A warm start computes them with two passes over
  // Z (after the deferred (u, rho) update it hands over); the initial iterate has
  // u = rho = 0.
  if (a.refresh) {
    const double rcoef0 = a.tau * sig_prev * sqmu * (1.0 - theta);
    for (int v = 0; v < 2; ++v) {
      CT* gp = reinterpret_cast<CT*>(uni);
      for (int k = 0; k < nmy; ++k) {
        const int64_t s = cta + (int64_t)k * grid;
        for (int j = threadIdx.x; j < TB; j += kThreads) {
          const int64_t gj = s * TB + j;
          double val = 0.0;
          if (gj < d) {
            if (v == 0 && pending) {
              const double g = a.g[gj];
              a.rho[gj] = (1.0 - a.tau) * a.rho[gj] - rcoef0 * g;
              a.u[gj] = theta * g;
            }
            val = v == 0 ? a.u[gj] : a.rho[gj];
          }
          gp[(size_t)k * TB + j] = (CT)val;
        }
      }
      __syncthreads();
      PassA<T> pa{gp, a.partial, TB, NB, Q, H};
      if (!stream_slabs<T>(L, rg, cta, grid, a.err, a.timeout_ns, &s_abort, pa)) return;
      GDWD_BARRIER(0);
      for (int t = warp; t < nrows; t += kWarps) {
        const int64_t i = r0 + t;
        const double bsum = reduce_partials<CT>(a.partial + (size_t)i * NB, NB, lane);
        if (lane == 0) (v == 0 ? a.Uu : a.Ur)[i] = a.sc[i] * bsum;
      }
      GDWD_BARRIER(0);   // the partials are rewritten by the next pass
    }
    pending = 0;
  } else {
    for (int t = threadIdx.x; t < nrows; t += kThreads) {
      a.Uu[r0 + t] = 0.0;
      a.Ur[r0 + t] = 0.0;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nrows; t += kThreads) {
    const int64_t i = r0 + t;
    RS(RS_R, t) = a.r[i];
    RS(RS_XI, t) = a.xi[i];
    RS(RS_AL, t) = a.alpha[i];
    RS(RS_B, t) = a.b[i];
    RS(RS_KC, t) = a.kc[i];
    RS(RS_UU, t) = a.Uu[i];
    RS(RS_UR, t) = a.Ur[i];
    RS(RS_Y, t) = a.y[i];
    RS(RS_P, t) = a.p[i];
    RS(RS_CE, t) = a.C * a.e[i];
    RS(RS_E, t) = a.e[i];
    RS(RS_OM, t) = a.omega[i];
    RS(RS_WT, t) = a.wt[i];
    RS(RS_SC, t) = a.sc[i];
  }
  for (int m = threadIdx.x; m < nmy * TB; m += kThreads) {
    const int k = m / TB, j = m - k * TB;
    const int64_t gj = (cta + (int64_t)k * grid) * TB + j;
    const bool in = gj < d;
    s_u[m] = df_from(in ? a.u[gj] : 0.0);
    s_rho[m] = df_from(in ? a.rho[gj] : 0.0);
    s_g[m] = df_from(in ? a.g[gj] : 0.0);
  }
  __syncthreads();

  int it = it0;
  bool dots_prev = false;   // the last pass B took the column dots Z~^T u
  bool fused = false;       // the last phase S formed the two products of the fused first solve
  double inv_sig = rcp_nr(sig);   // from the last phase S after the first iteration
  for (; it < a.max_iter; ++it) {
    const double gs_it = inv_sig * inv_sqmu;   // 1 / (sigma sqrt(mu)) of this iteration
    // this iteration's pass B takes the column dots Z~^T u every dots_every-th
    // iteration; otherwise it makes the products of the next fused first solve
    const bool dots_now = ((it - it0) % a.dots_every) == a.dots_every - 1;
    const bool fuse_next = can_fuse && !dots_now;
    bool use_fused = false;
    // ---------------- phase R (this CTA's rows): U_g = Z~^T g of the last iteration
    // from the pass-B column dots Z~^T u and (G - I) c; the deferred update
    // U_u = theta U_g, U_rho <- (1 - tau) U_rho - tau sigma' sqrt(mu) (1 - theta) U_g;
    // b = U_u + U_rho / (sigma sqrt(mu)); rhs1 = b + xi - r - alpha / sigma
    ring_prefetch(L, rg, cta, grid);   // this iteration's first Z chunks arrive during R, N1, N2
    double betabar;
    double xb_reg = 0.0;   // fused x-bar of this thread's row (at most one row per thread)
    {
      if (pending && dots_prev) {
        // the column dots Z~^T u of the last pass: one warp per row sums its slabs
        for (int t = warp; t < nrows; t += kWarps) {
          const double ug = RS(RS_SC, t) * reduce_partials<CT>(a.partial + (size_t)(r0 + t) * NB, NB, lane);
          if (lane == 0) s_ug[t] = ug;
        }
        __syncthreads();
      }
      // fused (sigma kept): x-bar = a1 X1 + XW from the last phase S's products,
      // a1 = theta - tau (1 - theta)
      use_fused = fused && sig == sig_prev;
      const double a1 = use_fused ? theta - a.tau * (1.0 - theta) : 0.0;
      if (use_fused) betabar = -(a1 * s_gx[nrows * 2] + s_gx[nrows * 2 + 1]) * a.inv_s;
      // the per-row work on consecutive threads (few warp instructions of FP64)
      for (int t = threadIdx.x; t < nrows; t += kThreads) {
        const int64_t i = r0 + t;
        double uu = RS(RS_UU, t), ur = RS(RS_UR, t);
        if (pending) {
          const double rcoef = a.tau * sig_prev * sqmu * (1.0 - theta);
          const double ug = (dots_prev ? s_ug[t] : uu) - RS(RS_KC, t);
          uu = theta * ug;
          ur = (1.0 - a.tau) * ur - rcoef * ug;
          RS(RS_UU, t) = uu;
          RS(RS_UR, t) = ur;
        }
        const double bi = uu + ur * gs_it;
        RS(RS_B, t) = bi;
        if (use_fused) {
          xb_reg = a1 * s_gx[t * 2] + s_gx[t * 2 + 1];
        } else {
          const double v = RS(RS_XI, t) - RS(RS_R, t) - RS(RS_AL, t) * inv_sig;
          const df r1 = df_from(bi + v);
          a.rhsA[i] = make_float2(r1.hi, r1.lo);
        }
      }
    }
    if (!use_fused) {
      GDWD_BARRIER(2);
      // ---------------- phase N1 (first solve): x-bar = G^{-1} rhs1, beta-bar
      GDWD_MARK(14);
      // G^{-1} rows of this CTA and, as one more row, p^T rhs1 for beta-bar (one
      // warp per row; rhs1 is read from L2, and from L1 after the SM's first warp)
      for (int t = warp; t <= nrows; t += kWarps) {
        const df x = row_dot(t < nrows ? a.P + (size_t)(r0 + t) * a.ldP : a.pdf, a.rhsA, npair);
        if (lane == 0) {
          s_xh[t] = x.hi;
          s_xl[t] = x.lo;
        }
      }
      __syncthreads();
      betabar = -((double)s_xh[nrows] + (double)s_xl[nrows]) * a.inv_s;
      GDWD_MARK(15);
    }
    // ---------------- phase N1 (rows): Step 1b prox, rhs2.  The per-row FP64 work
    // has one row per lane so each FP64 instruction serves up to 32 rows
    {
      if (use_fused) GDWD_MARK(2);
      for (int t = threadIdx.x; t < nrows; t += kThreads) {
        const int64_t i = r0 + t;
        const double xb = use_fused ? xb_reg : (double)s_xh[t] + (double)s_xl[t];
        const double cbar = xb + betabar * RS(RS_P, t);
        const double ri = RS(RS_R, t);
        const double rn = prox_root(cbar + ri, RS(RS_OM, t) * inv_sig, a.q, qcase, ri);
        GDWD_MARK(18);
        RS(RS_R, t) = rn;
        const double v = RS(RS_XI, t) - rn - RS(RS_AL, t) * inv_sig;
        const df r2 = df_from(RS(RS_B, t) + v);
        a.rhsB[i] = make_float2(r2.hi, r2.lo);
        s_rb[t] = make_float2(r2.hi, r2.lo);
      }
    }
    // the deferred d-space update of the last iteration's Steps 2-3 on this CTA's
    // slab rows, u+ = theta g, rho+ = (1 - tau) rho - tau sigma' sqrt(mu)
    // (1 - theta) g, made by warps 1.. while thread 0 waits at the barrier; the
    // pass over Z reads it from shared memory (u also in the compute type, for
    // the column dots)
    GDWD_BARRIER_SIDE(4, [&]() {
      // double-float on the FP32 pipes: each warp-level FP64 instruction occupies
      // the SM's FP64 unit for ~19 cycles, whatever the number of active lanes
      if (warp == 1 && lane < 5) {
        const double omt = 1.0 - theta;
        const double v = lane == 0 ? theta
                       : lane == 1 ? -a.tau * sig_prev * sqmu * omt
                       : lane == 2 ? a.tau * a.mu * sig * omt
                       : lane == 3 ? omt
                                   : gs_it;
        s_itdf[lane] = df_from(v);
      }
      asm volatile("bar.sync 1, %0;" ::"r"(kThreads - 32) : "memory");   // the side warps only
      const df th = s_itdf[0], mrc = s_itdf[1];
      for (int m = threadIdx.x - 32; m < nmy * TB; m += kThreads - 32) {
        const int k = m / TB, j = m - k * TB;
        const int64_t gj = (cta + (int64_t)k * grid) * TB + j;
        df uj = s_u[m];
        if (pending && gj < d) {
          const df g = s_g[m];
          s_rho[m] = df_sum(df_mul(omtau, s_rho[m]), df_mul(mrc, g));   // rho <- rho - tau sigma D (w - u+)
          uj = df_mul(th, g);                                            // u+ = Pi_B(g)
          s_u[m] = uj;
        }
        s_up[m] = (CT)((double)uj.hi + (double)uj.lo);
      }
    });

    // ---------------- phase N2: x, beta, c, Z~^T w; Step 2 (xi), Step 3 (alpha);
    // (G - I) c = rhs2 - x + beta (y - p) for the next U_g
    {
      GDWD_MARK(11);
      for (int t = warp; t <= nrows; t += kWarps) {
        const df x = row_dot(t < nrows ? a.P + (size_t)(r0 + t) * a.ldP : a.pdf, a.rhsB, npair);
        if (lane == 0) {
          s_xh[t] = x.hi;
          s_xl[t] = x.lo;
        }
      }
      __syncthreads();
      beta = -((double)s_xh[nrows] + (double)s_xl[nrows]) * a.inv_s;
      GDWD_MARK(12);
      for (int t = threadIdx.x; t < nrows; t += kThreads) {
        const int64_t i = r0 + t;
        {
          const double xv = (double)s_xh[t] + (double)s_xl[t];
          const double pi = RS(RS_P, t);
          const double c = xv + beta * pi;
          const double ri = RS(RS_R, t), al = RS(RS_AL, t), yi = RS(RS_Y, t), ce = RS(RS_CE, t);
          const double v = RS(RS_XI, t) - ri - al * inv_sig;
          const double zw = c - v - yi * beta;                                     // Z~^T w
          const double xin = dmax0(ri - zw - yi * beta + (al - ce) * inv_sig);  // Step 2
          const double res = zw + yi * beta + xin - ri;
          const double an = al - a.tau * sig * res;                                // Step 3
          RS(RS_XI, t) = xin;
          RS(RS_AL, t) = an;
          const double sci = RS(RS_SC, t);
          store_ct(a.cq + i, sci * c);
          store_ct(a.aq + i, sci * an);
          const float2 rb = s_rb[t];
          const double rh2 = (double)rb.x + (double)rb.y;
          const double kcn = rh2 - xv + beta * (yi - pi);
          RS(RS_KC, t) = kcn;
          if (fuse_next) {
            // right-hand sides of the next fused first solve: V1 = U_g and
            // W = ((1 - tau) U_rho / sqrt(mu) - alpha) / sigma + xi - r
            const df v1 = df_from(RS(RS_UU, t) - kcn);
            const df w = df_from(((1.0 - a.tau) * inv_sqmu * RS(RS_UR, t) - an) * inv_sig + (xin - ri));
            a.vrhs[i] = make_float2(v1.hi, v1.lo);
            a.vrhs[a.ldP + i] = make_float2(w.hi, w.lo);
          }
          RS(RS_RES, t) = res;
        }
      }
    }
    // the n-space KKT sums (read only by phase S, after the pass over Z) are
    // formed by warp 1 while thread 0 waits at the barrier: one lane per row
    // computes the row's nine terms, then lane k adds term k over the rows
    // through shared memory.  The objectives and y^T alpha (which cancels) are
    // summed in FP64; the terms that only feed a residual in FP32.
    GDWD_BARRIER_SIDE(6, [&]() {
      if (warp != 1) return;
      double* kt = reinterpret_cast<double*>(uni);         // [9][32] terms, then the 9 sums (free until phase B)
      for (int t0 = 0; t0 < nrows; t0 += 32) {
        const int t = t0 + lane;
        double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (t < nrows) {
          const double ri = RS(RS_R, t), an = RS(RS_AL, t), xin = RS(RS_XI, t), res = RS(RS_RES, t);
          const double yi = RS(RS_Y, t), ce = RS(RS_CE, t), om = RS(RS_OM, t);
          const double irq1 = rcp_nr(pow_q1(ri, a.q, qcase));
          const double cma = ce - an;                       // C e_i - alpha_i
          const float resf = (float)res, dvf = (float)(an - om * irq1), cmaf = (float)cma;
          const float mn = fminf((float)an, 0.f), mx = fminf(cmaf, 0.f);   // min(alpha, 0), -max(alpha - Ce, 0)
          v[0] = (double)(resf * resf);
          v[1] = yi * an;
          v[2] = (double)((float)xin * cmaf);
          v[3] = (double)(dvf * dvf);
          v[4] = (double)(mn * mn);
          v[5] = (double)(mx * mx);
          v[6] = om * inv_q * ri * irq1;                    // wt^q r^-q
          v[7] = RS(RS_E, t) * xin;
          v[8] = dual_pow(RS(RS_WT, t) * an, a.q, qcase);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) kt[k * 32 + lane] = v[k];
        __syncwarp();
        if (lane < 9) {
          const int nr = min(32, nrows - t0);
          double acc = t0 == 0 ? 0.0 : kt[9 * 32 + lane];
          for (int u = 0; u < nr; ++u) acc += kt[lane * 32 + u];
          kt[9 * 32 + lane] = acc;
        }
        __syncwarp();
      }
      if (lane < 9) {   // as a double-float pair (summed on the FP32 pipes in phase S)
        const df p = df_from(nrows > 0 ? kt[9 * 32 + lane] : 0.0);
        reinterpret_cast<float2*>(a.scal)[(size_t)lane * grid + cta] = make_float2(p.hi, p.lo);
      }
    });


    // ---------------- phase B (the one pass over Z): deferred (u, rho) update;
    // t = Z~ c, ta = Z~ alpha, g = u - t / mu and the d-space sums; on the same
    // chunks the column dots of Z~^T u (for the next U_g)
    {
      // c and alpha (scaled, compute type) in 16-byte pieces: both vectors are
      // padded to a multiple of 16 bytes in global and shared memory
      const int64_t nv = (n * (int64_t)sizeof(CT) + 15) / 16;
      CT* cv = reinterpret_cast<CT*>(uni);
      CT* av = reinterpret_cast<CT*>(uni + nv * 16);
      const size_t off_red = (size_t)nv * 32;
      double* red = reinterpret_cast<double*>(uni + off_red);
      for (int64_t k = threadIdx.x; k < nv; k += kThreads) {
        reinterpret_cast<uint4*>(cv)[k] = reinterpret_cast<const uint4*>(a.cq)[k];
        reinterpret_cast<uint4*>(av)[k] = reinterpret_cast<const uint4*>(a.aq)[k];
      }
      __syncthreads();
      GDWD_MARK(16);
      IterEpi epi{s_u, s_rho, s_g, inv_mu_df, acoef_df, s_itdf[2], s_itdf[3], s_itdf[4]};
      PassB<T, IterEpi> pb;
      pb.cv = cv;
      pb.av = av;
      pb.red = red;
      pb.TB = TB;
      pb.Q = Q;
      pb.G = G;
      pb.d = d;
      pb.two = true;
      pb.epi = &epi;
      for (int kk = 0; kk < VEC; ++kk) {
        pb.rc[kk].reset();
        pb.ra[kk].reset();
      }
      // the column dots Z~^T u run on every dots_every-th iteration; in between
      // U_u follows its recurrence
      dots_prev = dots_now;
      if (dots_prev) {
        PassA2<T> pa{s_up, a.partial, TB, NB, Q};
        PassBA<T, IterEpi> pba{&pb, &pa};
        if (!stream_slabs<T>(L, rg, cta, grid, a.err, a.timeout_ns, &s_abort, pba)) return;
      } else {
        if (!stream_slabs<T>(L, rg, cta, grid, a.err, a.timeout_ns, &s_abort, pb)) return;
      }
      fused = fuse_next;
      GDWD_MARK(17);
      // the six d-space sums of every thread, one warp per sum, through the
      // phase-local region (free once the pass is over)
      const df vals[6] = {epi.sg2, epi.syg, epi.sy2, epi.sv2, epi.svg, epi.sta2};
      __syncthreads();
      rows_sum_df<6>(vals, reinterpret_cast<float2*>(uni), TB,
                     reinterpret_cast<float2*>(a.scal) + (size_t)S_G2 * grid + cta, grid);
    }
    // the operands of the next first solve's two G^-1 products (this CTA's rows
    // of G^-1, p^T and the right-hand sides N2 wrote before barrier 6) go into the
    // idle ring during the wait at barrier 8 and land while phase S runs
    if (fused) rg.prefetched = fx.nx;   // drained by an early exit
    GDWD_BARRIER_SIDE(8, [&]() {
      if (fused && threadIdx.x == kThreads - 32)
        for (int e = 0; e < fx.nx; ++e) fx.issue(e, rg.buf + (size_t)e * rg.stage_bytes, &rg.bars[e]);
    });

    // ---------------- phase S: totals, KKT, sigma rule, stop test (same in every CTA)
    grid_totals_df(reinterpret_cast<const float2*>(a.scal), grid, s_tot);
    __syncthreads();
    GDWD_MARK(13);
    if (fused) {
      // warps 0-3 run phase S while warps 4-7 form the two products of the next
      // iteration's x-bar (phase R) from the ring
      if (warp < kWarps / 2) {
        s_phase(s_tot, sq, sig, gs_it, it, beta, status, false, a.ctrl, s_pd, s_etaf, s_ctl, s_ictl, theta, true,
                kThreads / 2);
      } else {
        for (int e = 0; e < fx.nx; ++e) {
          if (!mbar_wait(&rg.bars[e], (rg.phase >> e) & 1u, a.err, a.timeout_ns)) s_abort = 1;
          fx.consume(e, rg.buf + (size_t)e * rg.stage_bytes, kWarps / 2, kWarps / 2);
        }
      }
      for (int e = 0; e < fx.nx; ++e) rg.phase ^= 1u << e;
      __syncthreads();
      if (*(volatile int*)&s_abort) {
        ring_drain(rg, 0, fx.nx, true, a.err, a.timeout_ns);
        return;
      }
      rg.prefetched = 0;
    } else {
      s_phase(s_tot, sq, sig, gs_it, it, beta, status, false, a.ctrl, s_pd, s_etaf, s_ctl, s_ictl, theta, true);
    }
    GDWD_MARK(10);
    sig_prev = sig;
    theta = s_ctl[0];
    sig = s_ctl[1];
    inv_sig = s_ctl[2];
    pending = 1;
    const bool done = s_ictl[0] != 0;
    status = s_ictl[1];
    if (done) {
      ++it;
      break;
    }
  }
  if (it >= a.max_iter && status != GDWD_OK) status = GDWD_EMAXITER;
  // the slab rows of u, rho and g back to global memory (the host forms w from
  // g and rho; a later launch starts from them)
  for (int m = threadIdx.x; m < nmy * TB; m += kThreads) {
    const int k = m / TB, j = m - k * TB;
    const int64_t gj = (cta + (int64_t)k * grid) * TB + j;
    if (gj < d) {
      a.u[gj] = df_to_double(s_u[m]);
      a.rho[gj] = df_to_double(s_rho[m]);
      a.g[gj] = df_to_double(s_g[m]);
    }
  }
  // the rows back to global memory (the host reads alpha; a later launch starts
  // from r, xi, alpha, U_u, U_rho and (G - I) c)
  for (int t = threadIdx.x; t < nrows; t += kThreads) {
    const int64_t i = r0 + t;
    a.r[i] = RS(RS_R, t);
    a.xi[i] = RS(RS_XI, t);
    a.alpha[i] = RS(RS_AL, t);
    a.b[i] = RS(RS_B, t);
    a.kc[i] = RS(RS_KC, t);
    a.Uu[i] = RS(RS_UU, t);
    a.Ur[i] = RS(RS_UR, t);
  }
  if (cta == 0 && threadIdx.x == 0) {
    Ctrl* c = a.ctrl;
    if (it > it0) s_report(c, beta, s_pd, s_etaf);   // the residuals of the last iteration
    c->sigma = sig;
    c->sigma_prev = sig_prev;
    c->theta = theta;
    c->pending = pending;
    c->it = it;
    c->status = status;
    c->done = 1;
    for (int k = 0; k < kPhaseSlots; ++k) c->phase_ns[k] = (double)s_tacc[k];
  }
#undef GDWD_BARRIER
#undef GDWD_BARRIER_SIDE
#undef GDWD_MARK
#undef RS
}

// Phase-local region of the streaming passes (pass A's vector, pass B's
// coefficients and row partials); the stand-alone product kernels need only this.
template <typename T>
static size_t pass_bytes(const Layout& L, int grid) {
  using CT = typename ElemTraits<T>::compute_t;
  constexpr int VEC = ElemTraits<T>::kVec;
  const int nmy = (L.NB + grid - 1) / grid;
  const int Q = L.TB / VEC;
  const int G = Q <= kThreads ? kThreads / Q : 1;
  const size_t a_bytes = (size_t)nmy * L.TB * sizeof(CT);
  const size_t b_bytes = (size_t)(L.n * sizeof(CT) + 15) / 16 * 32 + (size_t)2 * G * L.TB * sizeof(double) +
                         (size_t)nmy * L.TB * sizeof(CT);
  return ((a_bytes > b_bytes ? a_bytes : b_bytes) + 127) & ~(size_t)127;
}

// Phase-local region of the iteration kernel plus the resident row state ahead of it.
template <typename T>
static size_t union_bytes(const Layout& L, int grid) {
  size_t r_bytes = (size_t)10 * 32 * sizeof(double);                               // N2 KKT terms
  if (r_bytes < (size_t)6 * kThreads * sizeof(double)) r_bytes = (size_t)6 * kThreads * sizeof(double);   // B sums
  size_t u = pass_bytes<T>(L, grid);
  if (r_bytes > u) u = r_bytes;
  using CT = typename ElemTraits<T>::compute_t;
  const int nslab_rows = (L.NB + grid - 1) / grid * L.TB;
  return ((u + 127) & ~(size_t)127) + row_state_bytes((L.n + grid - 1) / grid) +
         slab_state_bytes(nslab_rows, (int)sizeof(CT));
}


// Raises a kernel's dynamic shared-memory limit to the device maximum once per
// process.  (Setting it per launch to the launch's own size races when several
// host threads launch the same kernel with different sizes.)
template <auto Kern>
static cudaError_t ensure_max_dyn_smem() {
  static std::once_flag once;
  static cudaError_t status = cudaSuccess;
  std::call_once(once, [] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    status = cudaFuncGetAttributes(&fa, Kern);
    if (status == cudaSuccess)
      status = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  });
  return status;
}

template <typename T>
static cudaError_t launch_iterate_t(const IterArgs<typename ElemTraits<T>::compute_t>& args, int stages,
                                    int stage_bytes, size_t smem, cudaStream_t st) {
  auto kern = iterate_kernel<T>;
  cudaError_t e = ensure_max_dyn_smem<iterate_kernel<T>>();
  if (e != cudaSuccess) return e;
  void* params[] = {(void*)&args, (void*)&stages, (void*)&stage_bytes};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(args.grid), dim3(kThreads), params, smem, st);
}

// Columns per streamed chunk, at least two stages next to the phase-local
// buffers.  Every chunk costs a fixed ~0.5 us of waits and barriers on top of its
// bytes, so chunks are large: about 96 KB (two or three stages) when the stored Z
// fits in L2 and the pass is served from there, about 64 KB (three or more stages,
// more copies in flight) when it streams from HBM (measured on the spiked FP32
// workload at d = 20000 and 40000).
// The dynamic shared memory the iteration kernel may plan with.  The host's
// limit leaves 8 KB below the per-block maximum for static shared memory; the
// kernel's own static size (queried once) is taken if it is larger.
template <typename T>
static int iter_smem_limit(int smem_limit) {
  static int stat = -1;
  if (stat < 0) {
    cudaFuncAttributes fa;
    stat = cudaFuncGetAttributes(&fa, iterate_kernel<T>) == cudaSuccess ? (int)fa.sharedSizeBytes : 16384;
  }
  return std::min(smem_limit, smem_limit + 8192 - stat - 256);
}

template <typename T>
static int choose_cw_t(const Layout& L, int grid, int smem_limit) {
  smem_limit = iter_smem_limit<T>(smem_limit);
  const int64_t ub = (int64_t)union_bytes<T>(L, grid);
  const int64_t col_bytes = (int64_t)L.TB * L.esize;
  const int64_t avail = (int64_t)smem_limit - ub - 1024;
  const int64_t z_bytes = (int64_t)L.NB * L.TB * L.n * L.esize;
  const int64_t target = z_bytes <= (96ll << 20) ? 98304 : 65536;
  int64_t cw = std::min<int64_t>(target / col_bytes, (avail / 2 - 128) / col_bytes);
  cw = std::max<int64_t>(cw, 1);
  cw = std::min<int64_t>(cw, L.n);
  return (int)cw;
}

// Chunk columns for the stand-alone product kernels alone (no iteration kernel).
template <typename T>
static int choose_cw_apply(const Layout& L, int grid, int smem_limit) {
  const int64_t col_bytes = (int64_t)L.TB * L.esize;
  const int64_t avail = (int64_t)smem_limit - (int64_t)pass_bytes<T>(L, grid) - 1024;
  int64_t cw = std::min<int64_t>(65536 / col_bytes, (avail / 2 - 128) / col_bytes);
  cw = std::max<int64_t>(cw, 1);
  return (int)std::min<int64_t>(cw, L.n);
}

int choose_chunk_cols(int store, const Layout& L, int grid, int smem_limit, bool wide) {
  if (wide && store == GDWD_F32) return choose_cw_apply<f32w>(L, grid, smem_limit);
  switch (store) {
    case GDWD_F64: return choose_cw_t<double>(L, grid, smem_limit);
    case GDWD_BF16: return choose_cw_t<__nv_bfloat16>(L, grid, smem_limit);
    case GDWD_F16: return choose_cw_t<__half>(L, grid, smem_limit);
    case GDWD_E4M3: return choose_cw_t<__nv_fp8_e4m3>(L, grid, smem_limit);
    default: return choose_cw_t<float>(L, grid, smem_limit);
  }
}

// Plans the ring (stage size, stage count) for the available shared memory next
// to the iteration kernel's phase-local region (apply = false) or the product
// kernels' smaller one (apply = true).
template <typename T>
static bool plan_ring(const Layout& L, int grid, int smem_limit, int& stages, int& stage_bytes, size_t& smem,
                      bool apply = false) {
  const size_t ub = apply ? pass_bytes<T>(L, grid) : union_bytes<T>(L, grid);
  stage_bytes = (int)(((size_t)L.CW * L.TB * L.esize + 127) & ~(size_t)127);
  const int64_t avail = (int64_t)smem_limit - (int64_t)ub - 1024;
  if (avail < 2 * (int64_t)stage_bytes) return false;
  stages = (int)std::min<int64_t>(kMaxStages, avail / stage_bytes);
  smem = (size_t)stages * stage_bytes + ub;
  return true;
}

cudaError_t run_iterate_f64(const IterArgs<double>& a, int smem_limit, cudaStream_t st) {
  int stages, sb;
  size_t smem;
  smem_limit = iter_smem_limit<double>(smem_limit);
  if (!plan_ring<double>(a.L, a.grid, smem_limit, stages, sb, smem)) return cudaErrorInvalidConfiguration;
  return launch_iterate_t<double>(a, stages, sb, smem, st);
}

template <typename T>
static cudaError_t run_iterate_ft(const IterArgs<float>& a, int smem_limit, cudaStream_t st) {
  int stages, sb;
  size_t smem;
  smem_limit = iter_smem_limit<T>(smem_limit);
  if (!plan_ring<T>(a.L, a.grid, smem_limit, stages, sb, smem)) return cudaErrorInvalidConfiguration;
  return launch_iterate_t<T>(a, stages, sb, smem, st);
}

// FP32, BF16, FP16 and E4M3 storage (all compute in FP32)
cudaError_t run_iterate_f32(int store, const IterArgs<float>& a, int smem_limit, cudaStream_t st) {
  switch (store) {
    case GDWD_BF16: return run_iterate_ft<__nv_bfloat16>(a, smem_limit, st);
    case GDWD_F16: return run_iterate_ft<__half>(a, smem_limit, st);
    case GDWD_E4M3: return run_iterate_ft<__nv_fp8_e4m3>(a, smem_limit, st);
    default: return run_iterate_ft<float>(a, smem_limit, st);
  }
}

// ---------------------------------------------------------------------------
// stand-alone products with the stored data (gdwd_apply): same passes
// ---------------------------------------------------------------------------
struct ApplyEpi {
  double* out;
  __device__ void row(int64_t j, int, df t, df) { out[j] = df_to_double(t); }
};

template <typename T>
__global__ void __launch_bounds__(kThreads) applyA_kernel(Layout L, const double* x, typename ElemTraits<T>::compute_t* partial,
                                                          int stages, int stage_bytes, int* err, uint64_t tmo) {
  using CT = typename ElemTraits<T>::compute_t;
  constexpr int VEC = ElemTraits<T>::kVec;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t s_bars[kMaxStages];
  __shared__ int s_abort;
  Ring rg{smem, s_bars, stages, stage_bytes, 0};
  if (threadIdx.x == 0) s_abort = 0;
  ring_init(rg);
  CT* gp = reinterpret_cast<CT*>(smem + (size_t)stages * stage_bytes);
  const int cta = blockIdx.x, grid = gridDim.x;
  const int nmy = (L.NB > cta) ? (L.NB - cta + grid - 1) / grid : 0;
  for (int k = 0; k < nmy; ++k) {
    const int64_t s = cta + (int64_t)k * grid;
    for (int j = threadIdx.x; j < L.TB; j += kThreads) {
      const int64_t gj = s * L.TB + j;
      gp[(size_t)k * L.TB + j] = (CT)(gj < L.d ? x[gj] : 0.0);
    }
  }
  __syncthreads();
  PassA<T> pa{gp, partial, L.TB, L.NB, L.TB / VEC, kThreads / L.CW};
  stream_slabs<T>(L, rg, cta, grid, err, tmo, &s_abort, pa);
}

template <typename CT>
__global__ void applyA_reduce(const CT* partial, const double* sc, int64_t n, int NB, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < n; i += nw) {
    double acc = 0.0;
    for (int s = lane; s < NB; s += 32) acc += (double)partial[(size_t)i * NB + s];
    acc = warp_sum(acc);
    if (lane == 0) out[i] = sc[i] * acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) applyB_kernel(Layout L, const double* x, const double* sc, double* out,
                                                          int stages, int stage_bytes, int* err, uint64_t tmo) {
  using CT = typename ElemTraits<T>::compute_t;
  constexpr int VEC = ElemTraits<T>::kVec;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t s_bars[kMaxStages];
  __shared__ int s_abort;
  Ring rg{smem, s_bars, stages, stage_bytes, 0};
  if (threadIdx.x == 0) s_abort = 0;
  ring_init(rg);
  uint8_t* uni = smem + (size_t)stages * stage_bytes;
  CT* cv = reinterpret_cast<CT*>(uni);
  double* red = reinterpret_cast<double*>(uni + ((2 * L.n * sizeof(CT) + 15) & ~(size_t)15));
  for (int64_t i = threadIdx.x; i < L.n; i += kThreads) cv[i] = (CT)(sc[i] * x[i]);
  __syncthreads();
  const int Q = L.TB / VEC;
  ApplyEpi epi{out};
  PassB<T, ApplyEpi> pb;
  pb.cv = cv;
  pb.av = cv;
  pb.red = red;
  pb.TB = L.TB;
  pb.Q = Q;
  pb.G = Q <= kThreads ? kThreads / Q : 1;
  pb.d = L.d;
  pb.two = false;
  pb.epi = &epi;
  for (int kk = 0; kk < VEC; ++kk) {
    pb.rc[kk].reset();
    pb.ra[kk].reset();
  }
  stream_slabs<T>(L, rg, blockIdx.x, gridDim.x, err, tmo, &s_abort, pb);
}

template <typename T>
static cudaError_t run_apply_t(const Layout& L, int trans, const double* x, const double* sc, double* out,
                               void* partial, int grid, int smem_limit, int* err, uint64_t tmo, cudaStream_t st) {
  using CT = typename ElemTraits<T>::compute_t;
  int stages, sb;
  size_t smem;
  if (!plan_ring<T>(L, grid, smem_limit, stages, sb, smem, true)) return cudaErrorInvalidConfiguration;
  if (trans) {
    auto k = applyA_kernel<T>;
    cudaError_t e = ensure_max_dyn_smem<applyA_kernel<T>>();
    if (e != cudaSuccess) return e;
    k<<<grid, kThreads, smem, st>>>(L, x, (CT*)partial, stages, sb, err, tmo);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    applyA_reduce<CT><<<(int)std::min<int64_t>((L.n * 32 + 255) / 256, 1024), 256, 0, st>>>((const CT*)partial, sc, L.n,
                                                                                      L.NB, out);
    return cudaGetLastError();
  }
  auto k = applyB_kernel<T>;
  cudaError_t e = ensure_max_dyn_smem<applyB_kernel<T>>();
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(L, x, sc, out, stages, sb, err, tmo);
  return cudaGetLastError();
}

cudaError_t run_apply(int store, const Layout& L, int trans, const double* x, const double* sc, double* out,
                      void* partial, int grid, int smem_limit, int* err, uint64_t tmo, cudaStream_t st, bool wide) {
  if (wide && store == GDWD_F32)
    return run_apply_t<f32w>(L, trans, x, sc, out, partial, grid, smem_limit, err, tmo, st);
  switch (store) {
    case GDWD_F64: return run_apply_t<double>(L, trans, x, sc, out, partial, grid, smem_limit, err, tmo, st);
    case GDWD_BF16: return run_apply_t<__nv_bfloat16>(L, trans, x, sc, out, partial, grid, smem_limit, err, tmo, st);
    case GDWD_F16: return run_apply_t<__half>(L, trans, x, sc, out, partial, grid, smem_limit, err, tmo, st);
    case GDWD_E4M3: return run_apply_t<__nv_fp8_e4m3>(L, trans, x, sc, out, partial, grid, smem_limit, err, tmo, st);
    default: return run_apply_t<float>(L, trans, x, sc, out, partial, grid, smem_limit, err, tmo, st);
  }
}

}  // namespace gdwd
