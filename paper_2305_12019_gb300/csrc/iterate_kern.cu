// Kernelized n-space iteration of libgdwd: the loop of Algorithm 1 (Sec. 3) for
// one value of C run on the Gram matrix alone, in ONE cooperative launch with
// one CTA per SM and bounded grid barriers between its phases.
//
// From the initial iterate w = u = rho = 0 (reading R3) every d-space iterate
// stays in the range of Z~.  The solution of eq-linsys (SMW2 form, Sec. 3.3.2,
// solved in n-space as in the Z-streaming kernel) has w = g' - Z~ c / mu, Step 2
// projects g = u - Z~ c / mu onto the ball (a scaling by theta) and Step 3 moves
// rho by a multiple of the same g.  So u = Z~ a_u, rho = Z~ a_rho, g = Z~ a_g with
//     a_g = a_u - c / mu,   a_u+ = theta a_g,
//     a_rho+ = (1 - tau) a_rho - tau sigma sqrt(mu) (1 - theta) a_g,
// and every d-space quantity the iteration reads is an n-space product with
// K = Z~^T Z~:
//     b = Z~^T g' = K a_u + K a_rho / (sigma sqrt(mu)),
//     ||g||^2 = a_g^T K a_g,  <g, rho> = a_rho^T K a_g,  ||rho||^2 = a_rho^T K a_rho,
//     ||Z~ alpha||^2 = alpha^T K alpha,  <Z~ alpha, rho> = alpha^T K a_rho,
//     <Z~ alpha, g> = alpha^T K a_g.
// One double-float GEMV with K and the three right-hand sides alpha, a_g, a_rho
// per iteration gives all six products; K a_u and K a_rho of the next iteration
// follow from K a_g and K a_rho by the coefficients' own update, so no product
// is carried by a recurrence.  w = Z~ (a_g + a_rho / (sigma sqrt(mu))) is formed
// once, after the loop, by one pass over Z.  An iteration costs two G^{-1} GEMVs
// and one three-column K GEMV, O(n^2), and reads no Z.
//
//   prologue   a stored iterate: its deferred coefficient update, then U_u = K a_u,
//              U_rho = K a_rho (two-column GEMV); the initial iterate: zeros
//   phase R    this CTA's rows: the deferred update of a_u, a_rho, U_u, U_rho;
//              b = U_u + U_rho / (sigma sqrt(mu)); rhs1 = b + v-bar
//   phase N1   x-bar = G^{-1} rhs1 (double-float GEMV), beta-bar, Step 1b prox,
//              rhs2 = b + v
//   phase N2   x = G^{-1} rhs2, beta, c, Z~^T w; Step 2 xi, Step 3 alpha (n part);
//              a_g; the n-space KKT sums
//   phase K    K [alpha, a_g, a_rho] for this CTA's rows and the six products
//   phase S    totals, KKT residuals (Sec. 4.3), duality gap, sigma rule
//              (Sec. 4.4), stop test; identical in every CTA
#include <algorithm>
#include <mutex>

#include "iterate_kern.cuh"
#include "nspace.cuh"

namespace gdwd {

// Phase K's sums, in the slots S_G2 .. S_TA2 that phase S reads.  The d-space
// vectors are Z~ times coefficient vectors (g = Z~ a_g, rho = Z~ a_rho), so each
// norm is a quadratic form in K summed row by row.  The two small residuals are
// taken about the last iteration's theta_prev, as in the streaming iteration:
// y = (1 - theta_prev) g + rho / (sigma sqrt(mu)) and v = a - khat g, with
// a = Z~ alpha + sqrt(mu)(1 - tau) rho and khat = tau mu sigma (1 - theta_prev),
// their coefficient vectors formed per row before the products.
enum KernScal {
  KS_G2 = S_G2,     // ||g||^2
  KS_YG,            // <y, g>
  KS_Y2,            // ||y||^2
  KS_V2,            // ||v||^2
  KS_VG,            // <v, g>
  KS_TA2            // ||Z~ alpha||^2
};
static_assert((int)KS_TA2 < (int)S_COUNT && (int)KS_YG == (int)S_GRHO && (int)KS_Y2 == (int)S_RHO2 &&
                  (int)KS_V2 == (int)S_A2 && (int)KS_VG == (int)S_AG && (int)KS_TA2 == (int)S_TA2,
              "phase-K sums sit in the slots phase S reads");

// Three products of one double-float row of K with three double-float vectors
// (one warp; results in every lane).
__device__ __forceinline__ void row_dot3(const float2* __restrict__ Krow, const float2* v0, const float2* v1,
                                         const float2* v2, int npair, double& o0, double& o1, double& o2) {
  const float4* K4 = reinterpret_cast<const float4*>(Krow);
  const float4* A4 = reinterpret_cast<const float4*>(v0);
  const float4* B4 = reinterpret_cast<const float4*>(v1);
  const float4* C4 = reinterpret_cast<const float4*>(v2);
  df a0{0.f, 0.f}, a1{0.f, 0.f}, b0{0.f, 0.f}, b1{0.f, 0.f}, c0{0.f, 0.f}, c1{0.f, 0.f};
  const int lane = threadIdx.x & 31;
  int j = lane;
  for (; j + 32 < npair; j += 64) {
    const float4 k0 = __ldg(K4 + j), k1 = __ldg(K4 + j + 32);
    float4 r = A4[j];
    df_fma(a0, df{k0.x, k0.y}, df{r.x, r.y});
    df_fma(a1, df{k0.z, k0.w}, df{r.z, r.w});
    r = B4[j];
    df_fma(b0, df{k0.x, k0.y}, df{r.x, r.y});
    df_fma(b1, df{k0.z, k0.w}, df{r.z, r.w});
    r = C4[j];
    df_fma(c0, df{k0.x, k0.y}, df{r.x, r.y});
    df_fma(c1, df{k0.z, k0.w}, df{r.z, r.w});
    r = A4[j + 32];
    df_fma(a0, df{k1.x, k1.y}, df{r.x, r.y});
    df_fma(a1, df{k1.z, k1.w}, df{r.z, r.w});
    r = B4[j + 32];
    df_fma(b0, df{k1.x, k1.y}, df{r.x, r.y});
    df_fma(b1, df{k1.z, k1.w}, df{r.z, r.w});
    r = C4[j + 32];
    df_fma(c0, df{k1.x, k1.y}, df{r.x, r.y});
    df_fma(c1, df{k1.z, k1.w}, df{r.z, r.w});
  }
  for (; j < npair; j += 32) {
    const float4 k0 = __ldg(K4 + j);
    float4 r = A4[j];
    df_fma(a0, df{k0.x, k0.y}, df{r.x, r.y});
    df_fma(a1, df{k0.z, k0.w}, df{r.z, r.w});
    r = B4[j];
    df_fma(b0, df{k0.x, k0.y}, df{r.x, r.y});
    df_fma(b1, df{k0.z, k0.w}, df{r.z, r.w});
    r = C4[j];
    df_fma(c0, df{k0.x, k0.y}, df{r.x, r.y});
    df_fma(c1, df{k0.z, k0.w}, df{r.z, r.w});
  }
  df_add(a0, a1);
  df_add(b0, b1);
  df_add(c0, c1);
  o0 = df_to_double(df_warp_sum(a0));
  o1 = df_to_double(df_warp_sum(b0));
  o2 = df_to_double(df_warp_sum(c0));
}

__device__ __forceinline__ float2 to_f2(double x) {
  const df v = df_from(x);
  return make_float2(v.hi, v.lo);
}

// One CTA owns a contiguous block of at most kThreads rows of the n-space and
// thread t holds row r0 + t of every n-vector in registers for the whole launch
// (consecutive rows share a warp: the per-row FP64 work of a CTA's few rows then
// issues as few warp instructions as possible);
// only the vectors other CTAs read (the right-hand sides of the GEMVs and the
// partial sums) go through global memory.  The GEMVs read their right-hand
// sides straight from L2 (every warp of the SM reads the same vector, so it is
// served from L1 after the first warp).
__global__ void __launch_bounds__(kThreads, 1) iterate_kern_kernel(KernArgs a) {
  __shared__ int s_flag;
  __shared__ double s_tot[S_COUNT];
  __shared__ double s_ctl[15];
  __shared__ double s_pd[4];     // pobj, dobj, theta, ||w||
  __shared__ float s_etaf[11];   // gap, the nine residuals, kkt
  __shared__ int s_ictl[2];      // done, status
  __shared__ double s_rows[9 * kMaxRowsPerCta];    // per-row partial sums
  __shared__ double s_x[kMaxRowsPerCta + 1];      // GEMV results of the CTA's rows (+ the p^T rhs row)
  __shared__ double s_k[3][kMaxRowsPerCta];
  static_assert(kMaxRowsPerCta <= kThreads, "one row per thread");

  const int cta = blockIdx.x, grid = a.grid;
  const int64_t n = a.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t rpc = (n + grid - 1) / grid;
  const int64_t r0 = ((int64_t)cta * rpc < n) ? (int64_t)cta * rpc : n;
  const int nrows = (int)(((r0 + rpc < n) ? r0 + rpc : n) - r0);
  const int npair = (int)((n + 1) / 2);
  const int ldP = a.ldP;
  const int qcase = q_case(a.q);
  const double sqmu = sqrt(a.mu), inv_mu = 1.0 / a.mu;
  const double den = 1.0 + a.C;
  const double inv_q = 1.0 / a.q;
  const float inv_den = (float)(1.0 / den);
  const double sqrt_tol = sqrt(a.tol);
  const SPhaseArgs sq{a.C, a.kappa, a.R, a.mu, a.tau, sqmu, a.tol, sqrt_tol, inv_den, a.stop_rule, float_at_most(a.tol)};
  const double ac = sqmu * (1.0 - a.tau);              // Z~ alpha + ac rho enters eta_D3

  // this thread's row
  const int tr = threadIdx.x;
  const bool mine = tr < nrows;
  const int64_t i = r0 + tr;
  double yi = 0, pi = 0, ce = 0, omi = 0, wti = 0, ei = 0;
  double ri = 0, xii = 0, ali = 0, bi = 0;
  double Uu = 0, Ur = 0, au = 0, ar = 0, ag = 0, KG = 0, KR = 0;
  if (mine) {
    yi = a.y[i];
    pi = a.p[i];
    ei = a.e[i];
    ce = a.C * ei;
    omi = a.omega[i];
    wti = a.wt[i];
    ri = a.r[i];
    xii = a.xi[i];
    ali = a.alpha[i];
  }

  unsigned gen = 0;
  __shared__ unsigned long long s_tacc[kPhaseSlots], s_tprev;
  const bool timing = (cta == 0 && threadIdx.x == 0);
  if (timing) {
    for (int k = 0; k < kPhaseSlots; ++k) s_tacc[k] = 0;
    s_tprev = globaltimer();
  }
  double sig = a.ctrl->sigma, sig_prev = a.ctrl->sigma_prev, theta = a.ctrl->theta;
  int pending = a.ctrl->pending;
  const int it0 = a.ctrl->it;
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
#define GDWD_BARRIER(k)                                                                   \
  do {                                                                                    \
    GDWD_MARK(k);                                                                         \
    if (!grid_barrier(a.bar, (unsigned)grid, gen, a.err, a.timeout_ns, &s_flag)) return; \
    GDWD_MARK(k + 1);                                                                     \
  } while (0)

  // ---------------- prologue
  if (a.refresh) {
    // a stored iterate: its pending coefficient update, then U_u = K a_u and
    // U_rho = K a_rho by a two-column GEMV
    if (mine) {
      au = a.au[i];
      ar = a.ar[i];
      if (pending) {
        const double rcoef0 = a.tau * sig_prev * sqmu * (1.0 - theta);
        const double agi = a.ag[i];
        au = theta * agi;
        ar = (1.0 - a.tau) * ar - rcoef0 * agi;
      }
      a.vdf[i] = to_f2(au);
      a.vdf[ldP + i] = to_f2(ar);
    }
    GDWD_BARRIER(0);
    for (int t = warp; t < nrows; t += kWarps) {
      double ku, kr, unused;
      row_dot3(a.Kd + (size_t)(r0 + t) * ldP, a.vdf, a.vdf + ldP, a.vdf + ldP, npair, ku, kr, unused);
      if (lane == 0) {
        s_k[0][t] = ku;
        s_k[1][t] = kr;
      }
    }
    __syncthreads();
    if (mine) {
      Uu = s_k[0][tr];
      Ur = s_k[1][tr];
    }
    pending = 0;
  }

  int it = it0;
  for (; it < a.max_iter; ++it) {
    const double inv_sig = rcp_nr(sig);
    const double gs_it = rcp_nr(sig * sqmu);   // 1 / (sigma sqrt(mu)) of this iteration
    // ---------------- phase R (this thread's row): the deferred update
    // a_u = theta a_g, a_rho <- (1 - tau) a_rho - tau sigma' sqrt(mu) (1 - theta) a_g
    // and the same update of their images U_u = K a_u, U_rho = K a_rho from the
    // last phase K's products; b = U_u + U_rho / (sigma sqrt(mu)); rhs1 = b + v
    if (mine) {
      if (pending) {
        const double rcoef = a.tau * sig_prev * sqmu * (1.0 - theta);
        Uu = theta * KG;
        Ur = (1.0 - a.tau) * KR - rcoef * KG;
        au = theta * ag;
        ar = (1.0 - a.tau) * ar - rcoef * ag;
      }
      bi = Uu + Ur * gs_it;
      a.rhsA[i] = to_f2(bi + (xii - ri - ali * inv_sig));
    }
    GDWD_BARRIER(2);

    // ---------------- phase N1: x-bar, beta-bar, Step 1b prox, rhs2
    {
      GDWD_MARK(14);
      for (int t = warp; t <= nrows; t += kWarps) {
        const df x = row_dot(t < nrows ? a.P + (size_t)(r0 + t) * ldP : a.pdf, a.rhsA, npair);
        if (lane == 0) s_x[t] = df_to_double(x);
      }
      __syncthreads();
      GDWD_MARK(15);
      if (mine) {
        const double betabar = -s_x[nrows] * a.inv_s;
        const double cbar = s_x[tr] + betabar * pi;
        ri = prox_root(cbar + ri, omi * inv_sig, a.q, qcase, ri);
        a.rhsB[i] = to_f2(bi + (xii - ri - ali * inv_sig));
      }
    }
    GDWD_BARRIER(4);

    // ---------------- phase N2: x, beta, c, Z~^T w; Step 2 (xi), Step 3 (alpha);
    // a_g = a_u - c / mu; the right-hand sides of phase K
    {
      GDWD_MARK(11);
      for (int t = warp; t <= nrows; t += kWarps) {
        const df x = row_dot(t < nrows ? a.P + (size_t)(r0 + t) * ldP : a.pdf, a.rhsB, npair);
        if (lane == 0) s_x[t] = df_to_double(x);
      }
      __syncthreads();
      beta = -s_x[nrows] * a.inv_s;
      GDWD_MARK(12);
      double s_res2 = 0, s_ya = 0, s_xica = 0, s_ams2 = 0, s_amin2 = 0, s_amax2 = 0, s_pr = 0, s_px = 0, s_du = 0;
      if (mine) {
        const double c = s_x[tr] + beta * pi;
        const double v = xii - ri - ali * inv_sig;
        const double zw = c - v - yi * beta;                                      // Z~^T w
        const double xin = fmax(0.0, ri - zw - yi * beta + (ali - ce) * inv_sig);  // Step 2
        const double res = zw + yi * beta + xin - ri;
        const double an = ali - a.tau * sig * res;                                // Step 3
        xii = xin;
        ali = an;
        ag = au - c * inv_mu;                                                     // g = u - Z~ c / mu
        a.vdf[i] = to_f2(an);
        a.vdf[ldP + i] = to_f2(ag);
        a.vdf[2 * ldP + i] = to_f2(ar);
        const double irq1 = rcp_nr(pow_q1(ri, a.q, qcase));
        s_res2 = res * res;
        s_ya = yi * an;
        s_xica = xin * (ce - an);
        const double dv = an - omi * irq1;
        s_ams2 = dv * dv;
        const double mn = fmin(0.0, an), mx = fmax(0.0, an - ce);
        s_amin2 = mn * mn;
        s_amax2 = mx * mx;
        s_pr = omi * inv_q * ri * irq1;           // wt^q r^-q
        s_px = ei * xin;
        s_du = dual_pow(wti * an, a.q, qcase);
      }
      const double vals[9] = {s_res2, s_ya, s_xica, s_ams2, s_amin2, s_amax2, s_pr, s_px, s_du};
      rows_sum<9>(vals, tr, mine, nrows, s_rows, kMaxRowsPerCta, a.scal + cta, grid);
    }
    GDWD_BARRIER(6);

    // ---------------- phase K: K alpha, K a_g, K a_rho for this CTA's rows and the
    // six products of the d-space norms
    {
      for (int t = warp; t < nrows; t += kWarps) {
        double ka, kg, kr;
        row_dot3(a.Kd + (size_t)(r0 + t) * ldP, a.vdf, a.vdf + ldP, a.vdf + 2 * ldP, npair, ka, kg, kr);
        if (lane == 0) {
          s_k[0][t] = ka;
          s_k[1][t] = kg;
          s_k[2][t] = kr;
        }
      }
      __syncthreads();
      double g2 = 0, yg = 0, y2 = 0, v2 = 0, vg = 0, ta2 = 0;
      if (mine) {
        const double ka = s_k[0][tr];
        KG = s_k[1][tr];
        KR = s_k[2][tr];
        const double omp = 1.0 - theta, khat = a.tau * a.mu * sig * omp;
        const double cy = omp * ag + gs_it * ar, kcy = omp * KG + gs_it * KR;       // y's coefficients, K times them
        const double cv = ali + ac * ar - khat * ag, kcv = ka + ac * KR - khat * KG;  // v's
        g2 = ag * KG;
        yg = cy * KG;
        y2 = cy * kcy;
        v2 = cv * kcv;
        vg = cv * KG;
        ta2 = ali * ka;
      }
      const double vals[6] = {g2, yg, y2, v2, vg, ta2};
      rows_sum<6>(vals, tr, mine, nrows, s_rows, kMaxRowsPerCta, a.scal + (size_t)KS_G2 * grid + cta, grid);
    }
    GDWD_BARRIER(8);

    // ---------------- phase S: totals, KKT, sigma rule, stop test (same in every CTA)
    grid_totals(a.scal, grid, KS_TA2 + 1, s_tot);
    __syncthreads();
    GDWD_MARK(13);
    s_phase(s_tot, sq, sig, gs_it, it, beta, status, false, a.ctrl, s_pd, s_etaf, s_ctl, s_ictl, theta, true);
    GDWD_MARK(10);
    sig_prev = sig;
    theta = s_ctl[0];
    sig = s_ctl[1];
    pending = 1;
    const bool done = s_ictl[0] != 0;
    status = s_ictl[1];
    if (done) {
      ++it;
      break;
    }
  }
  if (it >= a.max_iter && status != GDWD_OK) status = GDWD_EMAXITER;
  // the rows back to global memory: the next launch's starting iterate and the
  // coefficients of w
  if (mine) {
    a.r[i] = ri;
    a.xi[i] = xii;
    a.alpha[i] = ali;
    a.b[i] = bi;
    a.Uu[i] = Uu;
    a.Ur[i] = Ur;
    a.au[i] = au;
    a.ar[i] = ar;
    a.ag[i] = ag;
    a.KG[i] = KG;
    a.KR[i] = KR;
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
#undef GDWD_MARK
}

int64_t kern_max_n(int grid, int) { return (int64_t)grid * kMaxRowsPerCta; }

cudaError_t run_iterate_kern(const KernArgs& a, int, cudaStream_t st) {
  if ((a.n + a.grid - 1) / a.grid > kMaxRowsPerCta) return cudaErrorInvalidConfiguration;
  KernArgs args = a;
  void* params[] = {(void*)&args};
  return cudaLaunchCooperativeKernel((const void*)iterate_kern_kernel, dim3(a.grid), dim3(kThreads), params, 0, st);
}

__global__ void kern_matrix_kernel(const double* G, int64_t n, int ldP, double mu, float2* Kd) {
  const int64_t total = n * ldP;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ldP, j = t % ldP;
    float2 v = make_float2(0.f, 0.f);
    if (j < n) v = to_f2(mu * (G[i * n + j] - (i == j ? 1.0 : 0.0)));
    Kd[t] = v;
  }
}

cudaError_t run_kern_matrix(const double* G, int64_t n, int ldP, double mu, float2* Kd, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n * ldP + 255) / 256, 4096);
  kern_matrix_kernel<<<blocks, 256, 0, st>>>(G, n, ldP, mu, Kd);
  return cudaGetLastError();
}

__global__ void kern_wcoef_kernel(const double* ag, const double* ar, const Ctrl* ctrl, double sqmu, double zscale,
                                  int64_t n, double* x) {
  const double gs = 1.0 / (ctrl->sigma_prev * sqmu);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (ag[i] + ar[i] * gs) / zscale;
}

cudaError_t run_kern_wcoef(const double* ag, const double* ar, const Ctrl* ctrl, double sqmu, double zscale, int64_t n,
                           double* x, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  kern_wcoef_kernel<<<blocks, 256, 0, st>>>(ag, ar, ctrl, sqmu, zscale, n, x);
  return cudaGetLastError();
}

}  // namespace gdwd
