// The inexact solver of eq-linsys for d and n both large (solver = 2; Sec. 3.3.3
// with T = 0, Algorithm 1 Steps 1a-1c with eq-linsys-tol): the element-wise
// kernels, the deterministic block reductions and the host-driven loop.
//
// Every product with A = U U^T + diag(mu I, 0), U = [Z~; y^T], is two passes of the
// streaming product kernels over the stored Z (Z~^T p_w, then Z~ t with
// t = Z~^T p_w + y p_beta), 4nd flops like the paper's PSQMR step.  The paper's
// Krylov solver is PSQMR, described in an appendix that is not part of the text;
// A is symmetric positive definite, so the conjugate-gradient method of the same
// family is used, preconditioned by diag(A) (Jacobi).  Z~^T w is carried through
// the CG updates and recomputed by one pass at the start of every Step 1a.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "inexact.cuh"
#include "nspace.cuh"

namespace gdwd {
namespace {

constexpr int kIxThreads = 256;

// K values of every thread summed over the block in a fixed order; value k goes
// to part[k * kIxBlocks + blockIdx.x].
template <int K>
__device__ __forceinline__ void block_store(const double (&v)[K], double* part) {
  __shared__ double s[kIxThreads / 32][K > 0 ? K : 1];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double t = warp_sum(v[k]);
    if (l == 0) s[w][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int i = 0; i < kIxThreads / 32; ++i) t += s[i][threadIdx.x];
    part[(size_t)threadIdx.x * kIxBlocks + blockIdx.x] = t;
  }
}

#define IX_LOOP(i, len) for (int64_t i = blockIdx.x * (int64_t)kIxThreads + threadIdx.x; i < (len); i += (int64_t)kIxBlocks * kIxThreads)

// diag(Z~ Z~^T) + mu, one thread per row of a slab
template <typename T>
__global__ void row_sumsq_kernel(Layout L, const double* sc, double mu, double* mw) {
  const T* Z = reinterpret_cast<const T*>(L.Z);
  for (int s = blockIdx.x; s < L.NB; s += gridDim.x) {
    const T* slab = Z + (size_t)s * L.n * L.TB;
    for (int j = threadIdx.x; j < L.TB; j += blockDim.x) {
      const int64_t gj = (int64_t)s * L.TB + j;
      if (gj >= L.d) continue;
      double acc = 0.0;
      for (int64_t i = 0; i < L.n; ++i) {
        const double z = sc[i] * (double)slab[(size_t)i * L.TB + j];
        acc = fma(z, z, acc);
      }
      mw[gj] = acc + mu;
    }
  }
}

// v = xi - r - alpha / sigma; sum y^T v
__global__ void ix_v_kernel(int64_t n, const double* xi, const double* r, const double* alpha, const double* y,
                            double inv_sig, double* v, double* part) {
  double s[1] = {0.0};
  IX_LOOP(i, n) {
    const double vi = xi[i] - r[i] - alpha[i] * inv_sig;
    v[i] = vi;
    s[0] = fma(y[i], vi, s[0]);
  }
  block_store<1>(s, part);
}

// hw = -td + mu u + crho rho  (the w block of the right-hand side of eq-linsys)
__global__ void ix_hw_kernel(int64_t d, const double* td, const double* u, const double* rho, double mu, double crho,
                             double* hw) {
  IX_LOOP(j, d) hw[j] = -td[j] + mu * u[j] + crho * rho[j];
}

// out = a + y s; sum y^T out
__global__ void ix_add_y_kernel(int64_t n, const double* a, const double* y, double s, double* out, double* part) {
  double v[1] = {0.0};
  IX_LOOP(i, n) {
    const double o = a[i] + y[i] * s;
    out[i] = o;
    v[0] = fma(y[i], o, v[0]);
  }
  block_store<1>(v, part);
}

// CG start from x = [w; beta]: r = hw - (td + mu w) (td = Z~ t), z = r / m, p = z;
// sums r.z and r.r (the beta component is handled on the host).  With hw == null
// the residual r is given (the continuation of Step 1c).
__global__ void ix_cg_init_kernel(int64_t d, const double* hw, const double* td, const double* w, double mu,
                                  const double* m, double* r, double* z, double* p, double* part) {
  double s[2] = {0.0, 0.0};
  IX_LOOP(j, d) {
    const double rj = hw ? hw[j] - (td[j] + mu * w[j]) : r[j];
    const double zj = rj / m[j];
    r[j] = rj;
    z[j] = zj;
    p[j] = zj;
    s[0] = fma(rj, zj, s[0]);
    s[1] = fma(rj, rj, s[1]);
  }
  block_store<2>(s, part);
}

// Ap = td + mu p (td = Z~ t_p); sum p.Ap
__global__ void ix_cg_ap_kernel(int64_t d, const double* td, const double* p, double mu, double* ap, double* part) {
  double s[1] = {0.0};
  IX_LOOP(j, d) {
    const double a = td[j] + mu * p[j];
    ap[j] = a;
    s[0] = fma(p[j], a, s[0]);
  }
  block_store<1>(s, part);
}

// w += a p; r -= a Ap; z = r / m; sums r.z, r.r
__global__ void ix_cg_step_kernel(int64_t d, double a, const double* p, const double* ap, const double* m, double* w,
                                  double* r, double* z, double* part) {
  double s[2] = {0.0, 0.0};
  IX_LOOP(j, d) {
    w[j] = fma(a, p[j], w[j]);
    const double rj = fma(-a, ap[j], r[j]);
    const double zj = rj / m[j];
    r[j] = rj;
    z[j] = zj;
    s[0] = fma(rj, zj, s[0]);
    s[1] = fma(rj, rj, s[1]);
  }
  block_store<2>(s, part);
}

// x += a y (n-vector update of Z~^T w)
__global__ void ix_axpy_kernel(int64_t n, double a, const double* x, double* y) {
  IX_LOOP(i, n) y[i] = fma(a, x[i], y[i]);
}

// p = z + b p
__global__ void ix_cg_dir_kernel(int64_t d, double b, const double* z, double* p) {
  IX_LOOP(j, d) p[j] = fma(b, p[j], z[j]);
}

// Step 1b: c = Z~^T w-bar + y beta-bar + xi - alpha / sigma, r+ = prox(c), dr = r+ - r;
// sum y^T dr
__global__ void ix_prox_kernel(int64_t n, const double* ztw, const double* y, double beta, const double* xi,
                               const double* alpha, const double* omega, double inv_sig, double q, double* r,
                               double* dr, double* part) {
  const int qc = q_case(q);
  double s[1] = {0.0};
  IX_LOOP(i, n) {
    const double c = ztw[i] + y[i] * beta + xi[i] - alpha[i] * inv_sig;
    const double ri = r[i];
    const double rn = prox_root(c, omega[i] * inv_sig, q, qc, ri);
    r[i] = rn;
    dr[i] = rn - ri;
    s[0] = fma(y[i], rn - ri, s[0]);
  }
  block_store<1>(s, part);
}

// r += td; sum r.r (residual of Step 1a's solution for Step 1c's right-hand side)
__global__ void ix_addres_kernel(int64_t d, const double* td, double* r, double* part) {
  double s[1] = {0.0};
  IX_LOOP(j, d) {
    const double rj = r[j] + td[j];
    r[j] = rj;
    s[0] = fma(rj, rj, s[0]);
  }
  block_store<1>(s, part);
}

// g = w - rho gs into g; sum g.g
__global__ void ix_g_kernel(int64_t d, const double* w, const double* rho, double gs, double* g, double* part) {
  double s[1] = {0.0};
  IX_LOOP(j, d) {
    const double gj = w[j] - rho[j] * gs;
    g[j] = gj;
    s[0] = fma(gj, gj, s[0]);
  }
  block_store<1>(s, part);
}

// Step 2 (u = theta g) and Step 3 (rho -= tau sigma sqrt(mu) (w - u)); sums
// ||w - u||^2 and ||w||^2
__global__ void ix_dupd_kernel(int64_t d, const double* w, const double* g, double theta, double crho, double* u,
                               double* rho, double* part) {
  double s[2] = {0.0, 0.0};
  IX_LOOP(j, d) {
    const double uj = theta * g[j];
    const double wj = w[j];
    u[j] = uj;
    rho[j] = fma(-crho, wj - uj, rho[j]);
    s[0] = fma(wj - uj, wj - uj, s[0]);
    s[1] = fma(wj, wj, s[1]);
  }
  block_store<2>(s, part);
}

// Step 2 (xi) and Step 3 (alpha) in n-space; the nine n-space KKT sums in the
// order of the Scal slots S_RES2 .. S_DUAL_A
__global__ void ix_nupd_kernel(int64_t n, const double* ztw, const double* y, double beta, const double* r,
                               const double* e, const double* omega, const double* wt, double C, double inv_sig,
                               double tau_sig, double q, double inv_q, double* xi, double* alpha, double* part) {
  const int qc = q_case(q);
  double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  IX_LOOP(i, n) {
    const double ce = C * e[i];
    const double ri = r[i], al = alpha[i], yi = y[i];
    const double zw = ztw[i] + yi * beta;
    const double xin = dmax0(ri - zw + (al - ce) * inv_sig);
    const double res = zw + xin - ri;
    const double an = al - tau_sig * res;
    xi[i] = xin;
    alpha[i] = an;
    const double irq1 = 1.0 / pow_q1(ri, q, qc);
    const double dv = an - omega[i] * irq1;
    const double mn = dmin0(an), mx = dmax0(an - ce);
    s[0] = fma(res, res, s[0]);
    s[1] = fma(yi, an, s[1]);
    s[2] = fma(xin, ce - an, s[2]);
    s[3] = fma(dv, dv, s[3]);
    s[4] = fma(mn, mn, s[4]);
    s[5] = fma(mx, mx, s[5]);
    s[6] += omega[i] * inv_q * ri * irq1;
    s[7] = fma(e[i], xin, s[7]);
    s[8] += dual_pow(wt[i] * an, q, qc);
  }
  block_store<9>(s, part);
}

// sums ||Z~ alpha + sqrt(mu) rho||^2 and ||Z~ alpha||^2 (td = Z~ alpha)
__global__ void ix_d3_kernel(int64_t d, const double* td, const double* rho, double sqmu, double* part) {
  double s[2] = {0.0, 0.0};
  IX_LOOP(j, d) {
    const double a = td[j] + sqmu * rho[j];
    s[0] = fma(a, a, s[0]);
    s[1] = fma(td[j], td[j], s[1]);
  }
  block_store<2>(s, part);
}

#undef IX_LOOP

}  // namespace

namespace {

// Sums of the first k slots of the block partials (fixed order: deterministic).
struct Reducer {
  double* part;
  double* hpart;
  cudaStream_t st;
  cudaError_t fetch(int k, double* out) {
    cudaError_t e = cudaMemcpyAsync(hpart, part, (size_t)k * kIxBlocks * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < k; ++s) {
      double t = 0.0;
      for (int b = 0; b < kIxBlocks; ++b) t += hpart[(size_t)s * kIxBlocks + b];
      out[s] = t;
    }
    return cudaSuccess;
  }
};

#define IX_CK(x)                              \
  do {                                        \
    const cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)
#define IX_GRID kIxBlocks, kIxThreads, 0, st

// Preconditioned CG on A [w; beta] = [hw; hb] from the current (w, beta) (init)
// or from the residual already in cr / rb (the continuation of Step 1c), until
// ||residual|| <= tol.  Keeps Z~^T w in ztw.  Returns the steps taken.
cudaError_t pcg(IxArgs& a, const IxPasses& ps, Reducer& red, cudaStream_t st, bool from_residual, double hb,
                double& rb, double tol, int64_t& steps) {
  const int64_t d = a.d, n = a.n;
  const double mb = (double)n;   // diag of the beta block: y^T y
  double s2[2];
  if (!from_residual) {
    // A x for x = (w, beta): t = Z~^T w + y beta (Z~^T w is recomputed, then carried)
    IX_CK(ps.apply(1, a.w, a.ztw, ps.ctx));
    ix_add_y_kernel<<<IX_GRID>>>(n, a.ztw, a.y, a.beta, a.tn, a.part);
    double yt;
    IX_CK(red.fetch(1, &yt));
    IX_CK(ps.apply(0, a.tn, a.td, ps.ctx));
    ix_cg_init_kernel<<<IX_GRID>>>(d, a.hw, a.td, a.w, a.mu, a.mw, a.cr, a.cz, a.cp, a.part);
    rb = hb - yt;
  } else {
    ix_cg_init_kernel<<<IX_GRID>>>(d, nullptr, nullptr, nullptr, a.mu, a.mw, a.cr, a.cz, a.cp, a.part);
  }
  IX_CK(red.fetch(2, s2));
  double zb = rb / mb, pb = zb;
  double rz = s2[0] + rb * zb, rr = s2[1] + rb * rb;
  for (int k = 0; k < 20000 && std::sqrt(rr) > tol; ++k) {   // bounded: 20000 steps per solve
    // A p: tp = Z~^T p_w + y p_beta, Ap = (Z~ tp + mu p_w, y^T tp)
    IX_CK(ps.apply(1, a.cp, a.zp, ps.ctx));
    ix_add_y_kernel<<<IX_GRID>>>(n, a.zp, a.y, pb, a.tn, a.part);
    double apb;
    IX_CK(red.fetch(1, &apb));
    IX_CK(ps.apply(0, a.tn, a.td, ps.ctx));
    ix_cg_ap_kernel<<<IX_GRID>>>(d, a.td, a.cp, a.mu, a.cap, a.part);
    double pap;
    IX_CK(red.fetch(1, &pap));
    pap += pb * apb;
    if (!(pap > 0.0)) break;    // A is SPD: a non-positive curvature means the residual is at rounding level
    const double al = rz / pap;
    ix_cg_step_kernel<<<IX_GRID>>>(d, al, a.cp, a.cap, a.mw, a.w, a.cr, a.cz, a.part);
    ix_axpy_kernel<<<IX_GRID>>>(n, al, a.zp, a.ztw);
    IX_CK(red.fetch(2, s2));
    a.beta += al * pb;
    rb -= al * apb;
    zb = rb / mb;
    const double rz_new = s2[0] + rb * zb;
    rr = s2[1] + rb * rb;
    ++steps;
    if (std::sqrt(rr) <= tol) break;
    const double b = rz_new / rz;
    ix_cg_dir_kernel<<<IX_GRID>>>(d, b, a.cz, a.cp);
    pb = zb + b * pb;
    rz = rz_new;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_row_sumsq(int store, const Layout& L, const double* sc, double mu, double* mw, cudaStream_t st) {
  const int blocks = std::min(L.NB, 4096);
  if (store == GDWD_F64) row_sumsq_kernel<double><<<blocks, 256, 0, st>>>(L, sc, mu, mw);
  else row_sumsq_kernel<float><<<blocks, 256, 0, st>>>(L, sc, mu, mw);
  return cudaGetLastError();
}

cudaError_t run_inexact(IxArgs& a, const IxPasses& ps, double sigma0, cudaStream_t st, IxResult* res) {
  const int64_t d = a.d, n = a.n;
  const double sqmu = std::sqrt(a.mu), den = 1.0 + a.C, inv_q = 1.0 / a.q;
  Reducer red{a.part, a.hpart, st};
  double sigma = sigma0;
  IxResult out{};
  out.status = GDWD_EMAXITER;
  int it = 0;
  for (; it < a.max_iter; ++it) {
    const double eps = a.eps_c / std::pow((double)it + 1.0, 1.5);   // eps_k
    const double inv_sig = 1.0 / sigma, gs = 1.0 / (sigma * sqmu);
    // ---- Step 1a: h-bar = [-Z~ v + mu u + sqrt(mu) rho / sigma; -y^T v], v = xi - r - alpha / sigma
    ix_v_kernel<<<IX_GRID>>>(n, a.xi, a.r, a.alpha, a.y, inv_sig, a.v, a.part);
    double yv;
    IX_CK(red.fetch(1, &yv));
    IX_CK(ps.apply(0, a.v, a.td, ps.ctx));
    ix_hw_kernel<<<IX_GRID>>>(d, a.td, a.u, a.rho, a.mu, sqmu * inv_sig, a.hw);
    double rb = 0.0;
    IX_CK(pcg(a, ps, red, st, false, -yv, rb, eps, out.cg_steps));
    const double beta_bar = a.beta;
    // ---- Step 1b: r^{k+1} by the prox at c = Z~^T w-bar + y beta-bar + xi - alpha / sigma
    ix_prox_kernel<<<IX_GRID>>>(n, a.ztw, a.y, beta_bar, a.xi, a.alpha, a.omega, inv_sig, a.q, a.r, a.dr, a.part);
    double ydr;
    IX_CK(red.fetch(1, &ydr));
    // ---- Step 1c: the residual of (w-bar, beta-bar) for h is the old one plus U (r+ - r)
    IX_CK(ps.apply(0, a.dr, a.td, ps.ctx));
    ix_addres_kernel<<<IX_GRID>>>(d, a.td, a.cr, a.part);
    double rr;
    IX_CK(red.fetch(1, &rr));
    rb += ydr;
    if (std::sqrt(rr + rb * rb) > 5.0 * eps) {
      IX_CK(pcg(a, ps, red, st, true, 0.0, rb, 5.0 * eps, out.cg_steps));
      ++out.step1c_solves;
    }
    // ---- Step 2: g = w - rho / (sigma sqrt(mu)), u = Pi_B(g); xi.  Step 3: alpha, rho
    ix_g_kernel<<<IX_GRID>>>(d, a.w, a.rho, gs, a.cz, a.part);
    double g2;
    IX_CK(red.fetch(1, &g2));
    const double gn = std::sqrt(g2);
    const double theta = gn <= a.R ? 1.0 : a.R / gn;
    ix_dupd_kernel<<<IX_GRID>>>(d, a.w, a.cz, theta, a.tau * sigma * sqmu, a.u, a.rho, a.part);
    double dsum[2];
    IX_CK(red.fetch(2, dsum));
    ix_nupd_kernel<<<IX_GRID>>>(n, a.ztw, a.y, a.beta, a.r, a.e, a.omega, a.wt, a.C, inv_sig, a.tau * sigma, a.q,
                                inv_q, a.xi, a.alpha, a.part);
    double ns[9];
    IX_CK(red.fetch(9, ns));
    IX_CK(ps.apply(0, a.alpha, a.td, ps.ctx));
    ix_d3_kernel<<<IX_GRID>>>(d, a.td, a.rho, sqmu, a.part);
    double d3[2];
    IX_CK(red.fetch(2, d3));
    // ---- KKT residuals and gap (Sec. 4.3; readings R6, R7, R9), stop test, sigma rule (Sec. 4.4)
    out.eta_c1 = std::fabs(ns[1]) / den;
    out.eta_c2 = std::fabs(ns[2]) / den;
    out.eta_c3 = std::sqrt(ns[3]) / den;
    out.eta_p1 = std::sqrt(ns[0]) / den;
    out.eta_p2 = sqmu * std::sqrt(dsum[0]) / den;
    out.eta_p3 = std::max(std::sqrt(dsum[1]) - a.R, 0.0) / den;
    out.eta_d1 = std::sqrt(ns[4]) / den;
    out.eta_d2 = std::sqrt(ns[5]) / den;
    out.eta_d3 = std::sqrt(d3[0]) / den;
    out.pobj = ns[6] + a.C * ns[7];
    out.dobj = a.kappa * ns[8] - a.R * std::sqrt(d3[1]);
    out.eta_gap = std::fabs(out.pobj - out.dobj) / (1.0 + std::fabs(out.pobj) + std::fabs(out.dobj));
    const double ep = std::max(out.eta_p1, std::max(out.eta_p2, out.eta_p3));
    const double ed = std::max(out.eta_d1, std::max(out.eta_d2, out.eta_d3));
    const double ec = std::max(out.eta_c1, std::max(out.eta_c2, out.eta_c3));
    out.kkt = std::max(std::max(ep, ed), std::max(ec, out.eta_gap));
    out.beta = a.beta;
    out.sigma = sigma;
    if (!std::isfinite(out.kkt)) {
      out.status = GDWD_ENUMERIC;
      ++it;
      break;
    }
    const bool stop = a.stop_rule == 0 ? out.kkt <= a.tol
                                       : (std::max(ep, ed) < a.tol && std::min(ec, out.eta_gap) < std::sqrt(a.tol) &&
                                          std::max(ec, out.eta_gap) < 0.05);
    if (stop) {
      out.status = GDWD_OK;
      ++it;
      break;
    }
    if (it >= 1 && std::min(ep, ed) > 1e-3 * a.tol) {
      const double chi = ep / std::max(ed, 1e-300);
      const double big = std::max(chi, 1.0 / std::max(chi, 1e-300));
      const double zeta = big > 500.0 ? 2.2 : (big > 50.0 ? 1.65 : 1.1);
      if (chi > 5.0) sigma *= zeta;
      else if (1.0 / std::max(chi, 1e-300) > 5.0) sigma /= zeta;
    }
  }
  out.iters = it;
  out.sigma = sigma;
  *res = out;
  return cudaGetLastError();
}

#undef IX_CK
#undef IX_GRID

}  // namespace gdwd
