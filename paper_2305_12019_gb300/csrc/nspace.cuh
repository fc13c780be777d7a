// n-space device helpers shared by the single- and multi-instance iteration
// kernels: the Step-1b prox (Newton, Sec. 3.2), the dual-objective power,
// deterministic block reductions and the double-float G^{-1} row products.
#pragma once

#include "passes.cuh"

namespace gdwd {

// ---------------------------------------------------------------------------
// r-subproblem (Step 1b, eq-varphi): the positive root of
// s^(q+1) (s - a) = kq,  kq = omega / sigma, by Newton's iteration of Sec. 3.2
// kept inside the bracket [max(a,0), max(a,0) + max(kq, 1)] (f < 0 at the left
// end, f >= 0 at the right end); steps that leave it are bisected.
//
// A dependent FP64 operation takes ~64 cycles on this part (an FP32 one ~5, an
// FP64 division ~1400), and the prox is on the critical path of every
// iteration.  So the same safeguarded iteration first runs in FP32 to ~2e-6
// relative.  Two FP64 corrections follow, written as s <- s - s f / den with
// f = s^(q+1)(s - a) - kq (Newton's step of Sec. 3.2 in correction form;
// den = kq (q+1) + s^(q+2)): f cancels and is evaluated in FP64, while the
// correction s f / den is a small number that needs only FP32 precision.  By
// quadratic convergence the first leaves ~1e-11 relative and the second
// ~1e-18 (plus ~1e-7 of the last correction from its FP32 quotient).  If the
// FP32 stage did not converge, or the corrections are not small and inside the
// bracket, the bracketed FP64 iteration runs instead.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pow_q1f(float s, float q, int qcase) {  // s^(q+1), FP32
  switch (qcase) {
    case 1: return s * s;
    case 2: return s * s * s;
    case 4: { float s2 = s * s; return s2 * s2 * s; }
    case 5: return s * sqrtf(s);
    default: return powf(s, q + 1.0f);
  }
}

__device__ __forceinline__ double pow_q1(double s, double q, int qcase) {  // s^(q+1)
  switch (qcase) {
    case 1: return s * s;
    case 2: return s * s * s;
    case 4: { double s2 = s * s; return s2 * s2 * s; }
    case 5: return s * sqrt_nr(s);   // q = 0.5
    default: return pow(s, q + 1.0);
  }
}

__device__ __forceinline__ int q_case(double q) {
  return q == 1.0 ? 1 : q == 2.0 ? 2 : q == 4.0 ? 4 : q == 0.5 ? 5 : 0;
}

__device__ inline double prox_root(double a, double kq, double q, int qcase, double r0) {
  // FP32 start, where every FP32 intermediate (up to a s^(q+1) and s^(q+2) with
  // s < hi) stays finite and normal; its bracket and eligibility tests are FP32
  // too (each FP64 instruction occupies this part's FP64 unit for many cycles)
  {
    const float af = (float)a, kf = (float)kq, qf = (float)q, r0f = (float)r0;
    const float lf0 = fmaxf(af, 0.f);
    const float hf0 = lf0 + fmaxf(kf, 1.f);
    if (fabsf(af) < 1e6f && kf > 1e-20f && kf < 1e6f && hf0 < 1e6f && q <= 4.0) {
      float lf = lf0, hf = hf0;
      float sf = (r0f > lf && r0f < hf) ? r0f : 0.5f * (lf + hf);
      bool conv = false;
      for (int it = 0; it < 30; ++it) {
        const float sq1 = pow_q1f(sf, qf, qcase);
        const float f = sq1 * (sf - af) - kf;
        if (f < 0.f) lf = sf;
        else if (f > 0.f) hf = sf;
        else {
          conv = true;
          break;
        }
        const float nt = sf * __fdividef(kf * (qf + 2.f) + af * sq1, kf * (qf + 1.f) + sq1 * sf);
        if (fabsf(nt - sf) <= 2e-6f * sf) {
          sf = nt;
          conv = true;
          break;
        }
        sf = (nt > lf && nt < hf) ? nt : 0.5f * (lf + hf);
      }
      if (conv && sf > 0.f) {
        const double kq1 = kq * (q + 1.0);
        double x = (double)sf;
        float dlf = 0.f, xf = sf;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const double sq1 = pow_q1(x, q, qcase);
          const double f = fma(sq1, x - a, -kq);
          const double den = fma(sq1, x, kq1);
          dlf = xf * __fdividef((float)f, (float)den);
          x -= (double)dlf;
          xf = (float)x;
        }
        // accepted when the last correction is below 1e-9 relative and the
        // root stays on the positive side of max(a, 0)
        if (fabsf(dlf) <= 1e-9f * sf && xf >= lf0) return x;
      }
    }
  }
  // bracketed FP64 iteration (inputs outside the FP32 range, or no FP32 convergence)
  double lo = dmax0(a);
  double hi = lo + (kq > 1.0 ? kq : 1.0);
  double s = (r0 > lo && r0 < hi) ? r0 : 0.5 * (lo + hi);
  for (int it = 0; it < 100; ++it) {
    const double sq1 = pow_q1(s, q, qcase);
    const double f = sq1 * (s - a) - kq;
    if (f < 0.0) lo = s;
    else if (f > 0.0) hi = s;
    else break;
    const double num = kq * (q + 2.0) + a * sq1, den = kq * (q + 1.0) + sq1 * s;
    // division by an FP32 seed and one FP64 correction (~1e-14) when den is in FP32 range
    const double nt = s * ((den > 1e-30 && den < 1e30) ? div_nr(num, den) : num / den);
    // converged when the correction is below 1e-9 relative (then taken): tested
    // before the safeguard, so rounding noise in f at the root cannot trigger a
    // bisection step
    if (fabs(nt - s) <= 1e-9 * s) {
      s = nt;
      break;
    }
    s = (nt > lo && nt < hi) ? nt : 0.5 * (lo + hi);
  }
  return s;
}

// (wt alpha)^(q/(q+1)) for the dual objective
__device__ __forceinline__ double dual_pow(double x, double q, int qcase) {
  if (x <= 0.0) return 0.0;
  switch (qcase) {
    case 1: return sqrt_nr(x);
    case 2: { double c = cbrt(x); return c * c; }
    case 5: return cbrt(x);
    default: return pow(x, q / (q + 1.0));
  }
}

// ---------------------------------------------------------------------------
// block-level deterministic reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* s_red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) s_red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kWarps; ++i) t += s_red[i];
    s_red[kWarps] = t;
  }
  __syncthreads();
  return s_red[kWarps];
}

__device__ __forceinline__ df block_sum_df(df v, float* s_red) {
  v = df_warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    s_red[2 * w] = v.hi;
    s_red[2 * w + 1] = v.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    df t{0.f, 0.f};
    for (int i = 0; i < kWarps; ++i) df_add(t, df{s_red[2 * i], s_red[2 * i + 1]});
    s_red[2 * kWarps] = t.hi;
    s_red[2 * kWarps + 1] = t.lo;
  }
  __syncthreads();
  return df{s_red[2 * kWarps], s_red[2 * kWarps + 1]};
}

// N values per thread summed over the first nw warps of the block: warp sums,
// then one thread per value adds the warp totals in a fixed order
// (deterministic); out[k * stride] receives value k.  Threads of warps >= nw
// must hold zeros.
template <int N>
__device__ __forceinline__ void block_sum_n(const double (&v)[N], int nw, double* s_part, double* out,
                                            int stride) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w < nw) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double t = warp_sum(v[k]);
      if (l == 0) s_part[w * N + k] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += s_part[i * N + threadIdx.x];
    out[(size_t)threadIdx.x * stride] = t;
  }
}

// Totals over the grid of the per-CTA partial sums of slots 0 .. nslots-1
// (nslots <= 16), in a fixed order: 16 threads per slot, each with all its loads
// in flight, then a 16-lane shuffle tree; s_tot[k] receives slot k.
__device__ __forceinline__ void grid_totals(const double* scal, int grid, int nslots, double* s_tot) {
  const int k = threadIdx.x >> 4, sub = threadIdx.x & 15;
  double acc = 0.0;
  if (k < nslots) {
    const double* part = scal + (size_t)k * grid;
    for (int base = 0; base < grid; base += 16 * 12) {
      double v[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const int c2 = base + sub + 16 * q;
        v[q] = c2 < grid ? part[c2] : 0.0;
      }
      // pairwise (depth 4 instead of a chain of 12 FP64 adds)
#pragma unroll
      for (int q = 0; q < 6; ++q) v[q] += v[q + 6];
      v[0] += v[3];
      v[1] += v[4];
      v[2] += v[5];
      acc += (v[0] + v[1]) + v[2];
    }
  }
#pragma unroll
  for (int m = 8; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  if (sub == 0 && k < nslots) s_tot[k] = acc;
}

// Grid totals when slots 0 .. S_DUAL_A hold double-float partials (float2 hi, lo
// in the 8-byte slots) and S_G2 .. S_TA2 FP64 ones.  Each warp-level FP64
// instruction occupies this part's FP64 unit for ~19 cycles whatever the number
// of active lanes, so the nine double-float slots are added on the FP32 pipes by
// warps 0-4 (16 lanes per slot) and the six FP64 slots by warps 5-7 only.  The
// order of the additions is fixed (deterministic).
__device__ __forceinline__ void grid_totals_mixed(const double* scal, int grid, double* s_tot) {
  const int t = threadIdx.x, sub = t & 15;
  if (t < 160) {
    const int k = t >> 4;                       // 0 .. 9; k = 9 (threads 144-159) holds no slot
    df acc{0.f, 0.f};
    if (k <= S_DUAL_A) {
      const float2* part = reinterpret_cast<const float2*>(scal + (size_t)k * grid);
      for (int c = sub; c < grid; c += 16) {
        const float2 v = part[c];
        df_add(acc, df{v.x, v.y});
      }
    }
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) df_add(acc, df_shfl_xor(acc, m));
    if (sub == 0 && k <= S_DUAL_A) s_tot[k] = df_to_double(acc);
  } else {
    const int k = S_G2 + ((t - 160) >> 4);      // 9 .. 14
    const double* part = scal + (size_t)k * grid;
    double acc = 0.0;
    for (int base = 0; base < grid; base += 16 * 12) {
      double v[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const int c2 = base + sub + 16 * q;
        v[q] = c2 < grid ? part[c2] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) v[q] += v[q + 6];
      v[0] += v[3];
      v[1] += v[4];
      v[2] += v[5];
      acc += (v[0] + v[1]) + v[2];
    }
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    if (sub == 0) s_tot[k] = acc;
  }
}

// Grid totals of double-float partials (float2 hi, lo in every 8-byte slot),
// added on the FP32 pipes in a fixed order (16 lanes per slot, then a fixed
// shuffle tree); warp 0 converts the 15 totals to FP64 (three FP64 instructions
// in all: each warp-level FP64 instruction occupies this part's FP64 unit for
// ~19 cycles whatever the number of active lanes).  s_tot is valid after the
// caller's next __syncthreads.
__device__ __forceinline__ void grid_totals_df(const float2* scal, int grid, double* s_tot) {
  __shared__ float2 s_totf[16];
  const int t = threadIdx.x, k = t >> 4, sub = t & 15;
  df acc{0.f, 0.f};
  if (k < S_COUNT - 1) {
    const float2* part = scal + (size_t)k * grid;
    for (int c = sub; c < grid; c += 16) {
      const float2 v = part[c];
      df_add(acc, df{v.x, v.y});
    }
  }
#pragma unroll
  for (int m = 8; m >= 1; m >>= 1) df_add(acc, df_shfl_xor(acc, m));
  if (sub == 0 && k < S_COUNT - 1) s_totf[k] = make_float2(acc.hi, acc.lo);
  __syncthreads();
  if (t < S_COUNT - 1) s_tot[t] = (double)s_totf[t].x + (double)s_totf[t].y;
}

// N double-float values per thread summed over the first nr threads of the block
// (deterministic): through shared memory s_rows (N x kThreads float2), warp k
// sums value k and lane 0 writes it to out[k * stride] as a double-float pair.
template <int N>
__device__ __forceinline__ void rows_sum_df(const df (&v)[N], float2* s_rows, int nr, float2* out, int stride) {
  nr = nr < kThreads ? nr : kThreads;
  if ((int)threadIdx.x < nr) {
#pragma unroll
    for (int k = 0; k < N; ++k) s_rows[k * kThreads + threadIdx.x] = make_float2(v[k].hi, v[k].lo);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < N; k += kWarps) {
    df acc{0.f, 0.f};
    for (int t = lane; t < nr; t += 32) {
      const float2 x = s_rows[k * kThreads + t];
      df_add(acc, df{x.x, x.y});
    }
    acc = df_warp_sum(acc);
    if (lane == 0) out[(size_t)k * stride] = make_float2(acc.hi, acc.lo);
  }
}

// N per-row values summed over the CTA's rows in row order (deterministic): the
// rows' values go to shared memory s_rows (N x ld doubles, ld >= nrows), then
// warp k sums value k (lanes over rows, then a fixed shuffle tree) and writes
// out[k * stride].  Each warp reduces one value, so the FP64 adds of the N
// reductions run on all warps instead of one after the other on the warp that
// holds the rows.
template <int N>
__device__ __forceinline__ void rows_sum(const double (&v)[N], int tr, bool mine, int nrows, double* s_rows, int ld,
                                         double* out, int stride) {
  if (mine) {
#pragma unroll
    for (int k = 0; k < N; ++k) s_rows[k * ld + tr] = v[k];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < N; k += kWarps) {
    double acc = 0.0;
    for (int t = lane; t < nrows; t += 32) acc += s_rows[k * ld + t];
    acc = warp_sum(acc);
    if (lane == 0) out[(size_t)k * stride] = acc;
  }
}

// The scalar part of phase S, identical in every CTA, once the totals are in
// s_tot (Scal layout): the KKT residuals of Sec. 4.3 (readings R6, R7, R9), the
// duality gap, the stop test (R8) and the sigma rule of Sec. 4.4 (R5, R5b).
// Three independent chains run on lane 0 of warps 0, 1 and 2: the projection and
// the w quantities (FP64 where cancellation needs it: theta, ||w - u||^2, the
// eta_D3 expansion, ||w|| - R), the objectives and the gap, and the plain norms
// (FP32: they are compared with tol).  The maxima, the stop test and the sigma
// rule are FP32.  On this part a dependent FP64 operation takes 64 cycles and an
// FP64 compare with its select about 200, an FP64 division ~1400: the chain to
// theta uses one FP32 rsqrt seed and one FP64 Newton step, the expansions are in
// Horner form, and the sigma rule multiplies by the reciprocal factors.
// gs = 1 / (sigma sqrt(mu)).  s_ctl (15 doubles) receives theta, sigma and
// 1 / sigma of the next iteration; s_ictl receives done and the status;
// s_etaf[10] the kkt value.
// With `report` thread 0 also writes the residuals to ctrl (s_report).
struct SPhaseArgs {
  double C, kappa, R, mu, tau, sqmu, tol, sqrt_tol;
  float inv_den;
  int stop_rule;
  float tolf;        // the largest float <= tol (kkt <= tolf implies kkt <= tol)
};

// the largest float not above tol
__device__ __forceinline__ float float_at_most(double tol) {
  float t = (float)tol;
  if ((double)t > tol) t = nextafterf(t, 0.f);
  return t;
}

__device__ __forceinline__ void s_report(Ctrl* ctrl, double beta, const double* s_pd, const float* s_etaf) {
  ctrl->beta = beta;
  ctrl->pobj = s_pd[0];
  ctrl->dobj = s_pd[1];
  ctrl->kkt = s_etaf[10];
  ctrl->eta_gap = s_etaf[0];
  ctrl->eta_p1 = s_etaf[1];
  ctrl->eta_d1 = s_etaf[2];
  ctrl->eta_d2 = s_etaf[3];
  ctrl->eta_c1 = s_etaf[4];
  ctrl->eta_c2 = s_etaf[5];
  ctrl->eta_c3 = s_etaf[6];
  ctrl->eta_p2 = s_etaf[7];
  ctrl->eta_p3 = s_etaf[8];
  ctrl->eta_d3 = s_etaf[9];
  ctrl->wnorm = s_pd[3];
}

// vsums: the d-space sums are taken about the last iteration's theta_prev
// (S_GRHO = <y, g>, S_RHO2 = ||y||^2, y = (1 - theta_prev) g + gs rho; S_AG =
// <v, g>, S_A2 = ||v||^2, v = a - tau mu sigma (1 - theta_prev) g), so the
// small residuals are expanded in theta_prev - theta; otherwise they are
// <g, rho>, ||rho||^2, <a, g>, ||a||^2.
__device__ __forceinline__ void s_phase(const double* s_tot, const SPhaseArgs& q, double sig, double gs, int it,
                                        double beta, int status, bool report, Ctrl* ctrl, double* s_pd,
                                        float* s_etaf, double* s_ctl, int* s_ictl, double theta_prev = 1.0,
                                        bool vsums = false, int nsync = kThreads) {
  // nsync < kThreads: only the first nsync threads take part (named barrier 2)
  auto sync = [nsync]() {
    if (nsync >= kThreads) __syncthreads();
    else asm volatile("bar.sync 2, %0;" ::"r"(nsync) : "memory");
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 3 && lane < 7) {
    // 1 / sigma' for each value the sigma rule can give (sigma times 1, 1.1, 1.65,
    // 2.2 or their reciprocals): ready before the rule picks one
    const double m = lane == 0 ? 1.0 : lane == 1 ? 1.1 : lane == 2 ? 1.65 : lane == 3 ? 2.2
                   : lane == 4 ? (1.0 / 1.1) : lane == 5 ? (1.0 / 1.65) : (1.0 / 2.2);
    s_ctl[8 + lane] = rcp_nr(sig * m);
  }
  if (lane == 0 && warp == 1) {
    const double pobj = s_tot[S_PRIM_R] + q.C * s_tot[S_PRIM_XI];
    const double dobj = q.kappa * s_tot[S_DUAL_A] - q.R * sqrt_nr(s_tot[S_TA2]);
    s_pd[0] = pobj;
    s_pd[1] = dobj;
    s_etaf[0] = __fdividef(fabsf((float)(pobj - dobj)), 1.f + fabsf((float)pobj) + fabsf((float)dobj));   // gap
  } else if (lane == 0 && warp == 2) {
    s_etaf[1] = fsqrt_approx((float)s_tot[S_RES2]) * q.inv_den;       // p1
    s_etaf[2] = fsqrt_approx((float)s_tot[S_AMIN2]) * q.inv_den;      // dd1
    s_etaf[3] = fsqrt_approx((float)s_tot[S_AMAX2]) * q.inv_den;      // dd2
    s_etaf[4] = fabsf((float)s_tot[S_YA]) * q.inv_den;                // c1
    s_etaf[5] = fabsf((float)s_tot[S_XICA]) * q.inv_den;              // c2
    s_etaf[6] = fsqrt_approx((float)s_tot[S_AMS2]) * q.inv_den;       // c3
  } else if (threadIdx.x == 0) {
    const double S1 = s_tot[S_G2];                                       // ||g||^2
    // Step 2 projection: theta = min(1, R / ||g||), R / ||g|| = R rsqrt(S1)
    const double r0 = (double)rsqrt_approx((float)S1);
    const double rs = r0 * fma(-0.5 * S1, r0 * r0, 1.5);
    const double th = (S1 <= q.R * q.R) ? 1.0 : q.R * rs;
    double w2, wu2, d3;
    if (vsums) {
      const double YG = s_tot[S_GRHO], Y2 = s_tot[S_RHO2];
      const double eps = theta_prev - th;
      w2 = fma(theta_prev, fma(theta_prev, S1, 2.0 * YG), Y2);          // ||y + theta_prev g||^2 = ||w||^2
      wu2 = fma(eps, fma(eps, S1, 2.0 * YG), Y2);                        // ||y + eps g||^2 = ||w - u+||^2
      const double dlt = (q.tau * q.mu) * sig * eps;                     // kap - khat
      d3 = fma(dlt, fma(dlt, S1, -2.0 * s_tot[S_AG]), s_tot[S_A2]);      // ||v - dlt g||^2 = ||a - kap g||^2
    } else {
      const double t2 = 2.0 * gs * s_tot[S_GRHO], t3 = gs * gs * s_tot[S_RHO2];
      w2 = S1 + t2 + t3;                                                 // ||w||^2
      const double om = 1.0 - th;
      wu2 = fma(om, fma(om, S1, t2), t3);                                // ||w - u+||^2
      const double kap = (q.tau * q.mu) * sig * om;
      d3 = fma(kap, fma(kap, S1, -2.0 * s_tot[S_AG]), s_tot[S_A2]);      // ||a - kap g||^2
    }
    const float wnf = fsqrt_approx((float)w2);
    const double wmr = (w2 - q.R * q.R) * (double)rcp_approx(wnf + (float)q.R);   // ||w|| - R
    s_pd[2] = th;
    s_pd[3] = (double)wnf;
    s_etaf[7] = fsqrt_approx((float)q.mu * (float)wu2) * q.inv_den;   // p2 (a rounding-negative square gives 0)
    s_etaf[8] = fmaxf((float)wmr, 0.f) * q.inv_den;                   // p3
    s_etaf[9] = fsqrt_approx((float)d3) * q.inv_den;                  // dd3
  }
  sync();
  if (threadIdx.x == 0) {
    const float gap = s_etaf[0], p1 = s_etaf[1], dd1 = s_etaf[2], dd2 = s_etaf[3], c1 = s_etaf[4], c2 = s_etaf[5],
                c3 = s_etaf[6], p2 = s_etaf[7], p3 = s_etaf[8], dd3 = s_etaf[9];
    const float ep = fmaxf(p1, fmaxf(p2, p3)), ed = fmaxf(dd1, fmaxf(dd2, dd3)), ec = fmaxf(c1, fmaxf(c2, c3));
    const float kkt = fmaxf(fmaxf(ep, ed), fmaxf(ec, gap));
    int done = 0;
    double mult = 1.0;
    int mi = 0;   // index of mult among the candidates of 1 / sigma'
    if (!(kkt == kkt) || isinf(kkt)) {
      done = 1;
      status = GDWD_ENUMERIC;
    } else if (q.stop_rule == 0 ? kkt <= q.tolf
                                : (fmaxf(ep, ed) < q.tolf && fminf(ec, gap) < (float)q.sqrt_tol && fmaxf(ec, gap) < 0.05f)) {
      done = 1;
      status = GDWD_OK;
    } else if (it >= 1 && fminf(ep, ed) > 1e-3f * q.tolf) {                          // sigma rule, Sec. 4.4
      const float chi = __fdividef(ep, fmaxf(ed, 1e-30f));
      const float ichi = __fdividef(ed, fmaxf(ep, 1e-30f));
      const float big = fmaxf(chi, ichi);
      const int zk = big > 500.f ? 2 : (big > 50.f ? 1 : 0);
      if (chi > 5.f) {
        mult = zk == 2 ? 2.2 : (zk == 1 ? 1.65 : 1.1);
        mi = 1 + zk;
      } else if (ichi > 5.f) {
        mult = zk == 2 ? (1.0 / 2.2) : (zk == 1 ? (1.0 / 1.65) : (1.0 / 1.1));
        mi = 4 + zk;
      }
    }
    s_ctl[0] = s_pd[2];
    s_ctl[1] = sig * mult;
    s_ctl[2] = s_ctl[8 + mi];   // 1 / sigma'
    s_ictl[0] = done;
    s_ictl[1] = status;
    s_etaf[10] = kkt;
    if (report) s_report(ctrl, beta, s_pd, s_etaf);
  }
  sync();
}

// x_i = sum_j P_ij rhs_j for one row, one warp, double-float (result in all lanes).
// Every load reads inside the row: an index past npair is clamped to the last
// pair and its value then zeroed.
__device__ __forceinline__ void row_pair_load(const float4* P4, const float4* R4, int j, int npair, float4& p,
                                              float4& r) {
  const int jj = j < npair ? j : npair - 1;
  p = __ldg(P4 + jj);
  r = R4[jj];
  if (j >= npair) {
    p = make_float4(0.f, 0.f, 0.f, 0.f);
    r = p;
  }
}

__device__ __forceinline__ df row_dot(const float2* __restrict__ Prow, const float2* rhs_s, int npair) {
  const float4* P4 = reinterpret_cast<const float4*>(Prow);
  const float4* R4 = reinterpret_cast<const float4*>(rhs_s);
  df a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
  const int lane = threadIdx.x & 31;
  // blocks of 512 pairs: all sixteen loads of P and of the right-hand side of a
  // lane are issued before any product, so a row of up to 1024 columns costs
  // one L2 round trip
  for (int base = 0; base < npair; base += 512) {
    float4 p[16], r[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) row_pair_load(P4, R4, base + lane + 32 * u, npair, p[u], r[u]);
#pragma unroll
    for (int u = 0; u < 16; u += 2) {
      df_fma(a0, df{p[u].x, p[u].y}, df{r[u].x, r[u].y});
      df_fma(a1, df{p[u].z, p[u].w}, df{r[u].z, r[u].w});
      df_fma(a2, df{p[u + 1].x, p[u + 1].y}, df{r[u + 1].x, r[u + 1].y});
      df_fma(a3, df{p[u + 1].z, p[u + 1].w}, df{r[u + 1].z, r[u + 1].w});
    }
  }
  df_add(a0, a1);
  df_add(a2, a3);
  df_add(a0, a2);
  return df_warp_sum(a0);
}

}  // namespace gdwd
