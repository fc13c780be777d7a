// Joint C-grid iteration: K values of C (K = 2 or 4) iterated in lock-step by
// one persistent cooperative kernel, so that each pass over Z serves all K
// instances.  The linear system eq-linsys does not depend on C or sigma
// (Sec. 3, Algorithm 1), so the instances share Z, G^{-1} and p and differ only
// in their ADMM state (r, xi, alpha, u, rho, sigma).  Every instance keeps its
// own sigma rule (Sec. 4.4) and its own stop test; a converged instance is
// frozen while the others continue.
//
// Per iteration, as in the single-instance kernel (see iterate.cu for the
// n-space reduction and for b_j = Z~^T g'_j without a pass of its own):
//   R   U_g from the column dots, deferred n-space updates, b_j, rhs1_j
//   N1  x-bar_j = G^{-1} rhs1_j (one read of each G^{-1} row for all j), Step 1b
//   N2  x_j, beta_j, c_j, Steps 2-3, (G - I) c_j, n-space sums
//   B   K deferred d-updates, Z~ [c_1 .. c_K], Z~ [alpha_1 .. alpha_K] and, every
//       dots_every-th iteration, the column dots Z~^T [u_1 .. u_K] (the one Z
//       read), d-space sums
//   S   per-instance KKT, sigma rule, stop test
#include <algorithm>
#include <mutex>

#include "nspace.cuh"

namespace gdwd {

constexpr int kMaxStagesM = 8;

// two consecutive stored elements -> compute type
__device__ __forceinline__ void load2(const double* p, double* v) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  v[0] = x.x;
  v[1] = x.y;
}
__device__ __forceinline__ void load2(const float* p, float* v) {
  const float2 x = *reinterpret_cast<const float2*>(p);
  v[0] = x.x;
  v[1] = x.y;
}
__device__ __forceinline__ void load2(const __nv_bfloat16* p, float* v) {
  bf16x2_to_float(*reinterpret_cast<const uint32_t*>(p), v);
}
__device__ __forceinline__ void load2(const __half* p, float* v) {
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(p));
  v[0] = f.x;
  v[1] = f.y;
}
__device__ __forceinline__ void load2(const __nv_fp8_e4m3* p, float* v) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(*reinterpret_cast<const __nv_fp8x2_storage_t*>(p), __NV_E4M3);
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h));
  v[0] = f.x;
  v[1] = f.y;
}

// pass A for K right-hand sides; each thread covers two columns per round so
// that every vector read from shared memory serves two Z vectors
template <typename T, int K>
struct PassAK {
  using CT = typename ElemTraits<T>::compute_t;
  static constexpr int VEC = ElemTraits<T>::kVec;
  const CT* gp;
  int gstride;
  CT* partial;
  int TB, NB, Q;
  int64_t n;

  __device__ void chunk(const T* buf, int k, int s, int col0, int cw) {
    const int h = threadIdx.x & 7, cl = threadIdx.x >> 3;
    for (int c0 = 0; c0 < cw; c0 += 2 * (kThreads / 8)) {
      const int ca = c0 + cl, cb = ca + kThreads / 8;
      const bool va = ca < cw, vb = cb < cw;
      CT acc[2][K];
#pragma unroll
      for (int j = 0; j < K; ++j) acc[0][j] = acc[1][j] = 0;
      const T* pa = buf + (size_t)(va ? ca : 0) * TB;
      const T* pb = buf + (size_t)(vb ? cb : 0) * TB;
      for (int v = h; v < Q; v += 8) {
        CT ea[VEC], eb[VEC];
        ElemTraits<T>::load(pa + v * VEC, ea);
        ElemTraits<T>::load(pb + v * VEC, eb);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          CT gv[VEC];
          load_ct<VEC>(gp + (size_t)j * gstride + (size_t)k * TB + v * VEC, gv);
#pragma unroll
          for (int kk = 0; kk < VEC; ++kk) {
            acc[0][j] = fma(ea[kk], gv[kk], acc[0][j]);
            acc[1][j] = fma(eb[kk], gv[kk], acc[1][j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          CT x = acc[c][j];
          x += __shfl_xor_sync(0xffffffffu, x, 4);
          x += __shfl_xor_sync(0xffffffffu, x, 2);
          x += __shfl_xor_sync(0xffffffffu, x, 1);
          acc[c][j] = x;
        }
        if (h == 0) {
          if (va) partial[((size_t)j * n + col0 + ca) * NB + s] = acc[0][j];
          if (vb) partial[((size_t)j * n + col0 + cb) * NB + s] = acc[1][j];
        }
      }
    }
  }
  __device__ void end_slab(int, int) {}
};

// pass-B row epilogue for instance j (compile-time j after unrolling)
template <int K>
struct EpiK {
  double* g;
  const double* u;
  const double* rho;
  int64_t dpad;
  double inv_mu, a_coef;
  double sums[K][6];
  template <int J>
  __device__ void row(int64_t gj, double t, double ta) {
    const int64_t idx = (int64_t)J * dpad + gj;
    const double gv = u[idx] - t * inv_mu;
    const double rj = rho[idx];
    const double aj = ta + a_coef * rj;
    g[idx] = gv;
    sums[J][0] = fma(gv, gv, sums[J][0]);
    sums[J][1] = fma(gv, rj, sums[J][1]);
    sums[J][2] = fma(rj, rj, sums[J][2]);
    sums[J][3] = fma(aj, aj, sums[J][3]);
    sums[J][4] = fma(aj, gv, sums[J][4]);
    sums[J][5] = fma(ta, ta, sums[J][5]);
  }
};

// pass B for K instances and, on the same chunks, the column dots Z~^T u_j
template <typename T, int K>
struct PassBAK;

// four consecutive stored elements (4-element aligned) -> compute type
__device__ __forceinline__ void load4r(const double* p, double* v) {
  const double2 x = *reinterpret_cast<const double2*>(p), y = *reinterpret_cast<const double2*>(p + 2);
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}
__device__ __forceinline__ void load4r(const float* p, float* v) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void load4r(const __nv_bfloat16* p, float* v) {
  const uint2 x = *reinterpret_cast<const uint2*>(p);
  bf16x2_to_float(x.x, v);
  bf16x2_to_float(x.y, v + 2);
}
__device__ __forceinline__ void load4r(const __half* p, float* v) {
  const uint2 x = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&x.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&x.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4r(const __nv_fp8_e4m3* p, float* v) {
  const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// the 2K pass-B coefficients of one column (sc c_j, then sc alpha_j), stored
// interleaved so that one column's are 16-byte vectors
template <int N>
__device__ __forceinline__ void load_coef(const float* p, float* v) {
#pragma unroll
  for (int k = 0; k < N; k += 4) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p + k));
    v[k] = x.x; v[k + 1] = x.y; v[k + 2] = x.z; v[k + 3] = x.w;
  }
}
template <int N>
__device__ __forceinline__ void load_coef(const double* p, double* v) {
#pragma unroll
  for (int k = 0; k < N; k += 2) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p + k));
    v[k] = x.x; v[k + 1] = x.y;
  }
}

// pass B for K instances x two right-hand sides (c_j, alpha_j).  Thread t owns
// rows 4q .. 4q+3 (q = t % Q4, Q4 = TB / 4) of the column group t / Q4, so the
// threads of a step read consecutive 4-element pieces of one column; the
// coefficients of a column are two (FP64: four) vector loads for all K; frozen
// instances are skipped.
template <typename T, int K>
struct PassBK {
  using CT = typename ElemTraits<T>::compute_t;
  const CT* coef;     // global [n][2K]
  double* red;        // shared 2 * G * TB
  int TB, Q4, G;
  int64_t n, d;
  unsigned act;       // bit j: instance j still iterating
  EpiK<K>* epi;
  RunAcc<CT> rc[K][4], ra[K][4];

  __device__ void chunk(const T* buf, int k, int s, int col0, int cw) {
    const int grp = threadIdx.x / Q4, q = threadIdx.x - grp * Q4;
    if (grp >= G) return;
    CT ac[K][4], aa[K][4];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) ac[j][r] = aa[j][r] = 0;
    const T* base = buf + 4 * q;
    int col = grp;
    // two columns per step: both columns' loads are in flight together
    for (; col + G < cw; col += 2 * G) {
      CT e0[4], e1[4], c0[2 * K], c1[2 * K];
      load4r(base + (size_t)col * TB, e0);
      load4r(base + (size_t)(col + G) * TB, e1);
      load_coef<2 * K>(coef + (size_t)(col0 + col) * 2 * K, c0);
      load_coef<2 * K>(coef + (size_t)(col0 + col + G) * 2 * K, c1);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        if (!(act & (1u << j))) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          ac[j][r] = fma(e0[r], c0[j], ac[j][r]);
          aa[j][r] = fma(e0[r], c0[K + j], aa[j][r]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          ac[j][r] = fma(e1[r], c1[j], ac[j][r]);
          aa[j][r] = fma(e1[r], c1[K + j], aa[j][r]);
        }
      }
    }
    if (col < cw) {
      CT e[4], cf[2 * K];
      load4r(base + (size_t)col * TB, e);
      load_coef<2 * K>(coef + (size_t)(col0 + col) * 2 * K, cf);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        if (!(act & (1u << j))) continue;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          ac[j][r] = fma(e[r], cf[j], ac[j][r]);
          aa[j][r] = fma(e[r], cf[K + j], aa[j][r]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (!(act & (1u << j))) continue;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        rc[j][r].fold(ac[j][r]);
        ra[j][r].fold(aa[j][r]);
      }
    }
  }

  template <int J>
  __device__ void finish_instance(int s) {
    if (!(act & (1u << J))) return;          // uniform across the CTA
    const int grp = threadIdx.x / Q4, q = threadIdx.x - grp * Q4;
    if (grp < G) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        red[(size_t)grp * TB + 4 * q + r] = rc[J][r].get();
        red[(size_t)(G + grp) * TB + 4 * q + r] = ra[J][r].get();
        rc[J][r].reset();
        ra[J][r].reset();
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < TB; j += blockDim.x) {
      double t = 0.0, ta = 0.0;
      for (int gq = 0; gq < G; ++gq) {
        t += red[(size_t)gq * TB + j];
        ta += red[(size_t)(G + gq) * TB + j];
      }
      const int64_t gj = (int64_t)s * TB + j;
      if (gj < d) epi->template row<J>(gj, t, ta);
    }
    __syncthreads();
  }

  __device__ void end_slab(int k, int s) {
    finish_instance<0>(s);
    if constexpr (K > 1) finish_instance<1>(s);
    if constexpr (K > 2) finish_instance<2>(s);
    if constexpr (K > 3) finish_instance<3>(s);
  }
};

template <typename T, int K>
struct PassBAK {
  PassBK<T, K>* b;
  PassAK<T, K>* a;
  __device__ void chunk(const T* buf, int k, int s, int col0, int cw) {
    b->chunk(buf, k, s, col0, cw);
    a->chunk(buf, k, s, col0, cw);
  }
  __device__ void end_slab(int k, int s) { b->end_slab(k, s); }
};

// K x N values per thread summed over the block; out[j * S_COUNT * grid + (k0 + k) * grid]
template <int K, int N>
__device__ __forceinline__ void block_sum_kn(const double (&v)[K][N], double* s_part, double* out, int grid,
                                             int k0) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double t = warp_sum(v[j][k]);
      if (l == 0) s_part[(w * K + j) * N + k] = t;
    }
  __syncthreads();
  for (int m = threadIdx.x; m < K * N; m += kThreads) {
    const int j = m / N, k = m - j * N;
    double t = 0.0;
    for (int i = 0; i < kWarps; ++i) t += s_part[(i * K + j) * N + k];
    out[((size_t)j * S_COUNT + k0 + k) * grid] = t;
  }
  __syncthreads();
}

template <typename T, int K>
__global__ void __launch_bounds__(kThreads, 1) iterate_multi_kernel(MultiArgs<typename ElemTraits<T>::compute_t> a,
                                                                    int stages, int stage_bytes) {
  using CT = typename ElemTraits<T>::compute_t;
  constexpr int VEC = ElemTraits<T>::kVec;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t s_bars[kMaxStagesM];
  __shared__ int s_flag, s_abort;
  __shared__ double s_red[2 * kWarps + 2];
  __shared__ double s_tot[K][S_COUNT];
  __shared__ double s_ctl[K][4];
  __shared__ double s_part[kWarps * K * 9];
  __shared__ float s_xh[K][kMaxRowsPerCta], s_xl[K][kMaxRowsPerCta];

  const Layout& L = a.L;
  const int cta = blockIdx.x, grid = a.grid;
  const int64_t n = L.n, d = L.d, dpad = a.dpad;
  const int TB = L.TB, NB = L.NB;
  const int Q = TB / VEC, Q4 = TB / 4;
  const int G4 = Q4 <= kThreads ? kThreads / Q4 : 1;
  const int nmy = (NB > cta) ? (NB - cta + grid - 1) / grid : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qcase = q_case(a.q);
  const double sqmu = sqrt(a.mu), inv_mu = 1.0 / a.mu;
  const double inv_q = 1.0 / a.q;
  const int64_t rpc = (n + grid - 1) / grid;
  const int64_t r0 = ((int64_t)cta * rpc < n) ? (int64_t)cta * rpc : n;
  const int nrows = (int)(((r0 + rpc < n) ? r0 + rpc : n) - r0);
  const int npair = (int)((n + 1) / 2);

  Ring rg;
  rg.buf = smem;
  rg.bars = s_bars;
  rg.stages = stages;
  rg.stage_bytes = stage_bytes;
  uint8_t* uni = smem + (size_t)stages * stage_bytes;
  if (threadIdx.x == 0) s_abort = 0;
  ring_init(rg);

  unsigned gen = 0;
  double sig[K], sig_prev[K], theta[K], beta[K];
  int status[K], iters[K];
  unsigned act = 0;
  int pending = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    sig[j] = a.ctrl[j].sigma;
    sig_prev[j] = a.ctrl[j].sigma_prev;
    theta[j] = a.ctrl[j].theta;
    beta[j] = 0.0;
    status[j] = GDWD_EMAXITER;
    iters[j] = 0;
    if (j < a.K) act |= 1u << j;
  }

  // per-phase timing by CTA 0, thread 0 (same slots as the single-instance kernel)
  __shared__ unsigned long long s_tacc[kPhaseSlots], s_tprev;
  const bool timing = (cta == 0 && threadIdx.x == 0);
  if (timing) {
    for (int k = 0; k < kPhaseSlots; ++k) s_tacc[k] = 0;
    s_tprev = globaltimer();
  }
#define MMARK(k)                           \
  do {                                     \
    if (timing) {                          \
      const uint64_t t_ = globaltimer();   \
      s_tacc[k] += t_ - s_tprev;           \
      s_tprev = t_;                        \
    }                                      \
  } while (0)
#define MBARRIER(k)                                                                       \
  do {                                                                                    \
    MMARK(k);                                                                             \
    if (!grid_barrier(a.bar, (unsigned)grid, gen, a.err, a.timeout_ns, &s_flag)) {       \
      ring_drain_prefetched(rg, a.err, a.timeout_ns);                                     \
      return;                                                                             \
    }                                                                                     \
    MMARK(k + 1);                                                                         \
  } while (0)

  // initial iterate: u = rho = 0, so Z~^T u = Z~^T rho = 0
  for (int m = threadIdx.x; m < K * nrows; m += kThreads) {
    const int j = m / nrows, t = m - j * nrows;
    a.Ur[(int64_t)j * n + r0 + t] = 0.0;
    a.Uu[(int64_t)j * n + r0 + t] = 0.0;
  }
  __syncthreads();

  float2* rhs_s = reinterpret_cast<float2*>(uni);
  const int rstride = 2 * npair;
  float* s_redf = reinterpret_cast<float*>(s_red);
  int it = 0;
  bool dots_prev = false;   // the last pass B took the column dots
  for (; it < a.max_iter && act && __popc(act) >= a.min_active; ++it) {
    ring_prefetch(L, rg, cta, grid);   // this iteration's first Z chunks arrive during R, N1, N2
    // ---------------- R (this CTA's rows, every active instance): U_g from the
    // pass-B column dots and (G - I) c, the deferred n-space update, b, rhs1
    // (see iterate.cu)
    for (int m = warp; m < K * nrows; m += kWarps) {
      const int j = m / nrows, t = m - j * nrows;
      if (!(act & (1u << j))) continue;
      const int64_t i = r0 + t, idx = (int64_t)j * n + i;
      double ug = 0.0;
      if (pending && dots_prev) {
        const CT* pp = a.partial + (size_t)idx * NB;
        double bsum;
        if constexpr (sizeof(CT) == 8) {
          double acc = 0.0;
          for (int s2 = lane; s2 < NB; s2 += 32) acc += (double)pp[s2];
          bsum = warp_sum(acc);
        } else {
          df acc{0.f, 0.f};
          for (int s2 = lane; s2 < NB; s2 += 32) df_add(acc, (float)pp[s2]);
          bsum = df_to_double(df_warp_sum(acc));
        }
        ug = a.sc[i] * bsum;
      }
      if (lane == 0) {
        double uu = a.Uu[idx], ur = a.Ur[idx];
        if (pending) {
          const double rcoef = a.tau * sig_prev[j] * sqmu * (1.0 - theta[j]);
          ug = (dots_prev ? ug : uu) - a.kc[idx];
          uu = theta[j] * ug;
          ur = (1.0 - a.tau) * ur - rcoef * ug;
          a.Uu[idx] = uu;
          a.Ur[idx] = ur;
        }
        const double bi = uu + ur * rcp_nr(sig[j] * sqmu);
        a.b[idx] = bi;
        const double v = a.xi[idx] - a.r[idx] - a.alpha[idx] * rcp_nr(sig[j]);
        const df r1 = df_from(bi + v);
        a.rhsA[idx] = make_float2(r1.hi, r1.lo);
      }
    }
    MBARRIER(2);

    // ---------------- N1 and N2 share the structure: load K right-hand sides,
    // beta_j = -p^T rhs_j / s, rows of G^{-1} against all K, per-row work
    for (int phase = 0; phase < 2; ++phase) {
      const float2* src = phase == 0 ? a.rhsA : a.rhsB;
      for (int64_t m = threadIdx.x; m < (int64_t)K * rstride; m += kThreads) {
        const int j = (int)(m / rstride);
        const int64_t i = m - (int64_t)j * rstride;
        rhs_s[m] = i < n ? src[(size_t)j * n + i] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      double bet[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        df pd{0.f, 0.f};
        for (int64_t i = threadIdx.x; i < n; i += kThreads) {
          const float2 pv = a.pdf[i];
          const float2 rv = rhs_s[(size_t)j * rstride + i];
          df_fma(pd, df{pv.x, pv.y}, df{rv.x, rv.y});
        }
        bet[j] = -df_to_double(block_sum_df(pd, s_redf)) * a.inv_s;
      }
      for (int t = warp; t < nrows; t += kWarps) {
        const float4* P4 = reinterpret_cast<const float4*>(a.P + (size_t)(r0 + t) * a.ldP);
        df acc[K][2];
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j][0] = acc[j][1] = df{0.f, 0.f};
        for (int jj = lane; jj < npair; jj += 32) {
          const float4 pv = __ldg(P4 + jj);
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const float4 rv = reinterpret_cast<const float4*>(rhs_s + (size_t)j * rstride)[jj];
            df_fma(acc[j][0], df{pv.x, pv.y}, df{rv.x, rv.y});
            df_fma(acc[j][1], df{pv.z, pv.w}, df{rv.z, rv.w});
          }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
          df_add(acc[j][0], acc[j][1]);
          const df x = df_warp_sum(acc[j][0]);
          if (lane == 0) {
            s_xh[j][t] = x.hi;
            s_xl[j][t] = x.lo;
          }
        }
      }
      __syncthreads();
      if (phase == 0) {
        for (int m = threadIdx.x; m < K * nrows; m += kThreads) {
          const int j = m / nrows, t = m - j * nrows;
          if (!(act & (1u << j))) continue;
          const int64_t i = r0 + t, idx = (int64_t)j * n + i;
          const double inv_sig = rcp_nr(sig[j]);
          const double cbar = ((double)s_xh[j][t] + (double)s_xl[j][t]) + bet[j] * a.p[i];
          const double ri = a.r[idx];
          const double rn = prox_root(cbar + ri, a.omega[i] * inv_sig, a.q, qcase, ri);
          a.r[idx] = rn;
          const double v = a.xi[idx] - rn - a.alpha[idx] * inv_sig;
          const df r2 = df_from(a.b[idx] + v);
          a.rhsB[idx] = make_float2(r2.hi, r2.lo);
        }
        MBARRIER(4);
      } else {
        double sums[K][9];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
          for (int k = 0; k < 9; ++k) sums[j][k] = 0.0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          beta[j] = bet[j];
          if (!(act & (1u << j))) continue;
          const double inv_sig = rcp_nr(sig[j]);
          for (int t = threadIdx.x; t < nrows; t += kThreads) {
            const int64_t i = r0 + t, idx = (int64_t)j * n + i;
            const double xv = (double)s_xh[j][t] + (double)s_xl[j][t];
            const double c = xv + bet[j] * a.p[i];
            const double ri = a.r[idx], al = a.alpha[idx], yi = a.y[i], ce = a.C[j] * a.e[i];
            const double v = a.xi[idx] - ri - al * inv_sig;
            const double zw = c - v - yi * bet[j];
            const double xin = fmax(0.0, ri - zw - yi * bet[j] + (al - ce) * inv_sig);
            const double res = zw + yi * bet[j] + xin - ri;
            const double an = al - a.tau * sig[j] * res;
            a.xi[idx] = xin;
            a.alpha[idx] = an;
            a.coef[(size_t)i * 2 * K + j] = (CT)(a.sc[i] * c);
            a.coef[(size_t)i * 2 * K + K + j] = (CT)(a.sc[i] * an);
            const float2 rv = rhs_s[(size_t)j * rstride + i];
            a.kc[idx] = ((double)rv.x + (double)rv.y) - xv + bet[j] * (yi - a.p[i]);   // (G - I) c
            const double rq1 = pow_q1(ri, a.q, qcase);
            const double irq1 = rcp_nr(rq1);
            const double om = a.omega[i];
            sums[j][0] = fma(res, res, sums[j][0]);
            sums[j][1] = fma(yi, an, sums[j][1]);
            sums[j][2] = fma(xin, ce - an, sums[j][2]);
            const double dv = an - om * irq1;
            sums[j][3] = fma(dv, dv, sums[j][3]);
            const double mn = fmin(0.0, an), mx = fmax(0.0, an - ce);
            sums[j][4] = fma(mn, mn, sums[j][4]);
            sums[j][5] = fma(mx, mx, sums[j][5]);
            sums[j][6] += om * inv_q * ri * irq1;
            sums[j][7] = fma(a.e[i], xin, sums[j][7]);
            sums[j][8] += dual_pow(a.wt[i] * an, a.q, qcase);
          }
        }
        block_sum_kn<K, 9>(sums, s_part, a.scal + cta, grid, 0);
        MBARRIER(6);
      }
    }

    // ---------------- B (the one Z read): K deferred d-updates, Z~ [c_1 .. c_K],
    // Z~ [alpha_1 .. alpha_K], d-space sums, column dots Z~^T [u_1 .. u_K]
    {
      const int gstride = nmy * TB;
      double* red = reinterpret_cast<double*>(uni);
      CT* up = reinterpret_cast<CT*>(uni + (size_t)2 * G4 * TB * sizeof(double));
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const bool on = act & (1u << j);
        const double rcoef = a.tau * sig_prev[j] * sqmu * (1.0 - theta[j]);
        for (int k = 0; k < nmy; ++k) {
          const int64_t s = cta + (int64_t)k * grid;
          for (int jl = threadIdx.x; jl < TB; jl += kThreads) {
            const int64_t gj = s * TB + jl;
            double uj = 0.0;
            if (on && gj < d) {
              const int64_t idx = (int64_t)j * dpad + gj;
              if (pending) {
                const double gv = a.g[idx];
                a.rho[idx] = (1.0 - a.tau) * a.rho[idx] - rcoef * gv;
                uj = theta[j] * gv;
                a.u[idx] = uj;
              } else {
                uj = a.u[idx];
              }
            }
            up[(size_t)j * gstride + (size_t)k * TB + jl] = (CT)uj;
          }
        }
      }
      __syncthreads();
      EpiK<K> epi;
      epi.g = a.g;
      epi.u = a.u;
      epi.rho = a.rho;
      epi.dpad = dpad;
      epi.inv_mu = inv_mu;
      epi.a_coef = sqmu * (1.0 - a.tau);
#pragma unroll
      for (int j = 0; j < K; ++j)
#pragma unroll
        for (int k = 0; k < 6; ++k) epi.sums[j][k] = 0.0;
      PassBK<T, K> pb;
      pb.coef = a.coef;
      pb.red = red;
      pb.TB = TB;
      pb.Q4 = Q4;
      pb.G = G4;
      pb.n = n;
      pb.d = d;
      pb.act = act;
      pb.epi = &epi;
#pragma unroll
      for (int j = 0; j < K; ++j)
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          pb.rc[j][x].reset();
          pb.ra[j][x].reset();
        }
      dots_prev = (it % a.dots_every) == a.dots_every - 1;
      if (dots_prev) {
        PassAK<T, K> pa{up, gstride, a.partial, TB, NB, Q, n};
        PassBAK<T, K> pba{&pb, &pa};
        if (!stream_slabs<T>(L, rg, cta, grid, a.err, a.timeout_ns, &s_abort, pba)) return;
      } else {
        if (!stream_slabs<T>(L, rg, cta, grid, a.err, a.timeout_ns, &s_abort, pb)) return;
      }
      block_sum_kn<K, 6>(epi.sums, s_part, a.scal + cta, grid, S_G2);
    }
    MBARRIER(8);

    // ---------------- S: per-instance totals, KKT, sigma rule, stop test
    for (int m = warp; m < K * (S_COUNT - 1); m += kWarps) {
      const int j = m / (S_COUNT - 1), k = m - j * (S_COUNT - 1);
      double acc = 0.0;
      for (int c2 = lane; c2 < grid; c2 += 32) acc += a.scal[((size_t)j * S_COUNT + k) * grid + c2];
      acc = warp_sum(acc);
      if (lane == 0) s_tot[j][k] = acc;
    }
    __syncthreads();
    MMARK(13);
    if (threadIdx.x < K && (act & (1u << threadIdx.x))) {
      const int j = threadIdx.x;
      const double* tt = s_tot[j];
      const double den = 1.0 + a.C[j];
      const float inv_den = (float)(1.0 / den);
      const double S1 = tt[S_G2], S2 = tt[S_GRHO], S3 = tt[S_RHO2];
      const double gs = rcp_nr(sig[j] * sqmu);
      const double gnorm = sqrt_nr(S1);
      const double th = (gnorm <= a.R) ? 1.0 : div_nr(a.R, gnorm);
      const double w2 = fmax(0.0, S1 + 2.0 * gs * S2 + gs * gs * S3);
      const double om = 1.0 - th;
      const double wu2 = fmax(0.0, om * om * S1 + 2.0 * om * gs * S2 + gs * gs * S3);
      const double kap = a.tau * sig[j] * a.mu * om;
      const double d3 = fmax(0.0, tt[S_A2] - 2.0 * kap * tt[S_AG] + kap * kap * S1);
      const float wnf = sqrtf((float)w2);
      const double wmr = (w2 - a.R * a.R) * (double)(1.0f / (wnf + (float)a.R));
      const double p1 = sqrtf((float)tt[S_RES2]) * inv_den;
      const double p2 = sqrtf((float)(a.mu * wu2)) * inv_den;
      const double p3 = fmax(wmr, 0.0) * inv_den;
      const double dd1 = sqrtf((float)tt[S_AMIN2]) * inv_den;
      const double dd2 = sqrtf((float)tt[S_AMAX2]) * inv_den;
      const double dd3 = sqrtf((float)d3) * inv_den;
      const double c1 = fabs(tt[S_YA]) * inv_den;
      const double c2 = fabs(tt[S_XICA]) * inv_den;
      const double c3 = sqrtf((float)tt[S_AMS2]) * inv_den;
      const double pobj = tt[S_PRIM_R] + a.C[j] * tt[S_PRIM_XI];
      const double dobj = a.kappa * tt[S_DUAL_A] - a.R * sqrt_nr(tt[S_TA2]);
      const double gap = (double)((float)fabs(pobj - dobj) / (float)(1.0 + fabs(pobj) + fabs(dobj)));
      const double ep = fmax(p1, fmax(p2, p3)), ed = fmax(dd1, fmax(dd2, dd3)), ec = fmax(c1, fmax(c2, c3));
      const double kkt = fmax(fmax(ep, ed), fmax(ec, gap));
      double done = 0.0, stat = GDWD_EMAXITER;
      double sig_next = sig[j];
      if (!(kkt == kkt) || isinf(kkt)) {
        done = 1.0;
        stat = GDWD_ENUMERIC;
      } else if (a.stop_rule == 0 ? kkt <= a.tol
                                  : (fmax(ep, ed) < a.tol && fmin(ec, gap) < sqrt_nr(a.tol) &&
                                     fmax(ec, gap) < 0.05)) {
        done = 1.0;
        stat = GDWD_OK;
      } else if (it >= 1 && fmin(ep, ed) > 1e-3 * a.tol) {
        const float chi = (float)ep / fmaxf((float)ed, 1e-30f);
        const float ichi = (float)ed / fmaxf((float)ep, 1e-30f);
        const float big = fmaxf(chi, ichi);
        const double zeta = big > 500.f ? 2.2 : (big > 50.f ? 1.65 : 1.1);
        if (chi > 5.f) sig_next = sig[j] * zeta;
        else if (ichi > 5.f) sig_next = sig[j] / zeta;
      }
      s_ctl[j][0] = th;
      s_ctl[j][1] = sig_next;
      s_ctl[j][2] = done;
      s_ctl[j][3] = stat;
      if (cta == 0) {
        Ctrl* c = a.ctrl + j;
        c->beta = beta[j];
        c->pobj = pobj;
        c->dobj = dobj;
        c->kkt = kkt;
        c->eta_p1 = p1; c->eta_p2 = p2; c->eta_p3 = p3;
        c->eta_d1 = dd1; c->eta_d2 = dd2; c->eta_d3 = dd3;
        c->eta_c1 = c1; c->eta_c2 = c2; c->eta_c3 = c3;
        c->eta_gap = gap;
        c->wnorm = (double)wnf;
        // the iterate this control block describes: the d-update of this
        // iteration is still pending and uses sigma and theta
        c->sigma = sig_next;
        c->sigma_prev = sig[j];
        c->theta = th;
        c->pending = 1;
        c->it = it + 1;
        c->status = (int)stat;
      }
    }
    __syncthreads();
    MMARK(10);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (!(act & (1u << j))) continue;
      sig_prev[j] = sig[j];
      theta[j] = s_ctl[j][0];
      sig[j] = s_ctl[j][1];
      iters[j] = it + 1;
      status[j] = (int)s_ctl[j][3];
      if (s_ctl[j][2] != 0.0) act &= ~(1u << j);
    }
    pending = 1;
  }
  if (cta == 0 && threadIdx.x == 0) {
    for (int j = 0; j < K; ++j) a.ctrl[j].done = 1;
    for (int k = 0; k < kPhaseSlots; ++k) a.ctrl[0].phase_ns[k] = (double)s_tacc[k];
  }
#undef MBARRIER
#undef MMARK
}

template <typename T>
static size_t union_bytes_multi(const Layout& L, int grid, int K) {
  const int Q4 = L.TB / 4;
  const int G4 = Q4 <= kThreads ? kThreads / Q4 : 1;
  using CT = typename ElemTraits<T>::compute_t;
  const int nmy = (L.NB + grid - 1) / grid;
  const size_t n_bytes = (size_t)K * ((L.n + 1) / 2) * 2 * sizeof(float2);
  const size_t b_bytes = (size_t)2 * G4 * L.TB * sizeof(double) + (size_t)K * nmy * L.TB * sizeof(CT);
  return (std::max(n_bytes, b_bytes) + 127) & ~(size_t)127;
}

template <auto Kern>
static cudaError_t ensure_max_dyn_smem_m() {
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

template <typename T, int K>
static cudaError_t run_multi_tk(const MultiArgs<typename ElemTraits<T>::compute_t>& args, int smem_limit,
                                cudaStream_t st) {
  if (args.L.TB / 2 > kThreads) return cudaErrorInvalidConfiguration;
  const size_t ub = union_bytes_multi<T>(args.L, args.grid, K);
  const int stage_bytes = (int)(((size_t)args.L.CW * args.L.TB * args.L.esize + 127) & ~(size_t)127);
  const int64_t avail = (int64_t)smem_limit - (int64_t)ub - 1024;
  if (avail < 2 * (int64_t)stage_bytes) return cudaErrorInvalidConfiguration;
  int stages = (int)std::min<int64_t>(kMaxStagesM, avail / stage_bytes);
  const size_t smem = (size_t)stages * stage_bytes + ub;
  cudaError_t e = ensure_max_dyn_smem_m<iterate_multi_kernel<T, K>>();
  if (e != cudaSuccess) return e;
  auto kern = iterate_multi_kernel<T, K>;
  MultiArgs<typename ElemTraits<T>::compute_t> a2 = args;
  void* params[] = {(void*)&a2, (void*)&stages, (void*)&stage_bytes};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(args.grid), dim3(kThreads), params, smem, st);
}

template <typename T>
static cudaError_t run_multi_t(int K, const MultiArgs<typename ElemTraits<T>::compute_t>& a, int smem_limit,
                               cudaStream_t st) {
  return K <= 2 ? run_multi_tk<T, 2>(a, smem_limit, st) : run_multi_tk<T, 4>(a, smem_limit, st);
}

// the largest K (2 or 4) whose per-instance shared buffers fit next to two stages
int multi_max_k(int store, const Layout& L, int grid, int smem_limit) {
  auto fits = [&](int K) {
    size_t ub;
    switch (store) {
      case GDWD_F64: ub = union_bytes_multi<double>(L, grid, K); break;
      case GDWD_BF16: ub = union_bytes_multi<__nv_bfloat16>(L, grid, K); break;
      case GDWD_F16: ub = union_bytes_multi<__half>(L, grid, K); break;
      case GDWD_E4M3: ub = union_bytes_multi<__nv_fp8_e4m3>(L, grid, K); break;
      default: ub = union_bytes_multi<float>(L, grid, K); break;
    }
    const int64_t stage = ((int64_t)L.CW * L.TB * L.esize + 127) & ~(int64_t)127;
    return (int64_t)smem_limit - (int64_t)ub - 1024 >= 2 * stage && L.TB / 4 <= kThreads &&
           (L.n + grid - 1) / grid <= kMaxRowsPerCta;
  };
  return fits(4) ? 4 : fits(2) ? 2 : 1;
}

cudaError_t run_multi_f64(int K, const MultiArgs<double>& a, int smem_limit, cudaStream_t st) {
  return run_multi_t<double>(K, a, smem_limit, st);
}

cudaError_t run_multi_f32(int store, int K, const MultiArgs<float>& a, int smem_limit, cudaStream_t st) {
  switch (store) {
    case GDWD_BF16: return run_multi_t<__nv_bfloat16>(K, a, smem_limit, st);
    case GDWD_F16: return run_multi_t<__half>(K, a, smem_limit, st);
    case GDWD_E4M3: return run_multi_t<__nv_fp8_e4m3>(K, a, smem_limit, st);
    default: return run_multi_t<float>(K, a, smem_limit, st);
  }
}

}  // namespace gdwd
