// The direct solver of Sec. 3.3.1 (T = 0, d << n): eq-linsys is solved in
// d-space through the (d+1) x (d+1) matrix A = [[M, Z~y], [(Z~y)^T, n]],
// M = Z~ Z~^T + mu I.  The set-up stores Z^T (FP32 or FP64) in the slab layout
// (samples as rows, features as columns), so the SIMT Gram of that storage is
// Z~ Z~^T, and factors G' = M / mu = I + Z~ Z~^T / mu with the same blocked
// Cholesky and inverse as the SMW path, with y replaced by b^ = Z~ y.  The
// border of A is then eliminated in closed form (a Schur complement):
//     beta = (h_beta - p^T h_w / mu) / (n - s / mu),   w = (P h_w - p beta) / mu,
// with P = G'^{-1}, p = P b^ and s = b^T p.
//
// One iteration (Algorithm 1) is a stream of kernels, each a no-op once the
// control block says the solve is done:
//   rhs -> G'^{-1} rows -> w-bar, beta-bar -> Z~^T w-bar (streaming pass) ->
//   Step 1b prox per sample -> Z~ dr (streaming pass) -> rhs -> G'^{-1} rows ->
//   w, beta -> Z~^T w -> Steps 2-3 per sample, n-space KKT sums ->
//   Z~ (xi - r), Z~ alpha (streaming passes) -> phase S (d-space norms, KKT,
//   sigma rule, the u / rho update).
// The d-space products use the identities h_w = mu g' - Z~ v with
// Z~ v = Z~ (xi - r) - Z~ alpha / sigma, the first two carried from the last
// iteration's pass and corrected by Z~ (r+ - r) after the prox (Step 1c).
#include <algorithm>

#include "direct.cuh"
#include "nspace.cuh"

namespace gdwd {


__global__ void transpose_kernel_f32(const float* __restrict__ in, int64_t d, int64_t n, int64_t ld, float* out) {
  __shared__ float t[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = j0 + threadIdx.x, i = i0 + k;
    if (j < d && i < n) t[k][threadIdx.x] = in[j + i * ld];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + threadIdx.x, j = j0 + k;
    if (j < d && i < n) out[i + j * n] = t[threadIdx.x][k];
  }
}

__global__ void transpose_kernel_f64(const double* __restrict__ in, int64_t d, int64_t n, int64_t ld, double* out) {
  __shared__ double t[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = j0 + threadIdx.x, i = i0 + k;
    if (j < d && i < n) t[k][threadIdx.x] = in[j + i * ld];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = i0 + threadIdx.x, j = j0 + k;
    if (j < d && i < n) out[i + j * n] = t[threadIdx.x][k];
  }
}

cudaError_t run_transpose(const void* Z, int zdt, int64_t d, int64_t n, int64_t ld, void* out, cudaStream_t st) {
  const dim3 grid((unsigned)((d + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  if (zdt == GDWD_F64)
    transpose_kernel_f64<<<grid, block, 0, st>>>((const double*)Z, d, n, ld, (double*)out);
  else
    transpose_kernel_f32<<<grid, block, 0, st>>>((const float*)Z, d, n, ld, (float*)out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The two products with the stored Z^T (slab layout, samples as rows): the
// direct solver's passes accumulate in double-float (FP32 storage) or FP64, so
// that sums over many samples keep their digits at d << n.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void acc_prod(df& acc, T z, df x);
template <>
__device__ __forceinline__ void acc_prod<float>(df& acc, float z, df x) {
  df_fma(acc, df{z, 0.f}, x);
}

// out_i = sum_j Z~_ji x_j (= Z~^T x) for every sample i: one thread per sample,
// reading its slab row across the d columns (consecutive threads, consecutive
// rows: coalesced)
// xs_j = sc_j x_j (double-float for FP32 storage, FP64 otherwise)
__global__ void dir_scale_kernel(const double* x, const double* sc, int64_t d, int f64, void* xs) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
    const double v = sc[j] * x[j];
    if (f64) {
      reinterpret_cast<double*>(xs)[j] = v;
    } else {
      const df t = df_from(v);
      reinterpret_cast<float2*>(xs)[j] = make_float2(t.hi, t.lo);
    }
  }
}

// FP32: a block takes 64 quads of consecutive samples (the slab height is a
// multiple of 4, so a column's quad is one 16-byte load and a warp reads 512
// contiguous bytes) and splits the d columns over blockDim / 64 groups (1 or
// 4; 4 when there are too few quads to fill the GPU), whose double-float
// partials are added in a fixed order.
constexpr int kRowQuads = 64, kRowGroups = 4;

__global__ void __launch_bounds__(kRowQuads * kRowGroups) dir_rowdot_f32(Layout L, const float2* __restrict__ xs,
                                                                         double* out) {
  const int ng = blockDim.x / kRowQuads;
  __shared__ float2 s_acc[kRowGroups][4][kRowQuads];
  const int64_t n = L.d, d = L.n;
  const int64_t qps = L.TB / 4;                       // quads per slab
  const int64_t nq = (int64_t)L.NB * qps;
  const int tq = threadIdx.x % kRowQuads, cg = threadIdx.x / kRowQuads;
  for (int64_t q0 = (int64_t)blockIdx.x * kRowQuads; q0 < nq; q0 += (int64_t)gridDim.x * kRowQuads) {
    const int64_t qd = q0 + tq;
    df a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
    int64_t s = 0, r = 0;
    if (qd < nq) {
      s = qd / qps;
      r = (qd - s * qps) * 4;
      const float4* col = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(L.Z) + (size_t)s * L.TB * d + r);
      const int64_t cs = L.TB / 4;                     // float4 stride between columns
      int64_t j = cg;
      for (; j + ng < d; j += 2 * ng) {
        const float4 z = col[(size_t)j * cs], z2 = col[(size_t)(j + ng) * cs];
        const float2 xv = __ldg(xs + j), xw = __ldg(xs + j + ng);
        const df x{xv.x, xv.y}, w{xw.x, xw.y};
        acc_prod<float>(a0, z.x, x);
        acc_prod<float>(a1, z.y, x);
        acc_prod<float>(a2, z.z, x);
        acc_prod<float>(a3, z.w, x);
        acc_prod<float>(a0, z2.x, w);
        acc_prod<float>(a1, z2.y, w);
        acc_prod<float>(a2, z2.z, w);
        acc_prod<float>(a3, z2.w, w);
      }
      if (j < d) {
        const float4 z = col[(size_t)j * cs];
        const float2 xv = __ldg(xs + j);
        const df x{xv.x, xv.y};
        acc_prod<float>(a0, z.x, x);
        acc_prod<float>(a1, z.y, x);
        acc_prod<float>(a2, z.z, x);
        acc_prod<float>(a3, z.w, x);
      }
    }
    s_acc[cg][0][tq] = make_float2(a0.hi, a0.lo);
    s_acc[cg][1][tq] = make_float2(a1.hi, a1.lo);
    s_acc[cg][2][tq] = make_float2(a2.hi, a2.lo);
    s_acc[cg][3][tq] = make_float2(a3.hi, a3.lo);
    __syncthreads();
    if (cg == 0 && qd < nq) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        df t{s_acc[0][k][tq].x, s_acc[0][k][tq].y};
        for (int g = 1; g < ng; ++g) df_add(t, df{s_acc[g][k][tq].x, s_acc[g][k][tq].y});
        const int64_t i = s * L.TB + r + k;
        if (i < n) out[i] = df_to_double(t);
      }
    }
    __syncthreads();
  }
}

__global__ void dir_rowdot_f64(Layout L, const double* __restrict__ xs, double* out) {
  const int64_t n = L.d, d = L.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / L.TB, r = i - s * L.TB;
    const double* base = reinterpret_cast<const double*>(L.Z) + (size_t)s * L.TB * d + r;
    double acc = 0.0;
    for (int64_t j = 0; j < d; ++j) acc = fma(base[(size_t)j * L.TB], __ldg(xs + j), acc);
    out[i] = acc;
  }
}

// part[j * NB + s] = sum over the samples of slab s of Zq_ij v_i: one CTA per
// slab, one warp per column (lanes over the slab's rows, coalesced)
// FP32: lanes over 16-byte quads of the column (512 contiguous bytes per warp
// per load, two loads in flight)
__global__ void dir_coldot_f32(Layout L, const double* __restrict__ v, double* part) {
  extern __shared__ float2 vs_d[];
  const int64_t s = blockIdx.x;
  const int64_t n = L.d, d = L.n;
  for (int r = threadIdx.x; r < L.TB; r += blockDim.x) {
    const int64_t i = s * L.TB + r;
    const df t = df_from(i < n ? v[i] : 0.0);
    vs_d[r] = make_float2(t.hi, t.lo);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int quads = L.TB / 4;
  const float* base = reinterpret_cast<const float*>(L.Z) + (size_t)s * L.TB * d;
  for (int64_t j = warp; j < d; j += nw) {
    const float4* col = reinterpret_cast<const float4*>(base + (size_t)j * L.TB);
    df a0{0.f, 0.f}, a1{0.f, 0.f};
    int q = lane;
    for (; q + 32 < quads; q += 64) {
      const float4 z = col[q], z2 = col[q + 32];
      const int r = 4 * q, r2 = 4 * (q + 32);
      acc_prod<float>(a0, z.x, df{vs_d[r].x, vs_d[r].y});
      acc_prod<float>(a0, z.y, df{vs_d[r + 1].x, vs_d[r + 1].y});
      acc_prod<float>(a0, z.z, df{vs_d[r + 2].x, vs_d[r + 2].y});
      acc_prod<float>(a0, z.w, df{vs_d[r + 3].x, vs_d[r + 3].y});
      acc_prod<float>(a1, z2.x, df{vs_d[r2].x, vs_d[r2].y});
      acc_prod<float>(a1, z2.y, df{vs_d[r2 + 1].x, vs_d[r2 + 1].y});
      acc_prod<float>(a1, z2.z, df{vs_d[r2 + 2].x, vs_d[r2 + 2].y});
      acc_prod<float>(a1, z2.w, df{vs_d[r2 + 3].x, vs_d[r2 + 3].y});
    }
    if (q < quads) {
      const float4 z = col[q];
      const int r = 4 * q;
      acc_prod<float>(a0, z.x, df{vs_d[r].x, vs_d[r].y});
      acc_prod<float>(a0, z.y, df{vs_d[r + 1].x, vs_d[r + 1].y});
      acc_prod<float>(a0, z.z, df{vs_d[r + 2].x, vs_d[r + 2].y});
      acc_prod<float>(a0, z.w, df{vs_d[r + 3].x, vs_d[r + 3].y});
    }
    df_add(a0, a1);
    a0 = df_warp_sum(a0);
    if (lane == 0) part[(size_t)j * L.NB + s] = df_to_double(a0);
  }
}

// Two right-hand sides in one read of the slab: part[j * NB + s] and
// part2[j * NB + s] for v and v2 (FP32 storage)
__global__ void dir_coldot2_f32(Layout L, const double* __restrict__ v, const double* __restrict__ v2, double* part,
                                double* part2) {
  extern __shared__ float2 vs_d[];                    // TB entries of v, then TB of v2
  float2* vs2 = vs_d + L.TB;
  const int64_t s = blockIdx.x;
  const int64_t n = L.d, d = L.n;
  for (int r = threadIdx.x; r < L.TB; r += blockDim.x) {
    const int64_t i = s * L.TB + r;
    const df t = df_from(i < n ? v[i] : 0.0), t2 = df_from(i < n ? v2[i] : 0.0);
    vs_d[r] = make_float2(t.hi, t.lo);
    vs2[r] = make_float2(t2.hi, t2.lo);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int quads = L.TB / 4;
  const float* base = reinterpret_cast<const float*>(L.Z) + (size_t)s * L.TB * d;
  for (int64_t j = warp; j < d; j += nw) {
    const float4* col = reinterpret_cast<const float4*>(base + (size_t)j * L.TB);
    df a0{0.f, 0.f}, b0{0.f, 0.f};
    for (int q = lane; q < quads; q += 32) {
      const float4 z = col[q];
      const int r = 4 * q;
      acc_prod<float>(a0, z.x, df{vs_d[r].x, vs_d[r].y});
      acc_prod<float>(a0, z.y, df{vs_d[r + 1].x, vs_d[r + 1].y});
      acc_prod<float>(a0, z.z, df{vs_d[r + 2].x, vs_d[r + 2].y});
      acc_prod<float>(a0, z.w, df{vs_d[r + 3].x, vs_d[r + 3].y});
      acc_prod<float>(b0, z.x, df{vs2[r].x, vs2[r].y});
      acc_prod<float>(b0, z.y, df{vs2[r + 1].x, vs2[r + 1].y});
      acc_prod<float>(b0, z.z, df{vs2[r + 2].x, vs2[r + 2].y});
      acc_prod<float>(b0, z.w, df{vs2[r + 3].x, vs2[r + 3].y});
    }
    a0 = df_warp_sum(a0);
    b0 = df_warp_sum(b0);
    if (lane == 0) {
      part[(size_t)j * L.NB + s] = df_to_double(a0);
      part2[(size_t)j * L.NB + s] = df_to_double(b0);
    }
  }
}

__global__ void dir_coldot_f64(Layout L, const double* __restrict__ v, double* part) {
  extern __shared__ float2 vs_d[];
  double* vd = reinterpret_cast<double*>(vs_d);
  const int64_t s = blockIdx.x;
  const int64_t n = L.d, d = L.n;
  for (int r = threadIdx.x; r < L.TB; r += blockDim.x) {
    const int64_t i = s * L.TB + r;
    vd[r] = i < n ? v[i] : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const double* base = reinterpret_cast<const double*>(L.Z) + (size_t)s * L.TB * d;
  for (int64_t j = warp; j < d; j += nw) {
    double acc = 0.0;
    for (int r = lane; r < L.TB; r += 32) acc = fma(base[(size_t)j * L.TB + r], vd[r], acc);
    acc = warp_sum(acc);
    if (lane == 0) part[(size_t)j * L.NB + s] = acc;
  }
}

// out_j = sc_j * sum_s part[j * NB + s] (fixed order; one warp per column)
__global__ void dir_colsum_kernel(const double* part, const double* sc, int64_t d, int NB, double* out) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w0; j < d; j += nw) {
    double acc = 0.0;
    for (int s = lane; s < NB; s += 32) acc += part[(size_t)j * NB + s];
    acc = warp_sum(acc);
    if (lane == 0) out[j] = sc[j] * acc;
  }
}

cudaError_t run_dir_product2(const Layout& L, int store, const double* x, const double* x2, const double* sc,
                             double* out, double* out2, double* part, double* part2, cudaStream_t st) {
  if (store != GDWD_F32 || L.TB % 4) {   // FP64 storage: two single products
    cudaError_t e = run_dir_product(L, store, 1, x, sc, out, part, st);
    return e != cudaSuccess ? e : run_dir_product(L, store, 1, x2, sc, out2, part2, st);
  }
  dir_coldot2_f32<<<L.NB, 256, (size_t)L.TB * 16, st>>>(L, x, x2, part, part2);
  const int rb = (int)std::min<int64_t>((L.n * 32 + 255) / 256, 4096);
  dir_colsum_kernel<<<rb, 256, 0, st>>>(part, sc, L.n, L.NB, out);
  dir_colsum_kernel<<<rb, 256, 0, st>>>(part2, sc, L.n, L.NB, out2);
  return cudaGetLastError();
}

cudaError_t run_dir_product(const Layout& L, int store, int trans, const double* x, const double* sc, double* out,
                            double* part, cudaStream_t st) {
  if (store != GDWD_F32 && store != GDWD_F64) return cudaErrorInvalidValue;
  const bool f64 = store == GDWD_F64;
  if (trans == 0) {   // part holds the scaled x (d entries of 8 bytes)
    dir_scale_kernel<<<(int)std::min<int64_t>((L.n + 255) / 256, 1024), 256, 0, st>>>(x, sc, L.n, f64 ? 1 : 0, part);
    const int blocks = (int)std::min<int64_t>((L.d + 255) / 256, 65535);
    if (f64) {
      dir_rowdot_f64<<<blocks, 256, 0, st>>>(L, part, out);
    } else {
      if (L.TB % 4) return cudaErrorInvalidValue;
      const int64_t nq = (int64_t)L.NB * (L.TB / 4);
      const int ng = nq < (int64_t)152 * 1024 ? kRowGroups : 1;   // fewer quads than ~1024 per SM: split d
      const int qb = (int)std::min<int64_t>((nq + kRowQuads - 1) / kRowQuads, 65535);
      dir_rowdot_f32<<<qb, kRowQuads * ng, 0, st>>>(L, reinterpret_cast<const float2*>(part), out);
    }
    return cudaGetLastError();
  }
  const size_t smem = (size_t)L.TB * 8;
  if (f64) {
    dir_coldot_f64<<<L.NB, 256, smem, st>>>(L, x, part);
  } else {
    if (L.TB % 4) return cudaErrorInvalidValue;
    dir_coldot_f32<<<L.NB, 256, smem, st>>>(L, x, part);
  }
  const int rb = (int)std::min<int64_t>((L.n * 32 + 255) / 256, 4096);
  dir_colsum_kernel<<<rb, 256, 0, st>>>(part, sc, L.n, L.NB, out);
  return cudaGetLastError();
}

// h_w = mu (u + rho / (sigma sqrt(mu))) - Z~ v as double-float, with
// Z~ v = Zxr - Zdr - Za / sigma (Zdr = 0 for Step 1a)
__global__ void dir_rhs_kernel(DirArgs a, int step1c) {
  if (a.ctrl->done) return;
  const double sig = a.ctrl->sigma, sqmu = sqrt(a.mu);
  const double gs = 1.0 / (sig * sqmu), inv_sig = 1.0 / sig;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.d; j += (int64_t)gridDim.x * blockDim.x) {
    const double zv = a.Zxr[j] - (step1c ? a.Zdr[j] : 0.0) - a.Za[j] * inv_sig;
    const df h = df_from(a.mu * (a.u[j] + a.rho[j] * gs) - zv);
    a.hw[j] = make_float2(h.hi, h.lo);
  }
}

// x = P h_w (one warp per row) and, as row d, p^T h_w
__global__ void dir_gemv_kernel(DirArgs a) {
  if (a.ctrl->done) return;
  const int npair = (int)((a.d + 1) / 2);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i <= a.d; i += nw) {
    const df x = row_dot(i < a.d ? a.P + (size_t)i * a.ldP : a.pdf, a.hw, npair);
    if (lane == 0) a.x[i] = df_to_double(x);
  }
}

// total of one slot of the per-block partial sums (one warp, fixed order; the
// result in every lane)
__device__ __forceinline__ double block_total(const double* part, int nblk, int lane) {
  double acc = 0.0;
  for (int b = lane; b < nblk; b += 32) acc += part[b];
  return warp_sum(acc);
}

// beta and w from x = P h_w and p^T h_w (border elimination); h_beta = -y^T v
// with y^T v = y^T (xi - r) - y^T dr - y^T alpha / sigma from the block sums
__global__ void dir_wsolve_kernel(DirArgs a, int step1c) {
  if (a.ctrl->done) return;
  __shared__ double s_hb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    const double yxr = block_total(a.scal + (size_t)DS_YXR * a.nblk, a.nblk, lane);
    const double ya = block_total(a.scal + (size_t)DS_YA * a.nblk, a.nblk, lane);
    const double ydr = step1c ? block_total(a.dscal, a.nblk, lane) : 0.0;
    if (lane == 0) s_hb = -(yxr - ydr - ya / a.ctrl->sigma);
  }
  __syncthreads();
  const double ptw = a.x[a.d];
  const double beta = (s_hb - ptw / a.mu) / ((double)a.n - a.s / a.mu);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.d; j += (int64_t)gridDim.x * blockDim.x)
    a.w[j] = (a.x[j] - a.p[j] * beta) / a.mu;
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->beta = beta;
}

// Step 1b per sample: c-bar_i = (Z~^T w-bar)_i + y_i beta-bar + v-bar_i, the prox
// at c-bar_i + r_i, dr_i = r+_i - r_i; block sums of y^T dr
__global__ void dir_prox_kernel(DirArgs a) {
  if (a.ctrl->done) return;
  __shared__ double s_red[kWarps];
  const double sig = a.ctrl->sigma, inv_sig = 1.0 / sig, beta = a.ctrl->beta;
  const int qc = q_case(a.q);
  double ydr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = a.r[i], yi = a.y[i];
    const double vb = a.xi[i] - ri - a.alpha[i] * inv_sig;
    const double cb = a.t[i] + yi * beta + vb;
    const double rn = prox_root(cb + ri, a.omega[i] * inv_sig, a.q, qc, ri);
    a.r[i] = rn;
    a.dv[i] = rn - ri;
    ydr = fma(yi, rn - ri, ydr);
  }
  ydr = warp_sum(ydr);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = ydr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kWarps; ++k) t += s_red[k];
    a.dscal[blockIdx.x] = t;
  }
}

// Steps 2-3 per sample with Z~^T w = t: xi, alpha; the n-space KKT sums and
// y^T (xi - r), y^T alpha (block partials); xi - r and alpha for the passes
__global__ void dir_step23_kernel(DirArgs a) {
  if (a.ctrl->done) return;
  __shared__ double s_part[kWarps * DS_COUNT];
  const double sig = a.ctrl->sigma, inv_sig = 1.0 / sig, beta = a.ctrl->beta;
  const int qc = q_case(a.q);
  const double inv_q = 1.0 / a.q;
  double v[DS_COUNT];
#pragma unroll
  for (int k = 0; k < DS_COUNT; ++k) v[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = a.r[i], al = a.alpha[i], yi = a.y[i], ce = a.C * a.e[i];
    const double zw = a.t[i];
    const double xin = fmax(0.0, ri - zw - yi * beta + (al - ce) * inv_sig);   // Step 2
    const double res = zw + yi * beta + xin - ri;
    const double an = al - a.tau * sig * res;                                 // Step 3
    a.xi[i] = xin;
    a.alpha[i] = an;
    a.dv[i] = xin - ri;
    a.dv2[i] = an;
    const double om = a.omega[i];
    const double irq1 = 1.0 / pow_q1(ri, a.q, qc);
    v[S_RES2] = fma(res, res, v[S_RES2]);
    v[S_YA] = fma(yi, an, v[S_YA]);
    v[S_XICA] = fma(xin, ce - an, v[S_XICA]);
    const double dvv = an - om * irq1;
    v[S_AMS2] = fma(dvv, dvv, v[S_AMS2]);
    const double mn = fmin(0.0, an), mx = fmax(0.0, an - ce);
    v[S_AMIN2] = fma(mn, mn, v[S_AMIN2]);
    v[S_AMAX2] = fma(mx, mx, v[S_AMAX2]);
    v[S_PRIM_R] += om * inv_q * ri * irq1;
    v[S_PRIM_XI] = fma(a.e[i], xin, v[S_PRIM_XI]);
    v[S_DUAL_A] += dual_pow(a.wt[i] * an, a.q, qc);
    v[DS_YXR] = fma(yi, xin - ri, v[DS_YXR]);
    v[DS_YA] = fma(yi, an, v[DS_YA]);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < DS_COUNT; ++k) {
    const double t = warp_sum(v[k]);
    if (l == 0) s_part[w * DS_COUNT + k] = t;
  }
  __syncthreads();
  if (threadIdx.x < DS_COUNT) {
    double t = 0.0;
    for (int k = 0; k < kWarps; ++k) t += s_part[k * DS_COUNT + threadIdx.x];
    a.scal[(size_t)threadIdx.x * a.nblk + blockIdx.x] = t;
  }
}

// Phase S on one CTA: the totals, the d-space norms of g = w - rho / (sigma sqrt(mu)),
// rho and a = Z~ alpha + sqrt(mu)(1 - tau) rho, then KKT, gap, sigma rule and stop
// (the shared s_phase), then u+ = theta g, rho+ = (1 - tau) rho - tau sigma sqrt(mu)
// (1 - theta) g and the iteration count.
__global__ void __launch_bounds__(kThreads) dir_s_kernel(DirArgs a) {
  Ctrl* c = a.ctrl;
  if (c->done) return;
  __shared__ double s_tot[S_COUNT];
  __shared__ double s_pd[4];
  __shared__ float s_etaf[11];
  __shared__ int s_ictl[2];
  __shared__ double s_ctl[15];
  __shared__ double s_part[kWarps * 6];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double sig = c->sigma, sqmu = sqrt(a.mu);
  const double gs = 1.0 / (sig * sqmu);
  const double ac = sqmu * (1.0 - a.tau);
  for (int k = warp; k < S_G2; k += kWarps) {
    const double t = block_total(a.scal + (size_t)k * a.nblk, a.nblk, lane);
    if (lane == 0) s_tot[k] = t;
  }
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t j = threadIdx.x; j < a.d; j += kThreads) {
    const double rj = a.rho[j];
    const double gj = a.w[j] - rj * gs;
    const double zaj = a.Za[j];
    const double aj = zaj + ac * rj;
    a.g[j] = gj;
    v[0] = fma(gj, gj, v[0]);
    v[1] = fma(gj, rj, v[1]);
    v[2] = fma(rj, rj, v[2]);
    v[3] = fma(aj, aj, v[3]);
    v[4] = fma(aj, gj, v[4]);
    v[5] = fma(zaj, zaj, v[5]);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double t = warp_sum(v[k]);
    if (lane == 0) s_part[warp * 6 + k] = t;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int k = 0; k < kWarps; ++k) t += s_part[k * 6 + threadIdx.x];
    s_tot[S_G2 + threadIdx.x] = t;   // S_G2, S_GRHO, S_RHO2, S_A2, S_AG, S_TA2
  }
  __syncthreads();
  const SPhaseArgs sq{a.C, a.kappa, a.R, a.mu, a.tau, sqmu, a.tol, sqrt(a.tol), (float)(1.0 / (1.0 + a.C)),
                      a.stop_rule, float_at_most(a.tol)};
  const int it = c->it;
  s_phase(s_tot, sq, sig, gs, it, c->beta, GDWD_EMAXITER, true, c, s_pd, s_etaf, s_ctl, s_ictl);
  const double th = s_ctl[0];
  const double rcoef = a.tau * sig * sqmu * (1.0 - th);
  for (int64_t j = threadIdx.x; j < a.d; j += kThreads) {
    const double gj = a.g[j];
    a.u[j] = th * gj;
    a.rho[j] = (1.0 - a.tau) * a.rho[j] - rcoef * gj;
  }
  if (threadIdx.x == 0) {
    c->sigma_prev = sig;
    c->sigma = s_ctl[1];
    c->theta = th;
    c->it = it + 1;
    c->status = s_ictl[1];
    if (s_ictl[0] != 0) c->done = 1;
    else if (it + 1 >= a.max_iter) {
      c->done = 1;
      c->status = GDWD_EMAXITER;
    }
  }
}

// w of the last iterate in the original scale: w / Z_scale
__global__ void dir_finish_kernel(const double* w, double zscale, int64_t d, double* out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = w[j] / zscale;
}

cudaError_t run_dir_finish(const double* w, double zscale, int64_t d, double* out, cudaStream_t st) {
  dir_finish_kernel<<<(int)std::min<int64_t>((d + 255) / 256, 1024), 256, 0, st>>>(w, zscale, d, out);
  return cudaGetLastError();
}

int dir_blocks(int64_t n) { return (int)std::min<int64_t>((n + kThreads - 1) / kThreads, kDirMaxBlocks); }

cudaError_t run_dir_iteration(const DirArgs& a, const DirPasses& ps, cudaStream_t st) {
  const int nb = a.nblk;
  const int db = (int)std::min<int64_t>((a.d + 255) / 256, 1024);
  const int gb = (int)std::min<int64_t>((a.d + 1 + kWarps - 1) / kWarps, 4096);
  cudaError_t e;
  for (int step1c = 0; step1c < 2; ++step1c) {
    dir_rhs_kernel<<<db, 256, 0, st>>>(a, step1c);
    dir_gemv_kernel<<<gb, kThreads, 0, st>>>(a);
    dir_wsolve_kernel<<<db, 256, 0, st>>>(a, step1c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = ps.apply(0, a.w, a.t, ps.ctx)) != cudaSuccess) return e;          // t = Z~^T w
    if (step1c == 0) {
      dir_prox_kernel<<<nb, kThreads, 0, st>>>(a);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = ps.apply(1, a.dv, a.Zdr, ps.ctx)) != cudaSuccess) return e;    // Z~ (r+ - r)
    }
  }
  dir_step23_kernel<<<nb, kThreads, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = ps.apply2(a.dv, a.dv2, a.Zxr, a.Za, ps.ctx)) != cudaSuccess) return e;   // Z~ (xi - r), Z~ alpha
  dir_s_kernel<<<1, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace gdwd
