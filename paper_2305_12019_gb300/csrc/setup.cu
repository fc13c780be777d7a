// Set-up kernels of libgdwd (everything that does not depend on sigma or C):
//
//   ingest   ||Z||_F, finiteness check, copy into the slab layout (Sec. 4.2 scaling
//            is carried by the per-column scale sc_i = 1 / Z_scale)
//   gram     K = Zq^T Zq from the stored values, lower-triangular 64x64 tiles,
//            FP32 products summed over 16-row chunks then folded into a
//            double-float accumulator (FP64 for FP64 storage), deterministic
//            split over d; G = I + sc_i sc_j K_ij / mu in FP64 (first block of J,
//            eq-H, Sec. 3.3.2)
//   factor   one cooperative launch: blocked right-looking FP64 Cholesky
//            G = L L^T (32x32 tiles), X = L^{-1} by blocked forward substitution,
//            P = X^T X = G^{-1}; p = P y, s = y^T p; P and p also stored as
//            double-float pairs for the per-iteration solves
#include <algorithm>

#include "solver.cuh"

namespace gdwd {

// ------------------------------------------------------------------ ingest
template <typename TI>
__global__ void sumsq_kernel(const TI* __restrict__ Z, int64_t d, int64_t n, int64_t ldz, double* part,
                             int* nonfinite) {
  double acc = 0.0;
  int bad = 0;
  const int64_t total = d * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / d, j = idx - i * d;
    const double v = (double)Z[i * ldz + j];
    if (!isfinite(v)) bad = 1;
    acc = fma(v, v, acc);
  }
  __shared__ double s[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    part[blockIdx.x] = t;
  }
  if (bad) atomicOr(nonfinite, 1);
}

// The block partials summed by one warp in a fixed order (lane l takes parts l,
// l + 32, ...; then a fixed shuffle tree), so every caller gets the same bits.
__device__ __forceinline__ double sum_parts_warp(const double* part, int np) {
  const int lane = threadIdx.x & 31;
  double t = 0.0;
  for (int i = lane; i < np; i += 32) t += part[i];
  return warp_sum(t);
}

__global__ void sum_parts_kernel(const double* part, int np, double* out) {
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  const double t = sum_parts_warp(part, np);
  if (threadIdx.x == 0) *out = t;
}

// FP32 / FP64 storage in one pass over the caller's column-major Z: the slab
// copy, the squares summed for ||Z||_F (FP32 input: exact squares, fmaf, added
// in double-float; FP64 input: FP64) and the finiteness check.  Work item =
// (slab, group of kIngCols columns); the item's output is one contiguous run.
constexpr int kIngCols = 32;

template <typename TI>
struct SqAcc;
template <>
struct SqAcc<float> {
  df a{0.f, 0.f};
  __device__ __forceinline__ void add(float v) {
    const float p = v * v;
    const float e = fmaf(v, v, -p);
    float s, e2;
    two_sum(a.hi, p, s, e2);
    a.lo += e2 + e;
    a.hi = s;
  }
  __device__ __forceinline__ double get() const { return df_to_double(a); }
};
template <>
struct SqAcc<double> {
  double a = 0.0;
  __device__ __forceinline__ void add(double v) { a = fma(v, v, a); }
  __device__ __forceinline__ double get() const { return a; }
};

template <typename TI, typename TS>
__global__ void __launch_bounds__(256) ingest_kernel(const TI* __restrict__ Z, int64_t ldz, Layout L,
                                                     TS* __restrict__ out, double* part, int* nonfinite) {
  const int ngrp = (int)((L.n + kIngCols - 1) / kIngCols);
  const int64_t items = (int64_t)L.NB * ngrp;
  const int64_t per_slab = (int64_t)L.TB * L.n;
  SqAcc<TI> acc;
  bool bad = false;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const int s = (int)(w / ngrp), g = (int)(w - (int64_t)s * ngrp);
    const int64_t i0 = (int64_t)g * kIngCols;
    const int nc = (int)(L.n - i0 < kIngCols ? L.n - i0 : kIngCols);
    const int64_t j0 = (int64_t)s * L.TB;
    const int rows = (int)(L.d - j0 < L.TB ? L.d - j0 : L.TB);   // valid rows of this slab (>= 1)
    TS* o = out + s * per_slab + i0 * L.TB;
    const TI* zin = Z + i0 * ldz + j0;
    const int total = nc * L.TB;
    for (int e = threadIdx.x; e < total; e += 256) {
      const int c = e / L.TB, jl = e - c * L.TB;
      TI v = (TI)0;
      if (jl < rows) {
        v = zin[(int64_t)c * ldz + jl];
        bad |= !isfinite(v);
        acc.add(v);
      }
      o[e] = (TS)v;
    }
  }
  __shared__ double sred[8];
  const double t = warp_sum(acc.get());
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int k = 0; k < 8; ++k) u += sred[k];
    part[blockIdx.x] = u;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(nonfinite, 1);
}

// ||Z||_F^2 from the ingest partials (every block sums them the same way), then
// sc_i = 1 / Z_scale with Z_scale = sqrt(||Z||_F); block 0 stores both scalars.
__global__ void ingest_scale_kernel(const double* part, int np, int64_t n, double* sumsq, double* sc,
                                    double* zscale) {
  __shared__ double s_zs;
  if (threadIdx.x < 32) {
    const double t = sum_parts_warp(part, np);
    if (threadIdx.x == 0) {
      s_zs = sqrt(sqrt(t));
      if (blockIdx.x == 0) {
        *sumsq = t;
        *zscale = s_zs;
      }
    }
  }
  __syncthreads();
  const double inv = 1.0 / s_zs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sc[i] = inv;
}

template <typename TI, typename TS>
__global__ void to_slabs_kernel(const TI* __restrict__ Z, int64_t ldz, Layout L, TS* __restrict__ out) {
  const int64_t per_slab = (int64_t)L.TB * L.n;
  const int64_t total = per_slab * L.NB;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / per_slab, rem = idx - s * per_slab;
    const int64_t i = rem / L.TB, jl = rem - i * L.TB;
    const int64_t j = s * L.TB + jl;
    out[idx] = (j < L.d) ? (TS)Z[i * ldz + j] : (TS)0;
  }
}

// sc_i = 1 / Z_scale, Z_scale = sqrt(||Z||_F)
__global__ void scale_kernel(const double* sumsq, int64_t n, double* sc, double* zscale) {
  const double zs = sqrt(sqrt(*sumsq));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sc[i] = 1.0 / zs;
  if (blockIdx.x == 0 && threadIdx.x == 0) *zscale = zs;
}

// Per-column absolute maximum of the input (one block per column, FP64).
template <typename TI>
__global__ void col_absmax_kernel(const TI* __restrict__ Z, int64_t d, int64_t ldz, double* amax) {
  const int64_t i = blockIdx.x;
  double m = 0.0;
  for (int64_t j = threadIdx.x; j < d; j += blockDim.x) m = fmax(m, fabs((double)Z[i * ldz + j]));
  for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, s[w]);
    amax[i] = t;
  }
}

// Largest stored magnitude used by the per-column scale of each format.
__host__ __device__ inline double fmt_max(int store) {
  return store == GDWD_E4M3 ? 448.0 : store == GDWD_F16 ? 32768.0 : 1.0;
}

// s_i = absmax_i / fmt_max (1 for an all-zero column), stored in colscale.
__global__ void colscale_kernel(const double* amax, int64_t n, double fmax_v, double* colscale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    colscale[i] = amax[i] > 0.0 ? amax[i] / fmax_v : 1.0;
}

__device__ __forceinline__ void to_store(double v, __nv_bfloat16* o) { *o = __double2bfloat16(v); }
__device__ __forceinline__ void to_store(double v, __half* o) { *o = __double2half(v); }
__device__ __forceinline__ void to_store(double v, __nv_fp8_e4m3* o) {
  o->__x = __nv_cvt_double_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// Zq_ji = round(Z_ji / s_i) in the storage format (round to nearest even,
// saturating for E4M3), written into the slab layout.
template <typename TI, typename TS>
__global__ void quantize_slabs_kernel(const TI* __restrict__ Z, int64_t ldz, Layout L, const double* colscale,
                                      TS* __restrict__ out) {
  const int64_t per_slab = (int64_t)L.TB * L.n;
  const int64_t total = per_slab * L.NB;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / per_slab, rem = idx - s * per_slab;
    const int64_t i = rem / L.TB, jl = rem - i * L.TB;
    const int64_t j = s * L.TB + jl;
    to_store(j < L.d ? (double)Z[i * ldz + j] / colscale[i] : 0.0, out + idx);
  }
}

// sc_i = s_i / Z_scale for quantized storage
__global__ void scale_q_kernel(const double* sumsq, const double* colscale, int64_t n, double* sc, double* zscale) {
  const double zs = sqrt(sqrt(*sumsq));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sc[i] = colscale[i] / zs;
  if (blockIdx.x == 0 && threadIdx.x == 0) *zscale = zs;
}

template <typename TI, typename TS>
static void quantize_t(const TI* Z, int64_t ldz, const Layout& L, void* out, double* amax, double* colscale,
                       int store, cudaStream_t st) {
  col_absmax_kernel<TI><<<(unsigned)L.n, 256, 0, st>>>(Z, L.d, ldz, amax);
  colscale_kernel<<<(int)std::min<int64_t>((L.n + 255) / 256, 1024), 256, 0, st>>>(amax, L.n, fmt_max(store), colscale);
  quantize_slabs_kernel<TI, TS><<<152 * 8, 256, 0, st>>>(Z, ldz, L, colscale, (TS*)out);
}

cudaError_t run_ingest(const void* Z, int zdt, int64_t ldz, const Layout& L, void* out, int store, double* part,
                       int nparts, double* sumsq, int* nonfinite, double* sc, double* zscale, double* amax,
                       double* colscale, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((L.n + 255) / 256, 1024);
  if (store == GDWD_F64 || store == GDWD_F32) {
    const int64_t items = (int64_t)L.NB * ((L.n + kIngCols - 1) / kIngCols);
    const int blocks = (int)std::min<int64_t>(items, nparts);
    if (zdt == GDWD_F64 && store == GDWD_F64)
      ingest_kernel<double, double><<<blocks, 256, 0, st>>>((const double*)Z, ldz, L, (double*)out, part, nonfinite);
    else if (zdt == GDWD_F64 && store == GDWD_F32)
      ingest_kernel<double, float><<<blocks, 256, 0, st>>>((const double*)Z, ldz, L, (float*)out, part, nonfinite);
    else if (zdt == GDWD_F32 && store == GDWD_F64)
      ingest_kernel<float, double><<<blocks, 256, 0, st>>>((const float*)Z, ldz, L, (double*)out, part, nonfinite);
    else
      ingest_kernel<float, float><<<blocks, 256, 0, st>>>((const float*)Z, ldz, L, (float*)out, part, nonfinite);
    ingest_scale_kernel<<<nb, 256, 0, st>>>(part, blocks, L.n, sumsq, sc, zscale);
    return cudaGetLastError();
  }
  if (zdt == GDWD_F64)
    sumsq_kernel<double><<<nparts, 256, 0, st>>>((const double*)Z, L.d, L.n, ldz, part, nonfinite);
  else
    sumsq_kernel<float><<<nparts, 256, 0, st>>>((const float*)Z, L.d, L.n, ldz, part, nonfinite);
  sum_parts_kernel<<<1, 32, 0, st>>>(part, nparts, sumsq);
  const bool f64 = zdt == GDWD_F64;
  switch (store) {
    case GDWD_BF16:
      if (f64) quantize_t<double, __nv_bfloat16>((const double*)Z, ldz, L, out, amax, colscale, store, st);
      else quantize_t<float, __nv_bfloat16>((const float*)Z, ldz, L, out, amax, colscale, store, st);
      break;
    case GDWD_F16:
      if (f64) quantize_t<double, __half>((const double*)Z, ldz, L, out, amax, colscale, store, st);
      else quantize_t<float, __half>((const float*)Z, ldz, L, out, amax, colscale, store, st);
      break;
    default:
      if (f64) quantize_t<double, __nv_fp8_e4m3>((const double*)Z, ldz, L, out, amax, colscale, store, st);
      else quantize_t<float, __nv_fp8_e4m3>((const float*)Z, ldz, L, out, amax, colscale, store, st);
      break;
  }
  scale_q_kernel<<<nb, 256, 0, st>>>(sumsq, colscale, L.n, sc, zscale);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ gram
constexpr int kGT = 64;   // output tile
constexpr int kGK = 16;   // rows per chunk

// compute type of the Gram tiles: FP64 for FP64 storage, FP32 otherwise (the
// products of two BF16, FP16 or E4M3 values are exact in FP32)
template <typename T>
struct GramType {
  using type = float;
};
template <>
struct GramType<double> {
  using type = double;
};

template <typename G>
struct GramAcc;
template <>
struct GramAcc<float> {
  float c[4][4];
  df s[4][4];
  __device__ void zero() {
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) { c[a][b] = 0.f; s[a][b] = df{0.f, 0.f}; }
  }
  __device__ void fold() {
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) { df_add(s[a][b], c[a][b]); c[a][b] = 0.f; }
  }
  __device__ double get(int a, int b) const { return df_to_double(s[a][b]); }
};
template <>
struct GramAcc<double> {
  double c[4][4];
  __device__ void zero() {
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) c[a][b] = 0.0;
  }
  __device__ void fold() {}
  __device__ double get(int a, int b) const { return c[a][b]; }
};

// four consecutive stored elements (4-element aligned) converted to the Gram type
__device__ __forceinline__ void load4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float* v) {
  const uint2 a = *reinterpret_cast<const uint2*>(p);
  bf16x2_to_float(a.x, v);
  bf16x2_to_float(a.y, v + 2);
}
__device__ __forceinline__ void load4(const __half* p, float* v) {
  const uint2 a = *reinterpret_cast<const uint2*>(p);
  const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
  const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
  v[0] = f0.x; v[1] = f0.y; v[2] = f1.x; v[3] = f1.y;
}
__device__ __forceinline__ void load4(const __nv_fp8_e4m3* p, float* v) {
  const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Loads rows [r0, r0+16) of columns [c0, c0+64) of one slab into sm[16][64].
template <typename T, typename GT>
__device__ __forceinline__ void gram_load(const T* slab, const Layout& L, int r0, int64_t c0, GT (*sm)[kGT]) {
  const int t = threadIdx.x;
  const int col = t >> 2;              // 0..63
  const int k0 = (t & 3) * 4;          // 0, 4, 8, 12
  const int64_t gc = c0 + col;
  const int rr = r0 + k0;
  GT e[4];
  if (gc < L.n && rr < L.TB) {         // TB is a multiple of 4: rows rr..rr+3 all valid
    load4(slab + gc * L.TB + rr, e);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) e[q] = (GT)0;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sm[k0 + q][col] = e[q];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) gram_kernel(Layout L, int T_tiles, int ksplit, double* Kpart) {
  using GT = typename GramType<T>::type;
  __shared__ __align__(16) GT As[kGK][kGT];
  __shared__ __align__(16) GT Bs[kGK][kGT];
  const int tile = blockIdx.x / ksplit, sp = blockIdx.x % ksplit;
  // tile -> (I, J), I >= J, row-major over the lower triangle
  int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= tile) ++I;
  while (I * (I + 1) / 2 > tile) --I;
  const int J = tile - I * (I + 1) / 2;
  const int s0 = (int)((int64_t)L.NB * sp / ksplit), s1 = (int)((int64_t)L.NB * (sp + 1) / ksplit);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  GramAcc<GT> acc;
  acc.zero();
  const T* Zs = reinterpret_cast<const T*>(L.Z);
  for (int s = s0; s < s1; ++s) {
    const T* slab = Zs + (int64_t)s * L.TB * L.n;
    for (int r0 = 0; r0 < L.TB; r0 += kGK) {
      gram_load<T, GT>(slab, L, r0, (int64_t)I * kGT, As);
      gram_load<T, GT>(slab, L, r0, (int64_t)J * kGT, Bs);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kGK; ++k) {
        GT a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = As[k][ty * 4 + q];
          b[q] = Bs[k][tx * 4 + q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc.c[p][q] = fma(a[p], b[q], acc.c[p][q]);
      }
      acc.fold();
      __syncthreads();
    }
  }
  const int64_t n = L.n;
  double* out = Kpart + (int64_t)sp * n * n;
  for (int p = 0; p < 4; ++p)
    for (int q = 0; q < 4; ++q) {
      const int64_t i = (int64_t)I * kGT + ty * 4 + p, j = (int64_t)J * kGT + tx * 4 + q;
      if (i < n && j < n && i >= j) out[i * n + j] = acc.get(p, q);
    }
}

// FP32 storage: 128 x 64 output tiles (the lower triangle's tile row I and tile
// columns J <= 2I + 1), 8 x 4 outputs per thread, 16-row chunks staged through
// shared memory, FP32 sums of 32 rows folded into double-float (the rounding
// profile of gram_kernel<float> with twice the rows per fold, and twice the
// multiply-adds per shared-memory read).
constexpr int kG32I = 128, kG32J = 64, kG32K = 16;

__device__ __forceinline__ int g32_tiles_j(int I, int Tj) { return (2 * I + 2 < Tj) ? 2 * I + 2 : Tj; }

__global__ void __launch_bounds__(kThreads) gram32_kernel(Layout L, int Ti, int Tj, int ksplit, double* Kpart) {
  __shared__ __align__(16) float As[kG32K][kG32I];
  __shared__ __align__(16) float Bs[kG32K][kG32J];
  // tile index -> (I, J): tile rows I hold g32_tiles_j(I) tiles each
  int tile = blockIdx.x / ksplit;
  const int sp = blockIdx.x % ksplit;
  int I = 0;
  while (tile >= g32_tiles_j(I, Tj)) {
    tile -= g32_tiles_j(I, Tj);
    ++I;
  }
  const int J = tile;
  const int s0 = (int)((int64_t)L.NB * sp / ksplit), s1 = (int)((int64_t)L.NB * (sp + 1) / ksplit);
  const int t = threadIdx.x;
  const int ti = t >> 4, tj = t & 15;            // outputs rows ti*8.., columns tj*4..
  // loader roles: A: column t % 128, rows 8 (t / 128) .. +8; B: column t % 64, rows 4 (t / 64) .. +4
  const int ca = t & 127, ra = (t >> 7) * 8;
  const int cb = t & 63, rb = (t >> 6) * 4;
  const int64_t gca = (int64_t)I * kG32I + ca, gcb = (int64_t)J * kG32J + cb;
  const float* Zs = reinterpret_cast<const float*>(L.Z);
  float acc[8][4];
  df sum[8][4];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc[p][q] = 0.f;
      sum[p][q] = df{0.f, 0.f};
    }
  // chunk sequence: (slab s, first row r0) for s in [s0, s1), r0 = 0, 16, .. < TB; the
  // loads of the next chunk are issued before the current one is computed
  const int per = (L.TB + kG32K - 1) / kG32K;
  const int nchunk = (s1 - s0) * per;
  auto load = [&](int c, float4& a0, float4& a1, float4& b0) {
    a0 = make_float4(0.f, 0.f, 0.f, 0.f);
    a1 = a0;
    b0 = a0;
    if (c >= nchunk) return;
    const int s = s0 + c / per, r0 = (c % per) * kG32K;
    const float* slab = Zs + (int64_t)s * L.TB * L.n;
    // rows beyond the slab and columns beyond n are zero (TB is a multiple of 4)
    if (gca < L.n) {
      const float* pa = slab + gca * L.TB + r0 + ra;
      if (r0 + ra < L.TB) a0 = *reinterpret_cast<const float4*>(pa);
      if (r0 + ra + 4 < L.TB) a1 = *reinterpret_cast<const float4*>(pa + 4);
    }
    if (gcb < L.n && r0 + rb < L.TB) b0 = *reinterpret_cast<const float4*>(slab + gcb * L.TB + r0 + rb);
  };
  float4 a0, a1, b0;
  load(0, a0, a1, b0);
  int since_fold = 0;
  for (int c = 0; c < nchunk; ++c) {
    __syncthreads();   // the previous chunk's reads are done
    As[ra + 0][ca] = a0.x; As[ra + 1][ca] = a0.y; As[ra + 2][ca] = a0.z; As[ra + 3][ca] = a0.w;
    As[ra + 4][ca] = a1.x; As[ra + 5][ca] = a1.y; As[ra + 6][ca] = a1.z; As[ra + 7][ca] = a1.w;
    Bs[rb + 0][cb] = b0.x; Bs[rb + 1][cb] = b0.y; Bs[rb + 2][cb] = b0.z; Bs[rb + 3][cb] = b0.w;
    __syncthreads();
    load(c + 1, a0, a1, b0);
#pragma unroll
    for (int k = 0; k < kG32K; ++k) {
      const float4 x0 = *reinterpret_cast<const float4*>(&As[k][ti * 8]);
      const float4 x1 = *reinterpret_cast<const float4*>(&As[k][ti * 8 + 4]);
      const float4 y = *reinterpret_cast<const float4*>(&Bs[k][tj * 4]);
      const float av[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float bv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
    }
    since_fold += kG32K;
    if (since_fold >= 32) {
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          df_add(sum[p][q], acc[p][q]);
          acc[p][q] = 0.f;
        }
      since_fold = 0;
    }
  }
  const int64_t n = L.n;
  double* out = Kpart + (int64_t)sp * n * n;
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      df v = sum[p][q];
      df_add(v, acc[p][q]);
      const int64_t i = (int64_t)I * kG32I + ti * 8 + p, j = (int64_t)J * kG32J + tj * 4 + q;
      if (i < n && j < n && i >= j) out[i * n + j] = df_to_double(v);
    }
}

int gram32_ksplit(const Layout& L, int sms) {
  const int Ti = (int)((L.n + kG32I - 1) / kG32I), Tj = (int)((L.n + kG32J - 1) / kG32J);
  int tiles = 0;
  for (int I = 0; I < Ti; ++I) tiles += std::min(2 * I + 2, Tj);
  int ks = std::max(1, sms / tiles);   // one wave of CTAs (one per SM)
  ks = std::min(ks, std::max(1, L.NB));
  return std::min(ks, 16);
}

// G_ij = delta_ij + sc_i sc_j sum_split K_ij / mu, both triangles.
__global__ void gram_finish_kernel(const double* Kpart, int ksplit, const double* sc, int64_t n, double inv_mu,
                                   double* G) {
  const int64_t total = n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    if (j > i) continue;
    double k = 0.0;
    for (int s = 0; s < ksplit; ++s) k += Kpart[(int64_t)s * total + idx];
    const double g = (i == j ? 1.0 : 0.0) + sc[i] * sc[j] * k * inv_mu;
    G[i * n + j] = g;
    G[j * n + i] = g;
  }
}

int gram_ksplit(const Layout& L, int sms) {
  if (L.esize == 4) return gram32_ksplit(L, sms);
  const int Tt = (int)((L.n + kGT - 1) / kGT);
  const int tiles = Tt * (Tt + 1) / 2;
  int ks = std::max(1, (2 * sms + tiles - 1) / tiles);
  ks = std::min(ks, std::max(1, L.NB));
  return std::min(ks, 16);
}

cudaError_t run_gram(int store, const Layout& L, int ksplit, double* Kpart, const double* sc, double mu, double* G,
                     bool tensor_cores, void* scratch, int* err, uint64_t timeout_ns, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (tensor_cores) {
    e = run_gram_tc(store, L, ksplit, Kpart, scratch, err, timeout_ns, st);
  } else {
    const int Tt = (int)((L.n + kGT - 1) / kGT);
    const int tiles = Tt * (Tt + 1) / 2;
    const dim3 grid(tiles * ksplit);
    switch (store) {
      case GDWD_F64: gram_kernel<double><<<grid, kThreads, 0, st>>>(L, Tt, ksplit, Kpart); break;
      case GDWD_BF16: gram_kernel<__nv_bfloat16><<<grid, kThreads, 0, st>>>(L, Tt, ksplit, Kpart); break;
      case GDWD_F16: gram_kernel<__half><<<grid, kThreads, 0, st>>>(L, Tt, ksplit, Kpart); break;
      case GDWD_E4M3: gram_kernel<__nv_fp8_e4m3><<<grid, kThreads, 0, st>>>(L, Tt, ksplit, Kpart); break;
      default: {
        const int Ti = (int)((L.n + kG32I - 1) / kG32I), Tj = (int)((L.n + kG32J - 1) / kG32J);
        int tiles32 = 0;
        for (int I = 0; I < Ti; ++I) tiles32 += std::min(2 * I + 2, Tj);
        gram32_kernel<<<tiles32 * ksplit, kThreads, 0, st>>>(L, Ti, Tj, ksplit, Kpart);
        break;
      }
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  gram_finish_kernel<<<1024, 256, 0, st>>>(Kpart, ksplit, sc, L.n, 1.0 / mu, G);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ factor
// One cooperative launch computes G = L L^T, X = L^{-1} and P = X^T X = G^{-1}
// with 32x32 tiles.  The matrices live in double-float (float2 hi/lo, ~48-bit
// mantissa): FP64 issues at 1/58 of the FP32 rate on this part, so everything
// runs in double-float on the FP32 pipes -- the bulk tile updates (n^3/6
// multiply-adds in each of the three stages) and the small sequential pieces
// (the 32x32 diagonal Cholesky, the triangular solves against it).
constexpr int kNB = 32;   // tile

__device__ __forceinline__ double f2d(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ float2 d2f(double x) {
  const df h = df_from(x);
  return make_float2(h.hi, h.lo);
}

// tile index t of the lower triangle (row-major) -> (i, j), i >= j
__device__ __forceinline__ void tri_index(int t, int& i, int& j) {
  int ii = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);   // an estimate, corrected below
  while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
  while (ii * (ii + 1) / 2 > t) --ii;
  i = ii;
  j = t - ii * (ii + 1) / 2;
}

// The diagonal tiles and the triangular solves against them run in
// double-float too: FP64 issues at one warp instruction per 64 cycles per SM
// sub-partition, which made the 32-column pivot chain of a tile the factor's
// critical path.
__device__ __forceinline__ df df_of(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ float2 f2_of(df v) { return make_float2(v.hi, v.lo); }
__device__ __forceinline__ df df_shfl(df a, int src) {
  return df{__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
}
// a - b * c
__device__ __forceinline__ df df_fnma(df a, df b, df c) { return df_sum(a, df_neg(df_mul(b, c))); }

// r (1 + e) for a small FP32 e (the correction of a Newton step)
__device__ __forceinline__ df df_scale_1p(df r, float e) {
  const float c = r.hi * e;
  return df_sum(r, df{c, fmaf(r.hi, e, -c)});
}

// 1 / sqrt(p) and sqrt(p) of a positive double-float p inside the normal FP32
// range: an FP32 seed and two double-float Newton steps (~1e-14 relative).
__device__ __forceinline__ void df_rsqrt_sqrt(df p, df& inv, df& s) {
  df r{rsqrt_approx(p.hi), 0.f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df t = df_mul(p, df_mul(r, r));        // p r^2, close to 1
    const float e = (1.0f - t.hi) - t.lo;        // 1 - t.hi is exact there
    r = df_scale_1p(r, 0.5f * e);
  }
  inv = r;
  s = df_mul(p, r);
}

// 1 / b of a double-float b inside the normal FP32 range (two Newton steps).
__device__ __forceinline__ df df_rcp(df b) {
  df r{rcp_approx(b.hi), 0.f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df t = df_mul(b, r);
    r = df_scale_1p(r, (1.0f - t.hi) - t.lo);
  }
  return r;
}

// Pivot c of the tile: L_cc = sqrt(D_cc) into D, 1 / L_cc into Dinv.  A
// non-positive pivot records GDWD_ENOTPD (and continues with 1).
__device__ __forceinline__ void chol_pivot_df(float2 (*D)[kNB + 1], float2* Dinv, int c, int* err) {
  df p = df_of(D[c][c]);
  if (!(p.hi > 0.f) || !isfinite(p.hi)) {
    atomicCAS(err, 0, (int)GDWD_ENOTPD);
    p = df{1.f, 0.f};
  }
  df inv, sq;
  df_rsqrt_sqrt(p, inv, sq);
  D[c][c] = f2_of(sq);
  Dinv[c] = f2_of(inv);
}

// The lower triangle of a 32 x 32 tile as (row << 8 | column), column-major
// (column q's entries from off[q]): the entries with column >= q are a suffix.
struct TriTable {
  uint16_t rq[kNB * (kNB + 1) / 2];
  uint16_t off[kNB + 1];
  constexpr TriTable() : rq(), off() {
    int k = 0;
    for (int q = 0; q < kNB; ++q) {
      off[q] = (uint16_t)k;
      for (int r = q; r < kNB; ++r) rq[k++] = (uint16_t)(r << 8 | q);
    }
    off[kNB] = (uint16_t)k;
  }
};
__device__ const TriTable kTri;

// Cholesky of the 32 x 32 double-float tile D (lower triangle, in place) by all
// threads of the CTA, column by column, with a look-ahead of one column: after
// column c is scaled, warp 0 updates column c+1 alone and takes its pivot while
// the other warps update the rest of the trailing triangle (its entries taken
// from a table, so no thread idles on the upper half).  (One warp holding the
// rows in registers is slower: a single warp issues the whole trailing update.)
__device__ void chol_tile_df(float2 (*D)[kNB + 1], float2* Dinv, int* err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) chol_pivot_df(D, Dinv, 0, err);
  for (int c = 0; c < kNB; ++c) {
    __syncthreads();                                   // pivot c is in D[c][c], Dinv[c]
    if (threadIdx.x > c && threadIdx.x < kNB)
      D[threadIdx.x][c] = f2_of(df_mul(df_of(D[threadIdx.x][c]), df_of(Dinv[c])));
    __syncthreads();                                   // column c of L is complete
    if (c + 1 == kNB) break;
    if (warp == 0) {
      // column c+1 first, then its pivot
      if (lane >= c + 1) D[lane][c + 1] = f2_of(df_fnma(df_of(D[lane][c + 1]), df_of(D[lane][c]), df_of(D[c + 1][c])));
      __syncwarp();
      if (lane == 0) chol_pivot_df(D, Dinv, c + 1, err);
    } else {
      // the rest of the trailing triangle: D[r][q] -= L[r][c] L[q][c], c+2 <= q <= r
      const int e1 = kTri.off[kNB];
      for (int e = kTri.off[c + 2] + threadIdx.x - 32; e < e1; e += kThreads - 32) {
        const int rq = __ldg(&kTri.rq[e]), r = rq >> 8, q = rq & 255;
        D[r][q] = f2_of(df_fnma(df_of(D[r][q]), df_of(D[r][c]), df_of(D[q][c])));
      }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) factor_kernel(FactorArgs a) {
  __shared__ float2 T1[kNB][kNB + 1], T2[kNB][kNB + 1];
  __shared__ float2 D[kNB][kNB + 1];     // double-float diagonal tile
  __shared__ float2 Dinv[kNB];           // its inverse diagonal
  __shared__ int s_flag;
  __shared__ double s_red[kWarps + 1];
  const int64_t n = a.n;
  const int nb = (int)((n + kNB - 1) / kNB);
  const int cta = blockIdx.x, grid = a.grid;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* A = a.A;
  float2* X = a.X;
  unsigned gen = 0;
#define FBAR()                                                                          \
  do {                                                                                  \
    if (!grid_barrier(a.bar, (unsigned)grid, gen, a.err, a.timeout_ns, &s_flag)) return; \
  } while (0)

  // ---------------- df copy of G (lower triangle) and X = I
  for (int64_t idx = (int64_t)cta * kThreads + threadIdx.x; idx < n * n; idx += (int64_t)grid * kThreads) {
    const int64_t i = idx / n, j = idx - i * n;
    A[idx] = j <= i ? d2f(a.G[idx]) : make_float2(0.f, 0.f);
    X[idx] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  FBAR();

  // ---------------- Cholesky and X = L^{-1} in one sweep over tile columns k.
  // Phase 1: with the factored diagonal tile L_kk, the panel rows below it
  // (L_ik = A_ik L_kk^{-T}) and tile row k of X (X_kJ <- L_kk^{-1} X_kJ, J <= k; its
  // updates from the steps before k are complete) -- n warp tasks in all.
  // Phase 2: the trailing update of the Cholesky (A_IJ -= L_Ik L_Jk^T, k < J <= I)
  // and of the inverse (X_IJ -= L_Ik X_kJ, I > k >= J), tile-parallel; CTA 0
  // instead updates diagonal tile k+1 and factors it (all its threads), a
  // look-ahead of one tile that keeps the diagonal factor off the critical path
  // whenever the trailing update takes longer.  Two grid barriers per k.
  auto factor_diag = [&](int64_t k0) {    // CTA 0: D <- tile (k0, k0) of A, factor, store L
    for (int t = threadIdx.x; t < kNB * kNB; t += kThreads) {
      const int r = t / kNB, c = t % kNB;
      const int64_t gr = k0 + r, gc = k0 + c;
      D[r][c] = (gr < n && gc < n) ? A[gr * n + gc] : make_float2(gr == gc ? 1.f : 0.f, 0.f);
    }
    chol_tile_df(D, Dinv, a.err);
    for (int t = threadIdx.x; t < kNB * kNB; t += kThreads) {
      const int r = t / kNB, c = t % kNB;
      const int64_t gr = k0 + r, gc = k0 + c;
      if (gr < n && gc < n && c <= r) A[gr * n + gc] = D[r][c];
    }
    __syncthreads();
  };
  // forward substitution L_kk x = b on one warp (lane r holds entry r; double-float)
  auto trsv = [&](df x) {
    for (int c = 0; c < kNB; ++c) {
      const df xc = df_mul(df_shfl(x, c), df_of(Dinv[c]));
      if (lane == c) x = xc;
      if (lane > c) x = df_fnma(x, xc, df_of(D[lane][c]));
    }
    return x;
  };
  if (cta == 0) factor_diag(0);
  FBAR();
  for (int k = 0; k < nb; ++k) {
    const int64_t k0 = (int64_t)k * kNB;
    // the factored diagonal tile L_kk and the reciprocals of its diagonal
    for (int t = threadIdx.x; t < kNB * kNB; t += kThreads) {
      const int r = t / kNB, c = t % kNB;
      const int64_t gr = k0 + r, gc = k0 + c;
      D[r][c] = (gr < n && gc < n && c <= r) ? A[gr * n + gc] : make_float2(gr == gc ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    if (threadIdx.x < kNB) Dinv[threadIdx.x] = f2_of(df_rcp(df_of(D[threadIdx.x][threadIdx.x])));
    __syncthreads();
    // phase 1: panel rows i >= k0 + 32 of A, then columns j < min(n, k0 + 32) of X's tile row k
    {
      const int64_t npanel = (n > k0 + kNB) ? n - k0 - kNB : 0;
      const int64_t ncols = (n < k0 + kNB) ? n : k0 + kNB;
      for (int64_t q = (int64_t)cta * kWarps + warp; q < npanel + ncols; q += (int64_t)grid * kWarps) {
        if (q < npanel) {
          const int64_t i = k0 + kNB + q;
          const df x = trsv((k0 + lane < n) ? df_of(A[i * n + k0 + lane]) : df{0.f, 0.f});
          if (k0 + lane < n) A[i * n + k0 + lane] = f2_of(x);
        } else {
          const int64_t j = q - npanel;
          const df x = trsv((k0 + lane < n) ? df_of(X[(k0 + lane) * n + j]) : df{0.f, 0.f});
          if (k0 + lane < n) X[(k0 + lane) * n + j] = f2_of(x);
        }
      }
    }
    FBAR();
    // phase 2: tile 0 of the Cholesky update is the next diagonal tile (CTA 0);
    // the other Cholesky tiles and the inverse tiles go round-robin to the other
    // CTAs (to all CTAs on a grid of one)
    {
      const int m = nb - k - 1;
      const int ntc = m * (m + 1) / 2;        // Cholesky tiles (tile 0 = the next diagonal)
      const int nti = m * (k + 1);            // inverse tiles
      // A task updates one 32 x 32 tile C -= L_Ik B^T: a Cholesky tile (C = A_IJ,
      // B = L_Jk) or an inverse tile (C = X_IJ, B^T = X_kJ).  Each thread keeps its
      // four outputs (orow, oc0 + 8 q) in registers, and the operands of a CTA's
      // next task are loaded into registers while the current one is computed.
      constexpr int kPer = kNB * kNB / kThreads;
      const int orow = threadIdx.x >> 3, oc0 = threadIdx.x & 7;
      struct Fetched {
        float2 a[kPer], b[kPer], c[4];
        float2* C;
        int64_t I0, J0;
      };
      auto fetch = [&](int u, Fetched& f) {   // u < ntc: Cholesky tile u; then inverse tiles
        const bool chol = u < ntc;
        int64_t I0, J0;
        if (chol) {
          int ii, jj;
          tri_index(u, ii, jj);
          I0 = (int64_t)(k + 1 + ii) * kNB;
          J0 = (int64_t)(k + 1 + jj) * kNB;
        } else {
          const int t = u - ntc, ii = t / (k + 1), jj = t % (k + 1);
          I0 = (int64_t)(k + 1 + ii) * kNB;
          J0 = (int64_t)jj * kNB;
        }
        f.C = chol ? A : X;
        f.I0 = I0;
        f.J0 = J0;
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          const int q = threadIdx.x + e * kThreads;
          const int r = q / kNB, c = q % kNB;                      // row-major: consecutive threads, consecutive columns
          f.a[e] = (I0 + r < n && k0 + c < n) ? A[(I0 + r) * n + k0 + c] : make_float2(0.f, 0.f);
          if (chol) {
            f.b[e] = (J0 + r < n && k0 + c < n) ? A[(J0 + r) * n + k0 + c] : make_float2(0.f, 0.f);
          } else {
            const int rt = q % kNB, ct = q / kNB;                  // B[rt][ct] = X[k0 + ct][J0 + rt]
            f.b[e] = (k0 + ct < n && J0 + rt < n) ? X[(k0 + ct) * n + J0 + rt] : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t gi = I0 + orow, gj = J0 + oc0 + 8 * q;
          f.c[q] = (gi < n && gj < n) ? f.C[gi * n + gj] : make_float2(0.f, 0.f);
        }
      };
      // commit f's operands to T1 / T2 (B transposed for inverse tiles, as fetched)
      auto commit = [&](const Fetched& f, bool chol) {
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          const int q = threadIdx.x + e * kThreads;
          T1[q / kNB][q % kNB] = f.a[e];
          if (chol) T2[q / kNB][q % kNB] = f.b[e];
          else T2[q % kNB][q / kNB] = f.b[e];
        }
      };
      auto finish = [&](float2* C, int64_t I0, int64_t J0, const float2 (&c)[4]) {
        df acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
        for (int kk = 0; kk < kNB; ++kk) {
          const float2 av = T1[orow][kk];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 bv = T2[oc0 + 8 * q][kk];
            df_fma(acc[q], df{av.x, av.y}, df{bv.x, bv.y});
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t gi = I0 + orow, gj = J0 + oc0 + 8 * q;
          if (gi < n && gj < n) C[gi * n + gj] = f2_of(df_sum(df{c[q].x, c[q].y}, df_neg(acc[q])));
        }
      };
      const int ntask = (ntc > 0 ? ntc - 1 : 0) + nti;   // every tile but the next diagonal one
      if (m > 0 && cta == 0) {
        Fetched f;
        fetch(0, f);
        commit(f, true);
        __syncthreads();
        finish(f.C, f.I0, f.J0, f.c);
        __syncthreads();
        factor_diag(k0 + kNB);
      }
      const int first = grid > 1 ? cta - 1 : 0, stride = grid > 1 ? grid - 1 : 1;
      if (grid == 1 || cta > 0) {
        Fetched f;
        int u = first;
        if (u < ntask) fetch(u + 1, f);                  // task u is tile u + 1 (tile 0: CTA 0)
        while (u < ntask) {
          commit(f, u + 1 < ntc);
          const float2 cc[4] = {f.c[0], f.c[1], f.c[2], f.c[3]};
          float2* C = f.C;
          const int64_t I0 = f.I0, J0 = f.J0;
          __syncthreads();
          const int next = u + stride;
          if (next < ntask) fetch(next + 1, f);
          finish(C, I0, J0, cc);
          __syncthreads();
          u = next;
        }
      }
    }
    FBAR();
  }

  // ---------------- P = X^T X (X lower): P_IJ = sum_{M >= I} X_MI^T X_MJ, I >= J
  {
    const int ntile = nb * (nb + 1) / 2;
    for (int t = cta; t < ntile; t += grid) {
      int ii, jj;
      tri_index(t, ii, jj);
      const int64_t I0 = (int64_t)ii * kNB, J0 = (int64_t)jj * kNB;
      // the sum over M runs in registers (4 outputs per thread); the two X tiles
      // of step M + 1 are loaded into registers while step M is computed
      constexpr int kPer = kNB * kNB / kThreads;
      float2 pa[kPer], pb[kPer];
      auto fetch = [&](int M) {
        const int64_t M0 = (int64_t)M * kNB;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const int q = threadIdx.x + k * kThreads;
          const int r = q % kNB, c = q / kNB;                        // consecutive threads: consecutive columns of X
          const int64_t gm = M0 + c;
          pa[k] = (gm < n && I0 + r < n) ? X[gm * n + I0 + r] : make_float2(0.f, 0.f);
          pb[k] = (gm < n && J0 + r < n) ? X[gm * n + J0 + r] : make_float2(0.f, 0.f);
        }
      };
      const int orow = threadIdx.x >> 3, oc0 = threadIdx.x & 7;      // outputs (orow, oc0 + 8 q)
      df acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      fetch(ii);
      for (int M = ii; M < nb; ++M) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const int q = threadIdx.x + k * kThreads;
          T1[q % kNB][q / kNB] = pa[k];
          T2[q % kNB][q / kNB] = pb[k];
        }
        __syncthreads();
        if (M + 1 < nb) fetch(M + 1);
#pragma unroll 4
        for (int k = 0; k < kNB; ++k) {
          const float2 av = T1[orow][k];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 bv = T2[oc0 + 8 * q][k];
            df_fma(acc[q], df{av.x, av.y}, df{bv.x, bv.y});
          }
        }
        // renormalise after every 32 terms: df_fma lets lo grow, and a lo far
        // above ulp(hi) / 2 rounds away the low bits
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = df_sum(df{0.f, 0.f}, acc[q]);
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t gi = I0 + orow, gj = J0 + oc0 + 8 * q;
        if (gi < n && gj < n && gi >= gj) {
          const df v = df_sum(df{0.f, 0.f}, acc[q]);
          a.P[gi * a.ldP + gj] = f2_of(v);
          a.P[gj * a.ldP + gi] = f2_of(v);
        }
      }
    }
  }
  FBAR();
  // ---------------- p = P y (double-float), s = y^T p
  for (int64_t i = (int64_t)cta * kWarps + warp; i < n; i += (int64_t)grid * kWarps) {
    df acc{0.f, 0.f};
    for (int64_t j = lane; j < n; j += 32) {
      const float2 pv = a.P[i * a.ldP + j];
      df_fma(acc, df{pv.x, pv.y}, df_from(a.y[j]));
    }
    acc = df_warp_sum(acc);
    if (lane == 0) {
      a.p[i] = df_to_double(acc);
      a.pdf[i] = make_float2(acc.hi, acc.lo);
    }
  }
  FBAR();
  if (cta == 0) {
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) acc = fma(a.y[i], a.p[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += s_red[w];
      *a.s_out = t;
    }
  }
#undef FBAR
}

cudaError_t run_factor(const FactorArgs& a, cudaStream_t st) {
  FactorArgs args = a;
  void* params[] = {(void*)&args};
  return cudaLaunchCooperativeKernel((const void*)factor_kernel, dim3(a.grid), dim3(kThreads), params, 0, st);
}

}  // namespace gdwd
