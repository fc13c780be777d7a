// Shared device helpers of libgdwd: double-float arithmetic, bounded grid
// barrier, 1-D bulk-copy (TMA) ring with mbarriers, element traits.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/gdwd.h"

namespace gdwd {

constexpr int kThreads = 256;          // threads of every persistent / streaming CTA
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------------------
// double-float ("df"): a value hi + lo held in two floats, ~48-bit mantissa.
// FP64 issues at 1/58 of the FP32 rate on this part, so the per-iteration
// n-space solves run in df with exact FP32 products (fmaf) and two-sum adds.
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// acc += x (x a plain float)
__device__ __forceinline__ void df_add(df& acc, float x) {
  float s, e;
  two_sum(acc.hi, x, s, e);
  acc.lo += e;
  acc.hi = s;
}

// acc += (a.hi + a.lo)
__device__ __forceinline__ void df_add(df& acc, df a) {
  float s, e;
  two_sum(acc.hi, a.hi, s, e);
  e += acc.lo + a.lo;
  float t = s + e;
  acc.lo = e - (t - s);
  acc.hi = t;
}

// acc += a * b for df a, b (product error kept through fmaf)
__device__ __forceinline__ void df_fma(df& acc, df a, df b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, e2;
  two_sum(acc.hi, p, s, e2);
  acc.lo += e2 + e;
  acc.hi = s;
}

// a * b, normalized (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float t = p + e;
  return df{t, e - (t - p)};
}

// a + b, normalized
__device__ __forceinline__ df df_sum(df a, df b) {
  df_add(a, b);
  return a;
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_from(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_shfl_xor(df a, int m) {
  df r;
  r.hi = __shfl_xor_sync(0xffffffffu, a.hi, m);
  r.lo = __shfl_xor_sync(0xffffffffu, a.lo, m);
  return r;
}

__device__ __forceinline__ df df_warp_sum(df a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) df_add(a, df_shfl_xor(a, m));
  return a;
}

// Approximate FP32 reciprocal and reciprocal square root of the special-function
// unit (about 1 ulp; denormals flushed): seeds for the FP64 corrections below.
// The correctly rounded forms (__frcp_rn, __fsqrt_rn, IEEE division) are long
// instruction sequences on this part (~170 cycles against ~40).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// sqrt(x) of a non-negative FP32 value to about 2 ulp (0 for x <= 0)
__device__ __forceinline__ float fsqrt_approx(float x) { return x > 0.f ? x * rsqrt_approx(x) : 0.f; }

// max(x, 0) and min(x, 0) by a compare and a select (the FP64 min / max
// instructions are slower than both on this part); NaN gives 0, as fmax does.
__device__ __forceinline__ double dmax0(double x) { return x > 0.0 ? x : 0.0; }
__device__ __forceinline__ double dmin0(double x) { return x < 0.0 ? x : 0.0; }

// 1/b, a/b and sqrt(x) for FP64 operands whose magnitudes lie inside the normal
// FP32 range (b != 0, x >= 0): an FP32 seed from the special-function unit and
// one FP64 Newton correction, which squares the seed's ~2^-23 relative error to
// ~2^-46 (about 1.5e-14).  A dependent FP64 operation takes 64 cycles on this
// part, an FP64 division ~1400 and an FP64 square root ~870; these take three
// or four FP64 operations.
__device__ __forceinline__ double rcp_nr(double b) {
  const double r = (double)rcp_approx((float)b);
  return fma(r, fma(-b, r, 1.0), r);
}
__device__ __forceinline__ double div_nr(double a, double b) {
  const double r = (double)rcp_approx((float)b);
  const double q = a * r;
  return fma(r, fma(-b, q, a), q);
}
__device__ __forceinline__ double sqrt_nr(double x) {
  if (!(x > 0.0)) return 0.0;
  const double r = (double)rsqrt_approx((float)x);   // ~1 / sqrt(x)
  const double s = x * r;
  const double h = 0.5 * r;
  return fma(h, fma(-s, s, x), s);
}

// 1/sqrt(x) for x > 0 inside the normal FP32 range: an FP32 seed and one FP64
// Newton step (~3e-14 relative).
__device__ __forceinline__ double rsqrt_nr(double x) {
  const double r = (double)rsqrt_approx((float)x);
  const double h = 0.5 * r;
  return fma(h, fma(-x * r, r, 1.0), r);
}

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) a += __shfl_xor_sync(0xffffffffu, a, m);
  return a;
}

// ---------------------------------------------------------------------------
// time and bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Error word shared by all CTAs of a launch.  Non-zero = a gdwd_status.
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// counter only grows; barrier number `gen` (1, 2, ...) completes when it reaches
// gen * nblocks.  Every wait is bounded by timeout_ns: on expiry (or when
// another CTA has already flagged an error) the error word is set and false is
// returned to every thread of the CTA, which must then leave the kernel.
__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// `extra` arrivals beyond the grid are awaited as well: 0 in normal use; a test
// passes 1 to make the wait run out (no CTA ever supplies that arrival).
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned nblocks, unsigned& gen, int* err,
                                             uint64_t timeout_ns, int* s_flag, unsigned extra = 0) {
  __syncthreads();
  gen += 1;
  if (threadIdx.x == 0) {
    // the CTA barrier orders the block's writes before this release (cumulativity)
    red_add_release(counter, 1u);
    const unsigned target = gen * nblocks + extra;
    int ok = 1;
    uint64_t t0 = 0;
    unsigned polls = 0;
    while ((int)(ld_acquire(counter) - target) < 0) {
      if ((++polls & 31u) == 0) {
        if (ld_volatile(err) != 0) { ok = 0; break; }
        const uint64_t t = globaltimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > timeout_ns) {
          atomicCAS(err, 0, (int)GDWD_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    if (ld_volatile(err) != 0) ok = 0;
    *s_flag = ok;
  }
  __syncthreads();
  return *(volatile int*)s_flag != 0;
}

// The same barrier with work for the rest of the CTA while thread 0 waits: warps
// 1 .. kWarps-1 run side() between this CTA's arrival and the end of the wait
// (work that depends only on the CTA's own data and is not needed by the other
// CTAs before the next barrier; its global writes are ordered before that one).
template <typename F>
__device__ __forceinline__ bool grid_barrier_side(unsigned* counter, unsigned nblocks, unsigned& gen, int* err,
                                                  uint64_t timeout_ns, int* s_flag, unsigned extra, F&& side) {
  __syncthreads();
  gen += 1;
  if (threadIdx.x == 0) {
    red_add_release(counter, 1u);
    const unsigned target = gen * nblocks + extra;
    int ok = 1;
    uint64_t t0 = 0;
    unsigned polls = 0;
    while ((int)(ld_acquire(counter) - target) < 0) {
      if ((++polls & 31u) == 0) {
        if (ld_volatile(err) != 0) { ok = 0; break; }
        const uint64_t t = globaltimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > timeout_ns) {
          atomicCAS(err, 0, (int)GDWD_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    if (ld_volatile(err) != 0) ok = 0;
    *s_flag = ok;
  } else if (threadIdx.x >= 32) {
    side();
  }
  __syncthreads();
  return *(volatile int*)s_flag != 0;
}

// ---------------------------------------------------------------------------
// mbarrier + 1-D bulk async copy (cp.async.bulk, the untiled TMA form)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bytes and both addresses must be multiples of 16
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The same copy with an L2 eviction-priority hint (a policy from createpolicy).
__device__ __forceinline__ void bulk_g2s_hint(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 eviction priority of the stored Z's chunks: 0 the default, 1 evict_last
// (keep Z, the largest data reused every iteration, ahead of other lines),
// 2 evict_first.
#ifndef GDWD_Z_L2_HINT
#define GDWD_Z_L2_HINT 0
#endif
__device__ __forceinline__ uint64_t z_l2_policy() {
  uint64_t p = 0;
#if GDWD_Z_L2_HINT == 1
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
#elif GDWD_Z_L2_HINT == 2
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
#endif
  return p;
}
__device__ __forceinline__ void bulk_g2s_z(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
#if GDWD_Z_L2_HINT == 0
  bulk_g2s(dst_smem, src_gmem, bytes, bar);
#else
  bulk_g2s_hint(dst_smem, src_gmem, bytes, bar, z_l2_policy());
#endif
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and err set) after timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > timeout_ns) {
      atomicCAS(err, 0, (int)GDWD_ETIMEOUT);
      return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// element traits of the stored Z: 16-byte vectors converted to the compute type
// ---------------------------------------------------------------------------
template <typename T>
struct ElemTraits;

template <>
struct ElemTraits<double> {
  using compute_t = double;
  static constexpr int kVec = 2;
  __device__ __forceinline__ static void load(const void* p, double* v) {
    double2 x = *reinterpret_cast<const double2*>(p);
    v[0] = x.x;
    v[1] = x.y;
  }
};

template <>
struct ElemTraits<float> {
  using compute_t = float;
  static constexpr int kVec = 4;
  __device__ __forceinline__ static void load(const void* p, float* v) {
    float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
};

// FP32 storage read into FP64 arithmetic (the inexact solver's products, whose
// conjugate-gradient recurrences need more than FP32 products): four stored
// values per 16-byte vector, each widened to double.
struct f32w {
  float v;
};
template <>
struct ElemTraits<f32w> {
  using compute_t = double;
  static constexpr int kVec = 4;
  __device__ __forceinline__ static void load(const void* p, double* v) {
    float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
};

// 16-bit and 8-bit storage: products with FP32 operands, FP32 accumulation.
__device__ __forceinline__ void bf16x2_to_float(uint32_t w, float* v) {
  v[0] = __uint_as_float(w << 16);
  v[1] = __uint_as_float(w & 0xffff0000u);
}

template <>
struct ElemTraits<__nv_bfloat16> {
  using compute_t = float;
  static constexpr int kVec = 8;
  __device__ __forceinline__ static void load(const void* p, float* v) {
    const uint4 x = *reinterpret_cast<const uint4*>(p);
    bf16x2_to_float(x.x, v);
    bf16x2_to_float(x.y, v + 2);
    bf16x2_to_float(x.z, v + 4);
    bf16x2_to_float(x.w, v + 6);
  }
};

template <>
struct ElemTraits<__half> {
  using compute_t = float;
  static constexpr int kVec = 8;
  __device__ __forceinline__ static void load(const void* p, float* v) {
    const uint4 x = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  }
};

template <>
struct ElemTraits<__nv_fp8_e4m3> {
  using compute_t = float;
  static constexpr int kVec = 16;
  __device__ __forceinline__ static void load(const void* p, float* v) {
    const uint4 x = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] & 0xffffu), __NV_E4M3);
      const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] >> 16), __NV_E4M3);
      const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
      const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
      v[4 * k] = a.x;
      v[4 * k + 1] = a.y;
      v[4 * k + 2] = b.x;
      v[4 * k + 3] = b.y;
    }
  }
};

// n consecutive compute-type values from shared memory (n a multiple of 16 bytes)
template <int N>
__device__ __forceinline__ void load_ct(const float* p, float* v) {
#pragma unroll
  for (int k = 0; k < N; k += 4) {
    const float4 x = *reinterpret_cast<const float4*>(p + k);
    v[k] = x.x;
    v[k + 1] = x.y;
    v[k + 2] = x.z;
    v[k + 3] = x.w;
  }
}
template <int N>
__device__ __forceinline__ void load_ct(const double* p, double* v) {
#pragma unroll
  for (int k = 0; k < N; k += 2) {
    const double2 x = *reinterpret_cast<const double2*>(p + k);
    v[k] = x.x;
    v[k + 1] = x.y;
  }
}

// Element size and format limits of a gdwd_dtype (host and device).
__host__ __device__ inline int dtype_size(int dt) {
  return dt == GDWD_F64 ? 8 : dt == GDWD_F32 ? 4 : dt == GDWD_E4M3 ? 1 : 2;
}

}  // namespace gdwd
