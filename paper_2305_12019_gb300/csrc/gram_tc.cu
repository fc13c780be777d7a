// K = Zq^T Zq on the 5th-generation tensor cores, for BF16, FP16 and E4M3
// storage, and for FP32 storage through a three-term BF16 split.
//
// The Gram matrix of the stored codes is the one dense contraction of the
// method: the n x n block I + Z~^T Z~ / mu of the SMW2 solve (Sec. 3.2,
// eq-Ainv), formed once per data set, over the d rows.  With 16- or 8-bit codes
// every product of two codes is exact in FP32, so it runs on tcgen05.mma:
//
//   * one CTA per (128 x 128 lower-triangular output tile, k-range); the
//     k-ranges split the sequence of (slab, 128-byte row strip) steps;
//   * warp 0 (one thread) loads, per k-step, the strips of the two column tiles
//     (128 columns x 128 bytes each: 64 BF16/FP16 or 128 E4M3 rows) from the
//     slab layout with a 3-D tensor map and the 128-byte swizzle into a
//     six-stage shared-memory ring (cp.async.bulk.tensor, mbarrier complete_tx);
//     a diagonal tile loads its strip once and uses it as both operands;
//   * warp 1 allocates 256 columns of tensor memory; one of its threads issues
//     four tcgen05.mma (M = N = 128, 32 bytes of k each, FP32 accumulators in
//     tensor memory) per stage and returns the stage with tcgen05.commit;
//   * the accumulator has two 128-column buffers: after every k-step (one
//     strip) the MMA thread moves to the other buffer and warps 4-19 read the
//     finished one (tcgen05.ld, 32 lanes x 32 columns per warp) and add it into
//     double-float registers, so no FP32 sum spans more than one strip (warps
//     2-3 idle: the register budget is shared out per group of four warps);
//   * the epilogue writes the tile's FP64 partial; gram_finish_kernel sums the
//     k-splits in a fixed order and applies the column scales.
//
// FP32 storage: each value is split into three BF16 terms, z = h + m + l
// (h = bf16(z), m = bf16(z - h), l = bf16(z - h - m); both differences are exact
// in FP32), written by split3_kernel into a scratch slab layout of 128 rows per
// slab, term t in slabs [t NB2, (t+1) NB2).  A k-step then loads the three terms
// of both column tiles into three consecutive ring stages and issues the six
// products whose order is at most 2^-16 of z_i z_j (l h, h l, m m, m h, h m,
// h h; smallest first), 24 MMAs per strip of 64 rows, h h into an accumulator
// of its own.  The products are exact; the three dropped ones (m l, l m, l l)
// are below 2^-23 of |z_i z_j|, about the rounding of one FP32 product.
//
// Every wait is bounded: after timeout_ns without progress a CTA records
// GDWD_ETIMEOUT, the other roles of the CTA stop at their next wait, the
// producer waits (bounded) for its copies still in flight, the MMA thread for
// its MMAs, and warp 1 frees the tensor memory before the CTA returns.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "solver.cuh"

namespace gdwd {
namespace {

constexpr int kTT = 128;                       // output tile edge (M = N)
constexpr int kStrip = 128;                    // bytes of k per stage and column
constexpr int kStageBytes = kTT * kStrip;      // one operand of one stage: 16 KB
constexpr int kStages = 6;
constexpr int kEpiWarps = 16;                  // four per tensor-memory lane quarter
constexpr int kEpiWarp0 = 4;                   // warps 0-3: producer, MMA, two idle
constexpr int kThreadsTc = (kEpiWarp0 + kEpiWarps) * 32;
constexpr int kTmemCols = 2 * kTT;             // two FP32 accumulator buffers
// The split of FP32 storage keeps the h h products in their own accumulator
// (columns [256, 512)), so the FP32 sum of a strip's largest terms carries only
// the four roundings of its four MMAs; the five smaller products share the other.
constexpr int kTmemColsSplit = 4 * kTT;
// The tensor core adds each MMA's 16 (8-bit: 32) products into the FP32
// accumulator with one rounding relative to the running sum, so the rows summed
// in FP32 before a fold into double-float bound the error: one 128-byte strip
// per fold (64 rows of 16-bit codes, 128 of E4M3; four MMAs) keeps it within
// four FP32 roundings of the largest partial.
constexpr int kFoldSteps = 1;
constexpr int kSplitRows = 128;                // rows per slab of the BF16 split of FP32 storage
constexpr int64_t kSplitMaxRows = 65536;       // longest contraction the FP32 split serves

struct __align__(1024) TcShared {
  uint8_t a[kStages][kStageBytes];             // 1024-byte aligned (128-byte swizzle atoms)
  uint8_t b[kStages][kStageBytes];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};
constexpr size_t kTcSmem = sizeof(TcShared) + 1024;   // + alignment slack of the dynamic base

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with
// the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO),
// descriptor version 1 (bits 46-47), swizzle mode 2 = 128 B (bits 61-63).  The
// leading-byte offset is unused for swizzled K-major tiles and set to 16 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* tile) {
  const uint64_t addr = smem_u32(tile);
  return ((addr & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_mn128(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTT >> 3) << 17) | ((uint32_t)(kTT >> 4) << 24);
}

// kKind: 0 = FP16, 1 = BF16 (kind::f16, format codes 0 / 1), 2 = E4M3 (kind::f8f6f4, code 0),
// 3 = the BF16 terms of FP32 storage (kind::f16, BF16)
template <int kKind>
__device__ __forceinline__ void mma_128x128(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  constexpr uint32_t idesc = idesc_mn128((kKind == 1 || kKind == 3) ? 1u : 0u);
  if constexpr (kKind == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 8 consecutive FP32 columns: thread t gets lane (taddr.lane + t).
__device__ __forceinline__ void tmem_ld_x8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Waits for phase `parity` of bar.  Returns false when another role of the CTA
// has aborted, or after timeout_ns (then records GDWD_ETIMEOUT and aborts the CTA).
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, TcShared& S, int* err, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*(volatile int*)&S.abort) return false;
    if (globaltimer() - t0 > timeout_ns) {
      atomicCAS(err, 0, (int)GDWD_ETIMEOUT);
      *(volatile int*)&S.abort = 1;
      return false;
    }
  }
}

// ---------------------------------------------------------------- the kernel
template <int kKind>
__global__ void __launch_bounds__(kThreadsTc, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap zmap, int ksplit, int nstrips, int strip_rows,
                   int64_t ksteps, int fold, int tslabs, int64_t n, double* Kpart, int* err, uint64_t timeout_ns) {
  // terms per k-step: one for 16- and 8-bit storage, three for the split of FP32
  // (term t of k-step i in ring stage (i kTerms + t) mod kStages; tslabs = slabs per term)
  constexpr int kTerms = kKind == 3 ? 3 : 1;
  constexpr int kCols = kKind == 3 ? kTmemColsSplit : kTmemCols;
  static_assert(kStages % kTerms == 0, "the terms of a k-step occupy consecutive stages");
  extern __shared__ uint8_t smem_raw[];
  TcShared& S = *reinterpret_cast<TcShared*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x / ksplit, sp = blockIdx.x % ksplit;
  // tile -> (I, J), I >= J, row-major over the lower triangle
  int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= tile) ++I;
  while (I * (I + 1) / 2 > tile) --I;
  const int J = tile - I * (I + 1) / 2;
  const bool diag = (I == J);
  const int64_t k0 = ksteps * sp / ksplit, k1 = ksteps * (sp + 1) / ksplit;
  const int nsteps = (int)(k1 - k0);
  const int nchunks = (nsteps + fold - 1) / fold;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.acc_full[b], 1);
      mbar_init(&S.acc_empty[b], kEpiWarps * 32);
    }
    mbar_init(&S.drain, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = S.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&zmap)) : "memory");
      const uint32_t tx = diag ? (uint32_t)kStageBytes : 2u * kStageBytes;
      const int nsub = nsteps * kTerms;
      int issued = 0;
      for (int u = 0; u < nsub; ++u) {
        const int s = u % kStages;
        if (u >= kStages && !tc_wait(&S.empty[s], (uint32_t)((u / kStages) - 1) & 1u, S, err, timeout_ns)) break;
        const int i = u / kTerms, t = u - i * kTerms;
        const int64_t k = k0 + i;
        const int slab = (int)(k / nstrips);
        const int x = (int)(k - (int64_t)slab * nstrips) * strip_rows;
        mbar_expect_tx(&S.full[s], tx);
        tma_load_3d(S.a[s], &zmap, x, I * kTT, t * tslabs + slab, &S.full[s]);
        if (!diag) tma_load_3d(S.b[s], &zmap, x, J * kTT, t * tslabs + slab, &S.full[s]);
        issued = u + 1;
      }
      if (*(volatile int*)&S.abort) {   // let the copies still in flight land
        for (int u = issued > kStages ? issued - kStages : 0; u < issued; ++u)
          mbar_wait(&S.full[u % kStages], (uint32_t)(u / kStages) & 1u, err, timeout_ns);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int buf = c & 1;
        if (c >= 2 && !tc_wait(&S.acc_empty[buf], (uint32_t)((c >> 1) - 1) & 1u, S, err, timeout_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dt = tbase + (uint32_t)(buf * kTT);
        const int i0 = c * fold, i1 = (i0 + fold < nsteps) ? i0 + fold : nsteps;
        for (int i = i0; i < i1 && ok; ++i) {
          int st[kTerms];
#pragma unroll
          for (int t = 0; t < kTerms; ++t) {
            const int u = i * kTerms + t;
            st[t] = u % kStages;
            if (!tc_wait(&S.full[st[t]], (uint32_t)(u / kStages) & 1u, S, err, timeout_ns)) {
              ok = false;
              break;
            }
          }
          if (!ok) break;
          tc_fence_after();
          if constexpr (kTerms == 1) {
            const uint64_t da = smem_desc_sw128(S.a[st[0]]);
            const uint64_t db = diag ? da : smem_desc_sw128(S.b[st[0]]);
#pragma unroll
            for (int j = 0; j < kStrip / 32; ++j)   // 32 bytes of k per MMA: start address + 2j (16-byte units)
              mma_128x128<kKind>(dt, da + 2 * j, db + 2 * j, (i > i0 || j > 0) ? 1u : 0u);
          } else {
            // the products of the split terms (A term, B term), smallest first
            constexpr int kPa[6] = {2, 0, 1, 1, 0, 0}, kPb[6] = {0, 2, 1, 0, 1, 0};
#pragma unroll
            for (int p = 0; p < 6; ++p) {
              const int sa = st[kPa[p]], sb = st[kPb[p]];
              const uint64_t da = smem_desc_sw128(S.a[sa]);
              const uint64_t db = smem_desc_sw128(diag ? S.a[sb] : S.b[sb]);
              const bool hh = p == 5;                            // h h: its own accumulator
              const uint32_t acc_d = hh ? dt + 2 * kTT : dt;
#pragma unroll
              for (int j = 0; j < kStrip / 32; ++j)
                mma_128x128<kKind>(acc_d, da + 2 * j, db + 2 * j, (i > i0 || (!hh && p > 0) || j > 0) ? 1u : 0u);
            }
          }
          for (int t = 0; t < kTerms; ++t) mma_commit(&S.empty[st[t]]);
        }
        if (ok) mma_commit(&S.acc_full[buf]);
      }
      if (!ok) {   // no MMA may still run when the tensor memory is freed
        mma_commit(&S.drain);
        mbar_wait(&S.drain, 0, err, timeout_ns);
      }
    }
    __syncwarp();
  } else if (warp >= kEpiWarp0) {
    // ------------------------------------------------ epilogue: fold into double-float
    const int quarter = warp & 3;                // the TMEM lane quarter this warp may access
    const int cg = (warp - kEpiWarp0) >> 2;      // columns [32 cg, 32 cg + 32) of the tile
    df acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = df{0.f, 0.f};
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      // after an abort the loop runs out without waiting or reading (a loop
      // without an early exit keeps the accumulators in registers)
      ok = ok && tc_wait(&S.acc_full[buf], (uint32_t)(c >> 1) & 1u, S, err, timeout_ns);
      if (ok) {
        tc_fence_after();
        const uint32_t ta = tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kTT + cg * 32);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          float v[8];
          tmem_ld_x8(ta + 8 * g, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) df_add(acc[8 * g + q], v[q]);
          if constexpr (kKind == 3) {
            tmem_ld_x8(ta + 2 * kTT + 8 * g, v);                 // the h h accumulator
#pragma unroll
            for (int q = 0; q < 8; ++q) df_add(acc[8 * g + q], v[q]);
          }
        }
        tc_fence_before();
        mbar_arrive(&S.acc_empty[buf]);
      }
    }
    if (ok) {
      const int64_t i = (int64_t)I * kTT + quarter * 32 + lane;
      double* out = Kpart + (int64_t)sp * n * n;
      if (i < n) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int64_t j = (int64_t)J * kTT + cg * 32 + c;
          if (j < n && j <= i) out[i * n + j] = df_to_double(acc[c]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols) : "memory");
  }
}

// ---------------------------------------------------------------- host side
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

template <int kKind>
cudaError_t set_smem_once() {
  static cudaError_t e = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    e = cudaFuncSetAttribute(gram_tc_kernel<kKind>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  });
  return e;
}

template <int kKind>
cudaError_t launch_tc(const CUtensorMap& map, int tiles, int ksplit, int nstrips, int strip_rows, int64_t ksteps,
                      int fold, int tslabs, int64_t n, double* Kpart, int* err, uint64_t timeout_ns, cudaStream_t st) {
  cudaError_t e = set_smem_once<kKind>();
  if (e != cudaSuccess) return e;
  gram_tc_kernel<kKind><<<tiles * ksplit, kThreadsTc, kTcSmem, st>>>(map, ksplit, nstrips, strip_rows, ksteps, fold,
                                                                    tslabs, n, Kpart, err, timeout_ns);
  return cudaGetLastError();
}

// The three BF16 terms of a value (each difference exact in FP32).
__device__ __forceinline__ void split3(float x, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(bh);
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(bm);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}

// FP32 slab layout (TB rows per slab) -> three BF16 term arrays of kSplitRows
// rows per slab (NB2 slabs each, term t at slabs [t NB2, (t+1) NB2)); rows past d
// are zero.  Each thread writes 8 consecutive rows of one column of each term
// (one 16-byte store per term).
__global__ void split3_kernel(const float* __restrict__ Z, Layout L, int NB2, uint16_t* __restrict__ out) {
  const int64_t per_slab = (int64_t)kSplitRows * L.n;
  const int64_t term = (int64_t)NB2 * per_slab;
  const int64_t groups = term / 8;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g * 8;
    const int64_t s2 = e / per_slab, rem = e - s2 * per_slab;
    const int64_t i = rem / kSplitRows;
    const int64_t j0 = s2 * kSplitRows + (rem - i * kSplitRows);   // global row of the first of the 8
    int64_t s = j0 / L.TB, jl = j0 - s * L.TB;
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float x = (j0 + q < L.d) ? Z[(s * L.n + i) * L.TB + jl] : 0.f;
      if (++jl == L.TB) {
        jl = 0;
        ++s;
      }
      uint32_t a, b, c;
      split3(x, a, b, c);
      if (q & 1) {
        h[q >> 1] |= a << 16;
        m[q >> 1] |= b << 16;
        l[q >> 1] |= c << 16;
      } else {
        h[q >> 1] = a;
        m[q >> 1] = b;
        l[q >> 1] = c;
      }
    }
    *reinterpret_cast<uint4*>(out + e) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(out + term + e) = make_uint4(m[0], m[1], m[2], m[3]);
    *reinterpret_cast<uint4*>(out + 2 * term + e) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

int split_slabs(const Layout& L) { return (int)((L.d + kSplitRows - 1) / kSplitRows); }

// k-steps (strips of 128 bytes per column) of the operand the kernel reads
int64_t tc_ksteps(int store, const Layout& L) {
  if (store == GDWD_F32) return (int64_t)split_slabs(L) * (kSplitRows * 2 / kStrip);
  const int strip_rows = kStrip / L.esize;
  return (int64_t)L.NB * ((L.TB + strip_rows - 1) / strip_rows);
}

}  // namespace

bool gram_tc_supported(int store, const Layout& L) {
  if (store != GDWD_BF16 && store != GDWD_F16 && store != GDWD_E4M3 && store != GDWD_F32) return false;
  // FP32 storage: the tensor core's FP32 accumulation of a strip's h h products
  // need not round to nearest, so its error can add up with one sign from strip
  // to strip (about 1e-7 of the sum of the strips' magnitudes).  Over a long
  // contraction with cancellation (the d x d Gram of the direct solver over
  // n = 1e6 samples) that is far above the SIMT kernel's error, so the split
  // serves contractions of at most kSplitMaxRows rows.
  if (store == GDWD_F32 && L.d > kSplitMaxRows) return false;
  // tensor-map strides are multiples of 16 bytes; tile rows and the slab count fit int
  if (store != GDWD_F32 && ((int64_t)L.TB * L.esize) % 16 != 0) return false;
  if (L.n > (1LL << 30) || 3LL * split_slabs(L) > (1LL << 30)) return false;
  return encode_tiled() != nullptr;
}

size_t gram_tc_scratch_bytes(int store, const Layout& L) {
  return store == GDWD_F32 ? (size_t)3 * split_slabs(L) * kSplitRows * (size_t)L.n * sizeof(uint16_t) : 0;
}

int gram_tc_ksplit(int store, const Layout& L, int sms) {
  const int64_t Tt = (L.n + kTT - 1) / kTT;
  const int64_t tiles = Tt * (Tt + 1) / 2;
  const int64_t ksteps = tc_ksteps(store, L);
  // one CTA per SM (the ring takes most of shared memory): whole waves only,
  // since a partial second wave doubles the time of the splits in it
  int64_t ks = tiles < sms ? sms / tiles : 1;
  ks = std::min<int64_t>(ks, std::max<int64_t>(1, ksteps / 4));      // >= 4 k-steps per split
  return (int)std::max<int64_t>(1, std::min<int64_t>(ks, 32));
}

cudaError_t run_gram_tc(int store, const Layout& L, int ksplit, double* Kpart, void* scratch, int* err,
                        uint64_t timeout_ns, cudaStream_t st) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const bool split = store == GDWD_F32;
  if (split && !scratch) return cudaErrorInvalidValue;
  const int es = split ? 2 : L.esize;
  const int rows = split ? kSplitRows : L.TB;                       // rows per slab of the operand
  const int slabs = split ? split_slabs(L) : L.NB;                  // slabs per term
  const int strip_rows = kStrip / es;
  const int nstrips = (rows + strip_rows - 1) / strip_rows;
  const int64_t ksteps = (int64_t)slabs * nstrips;
  const int fold = kFoldSteps;
  const int64_t Tt = (L.n + kTT - 1) / kTT;
  const int tiles = (int)(Tt * (Tt + 1) / 2);
  if (split) {
    const int64_t groups = (int64_t)slabs * kSplitRows * L.n / 8;
    const int blocks = (int)std::min<int64_t>((groups + 255) / 256, 152 * 16);
    split3_kernel<<<blocks, 256, 0, st>>>(static_cast<const float*>(L.Z), L, slabs, static_cast<uint16_t*>(scratch));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // the operand in the slab layout as a 3-D tensor: rows within a slab
  // (contiguous), columns, slabs (for the split: the three terms' slabs in turn)
  CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)rows, (cuuint64_t)L.n, (cuuint64_t)slabs * (split ? 3 : 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)rows * es, (cuuint64_t)rows * es * (cuuint64_t)L.n};
  const cuuint32_t box[3] = {(cuuint32_t)strip_rows, (cuuint32_t)kTT, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  void* base = split ? scratch : const_cast<void*>(L.Z);
  const CUresult r = enc(&map, es == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, base, dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  switch (store) {
    case GDWD_F16: return launch_tc<0>(map, tiles, ksplit, nstrips, strip_rows, ksteps, fold, 0, L.n, Kpart, err,
                                       timeout_ns, st);
    case GDWD_BF16: return launch_tc<1>(map, tiles, ksplit, nstrips, strip_rows, ksteps, fold, 0, L.n, Kpart, err,
                                        timeout_ns, st);
    case GDWD_E4M3: return launch_tc<2>(map, tiles, ksplit, nstrips, strip_rows, ksteps, fold, 0, L.n, Kpart, err,
                                        timeout_ns, st);
    case GDWD_F32: return launch_tc<3>(map, tiles, ksplit, nstrips, strip_rows, ksteps, fold, slabs, L.n, Kpart,
                                       err, timeout_ns, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace gdwd
