// K = Zq^T Zq on the 5th-generation tensor cores, for BF16, FP16 and E4M3
// storage.
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
// The tensor core adds each MMA's 16 (8-bit: 32) products into the FP32
// accumulator with one rounding relative to the running sum, so the rows summed
// in FP32 before a fold into double-float bound the error: one 128-byte strip
// per fold (64 rows of 16-bit codes, 128 of E4M3; four MMAs) keeps it within
// four FP32 roundings of the largest partial.
constexpr int kFoldSteps = 1;

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

// kKind: 0 = FP16, 1 = BF16 (kind::f16, format codes 0 / 1), 2 = E4M3 (kind::f8f6f4, code 0)
template <int kKind>
__device__ __forceinline__ void mma_128x128(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  constexpr uint32_t idesc = idesc_mn128(kKind == 1 ? 1u : 0u);
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
                   int64_t ksteps, int fold, int64_t n, double* Kpart, int* err, uint64_t timeout_ns) {
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
                 "r"(kTmemCols)
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
      int issued = 0;
      for (int i = 0; i < nsteps; ++i) {
        const int s = i % kStages;
        if (i >= kStages && !tc_wait(&S.empty[s], (uint32_t)((i / kStages) - 1) & 1u, S, err, timeout_ns)) break;
        const int64_t k = k0 + i;
        const int slab = (int)(k / nstrips);
        const int x = (int)(k - (int64_t)slab * nstrips) * strip_rows;
        mbar_expect_tx(&S.full[s], tx);
        tma_load_3d(S.a[s], &zmap, x, I * kTT, slab, &S.full[s]);
        if (!diag) tma_load_3d(S.b[s], &zmap, x, J * kTT, slab, &S.full[s]);
        issued = i + 1;
      }
      if (*(volatile int*)&S.abort) {   // let the copies still in flight land
        for (int i = issued > kStages ? issued - kStages : 0; i < issued; ++i)
          mbar_wait(&S.full[i % kStages], (uint32_t)(i / kStages) & 1u, err, timeout_ns);
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
        for (int i = i0; i < i1; ++i) {
          const int s = i % kStages;
          if (!tc_wait(&S.full[s], (uint32_t)(i / kStages) & 1u, S, err, timeout_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t da = smem_desc_sw128(S.a[s]);
          const uint64_t db = diag ? da : smem_desc_sw128(S.b[s]);
#pragma unroll
          for (int j = 0; j < kStrip / 32; ++j)   // 32 bytes of k per MMA: start address + 2j (16-byte units)
            mma_128x128<kKind>(dt, da + 2 * j, db + 2 * j, (i > i0 || j > 0) ? 1u : 0u);
          mma_commit(&S.empty[s]);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
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
                      int fold, int64_t n, double* Kpart, int* err, uint64_t timeout_ns, cudaStream_t st) {
  cudaError_t e = set_smem_once<kKind>();
  if (e != cudaSuccess) return e;
  gram_tc_kernel<kKind><<<tiles * ksplit, kThreadsTc, kTcSmem, st>>>(map, ksplit, nstrips, strip_rows, ksteps, fold,
                                                                    n, Kpart, err, timeout_ns);
  return cudaGetLastError();
}

}  // namespace

bool gram_tc_supported(int store, const Layout& L) {
  if (store != GDWD_BF16 && store != GDWD_F16 && store != GDWD_E4M3) return false;
  // tensor-map strides are multiples of 16 bytes; tile rows and the slab count fit int
  if (((int64_t)L.TB * L.esize) % 16 != 0 || L.n > (1LL << 30)) return false;
  return encode_tiled() != nullptr;
}

int gram_tc_ksplit(const Layout& L, int sms) {
  const int64_t Tt = (L.n + kTT - 1) / kTT;
  const int64_t tiles = Tt * (Tt + 1) / 2;
  const int strip_rows = kStrip / L.esize;
  const int64_t ksteps = (int64_t)L.NB * ((L.TB + strip_rows - 1) / strip_rows);
  int64_t ks = (sms + tiles - 1) / tiles;                           // at least one wave of CTAs
  ks = std::min<int64_t>(ks, std::max<int64_t>(1, ksteps / 4));      // >= 4 k-steps per split
  return (int)std::max<int64_t>(1, std::min<int64_t>(ks, 32));
}

cudaError_t run_gram_tc(int store, const Layout& L, int ksplit, double* Kpart, int* err, uint64_t timeout_ns,
                        cudaStream_t st) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const int es = L.esize;
  const int strip_rows = kStrip / es;
  const int nstrips = (L.TB + strip_rows - 1) / strip_rows;
  const int64_t ksteps = (int64_t)L.NB * nstrips;
  const int fold = kFoldSteps;
  const int64_t Tt = (L.n + kTT - 1) / kTT;
  const int tiles = (int)(Tt * (Tt + 1) / 2);
  // Z in the slab layout as a 3-D tensor: rows within a slab (contiguous), columns, slabs
  CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)L.TB, (cuuint64_t)L.n, (cuuint64_t)L.NB};
  const cuuint64_t strides[2] = {(cuuint64_t)L.TB * es, (cuuint64_t)L.TB * es * (cuuint64_t)L.n};
  const cuuint32_t box[3] = {(cuuint32_t)strip_rows, (cuuint32_t)kTT, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(&map, es == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                         const_cast<void*>(L.Z), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  switch (store) {
    case GDWD_F16: return launch_tc<0>(map, tiles, ksplit, nstrips, strip_rows, ksteps, fold, L.n, Kpart, err,
                                       timeout_ns, st);
    case GDWD_BF16: return launch_tc<1>(map, tiles, ksplit, nstrips, strip_rows, ksteps, fold, L.n, Kpart, err,
                                        timeout_ns, st);
    case GDWD_E4M3: return launch_tc<2>(map, tiles, ksplit, nstrips, strip_rows, ksteps, fold, L.n, Kpart, err,
                                        timeout_ns, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace gdwd
