// The two streaming passes over the stored Z, shared by the persistent
// iteration kernel and the stand-alone product kernels (gdwd_apply).
//
//   pass A:  partial[i][s] = sum_{j in slab s} Zq_ji g'_j          (Z~^T g' before scaling)
//   pass B:  t_j = sum_i Zq_ji cq_i,  ta_j = sum_i Zq_ji aq_i      (Z~ c, Z~ alpha)
//
// A CTA owns whole slabs (see Layout).  Chunks of CW columns of a slab are
// contiguous in HBM and are fetched by one thread with cp.async.bulk into a
// ring of `stages` shared-memory buffers, each guarded by an mbarrier with
// transaction counting; all 256 threads consume a chunk, then thread 0 refills
// the freed buffer.  Every wait is bounded.
#pragma once

#include "solver.cuh"

namespace gdwd {

struct Ring {
  uint8_t* buf;        // stages * stage_bytes, 128-byte aligned
  uint64_t* bars;      // stages mbarriers
  int stages;
  int stage_bytes;
  uint32_t phase;      // parity bit per stage (identical in all threads)
  int prefetched;      // chunks of the next stream_slabs already issued (identical in all threads)
};

__device__ __forceinline__ void ring_init(Ring& rg) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < rg.stages; ++s) mbar_init(&rg.bars[s], 1);
    fence_mbar_init();
  }
  rg.phase = 0;
  rg.prefetched = 0;
  __syncthreads();
}

// A cursor over the Z chunks of this CTA's sequence (slab cta + k grid, chunk cc
// of CW columns within it), advanced one chunk at a time with no division: the
// address of the next copy is ready when the stage it refills frees up.
struct ZCursor {
  const uint8_t* slab;   // first byte of the current slab
  int64_t slab_step;     // bytes from one of this CTA's slabs to the next
  int64_t chunk_bytes;   // bytes of a full chunk (CW columns)
  int cc, nch, k;        // chunk within the slab, chunks per slab, slab ordinal
  uint32_t last_bytes;   // bytes of a slab's last chunk
  __device__ void init(const Layout& L, int cta, int grid, int first) {
    const int64_t col_bytes = (int64_t)L.TB * L.esize;
    nch = (int)((L.n + L.CW - 1) / L.CW);
    chunk_bytes = (int64_t)L.CW * col_bytes;
    last_bytes = (uint32_t)((L.n - (int64_t)(nch - 1) * L.CW) * col_bytes);
    slab_step = (int64_t)grid * L.n * col_bytes;
    k = first / nch;
    cc = first - k * nch;
    slab = reinterpret_cast<const uint8_t*>(L.Z) + ((int64_t)cta + (int64_t)k * grid) * L.n * col_bytes;
  }
  __device__ void get(const uint8_t*& src, uint32_t& bytes) const {
    src = slab + (int64_t)cc * chunk_bytes;
    bytes = cc == nch - 1 ? last_bytes : (uint32_t)chunk_bytes;
  }
  __device__ void advance() {
    if (++cc == nch) {
      cc = 0;
      ++k;
      slab += slab_step;
    }
  }
};

// Issues the first chunks of the next stream_slabs early (the ring must be idle:
// every chunk of the previous stream consumed), so that they arrive while the
// CTA does other work.
__device__ __forceinline__ void ring_prefetch(const Layout& L, Ring& rg, int cta, int grid) {
  const int nch = (int)((L.n + L.CW - 1) / L.CW);
  const int nmy = (L.NB > cta) ? (L.NB - cta + grid - 1) / grid : 0;
  const int pre = min(rg.stages, nmy * nch);
  // issued by the last warp: thread 0 holds the first n-space row of the phase
  // that runs meanwhile
  if (threadIdx.x == kThreads - 32) {
    ZCursor zc;
    zc.init(L, cta, grid, 0);
    for (int c = 0; c < pre; ++c) {
      const uint8_t* src;
      uint32_t bytes;
      zc.get(src, bytes);
      zc.advance();
      mbar_expect_tx(&rg.bars[c], bytes);
      bulk_g2s_z(rg.buf + (size_t)c * rg.stage_bytes, src, bytes, &rg.bars[c]);
    }
  }
  rg.prefetched = pre;
}

// Waits, bounded, until the bulk copies of chunks [c0, c1) of the current stream
// have landed (chunk c sits in stage c % stages; `flipped` marks a chunk c0
// whose stage parity was already toggled by the wait that gave up).  A CTA that
// leaves the kernel early calls this first, so that no copy it issued is still
// writing its shared memory when it exits.  Every wait is bounded by tmo; if
// one runs out the CTA leaves all the same (the error word is already set).
__device__ __forceinline__ void ring_drain(Ring& rg, int c0, int c1, bool flipped, int* err, uint64_t tmo) {
  if (threadIdx.x == 0) {
    for (int c = c0; c < c1; ++c) {
      const int st = c % rg.stages;
      uint32_t par = (rg.phase >> st) & 1u;
      if (flipped && c == c0) par ^= 1u;
      if (!mbar_wait(&rg.bars[st], par, err, tmo)) break;
    }
  }
  __syncthreads();
}

// Chunks issued by ring_prefetch and not yet streamed: drained before an early exit.
__device__ __forceinline__ void ring_drain_prefetched(Ring& rg, int* err, uint64_t tmo) {
  if (rg.prefetched > 0) ring_drain(rg, 0, rg.prefetched, false, err, tmo);
  rg.prefetched = 0;
}

// A stream without extra chunks.
struct NoExtra {
  __device__ int count() const { return 0; }
  __device__ void issue(int, uint8_t*, uint64_t*) const {}
  __device__ void consume(int, const uint8_t*) {}
};

// Streams every chunk of the slabs cta, cta+grid, ... through the ring and
// calls f.chunk / f.end_slab.  An optional source x adds x->count() extra chunks
// (other data the CTA needs during the pass): they take the ring right after
// the first min(stages, Z chunks) chunks of Z -- the ones ring_prefetch may
// have issued -- so their copies and their work overlap the rest of the pass.
// x->issue(e, dst, bar) sets the transaction count and issues the copies of
// extra chunk e (one thread); x->consume(e, buf) runs on all threads.  Returns
// false (all threads) on a timed-out wait, after the copies still in flight
// have landed.
template <typename T, typename F, typename X = NoExtra>
__device__ bool stream_slabs(const Layout& L, Ring& rg, int cta, int grid, int* err, uint64_t tmo, int* s_abort,
                             F& f, X* x = nullptr) {
  const int nch = (int)((L.n + L.CW - 1) / L.CW);
  const int nmy = (L.NB > cta) ? (L.NB - cta + grid - 1) / grid : 0;
  const int nz = nmy * nch;
  const int nx = x ? x->count() : 0;
  const int xpos = min(rg.stages, nz);
  const int total = nz + nx;

  // the issue side (thread 0) walks the Z chunks from the first one not yet
  // issued by ring_prefetch; the extra chunks sit at positions [xpos, xpos + nx)
  ZCursor iz;
  if (threadIdx.x == 0) iz.init(L, cta, grid, rg.prefetched);
  auto issue = [&](int c) {
    const int st = c % rg.stages;
    uint8_t* dst = rg.buf + (size_t)st * rg.stage_bytes;
    if (c >= xpos && c < xpos + nx) {
      x->issue(c - xpos, dst, &rg.bars[st]);
      return;
    }
    const uint8_t* src;
    uint32_t bytes;
    iz.get(src, bytes);
    iz.advance();
    mbar_expect_tx(&rg.bars[st], bytes);
    bulk_g2s_z(dst, src, bytes, &rg.bars[st]);
  };

  if (threadIdx.x == 0) {
    const int pre = min(rg.stages, total);
    for (int c = rg.prefetched; c < pre; ++c) issue(c);
  }
  rg.prefetched = 0;
  int k = 0, cc = 0;   // slab ordinal and chunk of the next Z chunk consumed
  for (int c = 0; c < total; ++c) {
    const int st = c % rg.stages;
    const bool extra = c >= xpos && c < xpos + nx;
    const int s = cta + k * grid;
    const int col0 = cc * L.CW;
    const int cw = (int)min((int64_t)L.CW, L.n - col0);
    if (!mbar_wait(&rg.bars[st], (rg.phase >> st) & 1u, err, tmo)) *s_abort = 1;
    rg.phase ^= 1u << st;
    const uint8_t* buf = rg.buf + (size_t)st * rg.stage_bytes;
    if (extra) x->consume(c - xpos, buf);
    else f.chunk(reinterpret_cast<const T*>(buf), k, s, col0, cw);
    __syncthreads();
    if (*(volatile int*)s_abort) {
      // chunks c .. min(c + stages, total) - 1 were issued and may be in flight
      ring_drain(rg, c, min(c + rg.stages, total), true, err, tmo);
      return false;
    }
    if (threadIdx.x == 0 && c + rg.stages < total) issue(c + rg.stages);
    if (!extra) {
      if (cc == nch - 1) f.end_slab(k, s);
      if (++cc == nch) {
        cc = 0;
        ++k;
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// pass A: dots down the columns of each chunk, 32 columns per round.  8 lanes
// share a column (8 consecutive lanes read 8 consecutive 16-byte vectors of one
// column: no shared-memory bank conflicts), two independent accumulators per
// lane, then a 3-step shuffle reduction.
// ---------------------------------------------------------------------------
template <typename T>
struct PassA {
  using CT = typename ElemTraits<T>::compute_t;
  static constexpr int VEC = ElemTraits<T>::kVec;
  const CT* gp;       // shared: my slabs' g' (slab k at gp + k * TB)
  CT* partial;        // global n x NB
  int TB, NB, Q, H;

  __device__ void chunk(const T* buf, int k, int s, int col0, int cw) {
    const int h = threadIdx.x & 7, cl = threadIdx.x >> 3;
    const CT* g = gp + (size_t)k * TB;
    for (int c0 = 0; c0 < cw; c0 += kThreads / 8) {
      const int col = c0 + cl;
      CT acc0 = 0, acc1 = 0;
      if (col < cw) {
        const T* cp = buf + (size_t)col * TB;
        int v = h;
        for (; v + 8 < Q; v += 16) {
          CT e0[VEC], e1[VEC], g0[VEC], g1[VEC];
          ElemTraits<T>::load(cp + v * VEC, e0);
          ElemTraits<T>::load(cp + (v + 8) * VEC, e1);
          load_ct<VEC>(g + v * VEC, g0);
          load_ct<VEC>(g + (v + 8) * VEC, g1);
#pragma unroll
          for (int kk = 0; kk < VEC; ++kk) {
            acc0 = fma(e0[kk], g0[kk], acc0);
            acc1 = fma(e1[kk], g1[kk], acc1);
          }
        }
        if (v < Q) {
          CT e0[VEC], g0[VEC];
          ElemTraits<T>::load(cp + v * VEC, e0);
          load_ct<VEC>(g + v * VEC, g0);
#pragma unroll
          for (int kk = 0; kk < VEC; ++kk) acc0 = fma(e0[kk], g0[kk], acc0);
        }
      }
      CT acc = acc0 + acc1;
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (h == 0 && col < cw) partial[(size_t)(col0 + col) * NB + s] = acc;
    }
  }
  __device__ void end_slab(int, int) {}
};

// Pass A with two columns per lane per round (64 columns per round): every
// vector of the right-hand side read from shared memory serves two Z vectors.
template <typename T>
struct PassA2 {
  using CT = typename ElemTraits<T>::compute_t;
  static constexpr int VEC = ElemTraits<T>::kVec;
  const CT* gp;       // shared: my slabs' right-hand side (slab k at gp + k * TB)
  CT* partial;        // global n x NB
  int TB, NB, Q;

  __device__ void chunk(const T* buf, int k, int s, int col0, int cw) {
    const int h = threadIdx.x & 7, cl = threadIdx.x >> 3;
    const CT* g = gp + (size_t)k * TB;
    for (int c0 = 0; c0 < cw; c0 += 2 * (kThreads / 8)) {
      const int ca = c0 + cl, cb = ca + kThreads / 8;
      const bool va = ca < cw, vb = cb < cw;
      const T* pa = buf + (size_t)(va ? ca : 0) * TB;
      const T* pb = buf + (size_t)(vb ? cb : 0) * TB;
      CT a0 = 0, a1 = 0, b0 = 0, b1 = 0;
      int v = h;
      for (; v + 8 < Q; v += 16) {
        CT ea0[VEC], ea1[VEC], eb0[VEC], eb1[VEC], g0[VEC], g1[VEC];
        ElemTraits<T>::load(pa + v * VEC, ea0);
        ElemTraits<T>::load(pa + (v + 8) * VEC, ea1);
        ElemTraits<T>::load(pb + v * VEC, eb0);
        ElemTraits<T>::load(pb + (v + 8) * VEC, eb1);
        load_ct<VEC>(g + v * VEC, g0);
        load_ct<VEC>(g + (v + 8) * VEC, g1);
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk) {
          a0 = fma(ea0[kk], g0[kk], a0);
          a1 = fma(ea1[kk], g1[kk], a1);
          b0 = fma(eb0[kk], g0[kk], b0);
          b1 = fma(eb1[kk], g1[kk], b1);
        }
      }
      if (v < Q) {
        CT ea[VEC], eb[VEC], g0[VEC];
        ElemTraits<T>::load(pa + v * VEC, ea);
        ElemTraits<T>::load(pb + v * VEC, eb);
        load_ct<VEC>(g + v * VEC, g0);
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk) {
          a0 = fma(ea[kk], g0[kk], a0);
          b0 = fma(eb[kk], g0[kk], b0);
        }
      }
      CT xa = a0 + a1, xb = b0 + b1;
      xa += __shfl_xor_sync(0xffffffffu, xa, 4);
      xb += __shfl_xor_sync(0xffffffffu, xb, 4);
      xa += __shfl_xor_sync(0xffffffffu, xa, 2);
      xb += __shfl_xor_sync(0xffffffffu, xb, 2);
      xa += __shfl_xor_sync(0xffffffffu, xa, 1);
      xb += __shfl_xor_sync(0xffffffffu, xb, 1);
      if (h == 0) {
        if (va) partial[(size_t)(col0 + ca) * NB + s] = xa;
        if (vb) partial[(size_t)(col0 + cb) * NB + s] = xb;
      }
    }
  }
  __device__ void end_slab(int, int) {}
};

// Running sums of pass B: FP64 storage accumulates in double, FP32 storage
// accumulates each chunk in float and folds it into a double-float.
template <typename CT>
struct RunAcc;
template <>
struct RunAcc<double> {
  using part_t = double;   // what the end-of-slab reduction stores per group
  double v = 0.0;
  __device__ void fold(double c) { v += c; }
  __device__ void merge(part_t p) { v += p; }
  __device__ part_t part() const { return v; }
  __device__ double get() const { return v; }
  __device__ df get_df() const { return df_from(v); }
  __device__ void reset() { v = 0.0; }
};
template <>
struct RunAcc<float> {
  using part_t = float2;   // (hi, lo): the groups are added in double-float, FP32 pipes only
  df v{0.f, 0.f};
  __device__ void fold(float c) { df_add(v, c); }
  __device__ void merge(part_t p) { df_add(v, df{p.x, p.y}); }
  __device__ part_t part() const { return make_float2(v.hi, v.lo); }
  __device__ double get() const { return df_to_double(v); }
  __device__ df get_df() const { return df_sum(df{0.f, 0.f}, v); }
  __device__ void reset() { v.hi = 0.f; v.lo = 0.f; }
};

// ---------------------------------------------------------------------------
// pass B: axpys across the columns of each chunk for two right-hand sides.
// Thread t owns vector qv = t % Q of the column group t / Q (Q = TB / VEC <= 256),
// so the threads of a step read consecutive 16-byte vectors (conflict-free).
// At the end of a slab the groups are summed through shared memory and the
// row epilogue Epi runs once per row j of the slab with t_j and ta_j as
// double-float values (given the global row and its index among the CTA's slab
// rows, k * TB + j for its k-th slab).
// ---------------------------------------------------------------------------
template <typename T, typename Epi>
struct PassB {
  using CT = typename ElemTraits<T>::compute_t;
  static constexpr int VEC = ElemTraits<T>::kVec;
  const CT* cv;       // shared n: coefficients of RHS 1
  const CT* av;       // shared n: coefficients of RHS 2 (may equal cv)
  double* red;        // shared 2 * G * TB
  int TB, Q, G;
  int64_t d;
  bool two;           // second right-hand side present
  Epi* epi;
  RunAcc<CT> rc[VEC], ra[VEC];

  __device__ void chunk(const T* buf, int k, int s, int col0, int cw) {
    const int grp = threadIdx.x / Q, qv = threadIdx.x - grp * Q;
    if (grp >= G) return;
    CT ac[VEC], aa[VEC];
#pragma unroll
    for (int kk = 0; kk < VEC; ++kk) ac[kk] = aa[kk] = 0;
    const T* base = buf + qv * VEC;
    if (two) {
      // four columns per step, two accumulator sets: the shared-memory loads of
      // a step are issued together and the FMA chains are half as long
      CT bc[VEC], ba[VEC];
#pragma unroll
      for (int kk = 0; kk < VEC; ++kk) bc[kk] = ba[kk] = 0;
      int col = grp;
      for (; col + 3 * G < cw; col += 4 * G) {
        CT e0[VEC], e1[VEC], e2[VEC], e3[VEC];
        ElemTraits<T>::load(base + (size_t)col * TB, e0);
        ElemTraits<T>::load(base + (size_t)(col + G) * TB, e1);
        ElemTraits<T>::load(base + (size_t)(col + 2 * G) * TB, e2);
        ElemTraits<T>::load(base + (size_t)(col + 3 * G) * TB, e3);
        const CT c0 = cv[col0 + col], a0 = av[col0 + col];
        const CT c1 = cv[col0 + col + G], a1 = av[col0 + col + G];
        const CT c2 = cv[col0 + col + 2 * G], a2 = av[col0 + col + 2 * G];
        const CT c3 = cv[col0 + col + 3 * G], a3 = av[col0 + col + 3 * G];
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk) {
          ac[kk] = fma(e0[kk], c0, ac[kk]);
          aa[kk] = fma(e0[kk], a0, aa[kk]);
          bc[kk] = fma(e1[kk], c1, bc[kk]);
          ba[kk] = fma(e1[kk], a1, ba[kk]);
        }
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk) {
          ac[kk] = fma(e2[kk], c2, ac[kk]);
          aa[kk] = fma(e2[kk], a2, aa[kk]);
          bc[kk] = fma(e3[kk], c3, bc[kk]);
          ba[kk] = fma(e3[kk], a3, ba[kk]);
        }
      }
      for (; col < cw; col += G) {
        CT e[VEC];
        ElemTraits<T>::load(base + (size_t)col * TB, e);
        const CT c = cv[col0 + col], a = av[col0 + col];
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk) {
          ac[kk] = fma(e[kk], c, ac[kk]);
          aa[kk] = fma(e[kk], a, aa[kk]);
        }
      }
#pragma unroll
      for (int kk = 0; kk < VEC; ++kk) {
        ac[kk] += bc[kk];
        aa[kk] += ba[kk];
      }
    } else {
      for (int col = grp; col < cw; col += G) {
        CT e[VEC];
        ElemTraits<T>::load(base + (size_t)col * TB, e);
        const CT c = cv[col0 + col];
#pragma unroll
        for (int kk = 0; kk < VEC; ++kk) ac[kk] = fma(e[kk], c, ac[kk]);
      }
    }
#pragma unroll
    for (int kk = 0; kk < VEC; ++kk) {
      rc[kk].fold(ac[kk]);
      ra[kk].fold(aa[kk]);
    }
  }

  __device__ void end_slab(int k, int s) {
    using P = typename RunAcc<CT>::part_t;
    P* redp = reinterpret_cast<P*>(red);   // 2 G TB parts (8 bytes each, like the doubles it was sized for)
    const int grp = threadIdx.x / Q, qv = threadIdx.x - grp * Q;
    if (grp < G) {
#pragma unroll
      for (int kk = 0; kk < VEC; ++kk) {
        redp[(size_t)grp * TB + qv * VEC + kk] = rc[kk].part();
        redp[(size_t)(G + grp) * TB + qv * VEC + kk] = ra[kk].part();
        rc[kk].reset();
        ra[kk].reset();
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < TB; j += blockDim.x) {
      RunAcc<CT> t, ta;
      for (int gq = 0; gq < G; ++gq) {
        t.merge(redp[(size_t)gq * TB + j]);
        ta.merge(redp[(size_t)(G + gq) * TB + j]);
      }
      const int64_t gj = (int64_t)s * TB + j;
      if (gj < d) epi->row(gj, k * TB + j, t.get_df(), ta.get_df());
    }
    __syncthreads();
  }
};

// pass B and, on the same chunks, pass A with another vector (one read of Z
// serves Z~ [c, alpha] and Z~^T u)
template <typename T, typename Epi>
struct PassBA {
  PassB<T, Epi>* b;
  PassA2<T>* a;
  __device__ void chunk(const T* buf, int k, int s, int col0, int cw) {
    b->chunk(buf, k, s, col0, cw);
    a->chunk(buf, k, s, col0, cw);
  }
  __device__ void end_slab(int k, int s) { b->end_slab(k, s); }
};

}  // namespace gdwd
