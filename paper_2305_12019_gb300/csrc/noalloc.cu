// gdwd_gram_noalloc: the Gram matrix K = Z^T Z of a caller's column-major FP32
// matrix, computed without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need the
// Gram matrix: code running under an allocator that must not be re-entered, or
// embedders that own all device memory and only hand out input and output
// buffers.  For them this
// entry point keeps its scratch -- the split-K partial products -- in a
// file-scope __device__ array of fixed size that every GPU which loads the
// library holds until the process exits.
//
// The split-K kernel below is a variant of the slab Gram kernel of setup.cu
// (same 64x64 lower-triangular tiles, FP32 products summed over 16-row chunks
// and folded into double-float accumulators) that reads the caller's
// column-major matrix directly.
#include <algorithm>
#include <mutex>

#include "solver.cuh"

namespace gdwd {
namespace {

constexpr int64_t kScratchDoubles = 4ll << 20;   // 32 MiB of FP64 partial products
constexpr int64_t kMaxN = 2048;                   // kMaxN * kMaxN == kScratchDoubles
constexpr int kTile = 64;
constexpr int kChunk = 16;

static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

// Loads rows [r0, r0+16) of columns [c0, c0+64) of a column-major matrix into sm[16][64].
__device__ __forceinline__ void load_cm(const float* Z, int64_t d, int64_t n, int64_t ldz, int64_t r0, int64_t r1,
                                        int64_t c0, float (*sm)[kTile]) {
  const int t = threadIdx.x;
  const int col = t >> 2, k0 = (t & 3) * 4;
  const int64_t gc = c0 + col;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t gr = r0 + k0 + q;
    sm[k0 + q][col] = (gc < n && gr < r1) ? Z[gc * ldz + gr] : 0.f;
  }
}

// blockIdx.x = tile * ksplit + split; split s covers rows [s * rows, (s+1) * rows)
__global__ void __launch_bounds__(kThreads) gram_cm_kernel(const float* __restrict__ Z, int64_t d, int64_t n,
                                                          int64_t ldz, int ksplit, int64_t rows, double* part) {
  __shared__ __align__(16) float As[kChunk][kTile];
  __shared__ __align__(16) float Bs[kChunk][kTile];
  const int tile = blockIdx.x / ksplit, sp = blockIdx.x % ksplit;
  int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= tile) ++I;
  while (I * (I + 1) / 2 > tile) --I;
  const int J = tile - I * (I + 1) / 2;
  const int64_t r0 = (int64_t)sp * rows;
  const int64_t r1 = (r0 + rows < d) ? r0 + rows : d;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float c[4][4] = {};
  df s[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) s[a][b] = df{0.f, 0.f};
  for (int64_t rr = r0; rr < r1; rr += kChunk) {
    load_cm(Z, d, n, ldz, rr, r1, (int64_t)I * kTile, As);
    load_cm(Z, d, n, ldz, rr, r1, (int64_t)J * kTile, Bs);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[k][ty * 4 + q];
        b[q] = Bs[k][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) c[p][q] = fmaf(a[p], b[q], c[p][q]);
    }
    for (int p = 0; p < 4; ++p)
      for (int q = 0; q < 4; ++q) {
        df_add(s[p][q], c[p][q]);
        c[p][q] = 0.f;
      }
    __syncthreads();
  }
  double* out = part + (int64_t)sp * n * n;
  for (int p = 0; p < 4; ++p)
    for (int q = 0; q < 4; ++q) {
      const int64_t i = (int64_t)I * kTile + ty * 4 + p, j = (int64_t)J * kTile + tx * 4 + q;
      if (i < n && j < n && i >= j) out[i * n + j] = df_to_double(s[p][q]);
    }
}

__global__ void gram_cm_finish(const double* part, int ksplit, int64_t n, double* K) {
  const int64_t total = n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    if (j > i) continue;
    double k = 0.0;
    for (int s = 0; s < ksplit; ++s) k += part[(int64_t)s * total + idx];
    K[i * n + j] = k;
    K[j * n + i] = k;
  }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached; host code must never use the symbol itself.
double* scratch_address(int dev, cudaError_t* err) {
  static std::mutex mu;
  static double* addr[64] = {};
  static bool done[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!done[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    addr[dev] = static_cast<double*>(p);
    done[dev] = true;
  }
  *err = cudaSuccess;
  return addr[dev];
}

}  // namespace
}  // namespace gdwd

using namespace gdwd;

extern "C" gdwd_status gdwd_gram_noalloc(const float* Z, int64_t d, int64_t n, int64_t ldz, double* K, void* stream) {
  if (!Z || !K || d < 1 || n < 1 || ldz < d) return GDWD_EINVAL;
  // n > 2048 is beyond the fixed scratch; n is bounded before it is squared
  if (n > kMaxN || n * n > kScratchDoubles) return GDWD_EINVAL;
  // an asynchronous error of earlier, unrelated work is left for its owner to
  // read: this call launches nothing on a context that already failed
  if (cudaPeekAtLastError() != cudaSuccess) return GDWD_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GDWD_ECUDA;
  cudaError_t e = cudaSuccess;
  double* scratch = scratch_address(dev, &e);
  if (!scratch) return GDWD_ECUDA;
  int sms = 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return GDWD_ECUDA;
  const int T = (int)((n + kTile - 1) / kTile);
  const int tiles = T * (T + 1) / 2;
  int ksplit = std::max(1, std::min<int>((2 * sms + tiles - 1) / tiles, 16));
  ksplit = (int)std::min<int64_t>(ksplit, kScratchDoubles / (n * n));
  ksplit = (int)std::min<int64_t>(ksplit, (d + kChunk - 1) / kChunk);
  ksplit = std::max(ksplit, 1);
  // rows per split: a multiple of the 16-row chunk
  const int64_t rows = ((d + ksplit - 1) / ksplit + kChunk - 1) / kChunk * kChunk;
  cudaStream_t st = (cudaStream_t)stream;
  gram_cm_kernel<<<tiles * ksplit, kThreads, 0, st>>>(Z, d, n, ldz, ksplit, rows, scratch);
  if (cudaGetLastError() != cudaSuccess) return GDWD_ECUDA;
  gram_cm_finish<<<(int)std::min<int64_t>((n * n + 255) / 256, 2048), 256, 0, st>>>(scratch, ksplit, n, K);
  if (cudaGetLastError() != cudaSuccess) return GDWD_ECUDA;
  return GDWD_OK;
}
