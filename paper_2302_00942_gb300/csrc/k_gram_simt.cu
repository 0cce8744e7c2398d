// Step a3, FP32 "plain" form: the reductions over N, K = Phi^T Phi (upper
// tiles) and Y' = Phi^T F, on SIMT FP32 FMA (Sec. 2.4: M = B^T A, Y = B^T F;
// the diagonal column scales are applied by the reduce kernel).
//
// Each CTA computes one split-K piece (GramUnit) of a 128 x 128 tile:
//   C[f, g] = sum_{n in [k0, k1)} Psi[i0 + f][n] * Psi[j0 + g][n].
// Psi is feature-major (n contiguous), so every row of a tile is a contiguous
// run of points: 16-point slabs are read with float4 loads and transposed
// into shared memory.  Each thread holds an 8 x 8 outer-product tile in
// registers; the next slab's loads are issued before the current slab's
// FMAs, so the global-memory latency hides behind 16 x 64 FMAs per thread.
//
// Accuracy: every 256 points each accumulator is folded into a running FP32
// sum by an exact TwoSum (Knuth), and the rounding error of that addition
// becomes the accumulator's starting value for the next 256 points: the
// compensated (Kahan-type) sum without a carry array, so the rounding error
// of a partial is ~sqrt(16) ulps of the partial instead of growing with N;
// the split-K partials are summed in a fixed order, compensated, by the
// reduce kernel.  The running sums live in shared memory ([entry][thread],
// 64 KB, conflict-free), so a thread holds only its 64 accumulators and the
// operands: ~100 registers, two CTAs (16 warps) per SM to hide latency.
#include <cuda_runtime.h>
#include "kernels.h"

namespace rfd {

namespace {

constexpr int kT = kSimtTile;   // 128
constexpr int kK = kSimtK;      // 16 points per slab
constexpr int kThreads = 256;   // 16 x 16 threads, 8 x 8 outputs each
constexpr int kFold = 16;       // slabs per Kahan fold (256 points)
constexpr int kSumBytes = 64 * kThreads * 4;  // running sums: 64 entries per thread

__global__ void __launch_bounds__(kThreads, 2)
gram_simt_kernel(const float* __restrict__ psi, int64_t n_pad, const GramUnit* __restrict__ units,
                 float* __restrict__ partials) {
  const GramUnit u = units[blockIdx.x];
  __shared__ __align__(16) float As[kK][kT + 4];
  __shared__ __align__(16) float Bs[kK][kT + 4];
  extern __shared__ float sum_s[];  // [64][kThreads]: entry (i, j) of thread t at (8 i + j) kThreads + t
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      acc[i][j] = 0.f;
      sum_s[(8 * i + j) * kThreads + threadIdx.x] = 0.f;
    }

  // loader mapping: 128 rows x 4 float4 per slab and operand -> 2 float4 per thread
  const int lrow = threadIdx.x >> 2;       // 0..63
  const int lq = threadIdx.x & 3;          // which float4 of the 16-point slab
  const float* arow0 = psi + (size_t)(u.i0 + lrow) * n_pad + lq * 4;
  const float* arow1 = psi + (size_t)(u.i0 + lrow + 64) * n_pad + lq * 4;
  const float* brow0 = psi + (size_t)(u.j0 + lrow) * n_pad + lq * 4;
  const float* brow1 = psi + (size_t)(u.j0 + lrow + 64) * n_pad + lq * 4;
  // The plan allocates Psi with whole 128-row blocks past every tile start, so
  // these rows always exist; rows beyond a tile's valid range only feed
  // output rows/columns that the reduce ignores.

  float4 va0, va1, vb0, vb1;  // the next slab, loaded one slab ahead
  if (u.k0 < u.k1) {
    va0 = __ldg(reinterpret_cast<const float4*>(arow0 + u.k0));
    va1 = __ldg(reinterpret_cast<const float4*>(arow1 + u.k0));
    vb0 = __ldg(reinterpret_cast<const float4*>(brow0 + u.k0));
    vb1 = __ldg(reinterpret_cast<const float4*>(brow1 + u.k0));
  }
  int slab = 0;
  for (int64_t k = u.k0; k < u.k1; k += kK, ++slab) {
    __syncthreads();  // every thread is done reading the previous slab
    As[lq * 4 + 0][lrow] = va0.x; As[lq * 4 + 1][lrow] = va0.y; As[lq * 4 + 2][lrow] = va0.z; As[lq * 4 + 3][lrow] = va0.w;
    As[lq * 4 + 0][lrow + 64] = va1.x; As[lq * 4 + 1][lrow + 64] = va1.y; As[lq * 4 + 2][lrow + 64] = va1.z; As[lq * 4 + 3][lrow + 64] = va1.w;
    Bs[lq * 4 + 0][lrow] = vb0.x; Bs[lq * 4 + 1][lrow] = vb0.y; Bs[lq * 4 + 2][lrow] = vb0.z; Bs[lq * 4 + 3][lrow] = vb0.w;
    Bs[lq * 4 + 0][lrow + 64] = vb1.x; Bs[lq * 4 + 1][lrow + 64] = vb1.y; Bs[lq * 4 + 2][lrow + 64] = vb1.z; Bs[lq * 4 + 3][lrow + 64] = vb1.w;
    __syncthreads();
    const int64_t kn = k + kK;
    if (kn < u.k1) {  // in flight during this slab's FMAs
      va0 = __ldg(reinterpret_cast<const float4*>(arow0 + kn));
      va1 = __ldg(reinterpret_cast<const float4*>(arow1 + kn));
      vb0 = __ldg(reinterpret_cast<const float4*>(brow0 + kn));
      vb1 = __ldg(reinterpret_cast<const float4*>(brow1 + kn));
    }
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      const float4 a_lo = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 a_hi = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
      const float4 b_lo = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float4 b_hi = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
      const float a[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
      const float b[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if ((slab + 1) % kFold == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // sum + acc = t + e exactly; e carries on in acc
          float& sm = sum_s[(8 * i + j) * kThreads + threadIdx.x];
          const float sv = sm;
          const float t = sv + acc[i][j];
          const float bp = t - sv;
          acc[i][j] = (sv - (t - bp)) + (acc[i][j] - bp);
          sm = t;
        }
    }
  }
  float* out = partials + u.out;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = (i < 4) ? (ty * 4 + i) : (64 + ty * 4 + i - 4);
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = sum_s[(8 * i + j) * kThreads + threadIdx.x] + acc[i][j];
    *reinterpret_cast<float4*>(out + (size_t)r * kT + tx * 4) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(out + (size_t)r * kT + 64 + tx * 4) = make_float4(v[4], v[5], v[6], v[7]);
  }
}

// A field tile of at most 16 columns (Y' = Phi^T F for up to 16 channel rows):
// 128 feature rows x 16 columns, each thread 8 rows x 1 column, so that a few
// channels do not cost a whole 128 x 128 tile.  Same slabs, the same
// compensated folding (in registers: 8 sums per thread), and the same partial
// layout (row stride 128) as the square kernel.
__global__ void __launch_bounds__(kThreads)
gram_simt_narrow_kernel(const float* __restrict__ psi, int64_t n_pad, const GramUnit* __restrict__ units,
                        float* __restrict__ partials) {
  constexpr int kN = kSimtNarrow;
  const GramUnit u = units[blockIdx.x];
  __shared__ __align__(16) float As[kK][kT + 4];
  __shared__ __align__(16) float Bs[kK][kN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // column tx, rows 8 ty .. 8 ty + 7
  float acc[8], sum[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = sum[i] = 0.f;
  const int lrow = threadIdx.x >> 2, lq = threadIdx.x & 3;  // A: rows lrow and lrow + 64, float4 lq
  const float* arow0 = psi + (size_t)(u.i0 + lrow) * n_pad + lq * 4;
  const float* arow1 = psi + (size_t)(u.i0 + lrow + 64) * n_pad + lq * 4;
  const bool bload = threadIdx.x < kN * 4;                   // B: 16 rows x 4 float4
  const float* brow = psi + (size_t)(u.j0 + (threadIdx.x >> 2)) * n_pad + lq * 4;
  float4 va0, va1, vb = make_float4(0.f, 0.f, 0.f, 0.f);
  if (u.k0 < u.k1) {
    va0 = __ldg(reinterpret_cast<const float4*>(arow0 + u.k0));
    va1 = __ldg(reinterpret_cast<const float4*>(arow1 + u.k0));
    if (bload) vb = __ldg(reinterpret_cast<const float4*>(brow + u.k0));
  }
  int slab = 0;
  for (int64_t k = u.k0; k < u.k1; k += kK, ++slab) {
    __syncthreads();
    As[lq * 4 + 0][lrow] = va0.x; As[lq * 4 + 1][lrow] = va0.y; As[lq * 4 + 2][lrow] = va0.z; As[lq * 4 + 3][lrow] = va0.w;
    As[lq * 4 + 0][lrow + 64] = va1.x; As[lq * 4 + 1][lrow + 64] = va1.y; As[lq * 4 + 2][lrow + 64] = va1.z; As[lq * 4 + 3][lrow + 64] = va1.w;
    if (bload) {
      const int br = threadIdx.x >> 2;
      Bs[lq * 4 + 0][br] = vb.x; Bs[lq * 4 + 1][br] = vb.y; Bs[lq * 4 + 2][br] = vb.z; Bs[lq * 4 + 3][br] = vb.w;
    }
    __syncthreads();
    const int64_t kn = k + kK;
    if (kn < u.k1) {
      va0 = __ldg(reinterpret_cast<const float4*>(arow0 + kn));
      va1 = __ldg(reinterpret_cast<const float4*>(arow1 + kn));
      if (bload) vb = __ldg(reinterpret_cast<const float4*>(brow + kn));
    }
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      const float4 a_lo = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a_hi = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float b = Bs[kk][tx];
      const float a[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] = fmaf(a[i], b, acc[i]);
    }
    if ((slab + 1) % kFold == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {  // sum + acc = t + e exactly; e carries on in acc
        const float t = sum[i] + acc[i];
        const float bp = t - sum[i];
        acc[i] = (sum[i] - (t - bp)) + (acc[i] - bp);
        sum[i] = t;
      }
    }
  }
  float* out = partials + u.out;
#pragma unroll
  for (int i = 0; i < 8; ++i) out[(size_t)(ty * 8 + i) * kT + tx] = sum[i] + acc[i];
}

}  // namespace

cudaError_t launch_gram_simt_narrow(const float* psi, int64_t n_pad, const GramUnit* units, int num_units,
                                    float* partials, cudaStream_t st) {
  if (num_units <= 0) return cudaSuccess;
  gram_simt_narrow_kernel<<<num_units, kThreads, 0, st>>>(psi, n_pad, units, partials);
  return launched();
}

cudaError_t launch_gram_simt(const float* psi, int64_t n_pad, const GramUnit* units, int num_units,
                             float* partials, cudaStream_t st) {
  if (num_units <= 0) return cudaSuccess;
  static const cudaError_t attr =  // once per process (thread-safe initialisation)
      cudaFuncSetAttribute(gram_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSumBytes);
  if (attr != cudaSuccess) return attr;
  gram_simt_kernel<<<num_units, kThreads, kSumBytes, st>>>(psi, n_pad, units, partials);
  return launched();
}

}  // namespace rfd
