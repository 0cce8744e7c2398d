// Step a2 of the RFD path: the random-feature map (Sec. 2.4, real part as in
// App. A.4).  For point x_n and frequency w_j (j < h = m/2):
//     Phi[n, j]     = cos(2 pi w_j^T x_n)
//     Phi[n, h + j] = sin(2 pi w_j^T x_n)
// The column scales s sgn r / s of A and B are applied later, outside the
// GEMMs (per-column scaling), so Phi's entries stay in [-1, 1].
//
// Layout: the kernels write Phi TRANSPOSED, feature-major: Psi[row][n] with
// row j in [0, m) and n contiguous (leading dimension n_pad, a multiple of
// 128).  Both operands of the Gram Phi^T Phi are then K-major (K = points),
// the layout TMA + tcgen05 consume without transposition.  Columns
// n in [N, n_pad) are written as zeros.  Rows [m, m + cpad) of the same
// buffer hold F^T (fill_field_rows), so B^T F comes out of the same pass.
//
// Angle reduction is done in cycles: t = w^T x, r = t - rint(t) in [-1/2, 1/2],
// then sin/cos of 2 pi r.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include "kernels.h"

namespace rfd {

namespace {

constexpr int kFeatThreads = 256;
constexpr int kPtsPerThread = 2;                           // 2 consecutive points -> vector stores
constexpr int kPtsPerBlock = kFeatThreads * kPtsPerThread;  // 512
constexpr int kFreqPerBlock = 32;

// BF16 form: FP32 angle, MUFU sin/cos (|2 pi r| <= pi keeps __sinf/__cosf in
// their accurate range, absolute error ~1e-6, far below BF16's 2^-9).
__global__ void __launch_bounds__(kFeatThreads)
features_bf16_kernel(const float* __restrict__ pts, int64_t n, int64_t n_pad,
                     const float* __restrict__ omega_hi, int h,
                     __nv_bfloat16* __restrict__ psi) {
  __shared__ float w_s[kFreqPerBlock][3];
  const int j0 = blockIdx.y * kFreqPerBlock;
  const int jn = min(kFreqPerBlock, h - j0);
  if (threadIdx.x < jn * 3) w_s[threadIdx.x / 3][threadIdx.x % 3] = omega_hi[(size_t)j0 * 3 + threadIdx.x];
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * kPtsPerBlock + (int64_t)threadIdx.x * kPtsPerThread;
  if (p0 >= n_pad) return;
  float x[kPtsPerThread][3];
  bool valid[kPtsPerThread];
#pragma unroll
  for (int q = 0; q < kPtsPerThread; ++q) {
    valid[q] = (p0 + q) < n;
#pragma unroll
    for (int d = 0; d < 3; ++d) x[q][d] = valid[q] ? pts[(p0 + q) * 3 + d] : 0.f;
  }
  const float two_pi = 6.283185307179586f;
  for (int jj = 0; jj < jn; ++jj) {
    const float w0 = w_s[jj][0], w1 = w_s[jj][1], w2 = w_s[jj][2];
    float c[kPtsPerThread], s[kPtsPerThread];
#pragma unroll
    for (int q = 0; q < kPtsPerThread; ++q) {
      float t = fmaf(w0, x[q][0], fmaf(w1, x[q][1], w2 * x[q][2]));
      float r = t - rintf(t);
      float a = two_pi * r;
      c[q] = valid[q] ? __cosf(a) : 0.f;
      s[q] = valid[q] ? __sinf(a) : 0.f;
    }
    const int j = j0 + jj;
    __nv_bfloat162 cv = __floats2bfloat162_rn(c[0], c[1]);
    __nv_bfloat162 sv = __floats2bfloat162_rn(s[0], s[1]);
    *reinterpret_cast<__nv_bfloat162*>(psi + (size_t)j * n_pad + p0) = cv;
    *reinterpret_cast<__nv_bfloat162*>(psi + (size_t)(h + j) * n_pad + p0) = sv;
  }
}

// Exact product a*b = hi + lo (FMA), and exact sum a+b = s + e (Knuth TwoSum).
__device__ __forceinline__ void two_prod(float a, float b, float& hi, float& lo) {
  hi = a * b;
  lo = fmaf(a, b, -hi);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// FP32 form: the angle in cycles is formed from double-float frequencies
// (w = w_hi + w_lo, ~48 significant bits) and FP32 points with error-free
// products and sums, so t is accurate to ~2^-44 relative; the fractional part
// r is exact up to that, and sincospif(2 r) evaluates sin, cos(2 pi r)
// without a rounded 2 pi factor.
__global__ void __launch_bounds__(kFeatThreads)
features_f32_kernel(const float* __restrict__ pts, int64_t n, int64_t n_pad,
                    const float* __restrict__ omega_hi, const float* __restrict__ omega_lo, int h,
                    float* __restrict__ psi) {
  __shared__ float wh_s[kFreqPerBlock][3];
  __shared__ float wl_s[kFreqPerBlock][3];
  const int j0 = blockIdx.y * kFreqPerBlock;
  const int jn = min(kFreqPerBlock, h - j0);
  if (threadIdx.x < jn * 3) {
    wh_s[threadIdx.x / 3][threadIdx.x % 3] = omega_hi[(size_t)j0 * 3 + threadIdx.x];
    wl_s[threadIdx.x / 3][threadIdx.x % 3] = omega_lo[(size_t)j0 * 3 + threadIdx.x];
  }
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * kPtsPerBlock + (int64_t)threadIdx.x * kPtsPerThread;
  if (p0 >= n_pad) return;
  float x[kPtsPerThread][3];
  bool valid[kPtsPerThread];
#pragma unroll
  for (int q = 0; q < kPtsPerThread; ++q) {
    valid[q] = (p0 + q) < n;
#pragma unroll
    for (int d = 0; d < 3; ++d) x[q][d] = valid[q] ? pts[(p0 + q) * 3 + d] : 0.f;
  }
  for (int jj = 0; jj < jn; ++jj) {
    float c[kPtsPerThread], s[kPtsPerThread];
#pragma unroll
    for (int q = 0; q < kPtsPerThread; ++q) {
      float ph[3], pl[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        two_prod(wh_s[jj][d], x[q][d], ph[d], pl[d]);
        pl[d] = fmaf(wl_s[jj][d], x[q][d], pl[d]);
      }
      float s01, e01, s012, e012;
      two_sum(ph[0], ph[1], s01, e01);
      two_sum(s01, ph[2], s012, e012);
      const float lo = (pl[0] + pl[1]) + (pl[2] + (e01 + e012));
      // fractional part of s012 + lo: s012 - rint(s012) is exact (|.| <= 1/2)
      float r = (s012 - rintf(s012)) + lo;
      r -= rintf(r);
      float sn, cs;
      sincospif(2.0f * r, &sn, &cs);
      c[q] = valid[q] ? cs : 0.f;
      s[q] = valid[q] ? sn : 0.f;
    }
    const int j = j0 + jj;
    *reinterpret_cast<float2*>(psi + (size_t)j * n_pad + p0) = make_float2(c[0], c[1]);
    *reinterpret_cast<float2*>(psi + (size_t)(h + j) * n_pad + p0) = make_float2(s[0], s[1]);
  }
}

// Rows [m, m + cpad) of Psi: F^T (channel-major), zero for channels >= c and
// points >= N.  A 32 x 32 shared-memory transpose keeps both sides coalesced.
template <typename T>
__global__ void fill_field_rows_kernel(const float* __restrict__ F, int64_t ldF, int c, int64_t n,
                                       int64_t n_pad, int cpad, T* __restrict__ rows) {
  __shared__ float tile[32][33];
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {  // i: point offset, threadIdx.x: channel offset
    const int64_t pn = n0 + i;
    const int ch = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (pn < n && ch < c) ? F[pn * ldF + ch] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {  // i: channel offset, threadIdx.x: point offset
    const int ch = c0 + i;
    const int64_t pn = n0 + threadIdx.x;
    if (ch < cpad && pn < n_pad) {
      const float v = tile[threadIdx.x][i];
      if constexpr (sizeof(T) == 2)
        rows[(size_t)ch * n_pad + pn] = __float2bfloat16_rn(v);
      else
        rows[(size_t)ch * n_pad + pn] = v;
    }
  }
}

}  // namespace

cudaError_t launch_features(const float* pts, int64_t n, int64_t n_pad, const float* omega_hi,
                            const float* omega_lo, int h, bool bf16, void* psi, cudaStream_t st) {
  if (n_pad % kPtsPerThread) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((n_pad + kPtsPerBlock - 1) / kPtsPerBlock), (unsigned)((h + kFreqPerBlock - 1) / kFreqPerBlock));
  if (bf16)
    features_bf16_kernel<<<grid, kFeatThreads, 0, st>>>(pts, n, n_pad, omega_hi, h,
                                                        static_cast<__nv_bfloat16*>(psi));
  else
    features_f32_kernel<<<grid, kFeatThreads, 0, st>>>(pts, n, n_pad, omega_hi, omega_lo, h,
                                                       static_cast<float*>(psi));
  return launched();
}

cudaError_t launch_fill_field_rows(const float* F, int64_t ldF, int c, int64_t n, int64_t n_pad, int cpad,
                                   bool bf16, void* rows, cudaStream_t st) {
  dim3 grid((unsigned)((n_pad + 31) / 32), (unsigned)((cpad + 31) / 32));
  dim3 block(32, 8);
  if (bf16)
    fill_field_rows_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(F, ldF, c, n, n_pad, cpad,
                                                                  static_cast<__nv_bfloat16*>(rows));
  else
    fill_field_rows_kernel<float><<<grid, block, 0, st>>>(F, ldF, c, n, n_pad, cpad, static_cast<float*>(rows));
  return launched();
}

}  // namespace rfd
