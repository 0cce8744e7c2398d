// Steps a3 (reduction of the split-K partials), a5 (Z = diag(s sgn r) G Y) and
// a6 (out = F + Phi Z) of the RFD path (Sec. 2.4: x + A(G(B^T x)), with
// A = Phi diag(s sgn r), B = Phi diag(s)).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include "kernels.h"

namespace rfd {

namespace {

// One thread per tile element; partials of one tile are summed in split order
// (deterministic for a given N, m and channel count), compensated FP32; the
// compensated sum is scaled by the column scales in FP64 (step a4's input).
__global__ void reduce_kernel(const GramTile* __restrict__ tiles, const float* __restrict__ partials,
                              int64_t slot_elems, const double* __restrict__ oa,
                              const double* __restrict__ ob, int m, int c, double* __restrict__ M,
                              double* __restrict__ Y, int tile_cols) {
  const GramTile t = tiles[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = e / tile_cols, col = e % tile_cols;
  if (r >= t.ni || col >= t.nj) return;
  Fp32Sum acc;
  for (int u = 0; u < t.unit_count; ++u)
    acc.add(partials[(int64_t)(t.unit_first + u) * slot_elems + (int64_t)r * t.ld + t.col_off + col]);
  const double s = acc.wide();
  const int f = t.i0 + r;
  if (t.kind == kTileGram) {
    const int g = t.j0 + col;
    if (f > g) return;  // the mirrored entry (g, f) is covered as (row g, column f)
    // M = diag(s) K diag(s sgn r) with the commutative product s_f s_g, so that
    // M diag(sgn r) is exactly symmetric
    const double v = s * (ob[f] * ob[g]);
    M[(size_t)f * m + g] = oa[g] < 0.0 ? -v : v;
    if (f != g) M[(size_t)g * m + f] = oa[f] < 0.0 ? -v : v;
  } else {
    if (col < c) Y[(size_t)f * c + col] = ob[f] * s;
  }
}

// Z[f, ch] = oa[f] * sum_g G[f, g] Y[g, ch]: FP32 products, compensated FP32
// sums, stored FP32.  Block (32 channels x 8 g-slices) per row f.
__global__ void small_product_kernel(const double* __restrict__ G, const double* __restrict__ Y,
                                     const double* __restrict__ oa, int m, int c, float* __restrict__ Z) {
  const int f = blockIdx.x;
  __shared__ float red[8][32][2];
  for (int ch0 = 0; ch0 < c; ch0 += 32) {
    const int ch = ch0 + threadIdx.x;
    Fp32Sum acc;
    if (ch < c)
      for (int g = threadIdx.y; g < m; g += 8) acc.add((float)G[(size_t)f * m + g] * (float)Y[(size_t)g * c + ch]);
    red[threadIdx.y][threadIdx.x][0] = acc.s;
    red[threadIdx.y][threadIdx.x][1] = acc.c;
    __syncthreads();
    if (threadIdx.y == 0 && ch < c) {
      Fp32Sum tot;
      for (int y = 0; y < 8; ++y) {
        tot.add(red[y][threadIdx.x][0]);
        tot.add(red[y][threadIdx.x][1]);
      }
      Z[(size_t)f * c + ch] = (float)oa[f] * tot.value();
    }
    __syncthreads();
  }
}

// out[n, ch] = F[n, ch] + sum_f Psi[f][n] Z[f, ch]: one point per thread (Psi
// reads coalesced along n), CG channels per thread, Z streamed through shared
// memory in 64-row chunks.  F is read before out is written, row by row, so
// out may alias F.
template <int CG, typename T>
__global__ void __launch_bounds__(256)
apply_simt_kernel(const T* __restrict__ psi, int64_t n, int64_t n_pad, int m, const float* __restrict__ Z, int c,
                  const float* F, int64_t ldF, float* out, int64_t ldOut) {
  constexpr int kChunk = 64;
  __shared__ float zs[kChunk][CG];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ch0 = blockIdx.y * CG;
  const int cg = min(CG, c - ch0);
  float acc[CG];
#pragma unroll
  for (int q = 0; q < CG; ++q) acc[q] = 0.f;
  for (int f0 = 0; f0 < m; f0 += kChunk) {
    const int fn = min(kChunk, m - f0);
    __syncthreads();
    for (int i = threadIdx.x; i < kChunk * CG; i += blockDim.x) {
      const int fr = i / CG, q = i % CG;
      zs[fr][q] = (fr < fn && q < cg) ? Z[(size_t)(f0 + fr) * c + ch0 + q] : 0.f;
    }
    __syncthreads();
    if (p < n) {
      for (int fr = 0; fr < fn; ++fr) {
        float v;
        if constexpr (sizeof(T) == 2)
          v = __bfloat162float(psi[(size_t)(f0 + fr) * n_pad + p]);
        else
          v = psi[(size_t)(f0 + fr) * n_pad + p];
#pragma unroll
        for (int q = 0; q < CG; ++q) acc[q] = fmaf(v, zs[fr][q], acc[q]);
      }
    }
  }
  if (p < n) {
    for (int q = 0; q < cg; ++q) {
      const float fv = F[p * ldF + ch0 + q];
      out[p * ldOut + ch0 + q] = fv + acc[q];
    }
  }
}

template <int CG>
cudaError_t apply_cg(const void* psi, bool bf16, int64_t n, int64_t n_pad, int m, const float* Z, int c,
                     const float* F, int64_t ldF, float* out, int64_t ldOut, cudaStream_t st) {
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)((c + CG - 1) / CG));
  if (bf16)
    apply_simt_kernel<CG, __nv_bfloat16><<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(psi), n, n_pad, m,
                                                               Z, c, F, ldF, out, ldOut);
  else
    apply_simt_kernel<CG, float><<<grid, 256, 0, st>>>(static_cast<const float*>(psi), n, n_pad, m, Z, c, F, ldF,
                                                       out, ldOut);
  return launched();
}

}  // namespace

cudaError_t launch_reduce(const GramTile* tiles, int num_tiles, const float* partials, int64_t slot_elems,
                          const double* oa, const double* ob, int m, int c, double* M, double* Y, int tile_rows,
                          int tile_cols, cudaStream_t st) {
  if (num_tiles <= 0) return cudaSuccess;
  dim3 grid((unsigned)((tile_rows * tile_cols + 255) / 256), (unsigned)num_tiles);
  reduce_kernel<<<grid, 256, 0, st>>>(tiles, partials, slot_elems, oa, ob, m, c, M, Y, tile_cols);
  return launched();
}

cudaError_t launch_small_product(const double* G, const double* Y, const double* oa, int m, int c, float* Z,
                                 cudaStream_t st) {
  small_product_kernel<<<m, dim3(32, 8), 0, st>>>(G, Y, oa, m, c, Z);
  return launched();
}

cudaError_t launch_apply_simt(const void* psi, bool bf16, int64_t n, int64_t n_pad, int m, const float* Z, int c,
                              const float* F, int64_t ldF, float* out, int64_t ldOut, cudaStream_t st) {
  if (c <= 4) return apply_cg<4>(psi, bf16, n, n_pad, m, Z, c, F, ldF, out, ldOut, st);
  if (c <= 8) return apply_cg<8>(psi, bf16, n, n_pad, m, Z, c, F, ldF, out, ldOut, st);
  if (c <= 16) return apply_cg<16>(psi, bf16, n, n_pad, m, Z, c, F, ldF, out, ldOut, st);
  return apply_cg<32>(psi, bf16, n, n_pad, m, Z, c, F, ldF, out, ldOut, st);
}

}  // namespace rfd
