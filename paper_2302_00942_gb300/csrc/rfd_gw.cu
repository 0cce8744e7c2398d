// Gromov-Wasserstein building blocks with implicit structure matrices
// (App. C.2): the structure matrix of a cloud is its RFD kernel
// C = exp(lambda W_hat), applied to wide matrices by the resident plan
// (rfd_integrate over column chunks of at most max_channels), never formed.
//
//   rfd_fm_apply           Y = C X for an N x ncols matrix X
//   rfd_gw_tensor_product  L = (C^{(.)2} p) 1^T + 1 (D^{(.)2} q)^T - 2 C T D^T
//                          (Algorithm tensor_prod, square loss; C^{(.)2} p =
//                          diag(C D_p C^T), Eq. sq)
//   rfd_gw_line_search     the optimal step of a conditional-gradient (F)GW
//                          iteration (Algorithm line_search)
//
// FP32 matrices on the first plan's stream (both plans must share it or be
// ordered by the caller); temporaries from the stream-ordered allocator.
#include <cuda_runtime.h>
#include <cmath>
#include <string>
#include "kernels.h"
#include "rfd_internal.h"
#include "rfd_plan.h"

namespace rfd {

namespace {

// B = A^T for A rows x cols (lda), B cols x rows (ldb); 32 x 8 threads per 32 x 32 tile
__global__ void transpose_f32_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                                     float* __restrict__ B, int64_t ldb) {
  __shared__ float tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (r < rows && c < cols) ? A[r * lda + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < rows) B[c * ldb + r] = tile[threadIdx.x][y];
  }
}

// X = diag(p) (n x n)
__global__ void diag_fill_kernel(const float* __restrict__ p, float* __restrict__ X, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int64_t i = e / n, j = e % n;
  X[e] = (i == j) ? p[i] : 0.f;
}

// v[i] = Z[i, i]
__global__ void diag_take_kernel(const float* __restrict__ Z, float* __restrict__ v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = Z[i * n + i];
}

// L[i, j] = v1[i] + v2[j] - 2 W[i, j]
__global__ void assemble_kernel(const float* __restrict__ v1, const float* __restrict__ v2,
                                const float* __restrict__ W, float* __restrict__ L, int64_t n1, int64_t n2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n1 * n2) return;
  L[e] = v1[e / n2] + v2[e % n2] - 2.0f * W[e];
}

// sums[0..4] += <a1, dG>, <a1, G>, <b1, dG>, <M, dG>, <v1 1^T + 1 v2^T, dG> (FP64 accumulation)
__global__ void line_search_sums_kernel(const float* __restrict__ a1, const float* __restrict__ b1,
                                        const float* __restrict__ G, const float* __restrict__ dG,
                                        const float* __restrict__ M, const float* __restrict__ v1,
                                        const float* __restrict__ v2, int64_t n1, int64_t n2,
                                        double* __restrict__ sums) {
  double s[5] = {0, 0, 0, 0, 0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n1 * n2; e += (int64_t)gridDim.x * blockDim.x) {
    const double d = dG[e];
    s[0] += (double)a1[e] * d;
    s[1] += (double)a1[e] * G[e];
    s[2] += (double)b1[e] * d;
    s[3] += (double)M[e] * d;
    s[4] += ((double)v1[e / n2] + v2[e % n2]) * d;
  }
  __shared__ double red[5][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 5; ++k) {
    double v = s[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    atomicAdd(&sums[threadIdx.x], v);
  }
}

// ---- low-rank form (both clouds with m <= 32) --------------------------------
// A cloud's structure matrix is C = I + Psi K Psi^T with Psi its FP32 features
// (N x m) and K = diag(s sgn r) G diag(s) (m x m).  With U = Psi K:
//   C^{(.)2} p:  v_i = p_i (1 + 2 U_i . Psi_i) + U_i^T S U_i,  S = Psi^T D_p Psi
//   C T D^T   :  T + U_C P' + Q U_D^T,  P = Psi_C^T T, Q = T Psi_D,
//                R = P Psi_D, P' = P + R U_D^T
// (the same sums as Eq. sq and Algorithm tensor_prod, re-associated through
// the factors), so the n1 x n2 matrices are read once for P and Q and once
// for the output, and every other step is O(N m^2).

constexpr int kTI = 32;    // rows of a projection tile
constexpr int kTA = 64;    // rows of an assembly tile (scalar form)
constexpr int kTJ = 256;   // columns of a tile (one per thread)
constexpr int kPLd = kTJ + 1;  // smem row stride of a projection tile: rows and columns both conflict-free

// The row groups of the projection and assembly grids: about four CTAs per SM
// in all (two resident per SM, two waves), at least one tile per group.
int row_groups(int64_t n1, int64_t n2, int tile_rows) {
  static const int sms = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 148;
    return v > 0 ? v : 148;
  }();
  const int64_t strips = (n2 + kTJ - 1) / kTJ, tiles = (n1 + tile_rows - 1) / tile_rows;
  const int64_t want = (4ll * sms + strips - 1) / strips;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, tiles));
}

// Pt[g][j][f] = sum_{i in group g} X[i][j] psc[i][f],  Qp[s][i][f] = sum_{j in strip s} X[i][j] psd[j][f]
// in one pass over X.  A CTA takes a strip of kTJ columns and a group of rows
// in tiles of kTI rows staged in shared memory (row stride kTJ + 1: conflict-
// free along rows and down columns); with 16-byte loads the next tile's loads
// are issued into registers before the current tile is computed, so they are
// in flight during its FMAs.
//   P: thread t owns column t, MF sums over the group's rows (per row one
//      shared load of X and MF / 4 broadcast 16-byte loads of psc).
//   Q: warp w owns the tile's kTI rows (lane = row) over the columns
//      32 w .. 32 w + 31 (per column one shared load of X, MF / 4 broadcast
//      loads of psd); the 8 warps' partial sums meet in shared memory.
template <int MF>
__global__ void __launch_bounds__(256, 2) gw_project_kernel(const float* __restrict__ X, int64_t n1, int64_t n2,
                                                            const float* __restrict__ psc,
                                                            const float* __restrict__ psd,
                                                            float* __restrict__ Pt_part, float* __restrict__ Q_part,
                                                            int rows_per_group) {
  static_assert(kTI == 32 && kTJ == 256, "lane = tile row, 8 warps x 32 columns");
  constexpr int RLd = MF + 1;  // row stride of the Q reduction buffer
  extern __shared__ __align__(16) float sm[];
  float* Ts = sm;                   // kTI x kPLd
  float* pc = Ts + kTI * kPLd;      // kTI x MF  (kTI * kPLd is a multiple of 4: 16-byte aligned)
  float* pd = pc + kTI * MF;        // kTJ x MF
  float* red = pd + kTJ * MF;       // 8 x kTI x RLd
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * kTJ;
  const int64_t ig0 = (int64_t)blockIdx.y * rows_per_group;
  const int64_t ig1 = min(n1, ig0 + rows_per_group);
  for (int e = t; e < kTJ * MF; e += 256) {
    const int64_t j = j0 + e / MF;
    pd[e] = j < n2 ? psd[j * MF + e % MF] : 0.f;
  }
  float accP[MF];
#pragma unroll
  for (int f = 0; f < MF; ++f) accP[f] = 0.f;
  // whole 16-byte column groups: rows start 16-byte aligned and a group never straddles n2
  const bool vec = (n2 & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  const int c4 = (t & 63) * 4, r0 = t >> 6;  // vec: rows r0 + 4u, columns c4 .. c4 + 3
  float4 v[kTI / 4];
  auto fetch = [&](int64_t i0) {
#pragma unroll
    for (int u = 0; u < kTI / 4; ++u) {
      const int64_t i = i0 + r0 + 4 * u, j = j0 + c4;
      v[u] = (i < ig1 && j < n2) ? *reinterpret_cast<const float4*>(X + i * n2 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (vec && ig0 < ig1) fetch(ig0);
  for (int64_t i0 = ig0; i0 < ig1; i0 += kTI) {
    __syncthreads();  // the previous tile and its reduction buffer are consumed
    if (vec) {
#pragma unroll
      for (int u = 0; u < kTI / 4; ++u) {
        float* d = Ts + (r0 + 4 * u) * kPLd + c4;
        d[0] = v[u].x;
        d[1] = v[u].y;
        d[2] = v[u].z;
        d[3] = v[u].w;
      }
    } else {
#pragma unroll 8
      for (int r = 0; r < kTI; ++r) {
        const int64_t i = i0 + r, j = j0 + t;
        Ts[r * kPLd + t] = (i < ig1 && j < n2) ? X[i * n2 + j] : 0.f;
      }
    }
    for (int e = t; e < kTI * MF; e += 256) {
      const int64_t i = i0 + e / MF;
      pc[e] = i < ig1 ? psc[i * MF + e % MF] : 0.f;
    }
    __syncthreads();
    if (vec && i0 + kTI < ig1) fetch(i0 + kTI);  // the next tile's loads fly during this tile's FMAs
#pragma unroll 4
    for (int r = 0; r < kTI; ++r) {  // P: column t over the tile's rows
      const float x = Ts[r * kPLd + t];
      const float4* pr = reinterpret_cast<const float4*>(pc + r * MF);
#pragma unroll
      for (int f4 = 0; f4 < MF / 4; ++f4) {
        const float4 w = pr[f4];
        accP[4 * f4] = fmaf(x, w.x, accP[4 * f4]);
        accP[4 * f4 + 1] = fmaf(x, w.y, accP[4 * f4 + 1]);
        accP[4 * f4 + 2] = fmaf(x, w.z, accP[4 * f4 + 2]);
        accP[4 * f4 + 3] = fmaf(x, w.w, accP[4 * f4 + 3]);
      }
    }
    float accQ[MF];
#pragma unroll
    for (int f = 0; f < MF; ++f) accQ[f] = 0.f;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {  // Q: row `lane` over the warp's 32 columns
      const int c = warp * 32 + k;
      const float x = Ts[lane * kPLd + c];
      const float4* pr = reinterpret_cast<const float4*>(pd + c * MF);
#pragma unroll
      for (int f4 = 0; f4 < MF / 4; ++f4) {
        const float4 w = pr[f4];
        accQ[4 * f4] = fmaf(x, w.x, accQ[4 * f4]);
        accQ[4 * f4 + 1] = fmaf(x, w.y, accQ[4 * f4 + 1]);
        accQ[4 * f4 + 2] = fmaf(x, w.z, accQ[4 * f4 + 2]);
        accQ[4 * f4 + 3] = fmaf(x, w.w, accQ[4 * f4 + 3]);
      }
    }
    float* rw = red + (warp * kTI + lane) * RLd;
#pragma unroll
    for (int f = 0; f < MF; ++f) rw[f] = accQ[f];
    __syncthreads();
    for (int e = t; e < kTI * MF; e += 256) {  // the warps' sums, in warp order
      const int r = e / MF, f = e % MF;
      float q = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) q += red[(w * kTI + r) * RLd + f];
      const int64_t i = i0 + r;
      if (i < ig1) Q_part[((int64_t)blockIdx.x * n1 + i) * MF + f] = q;
    }
  }
  const int64_t j = j0 + t;
  if (j < n2) {
    float4* o = reinterpret_cast<float4*>(Pt_part + ((int64_t)blockIdx.y * n2 + j) * MF);
#pragma unroll
    for (int f4 = 0; f4 < MF / 4; ++f4)
      o[f4] = make_float4(accP[4 * f4], accP[4 * f4 + 1], accP[4 * f4 + 2], accP[4 * f4 + 3]);
  }
}

// The same projections for MF = 16 with register tiles, so that a 16-byte
// shared load feeds 16 FMAs where the kernel above spends 9 wavefronts per
// warp on 16: the tile is stored with a row stride of kTJ + 4 floats (16-byte
// aligned rows, conflict-free 16-byte stores and loads along rows), and
//   P: thread (fq = t % 4, jq = t / 4) owns 4 features x 4 adjacent columns
//      (per row: one 16-byte load of X, one of psc, 16 FMAs);
//   Q: warp rq owns rows 4 rq .. 4 rq + 3; lane (ks = lane % 8, fq = lane / 8)
//      owns 4 features and the column quads ks, ks + 8, ... (per quad: four
//      16-byte loads of X rows, four of psd held transposed, 64 FMAs); the 8
//      column slices meet by shuffles, in a fixed order.
// The next tile's loads are issued into registers before the current tile is
// computed.  X with 16-byte rows only (n2 % 4 == 0, 16-byte aligned).
__global__ void __launch_bounds__(256, 2) gw_project16_kernel(const float* __restrict__ X, int64_t n1, int64_t n2,
                                                             const float* __restrict__ psc,
                                                             const float* __restrict__ psd,
                                                             float* __restrict__ Pt_part, float* __restrict__ Q_part,
                                                             int rows_per_group) {
  constexpr int MF = 16, TLd = kTJ + 4;
  static_assert(kTI == 32 && kTJ == 256, "8 warps x 4 rows, 64 column quads");
  extern __shared__ __align__(16) float sm[];
  float* Ts = sm;                // kTI x TLd
  float* pc = Ts + kTI * TLd;    // kTI x MF
  float* pdT = pc + kTI * MF;    // MF x kTJ: psd transposed, so that a column quad of one feature is 16 bytes
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * kTJ;
  const int64_t ig0 = (int64_t)blockIdx.y * rows_per_group;
  const int64_t ig1 = min(n1, ig0 + rows_per_group);
  for (int e = t; e < kTJ * MF; e += 256) {
    const int64_t j = j0 + e / MF;
    pdT[(e % MF) * kTJ + e / MF] = j < n2 ? psd[j * MF + e % MF] : 0.f;
  }
  const int pfq = t & 3, pjq = t >> 2;             // P: features 4 pfq.., columns 4 pjq..
  const int ks = lane & 7, qfq = lane >> 3;        // Q: column quads ks + 8 k, features 4 qfq..
  float accP[4][4];                                // [feature][column]
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) accP[a][b] = 0.f;
  const int c4 = (t & 63) * 4, r0 = t >> 6;        // loads: rows r0 + 4u, columns c4 .. c4 + 3
  float4 v[kTI / 4];
  auto fetch = [&](int64_t i0) {
#pragma unroll
    for (int u = 0; u < kTI / 4; ++u) {
      const int64_t i = i0 + r0 + 4 * u, j = j0 + c4;
      v[u] = (i < ig1 && j < n2) ? *reinterpret_cast<const float4*>(X + i * n2 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (ig0 < ig1) fetch(ig0);
  for (int64_t i0 = ig0; i0 < ig1; i0 += kTI) {
    __syncthreads();  // the previous tile is consumed
#pragma unroll
    for (int u = 0; u < kTI / 4; ++u) *reinterpret_cast<float4*>(Ts + (r0 + 4 * u) * TLd + c4) = v[u];
    for (int e = t; e < kTI * MF; e += 256) {
      const int64_t i = i0 + e / MF;
      pc[e] = i < ig1 ? psc[i * MF + e % MF] : 0.f;
    }
    __syncthreads();
    if (i0 + kTI < ig1) fetch(i0 + kTI);  // the next tile's loads fly during this tile's FMAs
#pragma unroll 4
    for (int r = 0; r < kTI; ++r) {  // P
      const float4 x = *reinterpret_cast<const float4*>(Ts + r * TLd + 4 * pjq);
      const float4 w = *reinterpret_cast<const float4*>(pc + r * MF + 4 * pfq);
      const float xs[4] = {x.x, x.y, x.z, x.w}, ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) accP[a][b] = fmaf(ws[a], xs[b], accP[a][b]);
    }
    float accQ[4][4];  // [row][feature]
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) accQ[a][b] = 0.f;
#pragma unroll 2
    for (int k = 0; k < kTJ / 32; ++k) {  // Q: column quad cq of this lane's slice
      const int cq = ks + 8 * k;
      float xr[4][4], wc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4 x = *reinterpret_cast<const float4*>(Ts + (4 * warp + a) * TLd + 4 * cq);
        xr[a][0] = x.x; xr[a][1] = x.y; xr[a][2] = x.z; xr[a][3] = x.w;
        const float4 w = *reinterpret_cast<const float4*>(pdT + (4 * qfq + a) * kTJ + 4 * cq);  // feature 4 qfq + a
        wc[0][a] = w.x; wc[1][a] = w.y; wc[2][a] = w.z; wc[3][a] = w.w;
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)        // row
#pragma unroll
        for (int c = 0; c < 4; ++c)      // column of the quad
#pragma unroll
          for (int b = 0; b < 4; ++b)    // feature
            accQ[a][b] = fmaf(xr[a][c], wc[c][b], accQ[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {  // the 8 column slices, in a fixed butterfly order
        float q = accQ[a][b];
        q += __shfl_xor_sync(0xffffffffu, q, 1);
        q += __shfl_xor_sync(0xffffffffu, q, 2);
        q += __shfl_xor_sync(0xffffffffu, q, 4);
        accQ[a][b] = q;
      }
    if (ks == 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + 4 * warp + a;
        if (i < ig1)
          *reinterpret_cast<float4*>(Q_part + ((int64_t)blockIdx.x * n1 + i) * MF + 4 * qfq) =
              make_float4(accQ[a][0], accQ[a][1], accQ[a][2], accQ[a][3]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int64_t j = j0 + 4 * pjq + b;
    if (j < n2)
      *reinterpret_cast<float4*>(Pt_part + ((int64_t)blockIdx.y * n2 + j) * MF + 4 * pfq) =
          make_float4(accP[0][b], accP[1][b], accP[2][b], accP[3][b]);
  }
}

// out[e] = sum_s part[s * stride + e], e < count (fixed order)
__global__ void sum_parts_kernel(const float* __restrict__ part, int parts, int64_t stride, int64_t count,
                                 float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  float s = 0.f;
  for (int k = 0; k < parts; ++k) s += part[k * stride + e];
  out[e] = s;
}

// point-major FP32 features: out[i][f] = psi[f][i] (f < m), 0 for m <= f < MF
__global__ void features_point_major_kernel(const float* __restrict__ psi, int64_t ldpsi, int m, int64_t n, int mf,
                                            float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * mf) return;
  const int64_t i = e / mf;
  const int f = (int)(e % mf);
  out[e] = f < m ? psi[(int64_t)f * ldpsi + i] : 0.f;
}

// K[f][g] = oa[f] G[f][g] ob[g] (zero padded to mf x mf)
__global__ void lowrank_k_kernel(const double* __restrict__ G, const double* __restrict__ oa,
                                 const double* __restrict__ ob, int m, int mf, float* __restrict__ K) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mf * mf) return;
  const int f = e / mf, g = e % mf;
  K[e] = (f < m && g < m) ? (float)(oa[f] * G[(size_t)f * m + g] * ob[g]) : 0.f;
}

// out[i][:] = A[i][:] B (+ add[i][:]); B mf x mf (transposed when tB)
__global__ void rowmat_kernel(const float* __restrict__ A, const float* __restrict__ B, int tB,
                              const float* __restrict__ add, int64_t n, int mf, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * mf) return;
  const int64_t i = e / mf;
  const int f = (int)(e % mf);
  float s = add ? add[e] : 0.f;
  for (int g = 0; g < mf; ++g) s = fmaf(A[i * mf + g], tB ? B[f * mf + g] : B[g * mf + f], s);
  out[e] = s;
}

// part[y][f][g] = sum_{i in chunk y} w_i A[i][f] B[i][g] (w = 1 when null); block (f, y);
// FP32 over a thread's rows, FP64 across threads
__global__ void weighted_gram_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                     const float* __restrict__ w, int64_t n, int mf, float* __restrict__ part) {
  const int f = blockIdx.x;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(n, r0 + per);
  __shared__ float red[8][33];
  float acc[32];
  for (int g = 0; g < 32; ++g) acc[g] = 0.f;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const float a = A[i * mf + f] * (w ? w[i] : 1.f);
    for (int g = 0; g < mf; ++g) acc[g] = fmaf(a, B[i * mf + g], acc[g]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g = 0; g < mf; ++g) {  // FP32 within a warp (the FP64 pipe is slow), FP64 across warps
    float v = acc[g];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][g] = v;
  }
  __syncthreads();
  if (threadIdx.x < mf) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[k][threadIdx.x];
    part[((size_t)blockIdx.y * mf + f) * mf + threadIdx.x] = (float)v;
  }
}

// v_i = p_i (1 + 2 U_i . Psi_i) + U_i^T S U_i
__global__ void hadamard_lowrank_kernel(const float* __restrict__ U, const float* __restrict__ Psi,
                                        const float* __restrict__ S, const float* __restrict__ p, int64_t n, int mf,
                                        float* __restrict__ v) {
  __shared__ float Ss[32 * 32];
  for (int e = threadIdx.x; e < mf * mf; e += blockDim.x) Ss[e] = S[e];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* u = U + i * mf;
  float d = 0.f, q = 0.f;
  for (int f = 0; f < mf; ++f) {
    d = fmaf(u[f], Psi[i * mf + f], d);
    float su = 0.f;
    for (int g = 0; g < mf; ++g) su = fmaf(Ss[f * mf + g], u[g], su);
    q = fmaf(u[f], su, q);
  }
  v[i] = p[i] * (1.f + 2.f * d) + q;
}

// L[i][j] = v1_i + v2_j - 2 (T_ij + Uc_i . Pp_j + Q_i . Ud_j); a column per thread
template <int MF>
__global__ void __launch_bounds__(256) gw_assemble_kernel(const float* __restrict__ T, const float* __restrict__ v1,
                                                          const float* __restrict__ v2, const float* __restrict__ Uc,
                                                          const float* __restrict__ Q, const float* __restrict__ Pp,
                                                          const float* __restrict__ Ud, int64_t n1, int64_t n2,
                                                          float* __restrict__ L) {
  __shared__ __align__(16) float rowf[kTA][2 * MF];  // (Uc_i, Q_i)
  const int t = threadIdx.x;
  const int64_t j = (int64_t)blockIdx.x * kTJ + t, i0 = (int64_t)blockIdx.y * kTA;
  for (int e = t; e < kTA * 2 * MF; e += 256) {
    const int r = e / (2 * MF), k = e % (2 * MF);
    const int64_t i = i0 + r;
    rowf[r][k] = i < n1 ? (k < MF ? Uc[i * MF + k] : Q[i * MF + k - MF]) : 0.f;
  }
  float colf[2 * MF];  // (Pp_j, Ud_j)
#pragma unroll
  for (int k = 0; k < MF; ++k) {
    colf[k] = j < n2 ? Pp[j * MF + k] : 0.f;
    colf[MF + k] = j < n2 ? Ud[j * MF + k] : 0.f;
  }
  const float vj = j < n2 ? v2[j] : 0.f;
  __syncthreads();
  if (j >= n2) return;
  const int rows = (int)(n1 - i0 < kTA ? n1 - i0 : kTA);
#pragma unroll 8
  for (int r = 0; r < rows; ++r) {
    const int64_t i = i0 + r;
    const float4* rf = reinterpret_cast<const float4*>(rowf[r]);
    float s = T[i * n2 + j];
#pragma unroll
    for (int k4 = 0; k4 < MF / 2; ++k4) {
      const float4 a = rf[k4];
      s = fmaf(a.x, colf[4 * k4], s);
      s = fmaf(a.y, colf[4 * k4 + 1], s);
      s = fmaf(a.z, colf[4 * k4 + 2], s);
      s = fmaf(a.w, colf[4 * k4 + 3], s);
    }
    L[i * n2 + j] = v1[i] + vj - 2.f * s;
  }
}

// The same assembly, 16-byte I/O (n2 % 4 == 0, aligned T, L, v2): a CTA keeps
// the (P'_j, Ud_j) of its 256 columns in shared memory, k-major, and walks
// row tiles of 16; a thread takes 4 rows x 4 adjacent columns (2 shared
// 16-byte loads per 16 FMAs).  The next tile's T and row factors (Uc_i, Q_i)
// are loaded into registers while the current tile is computed; the row
// factors pass through two shared buffers in turn, so one barrier per tile
// suffices.
template <int MF>
__global__ void __launch_bounds__(256, 2) gw_assemble4_kernel(const float* __restrict__ T, const float* __restrict__ v1,
                                                              const float* __restrict__ v2, const float* __restrict__ Uc,
                                                              const float* __restrict__ Q, const float* __restrict__ Pp,
                                                              const float* __restrict__ Ud, int64_t n1, int64_t n2,
                                                              float* __restrict__ L, int rows_per_group) {
  constexpr int K2 = 2 * MF, TR = 16;
  constexpr int RF = K2 * TR / 256;  // row-factor values a thread loads per tile
  static_assert(RF * 256 == K2 * TR, "whole row-factor tiles");
  extern __shared__ __align__(16) float sm[];
  float* colS = sm;               // [K2][kTJ]
  float* rowS = colS + K2 * kTJ;  // two buffers of [K2][TR]
  const int t = threadIdx.x, cg = t & 63, rg = t >> 6;
  const int64_t j0 = (int64_t)blockIdx.x * kTJ;
  for (int e = t; e < K2 * kTJ; e += 256) {
    const int k = e / kTJ, c = e % kTJ;
    const int64_t j = j0 + c;
    colS[e] = j < n2 ? (k < MF ? Pp[j * MF + k] : Ud[j * MF + k - MF]) : 0.f;
  }
  const int64_t jc = j0 + 4 * cg;
  const bool cols_ok = jc < n2;  // n2 % 4 == 0: all four or none
  const float4 w2 = cols_ok ? *reinterpret_cast<const float4*>(v2 + jc) : make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t ig0 = (int64_t)blockIdx.y * rows_per_group, ig1 = min(n1, ig0 + rows_per_group);
  float4 tv[4];
  float rf[RF];
  auto fetch = [&](int64_t i0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t i = i0 + 4 * rg + r;
      tv[r] = (cols_ok && i < ig1) ? *reinterpret_cast<const float4*>(T + i * n2 + jc) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < RF; ++q) {
      const int e = t + 256 * q, k = e / TR;
      const int64_t i = i0 + e % TR;
      rf[q] = i < ig1 ? (k < MF ? Uc[i * MF + k] : Q[i * MF + k - MF]) : 0.f;
    }
  };
  if (ig0 < ig1) fetch(ig0);
  int buf = 0;
  for (int64_t i0 = ig0; i0 < ig1; i0 += TR, buf ^= 1) {
    float* rs = rowS + buf * K2 * TR;
#pragma unroll
    for (int q = 0; q < RF; ++q) rs[t + 256 * q] = rf[q];
    float4 cur[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) cur[r] = tv[r];
    __syncthreads();  // this tile's row factors (and, the first time, colS) are in place
    if (i0 + TR < ig1) fetch(i0 + TR);
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 8
    for (int k = 0; k < K2; ++k) {
      const float4 cv = *reinterpret_cast<const float4*>(colS + k * kTJ + 4 * cg);
      const float4 ra = *reinterpret_cast<const float4*>(rs + k * TR + 4 * rg);
      const float rv[4] = {ra.x, ra.y, ra.z, ra.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc[r][0] = fmaf(rv[r], cv.x, acc[r][0]);
        acc[r][1] = fmaf(rv[r], cv.y, acc[r][1]);
        acc[r][2] = fmaf(rv[r], cv.z, acc[r][2]);
        acc[r][3] = fmaf(rv[r], cv.w, acc[r][3]);
      }
    }
    if (!cols_ok) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t i = i0 + 4 * rg + r;
      if (i < ig1) {
        const float vi = v1[i];
        float4 o;
        o.x = vi + w2.x - 2.f * (cur[r].x + acc[r][0]);
        o.y = vi + w2.y - 2.f * (cur[r].y + acc[r][1]);
        o.z = vi + w2.z - 2.f * (cur[r].z + acc[r][2]);
        o.w = vi + w2.w - 2.f * (cur[r].w + acc[r][3]);
        *reinterpret_cast<float4*>(L + i * n2 + jc) = o;
      }
    }
  }
}

// sum += sum_i A_i . (B_i Km)   (FP64)
__global__ void rowdot_kernel(const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ Km,
                              int64_t n, int mf, double* __restrict__ sum) {
  __shared__ float Ks[32 * 32];
  __shared__ double red[8];
  for (int e = threadIdx.x; e < mf * mf; e += blockDim.x) Ks[e] = Km[e];
  __syncthreads();
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float row = 0.f;  // FP32 within a row, FP64 across rows
    for (int f = 0; f < mf; ++f) {
      float bk = 0.f;
      for (int g = 0; g < mf; ++g) bk = fmaf(B[i * mf + g], Ks[g * mf + f], bk);
      row = fmaf(A[i * mf + f], bk, row);
    }
    acc += (double)row;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    atomicAdd(sum, v);
  }
}

// sums[0..3] += <dG, dG>, <dG, G>, <M, dG>, <v1 1^T + 1 v2^T, dG>  (FP64); rows
// strided over blocks, columns over threads
__global__ void gw_dots_kernel(const float* __restrict__ G, const float* __restrict__ dG, const float* __restrict__ M,
                               const float* __restrict__ v1, const float* __restrict__ v2, int64_t n1, int64_t n2,
                               double* __restrict__ sums) {
  double s[4] = {0, 0, 0, 0};
  const bool vec = (n2 & 3) == 0 && ((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(dG) |
                                       reinterpret_cast<uintptr_t>(M) | reinterpret_cast<uintptr_t>(v2)) & 15) == 0;
  for (int64_t i = blockIdx.x; i < n1; i += gridDim.x) {  // FP32 within a row, FP64 across rows
    const float vi = v1[i];
    float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
    if (vec) {
      const float4* d4 = reinterpret_cast<const float4*>(dG + i * n2);
      const float4* g4 = reinterpret_cast<const float4*>(G + i * n2);
      const float4* m4 = reinterpret_cast<const float4*>(M + i * n2);
      const float4* w4 = reinterpret_cast<const float4*>(v2);
#pragma unroll 2
      for (int64_t j = threadIdx.x; j < n2 / 4; j += blockDim.x) {
        const float4 d = d4[j], g = g4[j], m = m4[j], w = w4[j];
        r0 = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, r0))));
        r1 = fmaf(d.x, g.x, fmaf(d.y, g.y, fmaf(d.z, g.z, fmaf(d.w, g.w, r1))));
        r2 = fmaf(d.x, m.x, fmaf(d.y, m.y, fmaf(d.z, m.z, fmaf(d.w, m.w, r2))));
        r3 = fmaf(d.x, vi + w.x, fmaf(d.y, vi + w.y, fmaf(d.z, vi + w.z, fmaf(d.w, vi + w.w, r3))));
      }
    } else {
#pragma unroll 4
      for (int64_t j = threadIdx.x; j < n2; j += blockDim.x) {
        const int64_t e = i * n2 + j;
        const float d = dG[e];
        r0 = fmaf(d, d, r0);
        r1 = fmaf(d, G[e], r1);
        r2 = fmaf(d, M[e], r2);
        r3 = fmaf(d, vi + v2[j], r3);
      }
    }
    s[0] += r0;
    s[1] += r1;
    s[2] += r2;
    s[3] += r3;
  }
  __shared__ double red[4][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 4; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    atomicAdd(&sums[threadIdx.x], v);
  }
}

rfd_status cuda_err(const char* what, cudaError_t e) { return fail(RFD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)); }

// Y = C X on the plan (column chunks of at most max_channels)
rfd_status fm_apply(rfd_plan_t pl, const float* X, int64_t ncols, int64_t ldX, float* Y, int64_t ldY) {
  const int64_t cmax = pl->p.max_channels;
  for (int64_t j0 = 0; j0 < ncols; j0 += cmax) {
    const int c = (int)std::min<int64_t>(cmax, ncols - j0);
    const rfd_status s = rfd_integrate(pl, X + j0, c, ldX, Y + j0, ldY);
    if (s != RFD_OK) return s;
  }
  return RFD_OK;
}

rfd_status transpose(const float* A, int64_t rows, int64_t cols, float* B, cudaStream_t st) {
  const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose_f32_kernel<<<grid, dim3(32, 8), 0, st>>>(A, cols, rows, cols, B, rows);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RFD_OK : cuda_err("transpose", e);
}

// v = C^{(.)2} p = diag(C D_p C^T) (Eq. sq); work: 2 n^2 floats
rfd_status hadamard_square(rfd_plan_t pl, const float* p, float* v, float* work) {
  const int64_t n = pl->n;
  cudaStream_t st = pl->stream;
  float *X = work, *Y = work + n * n;
  diag_fill_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(p, X, n);
  count_launch();
  rfd_status s = fm_apply(pl, X, n, n, Y, n);                 // C D_p
  if (s == RFD_OK) s = transpose(Y, n, n, X, st);             // (C D_p)^T
  if (s == RFD_OK) s = fm_apply(pl, X, n, n, Y, n);           // C D_p C^T
  if (s != RFD_OK) return s;
  diag_take_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Y, v, n);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RFD_OK : cuda_err("hadamard square", e);
}

// W = C T D^T = (FM_D(FM_C(T)^T))^T for T n1 x n2; work: 2 n1 n2 floats
rfd_status sandwich(rfd_plan_t pc, rfd_plan_t pd, const float* T, float* W, float* work) {
  const int64_t n1 = pc->n, n2 = pd->n;
  cudaStream_t st = pc->stream;
  float *A = work, *B = work + n1 * n2;
  rfd_status s = fm_apply(pc, T, n2, n2, A, n2);     // C T          (n1 x n2)
  if (s == RFD_OK) s = transpose(A, n1, n2, B, st);  // (C T)^T      (n2 x n1)
  if (s == RFD_OK) s = fm_apply(pd, B, n1, n1, A, n1);  // D (C T)^T (n2 x n1)
  if (s == RFD_OK) s = transpose(A, n2, n1, W, st);  // C T D^T      (n1 x n2)
  return s;
}

rfd_status check_pair(rfd_plan_t pc, rfd_plan_t pd) {
  if (!pc || !pd) return fail(RFD_EINVAL, "null plan");
  if (!pc->have_G || !pd->have_G) return fail(RFD_EINVAL, "rfd_features (or rfd_gfi) must run on both plans first");
  if (pc->stream != pd->stream) return fail(RFD_EINVAL, "both plans must use the same stream");
  return RFD_OK;
}

// ---- low-rank form: host side ---------------------------------------------------
constexpr int kLowRankMaxM = 32;

unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

constexpr int kGramChunks = 32;

// out (mf x mf) = sum_i w_i A_i A_i^T-like reduction in kGramChunks row chunks; part: kGramChunks mf^2 floats
void wgram(const float* A, const float* B, const float* w, int64_t n, int mf, float* part, float* out,
           cudaStream_t st) {
  weighted_gram_kernel<<<dim3(mf, kGramChunks), 256, 0, st>>>(A, B, w, n, mf, part);
  sum_parts_kernel<<<blocks_for((int64_t)mf * mf, 256), 256, 0, st>>>(part, kGramChunks, (int64_t)mf * mf,
                                                                      (int64_t)mf * mf, out);
  count_launch(2);
}

// bump allocator over one stream-ordered block (64-float granules)
struct Carve {
  float* base = nullptr;
  size_t used = 0;
  float* take(size_t floats) {
    float* p = base + used;
    used += (floats + 63) & ~size_t(63);
    return p;
  }
};

struct LowRank {  // one cloud: Psi and U point-major (N x MF), K (MF x MF)
  float *psi, *U, *K;
};

rfd_status launched_or(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RFD_OK : cuda_err(what, e);
}

rfd_status lowrank_prepare(rfd_plan_t pl, int mf, const LowRank& lr, float* tmp_fm, cudaStream_t st) {
  const float* fm = static_cast<const float*>(pl->d_psi);
  if (pl->bf16) {  // FP32 features from the plan's copy of its points
    const cudaError_t e = launch_features(pl->d_xyz, pl->n, pl->n_pad, pl->d_omega_hi, pl->d_omega_lo, pl->h, false,
                                          tmp_fm, st);
    count_launch();
    if (e != cudaSuccess) return cuda_err("features", e);
    fm = tmp_fm;
  }
  const int64_t n = pl->n;
  features_point_major_kernel<<<blocks_for(n * mf, 256), 256, 0, st>>>(fm, pl->n_pad, pl->m, n, mf, lr.psi);
  lowrank_k_kernel<<<blocks_for((int64_t)mf * mf, 256), 256, 0, st>>>(pl->d_G, pl->d_oa, pl->d_ob, pl->m, mf, lr.K);
  rowmat_kernel<<<blocks_for(n * mf, 256), 256, 0, st>>>(lr.psi, lr.K, 0, nullptr, n, mf, lr.U);
  count_launch(3);
  return launched_or("low-rank factors");
}

// v = C^{(.)2} p in the low-rank form; S: mf x mf scratch
rfd_status lowrank_hadamard(rfd_plan_t pl, int mf, const LowRank& lr, const float* p, float* S, float* v,
                            cudaStream_t st) {
  wgram(lr.psi, lr.psi, p, pl->n, mf, S + mf * mf, S, st);
  hadamard_lowrank_kernel<<<blocks_for(pl->n, 256), 256, 0, st>>>(lr.U, lr.psi, S, p, pl->n, mf, v);
  count_launch();
  return launched_or("hadamard square");
}

struct Proj {  // projections of one n1 x n2 matrix X: Pt = (Psi_C^T X)^T, Q = X Psi_D, Pp = P'^T
  float *Pt, *Q, *Pp;
};

size_t project_parts_floats(int64_t n1, int64_t n2, int mf) {
  const int64_t groups = row_groups(n1, n2, kTI);
  const int64_t strips = (n2 + kTJ - 1) / kTJ;
  return (size_t)(groups * n2 * mf + 64) + (size_t)(strips * n1 * mf + 64);
}

template <int MF>
rfd_status project_mf(const float* X, int64_t n1, int64_t n2, const LowRank& c, const LowRank& d, const Proj& pr,
                      float* parts, float* R, cudaStream_t st) {
  const int64_t tiles = (n1 + kTI - 1) / kTI;
  const int groups = row_groups(n1, n2, kTI);
  const int rows_per_group = (int)(((tiles + groups - 1) / groups) * kTI);
  const int strips = (int)((n2 + kTJ - 1) / kTJ);
  float* Pt_part = parts;
  float* Q_part = parts + (((size_t)groups * n2 * MF + 63) & ~size_t(63));
  const bool vec16 = MF == 16 && (n2 & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  cudaError_t e = cudaSuccess;
  if (vec16) {  // register tiles (16-byte rows of X)
    const size_t smem = (size_t)(kTI * (kTJ + 4) + kTI * MF + kTJ * MF) * sizeof(float);
    e = cudaFuncSetAttribute(gw_project16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_err("projection attribute", e);
    gw_project16_kernel<<<dim3(strips, groups), 256, smem, st>>>(X, n1, n2, c.psi, d.psi, Pt_part, Q_part,
                                                                 rows_per_group);
  } else {
    const size_t smem = (size_t)(kTI * kPLd + kTI * MF + kTJ * MF + 8 * kTI * (MF + 1)) * sizeof(float);
    e = cudaFuncSetAttribute(gw_project_kernel<MF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_err("projection attribute", e);
    gw_project_kernel<MF><<<dim3(strips, groups), 256, smem, st>>>(X, n1, n2, c.psi, d.psi, Pt_part, Q_part,
                                                                    rows_per_group);
  }
  sum_parts_kernel<<<blocks_for(n2 * MF, 256), 256, 0, st>>>(Pt_part, groups, n2 * MF, n2 * MF, pr.Pt);
  sum_parts_kernel<<<blocks_for(n1 * MF, 256), 256, 0, st>>>(Q_part, strips, n1 * MF, n1 * MF, pr.Q);
  wgram(pr.Pt, d.psi, nullptr, n2, MF, R + MF * MF, R, st);                                  // R = P Psi_D
  rowmat_kernel<<<blocks_for(n2 * MF, 256), 256, 0, st>>>(d.U, R, 1, pr.Pt, n2, MF, pr.Pp);  // P'^T
  count_launch(4);
  return launched_or("projection");
}

rfd_status project(int mf, const float* X, int64_t n1, int64_t n2, const LowRank& c, const LowRank& d,
                   const Proj& pr, float* parts, float* R, cudaStream_t st) {
  return mf == 16 ? project_mf<16>(X, n1, n2, c, d, pr, parts, R, st)
                  : project_mf<32>(X, n1, n2, c, d, pr, parts, R, st);
}

// everything both entry points need: factors of both clouds, v1, v2
struct LowRankPair {
  int mf = 16;
  LowRank c{}, d{};
  float *v1 = nullptr, *v2 = nullptr, *S = nullptr, *R = nullptr, *parts = nullptr;
};

size_t lowrank_floats(rfd_plan_t pc, rfd_plan_t pd, int mf, int nproj) {
  const int64_t n1 = pc->n, n2 = pd->n;
  const size_t fm = std::max((size_t)pc->m * pc->n_pad, (size_t)pd->m * pd->n_pad);
  size_t f = fm + 64;
  f += 2 * ((size_t)n1 * mf + 64) + 2 * ((size_t)n2 * mf + 64) + 2 * ((size_t)mf * mf + 64) +
       2 * ((size_t)(1 + kGramChunks) * mf * mf + 64);
  f += (size_t)n1 + (size_t)n2 + 128;
  f += project_parts_floats(n1, n2, mf) + 64;
  f += (size_t)nproj * ((size_t)n2 * mf * 2 + (size_t)n1 * mf + 192);
  return f + 256;
}

rfd_status lowrank_setup(rfd_plan_t pc, rfd_plan_t pd, const float* p, const float* q, Carve& cv, LowRankPair& lp,
                         cudaStream_t st) {
  const int mf = lp.mf;
  const int64_t n1 = pc->n, n2 = pd->n;
  float* tmp_fm = cv.take(std::max((size_t)pc->m * pc->n_pad, (size_t)pd->m * pd->n_pad));
  lp.c = LowRank{cv.take(n1 * mf), cv.take(n1 * mf), cv.take((size_t)mf * mf)};
  lp.d = LowRank{cv.take(n2 * mf), cv.take(n2 * mf), cv.take((size_t)mf * mf)};
  lp.S = cv.take((size_t)(1 + kGramChunks) * mf * mf);
  lp.R = cv.take((size_t)(1 + kGramChunks) * mf * mf);
  lp.v1 = cv.take(n1);
  lp.v2 = cv.take(n2);
  lp.parts = cv.take(project_parts_floats(n1, n2, mf));
  rfd_status s = lowrank_prepare(pc, mf, lp.c, tmp_fm, st);
  if (s == RFD_OK) s = lowrank_prepare(pd, mf, lp.d, tmp_fm, st);
  if (s == RFD_OK) s = lowrank_hadamard(pc, mf, lp.c, p, lp.S, lp.v1, st);
  if (s == RFD_OK) s = lowrank_hadamard(pd, mf, lp.d, q, lp.S, lp.v2, st);
  return s;
}

Proj take_proj(Carve& cv, int64_t n1, int64_t n2, int mf) {
  return Proj{cv.take(n2 * mf), cv.take(n1 * mf), cv.take(n2 * mf)};
}

bool lowrank_ok(rfd_plan_t pc, rfd_plan_t pd) { return pc->m <= kLowRankMaxM && pd->m <= kLowRankMaxM; }
int lowrank_mf(rfd_plan_t pc, rfd_plan_t pd) { return std::max(pc->m, pd->m) <= 16 ? 16 : 32; }

rfd_status tensor_product_lowrank(rfd_plan_t pc, rfd_plan_t pd, const float* T, const float* p, const float* q,
                                  float* L) {
  cudaStream_t st = pc->stream;
  LowRankPair lp;
  lp.mf = lowrank_mf(pc, pd);
  const int64_t n1 = pc->n, n2 = pd->n;
  Carve cv;
  const size_t bytes = lowrank_floats(pc, pd, lp.mf, 1) * sizeof(float);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&cv.base), bytes, st);
  if (e != cudaSuccess) return fail(RFD_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  rfd_status s = lowrank_setup(pc, pd, p, q, cv, lp, st);
  const Proj pr = take_proj(cv, n1, n2, lp.mf);
  if (s == RFD_OK) s = project(lp.mf, T, n1, n2, lp.c, lp.d, pr, lp.parts, lp.R, st);
  if (s == RFD_OK) {
    const bool vec4 = (n2 & 3) == 0 && ((reinterpret_cast<uintptr_t>(T) | reinterpret_cast<uintptr_t>(L) |
                                          reinterpret_cast<uintptr_t>(lp.v2)) & 15) == 0;
    if (vec4) {
      const int64_t tiles = (n1 + 15) / 16;
      const int groups = row_groups(n1, n2, 16);
      const int rows_per_group = (int)(((tiles + groups - 1) / groups) * 16);
      const dim3 grid((unsigned)((n2 + kTJ - 1) / kTJ), (unsigned)groups);
      const size_t smem = (size_t)2 * lp.mf * (kTJ + 2 * 16) * sizeof(float);
      if (lp.mf == 16) {
        e = cudaFuncSetAttribute(gw_assemble4_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
          gw_assemble4_kernel<16><<<grid, 256, smem, st>>>(T, lp.v1, lp.v2, lp.c.U, pr.Q, pr.Pp, lp.d.U, n1, n2, L,
                                                           rows_per_group);
      } else {
        e = cudaFuncSetAttribute(gw_assemble4_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
          gw_assemble4_kernel<32><<<grid, 256, smem, st>>>(T, lp.v1, lp.v2, lp.c.U, pr.Q, pr.Pp, lp.d.U, n1, n2, L,
                                                           rows_per_group);
      }
      if (e != cudaSuccess) s = cuda_err("assembly attribute", e);
    } else {
      const dim3 grid((unsigned)((n2 + kTJ - 1) / kTJ), (unsigned)((n1 + kTA - 1) / kTA));
      if (lp.mf == 16)
        gw_assemble_kernel<16><<<grid, 256, 0, st>>>(T, lp.v1, lp.v2, lp.c.U, pr.Q, pr.Pp, lp.d.U, n1, n2, L);
      else
        gw_assemble_kernel<32><<<grid, 256, 0, st>>>(T, lp.v1, lp.v2, lp.c.U, pr.Q, pr.Pp, lp.d.U, n1, n2, L);
    }
    count_launch();
    if (s == RFD_OK) s = launched_or("tensor product");
  }
  cudaFreeAsync(cv.base, st);
  return s;
}

rfd_status line_search_lowrank(rfd_plan_t pc, rfd_plan_t pd, const float* G, const float* dG, const float* M,
                               const float* p, const float* q, double h[5]) {
  cudaStream_t st = pc->stream;
  LowRankPair lp;
  lp.mf = lowrank_mf(pc, pd);
  const int64_t n1 = pc->n, n2 = pd->n;
  Carve cv;
  const size_t bytes = lowrank_floats(pc, pd, lp.mf, 2) * sizeof(float) + 32 * sizeof(double);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&cv.base), bytes, st);
  if (e != cudaSuccess) return fail(RFD_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  rfd_status s = lowrank_setup(pc, pd, p, q, cv, lp, st);
  const Proj pdG = take_proj(cv, n1, n2, lp.mf), pG = take_proj(cv, n1, n2, lp.mf);
  double* sums = reinterpret_cast<double*>(cv.take(2 * 16));
  if (s == RFD_OK) s = project(lp.mf, dG, n1, n2, lp.c, lp.d, pdG, lp.parts, lp.R, st);
  if (s == RFD_OK) s = project(lp.mf, G, n1, n2, lp.c, lp.d, pG, lp.parts, lp.R, st);
  double hs[10] = {};
  if (s == RFD_OK) {
    e = cudaMemsetAsync(sums, 0, 10 * sizeof(double), st);
    if (e == cudaSuccess) {
      const int mf = lp.mf;
      gw_dots_kernel<<<(unsigned)std::min<int64_t>(n1, 152 * 8), 256, 0, st>>>(G, dG, M, lp.v1, lp.v2, n1, n2, sums);
      // <C X D^T, Y> = <X, Y> + sum_j Pp_X[j] . (Pt_Y[j] K_C) + sum_i Q_X[i] . (Q_Y[i] K_D)
      const unsigned b2 = blocks_for(n2, 256) > 304 ? 304 : blocks_for(n2, 256);
      const unsigned b1 = blocks_for(n1, 256) > 304 ? 304 : blocks_for(n1, 256);
      rowdot_kernel<<<b2, 256, 0, st>>>(pdG.Pp, pdG.Pt, lp.c.K, n2, mf, sums + 4);
      rowdot_kernel<<<b1, 256, 0, st>>>(pdG.Q, pdG.Q, lp.d.K, n1, mf, sums + 5);
      rowdot_kernel<<<b2, 256, 0, st>>>(pdG.Pp, pG.Pt, lp.c.K, n2, mf, sums + 6);
      rowdot_kernel<<<b1, 256, 0, st>>>(pdG.Q, pG.Q, lp.d.K, n1, mf, sums + 7);
      rowdot_kernel<<<b2, 256, 0, st>>>(pG.Pp, pdG.Pt, lp.c.K, n2, mf, sums + 8);
      rowdot_kernel<<<b1, 256, 0, st>>>(pG.Q, pdG.Q, lp.d.K, n1, mf, sums + 9);
      count_launch(7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_err("line search", e);
  }
  cudaFreeAsync(cv.base, st);
  if (s != RFD_OK) return s;
  h[0] = hs[0] + hs[4] + hs[5];  // <C dG D^T, dG>
  h[1] = hs[1] + hs[6] + hs[7];  // <C dG D^T, G>
  h[2] = hs[1] + hs[8] + hs[9];  // <C G D^T, dG>
  h[3] = hs[2];                  // <M, dG>
  h[4] = hs[3];                  // <c_CD, dG>
  return RFD_OK;
}

// The step of Algorithm line_search.  Along G + tau dG the (F)GW cost is a
// quadratic in tau, q(tau) = a tau^2 + b tau + q(0), whose coefficients are
// combinations of five inner products h = <C dG D^T, dG>, <C dG D^T, G>,
// <C G D^T, dG>, <M, dG>, <c_CD, dG> weighted by alpha (the quadratic part
// comes from the structure term only, the linear part from both terms).  The
// step is the minimiser of q on [0, 1]: the vertex clamped to the interval
// when q is convex, else whichever end costs less (q(1) - q(0) = a + b).
rfd_status finish_line_search(double alpha, const double h[5], double* out3) {
  const double a = -2.0 * alpha * h[0];
  const double b = (1.0 - alpha) * h[3] + alpha * h[4] - 2.0 * alpha * (h[1] + h[2]);
  const double tau = a > 0 ? std::min(1.0, std::max(0.0, -b / (2.0 * a))) : (a + b < 0 ? 1.0 : 0.0);
  out3[0] = tau;
  out3[1] = a;
  out3[2] = b;
  return RFD_OK;
}

}  // namespace

}  // namespace rfd

using namespace rfd;

extern "C" rfd_status rfd_fm_apply(rfd_plan_t pl, const float* d_X, int64_t ncols, int64_t ldX, float* d_Y,
                                   int64_t ldY) {
  if (!pl || !d_X || !d_Y) return fail(RFD_EINVAL, "null argument");
  if (ncols < 1 || ldX < ncols || ldY < ncols) return fail(RFD_EINVAL, "need 1 <= ncols <= ldX, ldY");
  if (!pl->have_G) return fail(RFD_EINVAL, "rfd_features (or rfd_gfi) must run before rfd_fm_apply");
  return fm_apply(pl, d_X, ncols, ldX, d_Y, ldY);
}

extern "C" rfd_status rfd_gw_tensor_product(rfd_plan_t pc, rfd_plan_t pd, const float* d_T, const float* d_p,
                                            const float* d_q, float* d_L) {
  rfd_status s = check_pair(pc, pd);
  if (s != RFD_OK) return s;
  if (!d_T || !d_p || !d_q || !d_L) return fail(RFD_EINVAL, "null argument");
  if (lowrank_ok(pc, pd)) return tensor_product_lowrank(pc, pd, d_T, d_p, d_q, d_L);
  const int64_t n1 = pc->n, n2 = pd->n, nn = std::max(n1, n2);
  cudaStream_t st = pc->stream;
  float* work = nullptr;
  const size_t elems = (size_t)(2 * nn * nn + 3 * n1 * n2 + n1 + n2);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&work), elems * sizeof(float), st);
  if (e != cudaSuccess) return fail(RFD_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  float* sq = work;                     // 2 nn^2: the Hadamard-square work
  float* W = sq + 2 * nn * nn;          // n1 n2: C T D^T
  float* sw = W + n1 * n2;              // 2 n1 n2: the sandwich work
  float* v1 = sw + 2 * n1 * n2;
  float* v2 = v1 + n1;
  s = hadamard_square(pc, d_p, v1, sq);
  if (s == RFD_OK) s = hadamard_square(pd, d_q, v2, sq);
  if (s == RFD_OK) s = sandwich(pc, pd, d_T, W, sw);
  if (s == RFD_OK) {
    assemble_kernel<<<(unsigned)((n1 * n2 + 255) / 256), 256, 0, st>>>(v1, v2, W, d_L, n1, n2);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_err("tensor product", e);
  }
  cudaFreeAsync(work, st);
  return s;
}

extern "C" rfd_status rfd_gw_line_search(rfd_plan_t pc, rfd_plan_t pd, double alpha, const float* d_G,
                                         const float* d_dG, const float* d_M, const float* d_p, const float* d_q,
                                         double* out3) {
  rfd_status s = check_pair(pc, pd);
  if (s != RFD_OK) return s;
  if (!d_G || !d_dG || !d_M || !d_p || !d_q || !out3) return fail(RFD_EINVAL, "null argument");
  if (!std::isfinite(alpha)) return fail(RFD_EINVAL, "alpha must be finite");
  double h[5] = {0, 0, 0, 0, 0};
  if (lowrank_ok(pc, pd)) {
    s = line_search_lowrank(pc, pd, d_G, d_dG, d_M, d_p, d_q, h);
    if (s != RFD_OK) return s;
    return finish_line_search(alpha, h, out3);
  }
  const int64_t n1 = pc->n, n2 = pd->n, nn = std::max(n1, n2);
  cudaStream_t st = pc->stream;
  float* work = nullptr;
  const size_t elems = (size_t)(2 * nn * nn + 4 * n1 * n2 + n1 + n2) + 16;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&work), elems * sizeof(float), st);
  if (e != cudaSuccess) return fail(RFD_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  float* sq = work;
  float* a1 = sq + 2 * nn * nn;
  float* b1 = a1 + n1 * n2;
  float* sw = b1 + n1 * n2;  // 2 n1 n2
  float* v1 = sw + 2 * n1 * n2;
  float* v2 = v1 + n1;
  double* sums = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(v2 + n2) + 15) & ~uintptr_t(15));
  s = hadamard_square(pc, d_p, v1, sq);  // c_CD = v1 1^T + 1 v2^T (steps 1 and 2 of tensor_prod)
  if (s == RFD_OK) s = hadamard_square(pd, d_q, v2, sq);
  if (s == RFD_OK) s = sandwich(pc, pd, d_dG, a1, sw);  // a1 = C dG D
  if (s == RFD_OK) s = sandwich(pc, pd, d_G, b1, sw);   // b1 = C G D
  if (s == RFD_OK) {
    e = cudaMemsetAsync(sums, 0, 5 * sizeof(double), st);
    if (e == cudaSuccess) {
      line_search_sums_kernel<<<152 * 4, 256, 0, st>>>(a1, b1, d_G, d_dG, d_M, v1, v2, n1, n2, sums);
      count_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_err("line search", e);
  }
  cudaFreeAsync(work, st);
  if (s != RFD_OK) return s;
  return finish_line_search(alpha, h, out3);
}
