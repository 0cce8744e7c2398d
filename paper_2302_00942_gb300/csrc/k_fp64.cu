// FP64 dense building blocks for step a4, G = lambda phi1(lambda M), on the
// m x m matrix M (Sec. 2.4: "cubic in the number of random features").  The
// Pade evaluation (rfd_phi1.cu) is written in terms of these: a GEMM, linear
// combinations, the 1-norm, and an LU factorisation with partial pivoting
// followed by triangular solves for the Pade denominator.
//
// GB300 runs FP64 at ~1 TFLOP/s (DFMA and DMMA alike), so every kernel here is
// FP64-pipe-bound at any reasonable tiling; tiles are small (32 x 32) so that a
// 1024 x 1024 product spreads over all SMs in ~7 balanced rounds.
#include <cuda_runtime.h>
#include <cstdint>
#include "kernels.h"

namespace rfd {

namespace {

constexpr int kGT = 32;   // output tile
constexpr int kGK = 32;   // k chunk
constexpr int kGThreads = 64;  // 8 x 8 threads, 4 x 4 outputs each

__global__ void __launch_bounds__(kGThreads)
dgemm_kernel(int M, int N, int K, double alpha, const double* __restrict__ A, int lda,
             const double* __restrict__ B, int ldb, double beta, double* C, int ldc) {
  __shared__ double As[kGK][kGT + 1];
  __shared__ double Bs[kGK][kGT + 1];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int row0 = blockIdx.y * kGT, col0 = blockIdx.x * kGT;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGK) {
    for (int i = threadIdx.x; i < kGT * kGK; i += kGThreads) {
      const int r = i / kGK, kk = i % kGK;          // A: row r, column k0 + kk
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[(size_t)gr * lda + gk] : 0.0;
      const int br = i / kGT, bc = i % kGT;         // B: row k0 + br, column col0 + bc
      const int gbr = k0 + br, gbc = col0 + bc;
      Bs[br][bc] = (gbr < K && gbc < N) ? B[(size_t)gbr * ldb + gbc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 8 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 8 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 8 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = col0 + tx + 8 * j;
      if (cc >= N) continue;
      double* p = C + (size_t)r * ldc + cc;
      *p = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *p);
    }
  }
}

__global__ void dcombine_kernel(int m, int n, double* D, int ldd, double a0, const double* X0, double a1,
                                const double* X1, double a2, const double* X2, double a3, const double* X3,
                                double diag, int ldx) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const size_t ix = (size_t)i * ldx + j;
  double v = (i == j) ? diag : 0.0;
  if (X0) v += a0 * X0[ix];
  if (X1) v += a1 * X1[ix];
  if (X2) v += a2 * X2[ix];
  if (X3) v += a3 * X3[ix];
  D[(size_t)i * ldd + j] = v;
}

// max over columns of the column abs-sum; non-negative doubles order like
// their bit patterns, so an integer atomicMax on the bits is exact.
// Block (32 columns x 32 row lanes): each thread sums every 32nd row of one
// column (coalesced across x), the 32 partial sums are reduced in shared memory.
__global__ void dnorm1_kernel(int m, const double* __restrict__ X, int ldx, unsigned long long* out) {
  __shared__ double part[32][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (j < m)
    for (int i = threadIdx.y; i < m; i += 32) s += fabs(X[(size_t)i * ldx + j]);
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < m) {
    double t = 0.0;
    for (int y = 0; y < 32; ++y) t += part[y][threadIdx.x];
    if (!(t == t)) t = __longlong_as_double(0x7FF0000000000000ll);  // NaN -> +inf
    atomicMax(out, (unsigned long long)__double_as_longlong(t));
  }
}

__global__ void dfinite_kernel(int m, int n, const double* __restrict__ X, int ldx, int* flag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * n) return;
  const double v = X[(size_t)(e / n) * ldx + e % n];
  if (!isfinite(v)) atomicExch(flag, 1);
}

// ---- LU with partial pivoting ---------------------------------------------------
constexpr int kNB = 16;          // panel width
constexpr int kPanelThreads = 1024;

// Factor the panel A[k0:m, k0:k0+nb] in place (one CTA; the panel is L2
// resident).  For each column: pivot = first row of largest |value| (ties to
// the smaller index), swap within the panel, scale, rank-1 update.
__global__ void __launch_bounds__(kPanelThreads)
panel_kernel(int m, double* A, int lda, int k0, int nb, int* ipiv, int* info) {
  __shared__ double red_v[kPanelThreads / 32];
  __shared__ int red_i[kPanelThreads / 32];
  __shared__ int piv_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int j = 0; j < nb; ++j) {
    const int col = k0 + j;
    double best = -1.0;
    int bi = m;
    for (int i = col + tid; i < m; i += kPanelThreads) {
      const double v = fabs(A[(size_t)i * lda + col]);
      if (v > best) { best = v; bi = i; }  // i increases within a thread: keeps the first max
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[wid] = best; red_i[wid] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = -1.0;
      int bidx = m;
      for (int w = 0; w < kPanelThreads / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bidx)) { bv = red_v[w]; bidx = red_i[w]; }
      if (bidx >= m || bv == 0.0) { bidx = col; if (*info == 0) *info = col + 1; }
      piv_s = bidx;
      ipiv[col] = bidx;
    }
    __syncthreads();
    const int p = piv_s;
    if (p != col && tid < nb) {
      double* r1 = A + (size_t)col * lda + k0;
      double* r2 = A + (size_t)p * lda + k0;
      const double t = r1[tid];
      r1[tid] = r2[tid];
      r2[tid] = t;
    }
    __syncthreads();
    const double d = A[(size_t)col * lda + col];
    const double inv = (d != 0.0) ? 1.0 / d : 0.0;
    for (int i = col + 1 + tid; i < m; i += kPanelThreads) A[(size_t)i * lda + col] *= inv;
    __syncthreads();
    const int rem = nb - j - 1;
    if (rem > 0) {
      const int rows = m - col - 1;
      for (int e = tid; e < rows * rem; e += kPanelThreads) {
        const int i = col + 1 + e / rem, jj = col + 1 + e % rem;
        A[(size_t)i * lda + jj] -= A[(size_t)i * lda + col] * A[(size_t)col * lda + jj];
      }
    }
    __syncthreads();
  }
}

// Apply the panel's row interchanges (ipiv[k0 .. k0+nb-1], in order) to the
// columns outside the panel.
__global__ void swap_outside_kernel(int m, double* A, int lda, const int* ipiv, int k0, int nb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m || (j >= k0 && j < k0 + nb)) return;
  for (int t = 0; t < nb; ++t) {
    const int r = k0 + t, p = ipiv[r];
    if (p != r) {
      const double x = A[(size_t)r * lda + j];
      A[(size_t)r * lda + j] = A[(size_t)p * lda + j];
      A[(size_t)p * lda + j] = x;
    }
  }
}

// Rows [k0, k0+nb) of B (columns [c0, c0+ncols)) <- L11^{-1} B, L11 unit lower
// (the diagonal block of the factor at rows/cols k0..).  One thread per column.
__global__ void trsm_lower_unit_kernel(const double* __restrict__ L, int ldl, int k0, int nb, double* B, int ldb,
                                       int c0, int ncols) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  double x[kNB];
  for (int i = 0; i < nb; ++i) {
    double v = B[(size_t)(k0 + i) * ldb + c0 + j];
    for (int t = 0; t < i; ++t) v -= L[(size_t)(k0 + i) * ldl + k0 + t] * x[t];
    x[i] = v;
    B[(size_t)(k0 + i) * ldb + c0 + j] = v;
  }
}

// Rows [k0, k0+nb) of B <- U11^{-1} B, U11 upper triangular with its diagonal.
__global__ void trsm_upper_kernel(const double* __restrict__ U, int ldu, int k0, int nb, double* B, int ldb,
                                  int ncols) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  double x[kNB];
  for (int i = nb - 1; i >= 0; --i) {
    double v = B[(size_t)(k0 + i) * ldb + j];
    for (int t = i + 1; t < nb; ++t) v -= U[(size_t)(k0 + i) * ldu + k0 + t] * x[t];
    v /= U[(size_t)(k0 + i) * ldu + k0 + i];
    x[i] = v;
    B[(size_t)(k0 + i) * ldb + j] = v;
  }
}

__global__ void apply_pivots_kernel(int m, const int* ipiv, double* B, int ldb, int ncols) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  for (int r = 0; r < m; ++r) {
    const int p = ipiv[r];
    if (p != r) {
      const double x = B[(size_t)r * ldb + j];
      B[(size_t)r * ldb + j] = B[(size_t)p * ldb + j];
      B[(size_t)p * ldb + j] = x;
    }
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t dgemm(int M, int N, int K, double alpha, const double* A, int lda, const double* B, int ldb,
                  double beta, double* C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(blocks_for(N, kGT), blocks_for(M, kGT));
  dgemm_kernel<<<grid, kGThreads, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  return launched();
}

cudaError_t dcombine(int m, int n, double* D, int ldd, double a0, const double* X0, double a1, const double* X1,
                     double a2, const double* X2, double a3, const double* X3, double diag, int ldx,
                     cudaStream_t st) {
  dcombine_kernel<<<blocks_for((int64_t)m * n, 256), 256, 0, st>>>(m, n, D, ldd, a0, X0, a1, X1, a2, X2, a3, X3,
                                                                    diag, ldx);
  return launched();
}

cudaError_t dnorm1(int m, const double* X, int ldx, double* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  dnorm1_kernel<<<blocks_for(m, 32), dim3(32, 32), 0, st>>>(m, X, ldx, reinterpret_cast<unsigned long long*>(out));
  return launched();
}

cudaError_t dfinite_check(int m, int n, const double* X, int ldx, int* flag, cudaStream_t st) {
  dfinite_kernel<<<blocks_for((int64_t)m * n, 256), 256, 0, st>>>(m, n, X, ldx, flag);
  return launched();
}

cudaError_t dgetrf(int m, double* A, int lda, int* ipiv, double* /*work*/, int* info, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  for (int k0 = 0; k0 < m; k0 += kNB) {
    const int nb = (m - k0 < kNB) ? (m - k0) : kNB;
    panel_kernel<<<1, kPanelThreads, 0, st>>>(m, A, lda, k0, nb, ipiv, info);
    swap_outside_kernel<<<blocks_for(m, 128), 128, 0, st>>>(m, A, lda, ipiv, k0, nb);
    count_launch(2);
    const int rest = m - k0 - nb;
    if (rest > 0) {
      count_launch(1);
      trsm_lower_unit_kernel<<<blocks_for(rest, 128), 128, 0, st>>>(A, lda, k0, nb, A, lda, k0 + nb, rest);
      e = dgemm(rest, rest, nb, -1.0, A + (size_t)(k0 + nb) * lda + k0, lda, A + (size_t)k0 * lda + k0 + nb, lda,
                1.0, A + (size_t)(k0 + nb) * lda + k0 + nb, lda, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t dgetrs(int m, int nrhs, const double* LU, int lda, const int* ipiv, double* B, int ldb,
                   cudaStream_t st) {
  apply_pivots_kernel<<<blocks_for(nrhs, 128), 128, 0, st>>>(m, ipiv, B, ldb, nrhs);
  count_launch(1);
  // forward: L y = P b  (unit lower), block by block
  for (int k0 = 0; k0 < m; k0 += kNB) {
    const int nb = (m - k0 < kNB) ? (m - k0) : kNB;
    trsm_lower_unit_kernel<<<blocks_for(nrhs, 128), 128, 0, st>>>(LU, lda, k0, nb, B, ldb, 0, nrhs);
    count_launch(1);
    const int rest = m - k0 - nb;
    if (rest > 0) {
      cudaError_t e = dgemm(rest, nrhs, nb, -1.0, LU + (size_t)(k0 + nb) * lda + k0, lda, B + (size_t)k0 * ldb, ldb,
                            1.0, B + (size_t)(k0 + nb) * ldb, ldb, st);
      if (e != cudaSuccess) return e;
    }
  }
  // backward: U x = y
  const int last = ((m - 1) / kNB) * kNB;
  for (int k0 = last; k0 >= 0; k0 -= kNB) {
    const int nb = (m - k0 < kNB) ? (m - k0) : kNB;
    trsm_upper_kernel<<<blocks_for(nrhs, 128), 128, 0, st>>>(LU, lda, k0, nb, B, ldb, nrhs);
    count_launch(1);
    if (k0 > 0) {
      cudaError_t e = dgemm(k0, nrhs, nb, -1.0, LU + k0, lda, B + (size_t)k0 * ldb, ldb, 1.0, B, ldb, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

}  // namespace rfd
