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
  double h[5] = {0, 0, 0, 0, 0};
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
  const double a = -2.0 * alpha * h[0];
  const double b = (1.0 - alpha) * h[3] + alpha * h[4] - 2.0 * alpha * (h[1] + h[2]);
  double tau;
  if (a > 0)
    tau = std::min(1.0, std::max(0.0, -b / (2.0 * a)));
  else
    tau = (a + b < 0) ? 1.0 : 0.0;
  out3[0] = tau;
  out3[1] = a;
  out3[2] = b;
  return RFD_OK;
}
