// Entropic Wasserstein barycenter on a resident plan (App. C, Algorithm
// wass_barycenter, after Solomon et al. 2015, Algorithm 2).  The kernel action
// x -> K x with K = exp(lambda W_hat) is rfd_integrate on the plan's resident
// features and G, applied to all k distributions at once (k field channels).
// Each pass is a round of Sinkhorn-type scalings: every input distribution
// gets a pair of scaling vectors (v^i, w^i); the barycenter estimate mu is the
// alpha-weighted geometric mean of the current marginals v^i K(a w^i), and the
// v^i are rescaled towards it.  A pass is two kernel actions (on a v^i and on
// a w^i, a the area weights) and two fused element-wise kernels around them;
// mu starts from 1 in every pass.
//
// Kernel outputs are lifted to kFloor before they divide or enter a power (the
// random-feature kernel need not be positive).  FP32 throughout, on the plan's
// stream; the temporaries come from the stream-ordered allocator.
#include <cuda_runtime.h>
#include <cmath>
#include <string>
#include "kernels.h"
#include "rfd_internal.h"
#include "rfd_plan.h"

namespace rfd {

namespace {

constexpr float kFloor = 1e-30f;
constexpr int kMaxK = 32;

struct Alpha {
  float a[kMaxK];
};

// v = 1 (N x k), F = a (the first pass's a v), out = 1
__global__ void bary_init_kernel(const float* __restrict__ area, float* __restrict__ v, float* __restrict__ F,
                                 float* __restrict__ out, int64_t n, int k) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  v[e] = 1.0f;
  F[e] = area[e / k];
  if (e % k == 0) out[e / k] = 1.0f;
}

// step 1: w = mu_in / max(H, floor); then F = a w for step 2
__global__ void bary_step1_kernel(const float* __restrict__ mu_in, int64_t ld_mu, const float* __restrict__ area,
                                  const float* __restrict__ H, float* __restrict__ w, float* __restrict__ F, int64_t n,
                                  int k) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t p = e / k;
  const int i = (int)(e % k);
  const float wv = mu_in[p * ld_mu + i] / fmaxf(H[e], kFloor);
  w[e] = wv;
  F[e] = area[p] * wv;
}

// steps 2-4 for one point: d^i = v^i max(H^i, floor), mu = exp(sum_i alpha_i log d^i),
// v^i <- v^i mu / d^i, and F = a v for the next pass; mu into out
__global__ void bary_step2_kernel(const float* __restrict__ area, const float* __restrict__ H, float* __restrict__ v,
                                  float* __restrict__ F, float* __restrict__ out, int64_t n, int k, Alpha alpha) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float d[kMaxK];
  float logmu = 0.f;
  for (int i = 0; i < k; ++i) {
    d[i] = fmaxf(v[p * k + i] * fmaxf(H[p * k + i], kFloor), kFloor);
    logmu = fmaf(alpha.a[i], logf(d[i]), logmu);
  }
  const float mu = expf(logmu);
  out[p] = mu;
  for (int i = 0; i < k; ++i) {
    const float vn = v[p * k + i] * mu / d[i];
    v[p * k + i] = vn;
    F[p * k + i] = area[p] * vn;
  }
}

}  // namespace

}  // namespace rfd

using namespace rfd;

extern "C" rfd_status rfd_barycenter(rfd_plan_t pl, const float* d_mu, int32_t k, int64_t ld_mu, const double* alpha,
                                     const float* d_area, int32_t iters, float* d_out) {
  if (!pl || !d_mu || !alpha || !d_area || !d_out) return fail(RFD_EINVAL, "null argument");
  if (k < 1 || k > kMaxK || k > pl->p.max_channels)
    return fail(RFD_EINVAL, "k must be in [1, min(32, max_channels)]");
  if (ld_mu < k) return fail(RFD_EINVAL, "ld_mu must be >= k");
  if (iters < 0) return fail(RFD_EINVAL, "iters must be >= 0");
  if (!pl->have_G) return fail(RFD_EINVAL, "rfd_features (or rfd_gfi) must run before rfd_barycenter");
  Alpha al{};
  for (int i = 0; i < k; ++i) {
    if (!std::isfinite(alpha[i]) || alpha[i] < 0.0) return fail(RFD_EINVAL, "alpha must be finite and >= 0");
    al.a[i] = (float)alpha[i];
  }
  const int64_t n = pl->n, nk = n * k;
  cudaStream_t st = pl->stream;
  float* buf = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), (size_t)nk * 4 * sizeof(float), st);
  if (e != cudaSuccess) return fail(RFD_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  float *v = buf, *w = buf + nk, *F = buf + 2 * nk, *H = buf + 3 * nk;
  const unsigned bk = (unsigned)((nk + 255) / 256), bp = (unsigned)((n + 255) / 256);
  rfd_status s = RFD_OK;
  bary_init_kernel<<<bk, 256, 0, st>>>(d_area, v, F, d_out, n, k);
  count_launch();
  e = cudaGetLastError();
  for (int it = 0; it < iters && s == RFD_OK && e == cudaSuccess; ++it) {
    s = rfd_integrate(pl, F, k, k, H, k);  // K (a v)
    if (s != RFD_OK) break;
    bary_step1_kernel<<<bk, 256, 0, st>>>(d_mu, ld_mu, d_area, H, w, F, n, k);
    count_launch();
    s = rfd_integrate(pl, F, k, k, H, k);  // K (a w)
    if (s != RFD_OK) break;
    bary_step2_kernel<<<bp, 256, 0, st>>>(d_area, H, v, F, d_out, n, k, al);
    count_launch();
    e = cudaGetLastError();
  }
  if (s == RFD_OK && e != cudaSuccess) s = fail(RFD_ECUDA, std::string("barycenter: ") + cudaGetErrorString(e));
  (void)w;
  cudaFreeAsync(buf, st);
  return s;
}
