// Eigenvalues of a cloud's RFD kernel exp(lambda W_hat) from its low-rank
// factors (Sec. 3.3, point-cloud classification by the kernel's k smallest
// eigenvalues; App. E, graph classification by the k largest; the
// factorisation route after Nakatsukasa 2019).
//
// W_hat = A B^T = Phi Omega_b Sigma Omega_b Phi^T, Sigma = diag(sgn r), is
// symmetric of rank <= m.  Its nonzero eigenvalues are those of the m x m
// matrix M = B^T A = P Sigma with P = Omega_b Phi^T Phi Omega_b = M Sigma
// (symmetric positive semidefinite).  With P = L L^T (Cholesky; a column whose
// pivot falls below the rounding level of P is dropped, the semidefinite
// case), eig(P Sigma) = eig(L^T Sigma L): a symmetric m x m matrix, here
// diagonalised by cyclic Jacobi rotations (round-robin ordering, m/2 disjoint
// rotations at a time).  exp(lambda W_hat) then has the eigenvalues
// exp(lambda mu) and, for the N - m directions W_hat annihilates, 1; when
// N < m, the m - N eigenvalues of smallest modulus belong to the rank
// deficiency and are dropped.
//
// One CTA per cloud, all in shared memory.  For an M from the FP32 plain form:
// the Cholesky factor in FP64, the Jacobi iteration in FP32 with its rotations
// accumulated, and each eigenvalue then taken as the FP64 Rayleigh quotient of
// its FP32 eigenvector on the FP64 factor (error second order in the
// eigenvector's, so the FP32 rotations do not limit the eigenvalues).  For an
// M from the BF16 form (good to ~1e-4), FP32 throughout: the Jacobi diagonal
// (~1e-6 of ||H||) is far inside that, and the slow FP64 pipe is not used.
// No device-side waits.
#include <cuda_runtime.h>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>
#include "kernels.h"
#include "rfd_internal.h"
#include "rfd_plan.h"

namespace rfd {

namespace {

constexpr int kEigThreads = 128;
constexpr int kEigMaxM = 128;
static_assert(kEigThreads >= kEigMaxM, "the spectrum ranks take one thread per eigenvalue");
constexpr int kMaxSweeps = 20;
// stop when off(H) <= kOffTol ||H||_F: the eigenvectors are then good to ~1e-5,
// and the FP64 Rayleigh quotients good to ~1e-10 relative (second order)
constexpr float kOffTol = 1e-5f;

struct EigJob {
  const double* M;   // m x m, row-major: M = B^T A
  const double* oa;  // column scales of A (sign of r)
  double lambda;
  int64_t n;
  int32_t m, pad_;
};

// shared memory: L (packed lower triangle; FP64 when refined, else FP32), the
// eigenvalue array, the Jacobi iterate H and (refined) the accumulated
// rotations V (FP32, m x (m+1)), then small arrays
size_t eig_smem_bytes(int m, bool refine) {
  const size_t ld = (size_t)m + 1, tri = (size_t)m * (m + 1) / 2;
  const size_t lbytes = (tri * (refine ? sizeof(double) : sizeof(float)) + 15) & ~size_t(15);
  return lbytes + (size_t)m * 2 * sizeof(double) + (refine ? 2 : 1) * m * ld * sizeof(float) +
         (size_t)(3 * m + 64) * sizeof(float) + (size_t)2 * m * sizeof(int);
}

__device__ float block_sum(float v, float* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// e / d and e % d for 0 <= e < 2^14, 1 <= d <= 2^7 by a multiply-high with ceil(2^32 / d):
// the error e (ceil(2^32/d) - 2^32/d) / 2^32 < 2^-18 stays below the gap 1/d to the next
// integer, so the quotient is exact (the loops below index flat m x m or t x t ranges).
struct FastDiv {
  uint32_t d, magic;
  __device__ explicit FastDiv(int dd) : d((uint32_t)dd), magic(dd > 1 ? 0xFFFFFFFFu / (uint32_t)dd + 1u : 0u) {}
  __device__ int quo(int e) const { return d > 1 ? (int)__umulhi((uint32_t)e, magic) : e; }
};
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i
__device__ __forceinline__ double root(double x) { return sqrt(x); }
__device__ __forceinline__ float root(float x) { return sqrtf(x); }

// All m eigenvalues of the symmetric H (m x m, row stride ld, FP32; overwritten)
// into mu[0..m): Householder reduction to tridiagonal form (m - 2 reflections,
// each a matrix-vector product and a rank-2 update over the CTA),
// then bisection on Sturm counts, one thread per eigenvalue with no barrier.
// Each reflection's norm, v and w come from one warp (shuffle sums), so a
// reflection takes four CTA barriers.  Backward stable in FP32: the
// eigenvalues carry an error of ~m 2^-24 ||H||.
// Scratch: vs, ps (m floats each), dg, e2 (m floats each), red (>= 2 floats).
__device__ void eig_tridiag_bisect(float* H, int ld, int m, double* mu, float* vs, float* ps, float* dg,
                                   float* e2, float* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k + 2 < m; ++k) {
    const int n = m - k - 1;  // the column below the diagonal: rows k + 1 .. m - 1
    if (warp == 0) {  // the reflection: norm, alpha, beta and v, by one warp (no block reduction)
      float ss = 0.f;
      for (int i = lane; i < n; i += 32) {
        const float x = H[(k + 1 + i) * ld + k];
        ss = fmaf(x, x, ss);
      }
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float x0 = H[(k + 1) * ld + k];
      const bool reflect = ss - x0 * x0 > 1e-30f * ss;  // anything below the subdiagonal
      const float alpha = reflect ? (x0 > 0.f ? -sqrtf(ss) : sqrtf(ss)) : x0;
      if (reflect)
        for (int i = lane; i < n; i += 32) vs[i] = H[(k + 1 + i) * ld + k] - (i == 0 ? alpha : 0.f);
      if (lane == 0) {
        red[0] = reflect ? 1.f / (ss - alpha * x0) : 0.f;  // beta = 2 / ||v||^2, v = x - alpha e1
        dg[k] = H[k * ld + k];                              // final since the previous step
        e2[k] = alpha * alpha;
      }
    }
    __syncthreads();
    const float beta = red[0];
    if (beta != 0.f) {
      for (int i = tid; i < n; i += nt) {  // p = beta H' v, H' the trailing block
        const float* row = H + (k + 1 + i) * ld + (k + 1);
        float acc = 0.f;
        for (int j = 0; j < n; ++j) acc = fmaf(row[j], vs[j], acc);
        ps[i] = beta * acc;
      }
      __syncthreads();
      if (warp == 0) {  // w = p - (beta v^T p / 2) v
        float vp = 0.f;
        for (int i = lane; i < n; i += 32) vp = fmaf(vs[i], ps[i], vp);
        for (int o = 16; o > 0; o >>= 1) vp += __shfl_xor_sync(0xffffffffu, vp, o);
        const float kk = 0.5f * beta * vp;
        for (int i = lane; i < n; i += 32) ps[i] = fmaf(-kk, vs[i], ps[i]);
      }
      __syncthreads();
      const FastDiv divn(n);
      for (int e = tid; e < n * n; e += nt) {  // H' -= v w^T + w v^T
        const int i = divn.quo(e), j = e - i * n;
        float* h = H + (k + 1 + i) * ld + (k + 1 + j);
        *h = fmaf(-vs[i], ps[j], fmaf(-ps[i], vs[j], *h));
      }
    }
    __syncthreads();  // the update is complete; red[0] and vs may be rewritten
  }
  if (tid == 0) {
    if (m >= 2) {
      dg[m - 2] = H[(m - 2) * ld + m - 2];
      const float e = H[(m - 1) * ld + m - 2];
      e2[m - 2] = e * e;
    }
    dg[m - 1] = H[(m - 1) * ld + m - 1];
    // Gershgorin bounds of the tridiagonal matrix, in red[0], red[1]
    float lo = 3.0e38f, hi = -3.0e38f;
    for (int i = 0; i < m; ++i) {
      const float r = (i > 0 ? sqrtf(e2[i - 1]) : 0.f) + (i + 1 < m ? sqrtf(e2[i]) : 0.f);
      lo = fminf(lo, dg[i] - r);
      hi = fmaxf(hi, dg[i] + r);
    }
    const float w = fmaxf(fabsf(lo), fabsf(hi));
    red[0] = lo - 1e-6f * w - 1e-30f;
    red[1] = hi + 1e-6f * w + 1e-30f;
  }
  __syncthreads();
  const float lo0 = red[0], hi0 = red[1];
  const float tnorm = fmaxf(fabsf(lo0), fabsf(hi0));
  const float pivmin = 1e-30f * fmaxf(1.f, tnorm);
  // an interval of 2^-24 ||T|| is below the reduction's own error (~m 2^-24 ||H||)
  const float tol = 5.96e-8f * tnorm;
  for (int i = tid; i < m; i += nt) {  // the (i + 1)-th smallest eigenvalue
    float a = lo0, b = hi0;
    for (int it = 0; it < 64 && b - a > tol; ++it) {
      const float x = 0.5f * (a + b);
      if (!(x > a && x < b)) break;  // no representable midpoint left
      int cnt = 0;                   // eigenvalues below x (Sturm sequence of T - x I)
      float q = dg[0] - x;
      if (fabsf(q) < pivmin) q = -pivmin;
      cnt += q < 0.f;
      for (int j = 1; j < m; ++j) {
        q = (dg[j] - x) - __fdividef(e2[j - 1], q);  // |q| >= pivmin, far below 2^126
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.f;
      }
      if (cnt > i)
        b = x;
      else
        a = x;
    }
    mu[i] = 0.5 * ((double)a + (double)b);
  }
  __syncthreads();
}

// REFINE: FP64 Cholesky and FP64 Rayleigh quotients of the FP32 eigenvectors
// (the FP32 plain form's M); otherwise FP32 throughout and the eigenvalues are
// the Jacobi diagonal, ~1e-6 of ||H|| (the BF16 form's M is good to ~1e-4).
template <int MAXM, bool REFINE>
__global__ void __launch_bounds__(kEigThreads) kernel_eigen_kernel(const EigJob* __restrict__ jobs, int k,
                                                                   int largest, float* __restrict__ out) {
  using TL = typename std::conditional<REFINE, double, float>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EigJob jb = jobs[blockIdx.x];
  const int m = jb.m, ld = m + 1, half = m / 2, tid = threadIdx.x, nt = blockDim.x;
  TL* L = reinterpret_cast<TL*>(smem_raw);              // P, then its Cholesky factor (packed lower)
  double* mu = reinterpret_cast<double*>(smem_raw + (((size_t)m * (m + 1) / 2 * sizeof(TL) + 15) & ~size_t(15)));
  float* H = reinterpret_cast<float*>(mu + 2 * m);      // L^T Sigma L, then the Jacobi iterate
  float* V = H + m * ld;                                // accumulated rotations (REFINE only)
  float* sig = REFINE ? V + m * ld : V;                 // Sigma
  float* cs = sig + m;                                  // rotation (c, s, t) of each pair
  float* red = cs + 2 * m;                              // 64 floats of reduction scratch
  int* pq = reinterpret_cast<int*>(red + 64);           // (p, q) of each pair

  // P = M Sigma, symmetrised (M Sigma is symmetric up to rounding), FP64
  for (int i = tid; i < m; i += nt) sig[i] = jb.oa[i] < 0.0 ? -1.f : 1.f;
  const FastDiv divm(m);
  for (int e = tid; e < m * m; e += nt) {
    const int i = divm.quo(e), j = e - i * m;
    if (j > i) continue;
    const double si = jb.oa[i] < 0.0 ? -1.0 : 1.0, sj = jb.oa[j] < 0.0 ? -1.0 : 1.0;
    L[tri(i, j)] = (TL)(0.5 * (jb.M[(size_t)i * m + j] * sj + jb.M[(size_t)j * m + i] * si));
  }
  __syncthreads();
  TL dmax = 0;
  for (int i = 0; i < m; ++i) dmax = max(dmax, L[tri(i, i)]);
  const TL tol = dmax * (TL)m * (TL)(REFINE ? 4e-16 : 2.4e-7);

  // Cholesky P = L L^T, right-looking; a pivot <= tol drops its column
  for (int j = 0; j < m; ++j) {
    const TL d = L[tri(j, j)];
    const TL piv = d > tol ? root(d) : (TL)0;
    __syncthreads();
    if (tid == 0) L[tri(j, j)] = piv;
    const TL inv = piv > (TL)0 ? (TL)1 / piv : (TL)0;
    for (int i = j + 1 + tid; i < m; i += nt) L[tri(i, j)] *= inv;
    __syncthreads();
    const int t = m - j - 1;
    const FastDiv divt(t > 0 ? t : 1);
    for (int e = tid; e < t * t; e += nt) {
      const int q = divt.quo(e), i = j + 1 + q, l = j + 1 + (e - q * t);
      if (l <= i) L[tri(i, l)] -= L[tri(i, j)] * L[tri(l, j)];
    }
    __syncthreads();
  }

  // H = L^T Sigma L in FP32 (refined: it only seeds the FP32 iteration, the
  // eigenvalues come from the FP64 factor; an FP32 copy of L in V's space first)
  const float* Lf = reinterpret_cast<const float*>(L);
  if constexpr (REFINE) {
    for (int e = tid; e < m * m; e += nt) {
      const int i = divm.quo(e), j = e - i * m;
      V[i * ld + j] = j <= i ? (float)L[tri(i, j)] : 0.f;
    }
    __syncthreads();
  }
  for (int e = tid; e < m * m; e += nt) {
    const int a = divm.quo(e), b = e - a * m;
    if (a > b) continue;
    float s = 0.f;
    if constexpr (REFINE)
      for (int i = b; i < m; ++i) s = fmaf(V[i * ld + a] * sig[i], V[i * ld + b], s);
    else
      for (int i = b, ia = tri(b, a), ib = tri(b, b); i < m; ia += i + 1, ib += i + 1, ++i)
        s = fmaf(Lf[ia] * sig[i], Lf[ib], s);
    H[a * ld + b] = s;
    H[b * ld + a] = s;
  }
  __syncthreads();
  if constexpr (!REFINE) {  // eigenvalues only: tridiagonal form and bisection
    eig_tridiag_bisect(H, ld, m, mu, cs, cs + m, reinterpret_cast<float*>(pq), reinterpret_cast<float*>(pq) + m, red);
  } else {
  if constexpr (REFINE) {
    for (int e = tid; e < m * m; e += nt) V[(e / m) * ld + e % m] = (e / m) == (e % m) ? 1.f : 0.f;
    __syncthreads();
  }

  // cyclic Jacobi in FP32, round-robin pairs: round r pairs (r, m-1) and
  // ((r + q) mod (m-1), (r - q) mod (m-1)) for q = 1 .. m/2 - 1.  The m/2
  // rotations of a round are disjoint, so H <- J^T H J splits into 2 x 2
  // blocks (pair a rows, pair b columns), each read and written by one thread
  // (the block of pairs (b, a) is the transpose); V <- V J likewise by rows.
  float fro = 0.f;
  for (int e = tid; e < m * m; e += nt) fro += H[(e / m) * ld + e % m] * H[(e / m) * ld + e % m];
  fro = block_sum(fro, red);
  // this thread's 2 x 2 blocks (a <= b, row-major over the upper triangle of
  // pair blocks), decoded once: (a << 16) | b, or -1
  const int nblk = half * (half + 1) / 2;
  constexpr int kBlk = ((MAXM / 2) * (MAXM / 2 + 1) / 2 + kEigThreads - 1) / kEigThreads;
  int blk[kBlk];
#pragma unroll
  for (int u = 0; u < kBlk; ++u) {
    const int e = tid + u * nt;
    blk[u] = -1;
    if (e < nblk) {
      int a = 0, rem = e;
      while (rem >= half - a) {
        rem -= half - a;
        ++a;
      }
      blk[u] = (a << 16) | (a + rem);
    }
  }
  // V <- V J: a fixed pair per thread, rows strided
  const int vgroups = nt / max(half, 1), vq = tid % max(half, 1), vi0 = tid / max(half, 1);
  for (int sweep = 0; sweep < kMaxSweeps && m > 1; ++sweep) {
    float off = 0.f;
    for (int e = tid; e < m * m; e += nt) {
      const int a = divm.quo(e), b = e - a * m;
      if (a != b) off += H[a * ld + b] * H[a * ld + b];
    }
    off = block_sum(off, red);
    if (off <= kOffTol * kOffTol * fro) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int q = tid; q < half; q += nt) {
        int p0, p1;
        if (q == 0) {
          p0 = r;
          p1 = m - 1;
        } else {
          p0 = (r + q) % (m - 1);
          p1 = (r - q + m - 1) % (m - 1);
        }
        const int p = min(p0, p1), qq = max(p0, p1);
        const float hpq = H[p * ld + qq];
        float c = 1.f, s = 0.f, t = 0.f;
        if (fabsf(hpq) > 1e-30f) {
          const float tau = (H[qq * ld + qq] - H[p * ld + p]) / (2.f * hpq);
          t = fabsf(tau) > 1e18f ? 0.5f / tau : copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
          c = rsqrtf(fmaf(t, t, 1.f));
          s = t * c;
        }
        pq[2 * q] = p;
        pq[2 * q + 1] = qq;
        cs[3 * q] = c;
        cs[3 * q + 1] = s;
        cs[3 * q + 2] = t;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kBlk; ++u) {
        if (blk[u] < 0) continue;
        const int a = blk[u] >> 16, b = blk[u] & 0xffff;
        const int pa = pq[2 * a], qa = pq[2 * a + 1], pb = pq[2 * b], qb = pq[2 * b + 1];
        const float ca = cs[3 * a], sa = cs[3 * a + 1];
        const float h00 = H[pa * ld + pb], h01 = H[pa * ld + qb], h10 = H[qa * ld + pb], h11 = H[qa * ld + qb];
        if (a == b) {
          const float ta = cs[3 * a + 2];
          H[pa * ld + pa] = h00 - ta * h01;
          H[qa * ld + qa] = h11 + ta * h01;
          H[pa * ld + qa] = 0.f;
          H[qa * ld + pa] = 0.f;
        } else {
          const float cb = cs[3 * b], sb = cs[3 * b + 1];
          const float x00 = ca * h00 - sa * h10, x01 = ca * h01 - sa * h11;
          const float x10 = sa * h00 + ca * h10, x11 = sa * h01 + ca * h11;
          const float y00 = cb * x00 - sb * x01, y01 = sb * x00 + cb * x01;
          const float y10 = cb * x10 - sb * x11, y11 = sb * x10 + cb * x11;
          H[pa * ld + pb] = y00;
          H[pa * ld + qb] = y01;
          H[qa * ld + pb] = y10;
          H[qa * ld + qb] = y11;
          H[pb * ld + pa] = y00;
          H[qb * ld + pa] = y01;
          H[pb * ld + qa] = y10;
          H[qb * ld + qa] = y11;
        }
      }
      if (REFINE && vi0 < vgroups) {
        const int p = pq[2 * vq], qq = pq[2 * vq + 1];
        const float c = cs[3 * vq], s = cs[3 * vq + 1];
        for (int i = vi0; i < m; i += vgroups) {
          const float vp = V[i * ld + p], vv = V[i * ld + qq];
          V[i * ld + p] = c * vp - s * vv;
          V[i * ld + qq] = s * vp + c * vv;
        }
      }
      __syncthreads();
    }
  }

  {
  // the eigenvectors to FP64, one padded row per vector (V64[a][j] = V[j][a]),
  // over the space of H and V: rows a < m/2 land in H's space; the columns
  // a >= m/2 of V are read into registers before their rows overwrite V's
  double* V64 = reinterpret_cast<double*>(H);
  for (int e = tid; e < half * m; e += nt) {
    const int a = e / m, j = e % m;
    V64[a * ld + j] = (double)V[j * ld + a];
  }
  constexpr int kHold = MAXM * MAXM / 2 / kEigThreads;
  float hold[kHold];
#pragma unroll
  for (int u = 0; u < kHold; ++u) {
    const int e = tid + u * nt;
    hold[u] = e < half * m ? V[(e % m) * ld + half + e / m] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kHold; ++u) {
    const int e = tid + u * nt;
    if (e < half * m) V64[(half + e / m) * ld + e % m] = (double)hold[u];
  }
  __syncthreads();

  // FP64 Rayleigh quotients of the FP32 eigenvectors on the FP64 factor:
  // mu_a = (L v)^T Sigma (L v) / v^T v, second order in the eigenvector error;
  // g = nt / m threads per vector (adjacent lanes), rows i dealt round-robin
  {
    const int g = min(8, max(1, nt / m));
    const int a = tid / g, sub = tid % g;
    double num = 0.0, den = 0.0;
    if (a < m) {
      const double* v = V64 + (size_t)a * ld;
      for (int i = sub; i < m; i += g) {
        double w = 0.0;
        for (int j = 0; j <= i; ++j) w = fma(L[tri(i, j)], v[j], w);
        num = fma((double)sig[i] * w, w, num);
        den = fma(v[i], v[i], den);
      }
    }
    for (int o = 1; o < g; o <<= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (a < m && sub == 0) mu[a] = den > 0.0 ? num / den : 0.0;
  }
  __syncthreads();

  }
  }  // REFINE

  // the spectrum of exp(lambda W_hat): drop the rank deficiency, sort, merge the
  // ones -- all by ranks (thread i counts the entries before entry i), no serial step
  const int drop = jb.n < m ? m - (int)jb.n : 0;  // the m - n of smallest modulus go (rank deficiency)
  double kap = 0.0;
  bool keep = false;
  if (tid < m) {
    const double x = mu[tid];
    int r = 0;
    for (int j = 0; j < m; ++j) {
      const double y = fabs(mu[j]);
      r += (y < fabs(x)) || (y == fabs(x) && j < tid);
    }
    keep = r >= drop;
    kap = REFINE ? exp(jb.lambda * x) : (double)expf((float)(jb.lambda * x));
  }
  __syncthreads();
  if (tid < m) mu[tid] = keep ? kap : INFINITY;  // dropped entries sort last and are never read
  __syncthreads();
  if (tid < m && keep) {
    int r = 0;
    for (int j = 0; j < m; ++j) r += (mu[j] < kap) || (mu[j] == kap && j < tid);
    mu[m + r] = kap;
  }
  const int cnt = m - drop;
  const int below = __syncthreads_count(tid < m && keep && kap < 1.0);
  const int above = __syncthreads_count(tid < m && keep && kap > 1.0);
  mu += m;  // the sorted kernel eigenvalues
  const int64_t ones = jb.n > m ? jb.n - m : 0;
  float* o = out + (size_t)blockIdx.x * k;
  for (int j = tid; j < k; j += nt) {
    double v;
    if (!largest) {  // ascending: kappa < 1, then the ones (with any kappa == 1), then kappa > 1
      if (j < below) v = mu[j];
      else if ((int64_t)j < (int64_t)(cnt - above) + ones) v = 1.0;
      else v = mu[(int64_t)j - ones];
    } else {  // descending
      if (j < above) v = mu[cnt - 1 - j];
      else if ((int64_t)j < (int64_t)(cnt - below) + ones) v = 1.0;
      else v = mu[cnt - 1 - ((int64_t)j - ones)];
    }
    o[j] = (float)v;
  }
}

template <int MAXM, bool REFINE>
rfd_status launch_eigen_t(const EigJob* d_jobs, int count, int max_m, int k, int largest, float* d_out,
                          cudaStream_t st) {
  const size_t smem = eig_smem_bytes(max_m, REFINE);
  cudaError_t e = cudaFuncSetAttribute(kernel_eigen_kernel<MAXM, REFINE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return fail(RFD_ECUDA, std::string("eigen attribute: ") + cudaGetErrorString(e));
  kernel_eigen_kernel<MAXM, REFINE><<<count, kEigThreads, smem, st>>>(d_jobs, k, largest, d_out);
  count_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? RFD_OK : fail(RFD_ECUDA, std::string("eigen launch: ") + cudaGetErrorString(e));
}

rfd_status launch_eigen(const EigJob* d_jobs, int count, int max_m, int k, int largest, bool refine, float* d_out,
                        cudaStream_t st) {
  if (max_m <= 64)
    return refine ? launch_eigen_t<64, true>(d_jobs, count, max_m, k, largest, d_out, st)
                  : launch_eigen_t<64, false>(d_jobs, count, max_m, k, largest, d_out, st);
  return refine ? launch_eigen_t<kEigMaxM, true>(d_jobs, count, max_m, k, largest, d_out, st)
                : launch_eigen_t<kEigMaxM, false>(d_jobs, count, max_m, k, largest, d_out, st);
}

rfd_status check_eigen_plan(const rfd_plan_s* pl, int k, int idx) {
  const std::string who = idx < 0 ? std::string() : "cloud " + std::to_string(idx) + ": ";
  if (pl->m > kEigMaxM) return fail(RFD_EINVAL, who + "m must be <= 128 for the kernel eigenvalues");
  if ((int64_t)k > pl->n) return fail(RFD_EINVAL, who + "k must be <= N");
  return RFD_OK;
}

EigJob job_of(const rfd_plan_s* pl) { return EigJob{pl->d_M, pl->d_oa, pl->p.lambda, pl->n, pl->m, 0}; }

// runs the kernel on host-built jobs (a temporary device table on the stream)
rfd_status run_jobs(const std::vector<EigJob>& jobs, int max_m, int k, int largest, bool refine, float* d_out,
                    cudaStream_t st) {
  EigJob* d_jobs = nullptr;
  const size_t bytes = jobs.size() * sizeof(EigJob);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_jobs), bytes, st);
  if (e != cudaSuccess) return fail(RFD_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(d_jobs, jobs.data(), bytes, cudaMemcpyHostToDevice, st);
  rfd_status s = e == cudaSuccess ? launch_eigen(d_jobs, (int)jobs.size(), max_m, k, largest, refine, d_out, st)
                                  : fail(RFD_ECUDA, std::string("job upload: ") + cudaGetErrorString(e));
  cudaFreeAsync(d_jobs, st);  // a pageable upload is staged before cudaMemcpyAsync returns
  return s;
}

}  // namespace

rfd_status batch_eigenvalues(rfd_plan_s* const* plans, int count, int k, int largest, float* d_out, cudaStream_t st,
                             Timing* tm) {
  std::vector<EigJob> jobs((size_t)count);
  int max_m = 2;
  bool refine = false;  // FP64 refinement when some cloud's M came from the FP32 plain form
  for (int i = 0; i < count; ++i) {
    jobs[i] = job_of(plans[i]);
    max_m = std::max(max_m, plans[i]->m);
    refine = refine || !plans[i]->bf16;
  }
  StepScope sc(tm, st, RFD_STEP_EIGEN);
  return run_jobs(jobs, max_m, k, largest, refine, d_out, st);
}

rfd_status check_eigen_args(rfd_plan_s* const* plans, int count, int k) {
  if (k < 1) return fail(RFD_EINVAL, "k must be >= 1");
  for (int i = 0; i < count; ++i) {
    rfd_status s = check_eigen_plan(plans[i], k, count > 1 ? i : -1);
    if (s != RFD_OK) return s;
  }
  return RFD_OK;
}

}  // namespace rfd

using namespace rfd;

extern "C" rfd_status rfd_eigenvalues(rfd_plan_t pl, int32_t k, int32_t largest, float* d_out) {
  if (!pl || !d_out) return fail(RFD_EINVAL, "null plan or output");
  if (largest != 0 && largest != 1) return fail(RFD_EINVAL, "largest must be 0 or 1");
  if (!pl->have_G) return fail(RFD_EINVAL, "rfd_features (or rfd_gfi) must run before rfd_eigenvalues");
  rfd_plan_s* one = pl;
  rfd_status s = check_eigen_args(&one, 1, k);
  if (s != RFD_OK) return s;
  return batch_eigenvalues(&one, 1, k, largest, d_out, pl->stream, nullptr);
}
