// Step a4: G = lambda phi1(lambda M) in FP64 on the device (Sec. 2.4: the
// factor [exp(lambda B^T A) - I](B^T A)^{-1}, which equals lambda phi1(lambda M)
// with phi1(X) = sum_k X^k/(k+1)! whenever M is invertible and stays defined
// when it is not; no inverse is formed).
//
// Method: phi1(X) is the top-right block of exp(Xa), Xa = [[X, I], [0, 0]].
// exp(Xa) is evaluated by scaling and squaring with the diagonal Pade
// approximant r_q(Xa) = (V - U)^{-1} (V + U), U the odd and V the even part of
// the numerator p_q; degree q and scaling s are chosen from ||X||_1 with the
// thresholds theta_q of Higham, "The scaling and squaring method for the matrix
// exponential revisited", SIAM J. Matrix Anal. Appl. 26 (2005), Table 2.3.
//
// Block structure.  Xa^k = [[X^k, X^{k-1}], [0, 0]] (k >= 1), so with
// Sp = sum_{k odd} b_k X^{k-1} (even powers of X only):
//   U = Xa sum_{k odd} b_k Xa^{k-1} = [[X Sp, Sp], [0, 0]],
//   V = sum_{k even} b_k Xa^k       = [[Vp, Vq], [0, b_0 I]],  Vp = sum_{k even} b_k X^k.
// Writing r_q(Xa) = [[E, F], [0, I]], the equations (V - U) r = V + U give
//   (Vp - X Sp) E = Vp + X Sp,      (Vp - X Sp) F = 2 Sp,
// E ~ e^{X}, F ~ phi1(X); Vq is never needed.  The evaluation therefore costs
// exactly the GEMMs of a plain Pade exponential (six for q = 13 with Higham's
// grouping X^6 (b13 X^6 + b11 X^4 + b9 X^2) + ..., four for q = 7) plus one LU
// factorisation; when s = 0 only the m right-hand sides of F are solved.
// The squaring phase uses phi1(2Y) = (e^Y phi1(Y) + phi1(Y))/2, e^{2Y} = (e^Y)^2.
//
// The 1-norm is brought to the host to pick (q, s): one stream
// synchronisation per call.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <vector>
#include "kernels.h"
#include "rfd_phi1.h"

namespace rfd {

namespace {

// Higham (2005), Table 2.3: largest ||X||_1 for which the degree-q diagonal
// Pade approximant meets double-precision backward error.
constexpr int kDegrees[5] = {3, 5, 7, 9, 13};
constexpr double kTheta[5] = {1.495585217958292e-2, 2.539398330063230e-1, 9.504178996162932e-1,
                              2.097847961257068e0, 5.371920351148152e0};

// Coefficients of the diagonal Pade numerator p_q(x) = sum_k b_k x^k,
// b_k = (2q-k)! q! / ((2q)! k! (q-k)!), normalised to b_0 = 1 by the ratio
// b_{k+1}/b_k = (q-k) / ((2q-k)(k+1)); the denominator is p_q(-x).
std::vector<double> pade_coeffs(int q) {
  std::vector<double> b(q + 1);
  b[0] = 1.0;
  for (int k = 0; k < q; ++k) b[k + 1] = b[k] * double(q - k) / (double(2 * q - k) * double(k + 1));
  return b;
}

}  // namespace

size_t phi1_workspace_doubles(int m) { return (size_t)m * m * 18 + (ozaki_workspace_bytes(m, m, m) + 7) / 8; }

int phi1_gemm_count(int q, int s) {
  const int powers = (q == 13) ? 3 : (q - 1) / 2;  // X^2, X^4, ... up to X^{q-1} (X^6 for q = 13)
  return powers + (q == 13 ? 2 : 0) + 1 + (s > 0 ? 2 * s - 1 : 0);
}

rfd_status phi1_fp64(int m, double lambda, const double* d_M, double* d_G, double* work, int* d_ipiv, int* d_info,
                     double* d_scalar, int* d_flag, int* d_err, bool emulated, cudaStream_t st, Phi1Info* info) {
  const size_t mm = (size_t)m * m;
  void* oz_work = work + mm * 18;
  const bool use_oz = emulated && m >= 256 && ozaki_supported(m);  // below m = 256 native FP64 is as fast
  // the m x m x m products: FP64-accurate emulation on the tensor cores, or native FP64
  auto mm3 = [&](double alpha, const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                 cudaStream_t s_) {
    ++info->gemms;
    return use_oz ? dgemm_ozaki(m, m, m, alpha, A, lda, B, ldb, beta, C, ldc, oz_work, d_err, s_)
                  : dgemm(m, m, m, alpha, A, lda, B, ldb, beta, C, ldc, s_);
  };
  *info = Phi1Info{};
  info->emulated = use_oz ? 1 : 0;
  info->degree = 0;
  info->squarings = 0;
  info->norm1 = 0.0;
  info->nonfinite = 0;
#define CK(x)                                \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return RFD_ECUDA; \
  } while (0)
  if (lambda == 0.0) {  // G = 0: out == F exactly
    CK(cudaMemsetAsync(d_G, 0, mm * sizeof(double), st));
    return RFD_OK;
  }
  double* X = work;                  // lambda M / 2^s
  double* Xp[5] = {nullptr, work + mm, work + 2 * mm, work + 3 * mm, work + 4 * mm};  // X^2, X^4, X^6, X^8
  double* T = work + 5 * mm;
  double* Sp = work + 6 * mm;        // odd part's top-right block  = sum_{k odd} b_k X^{k-1}
  double* Up = work + 7 * mm;        // X Sp
  double* Vp = work + 8 * mm;        // sum_{k even} b_k X^k
  double* LU = work + 9 * mm;
  double* RHS = work + 10 * mm;      // m x 2m: [E | F] (s > 0) or m x m: F (s = 0)
  double* Ea = work + 12 * mm;       // squaring phase
  double* Fsq = work + 13 * mm;
  double* Eb = work + 14 * mm;

  CK(dcombine(m, m, X, m, lambda, d_M, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
  CK(dnorm1(m, X, m, d_scalar, st));
  double nrm = 0.0;
  CK(cudaMemcpyAsync(&nrm, d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  info->norm1 = nrm;
  if (!std::isfinite(nrm)) {
    info->nonfinite = 1;
    return RFD_ENUMERIC;
  }
  if (nrm == 0.0) {  // phi1(0) = I
    CK(dcombine(m, m, d_G, m, 0, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, lambda, m, st));
    return RFD_OK;
  }
  // Degree and scaling.  Native path: Higham's cheapest degree (up to 13), LU
  // solve.  Emulated path: degree <= 5, so that the denominator residual
  // R = I - q_q(X) obeys ||R||_1 <= p_q(||X||_1) - 1 <= p_5(theta_5) - 1 < 0.14
  // and q_q(X)^{-1} = prod_j (I + R^(2^j)) converges in five factors: the whole
  // evaluation is then GEMMs, which the tensor-core emulation makes cheap.
  const int top = use_oz ? 1 : 4;  // index of the largest admissible degree
  int q = kDegrees[top], s = 0;
  bool chosen = false;
  for (int i = 0; i < top; ++i)
    if (nrm <= kTheta[i]) {
      q = kDegrees[i];
      chosen = true;
      break;
    }
  if (!chosen) {
    s = std::max(0, (int)std::ceil(std::log2(nrm / kTheta[top])));
    if (s > 1000) {
      info->nonfinite = 1;
      return RFD_ENUMERIC;
    }
  }
  info->degree = q;
  info->squarings = s;
  if (s > 0) CK(dcombine(m, m, X, m, std::ldexp(1.0, -s), X, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
  const std::vector<double> b = pade_coeffs(q);

  // even powers X^2, X^4, ... (X^6 at most for q = 13)
  const int kmax = (q == 13) ? 3 : (q - 1) / 2;
  CK(mm3(1.0, X, m, X, m, 0.0, Xp[1], m, st));
  if (kmax >= 2) CK(mm3(1.0, Xp[1], m, Xp[1], m, 0.0, Xp[2], m, st));
  if (kmax >= 3) CK(mm3(1.0, Xp[2], m, Xp[1], m, 0.0, Xp[3], m, st));
  if (kmax >= 4) CK(mm3(1.0, Xp[2], m, Xp[2], m, 0.0, Xp[4], m, st));

  if (q == 13) {
    // Sp = X^6 (b13 X^6 + b11 X^4 + b9 X^2) + b7 X^6 + b5 X^4 + b3 X^2 + b1 I
    CK(dcombine(m, m, T, m, b[13], Xp[3], b[11], Xp[2], b[9], Xp[1], 0, nullptr, 0.0, m, st));
    CK(dcombine(m, m, Sp, m, b[7], Xp[3], b[5], Xp[2], b[3], Xp[1], 0, nullptr, b[1], m, st));
    CK(mm3(1.0, Xp[3], m, T, m, 1.0, Sp, m, st));
    // Vp = X^6 (b12 X^6 + b10 X^4 + b8 X^2) + b6 X^6 + b4 X^4 + b2 X^2 + b0 I
    CK(dcombine(m, m, T, m, b[12], Xp[3], b[10], Xp[2], b[8], Xp[1], 0, nullptr, 0.0, m, st));
    CK(dcombine(m, m, Vp, m, b[6], Xp[3], b[4], Xp[2], b[2], Xp[1], 0, nullptr, b[0], m, st));
    CK(mm3(1.0, Xp[3], m, T, m, 1.0, Vp, m, st));
  } else {
    double so[4] = {0, 0, 0, 0}, se[4] = {0, 0, 0, 0};
    for (int k = 1; k <= kmax; ++k) {
      so[k - 1] = b[2 * k + 1];  // coefficient of X^{2k} in Sp
      se[k - 1] = b[2 * k];      // coefficient of X^{2k} in Vp
    }
    auto P = [&](int i) -> const double* { return i < kmax ? Xp[i + 1] : nullptr; };
    CK(dcombine(m, m, Sp, m, so[0], P(0), so[1], P(1), so[2], P(2), so[3], P(3), b[1], m, st));
    CK(dcombine(m, m, Vp, m, se[0], P(0), se[1], P(1), se[2], P(2), se[3], P(3), b[0], m, st));
  }
  CK(mm3(1.0, X, m, Sp, m, 0.0, Up, m, st));
  // F ~ phi1(X) from (Vp - Up) F = 2 Sp
  double* F = RHS;
  if (!use_oz) {
    CK(dcombine(m, m, LU, m, 1.0, Vp, -1.0, Up, 0, nullptr, 0, nullptr, 0.0, m, st));
    CK(dcombine(m, m, F, m, 2.0, Sp, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
    CK(dgetrf(m, LU, m, d_ipiv, nullptr, d_info, st));
    CK(dgetrs(m, m, LU, m, d_ipiv, F, m, st));
    info->lu = 1;
  } else {
    // R = I - (Vp - Up);  F = (I + R^(2^(k-1))) ... (I + R^2)(I + R) 2 Sp
    double rho = 0.0, xs = std::ldexp(nrm, -s), pw = 1.0;
    for (int k = 1; k <= q; ++k) rho += b[k] * (pw *= xs);
    // after nfac factors the error is R^(2^nfac) (I - R)^{-1}: stop once rho^(2^nfac)/(1 - rho) <= 2^-56
    int nfac = 1;
    for (double r2 = rho * rho; r2 / (1.0 - rho) > 0x1p-56 && nfac < 8; r2 *= r2) ++nfac;
    double* Pa = T;
    double* Pb = LU;
    double* Fb = RHS + mm;
    CK(dcombine(m, m, Pa, m, -1.0, Vp, 1.0, Up, 0, nullptr, 0, nullptr, 1.0, m, st));
    CK(dcombine(m, m, F, m, 2.0, Sp, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
    for (int j = 0; j < nfac; ++j) {
      CK(cudaMemcpyAsync(Fb, F, mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CK(mm3(1.0, Pa, m, F, m, 1.0, Fb, m, st));  // F <- F + R^(2^j) F
      std::swap(F, Fb);
      if (j + 1 < nfac) {
        CK(mm3(1.0, Pa, m, Pa, m, 0.0, Pb, m, st));  // R^(2^(j+1))
        std::swap(Pa, Pb);
      }
    }
    info->solve_factors = nfac;
  }
  if (s > 0) {
    // squaring phase: E = I + X F (the Pade quantities satisfy it exactly:
    // E - I = (Vp - Up)^{-1} 2 X Sp = X F), then F' = (E F + F)/2, E' = E E
    double* Fa = F;
    double* Fb = (F == RHS) ? Fsq : RHS;
    CK(dcombine(m, m, Ea, m, 0, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 1.0, m, st));
    CK(mm3(1.0, X, m, Fa, m, 1.0, Ea, m, st));
    for (int i = 0; i < s; ++i) {
      CK(dcombine(m, m, Fb, m, 0.5, Fa, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
      CK(mm3(0.5, Ea, m, Fa, m, 1.0, Fb, m, st));
      if (i + 1 < s) CK(mm3(1.0, Ea, m, Ea, m, 0.0, Eb, m, st));  // the last E is not needed
      std::swap(Ea, Eb);
      std::swap(Fa, Fb);
    }
    F = Fa;
  }
  // G = lambda phi1(X)
  CK(dcombine(m, m, d_G, m, lambda, F, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
  CK(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
  CK(dfinite_check(m, m, d_G, m, d_flag, st));
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (flag) {
    info->nonfinite = 1;
    return RFD_ENUMERIC;
  }
  return RFD_OK;
#undef CK
}

}  // namespace rfd
