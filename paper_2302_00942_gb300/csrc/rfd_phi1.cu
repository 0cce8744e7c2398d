// Step a4: G = lambda phi1(lambda M) in FP64 on the device (Sec. 2.4: the
// factor [exp(lambda B^T A) - I](B^T A)^{-1}, which equals lambda phi1(lambda M)
// with phi1(X) = sum_k X^k/(k+1)! whenever M is invertible and stays defined
// when it is not; no inverse is formed).
//
// Method: phi1(X) is the top-right block of exp(Xa), Xa = [[X, I], [0, 0]].
// exp(Xa) is evaluated by scaling and squaring with a diagonal Pade
// approximant r_q = q_q(Xa)^{-1} p_q(Xa), degree q and scaling s chosen from
// ||X||_1 with the thresholds theta_q of Higham, "The scaling and squaring
// method for the matrix exponential revisited", SIAM J. Matrix Anal. Appl. 26
// (2005), Table 2.3 (the backward-error bounds of the double-precision Pade
// approximants).  Every matrix met in the evaluation is block upper triangular
// [[P, Q], [0, a I]], so products cost two m x m GEMMs instead of eight:
//   [[P1, Q1], [0, a1]] [[P2, Q2], [0, a2]] = [[P1 P2, P1 Q2 + a2 Q1], [0, a1 a2]].
// The Pade denominator is solved with an LU factorisation (partial pivoting):
//   (V - U) [E | F] = [V_p + U_p | 2 U_q]  gives  E ~ e^{X/2^s}, F ~ phi1(X/2^s).
// The squaring phase uses phi1(2Y) = (e^Y phi1(Y) + phi1(Y))/2 and
// e^{2Y} = (e^Y)^2.
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

size_t phi1_workspace_doubles(int m) { return (size_t)m * m * 24; }

rfd_status phi1_fp64(int m, double lambda, const double* d_M, double* d_G, double* work, int* d_ipiv, int* d_info,
                     double* d_scalar, int* d_flag, cudaStream_t st, Phi1Info* info) {
  const size_t mm = (size_t)m * m;
  info->degree = 0;
  info->squarings = 0;
  info->norm1 = 0.0;
  info->nonfinite = 0;
#define CK(x)                                      \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) return RFD_ECUDA;       \
  } while (0)
  if (lambda == 0.0) {  // G = 0: out == F exactly
    CK(cudaMemsetAsync(d_G, 0, mm * sizeof(double), st));
    return RFD_OK;
  }
  double* X = work;             // lambda M / 2^s
  double* P[5];                 // P[k]: X^{2k}   (k = 1..4)
  double* Q[5];                 // Q[k]: X^{2k-1} (top-right block of Xa^{2k})
  for (int k = 1; k <= 4; ++k) {
    P[k] = work + mm * (2 * k - 1);
    Q[k] = work + mm * (2 * k);
  }
  double* Tp = work + mm * 9;
  double* Tq = work + mm * 10;
  double* Wp = work + mm * 11;
  double* Wq = work + mm * 12;
  double* Up = work + mm * 13;
  double* Uq = work + mm * 14;
  double* Vp = work + mm * 15;
  double* Vq = work + mm * 16;
  double* LU = work + mm * 17;
  double* RHS = work + mm * 18;   // m x 2m: [E | F] after the solve
  double* E2 = work + mm * 20;
  double* F2 = work + mm * 21;
  double* Tmp = work + mm * 22;

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
  int q = 13, s = 0;
  bool chosen = false;
  for (int i = 0; i < 4; ++i)
    if (nrm <= kTheta[i]) {
      q = kDegrees[i];
      chosen = true;
      break;
    }
  if (!chosen) {
    q = 13;
    s = std::max(0, (int)std::ceil(std::log2(nrm / kTheta[4])));
    if (s > 1000) {
      info->nonfinite = 1;
      return RFD_ENUMERIC;
    }
  }
  info->degree = q;
  info->squarings = s;
  if (s > 0) CK(dcombine(m, m, X, m, std::ldexp(1.0, -s), X, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
  const std::vector<double> b = pade_coeffs(q);

  // even powers of Xa: [[X^{2k}, X^{2k-1}], [0, 0]]
  const int kmax = (q == 13) ? 3 : (q - 1) / 2;
  CK(dgemm(m, m, m, 1.0, X, m, X, m, 0.0, P[1], m, st));
  CK(cudaMemcpyAsync(Q[1], X, mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (kmax >= 2) {
    CK(dgemm(m, m, m, 1.0, P[1], m, P[1], m, 0.0, P[2], m, st));
    CK(dgemm(m, m, m, 1.0, P[1], m, Q[1], m, 0.0, Q[2], m, st));
  }
  if (kmax >= 3) {
    CK(dgemm(m, m, m, 1.0, P[2], m, P[1], m, 0.0, P[3], m, st));
    CK(dgemm(m, m, m, 1.0, P[2], m, Q[1], m, 0.0, Q[3], m, st));
  }
  if (kmax >= 4) {
    CK(dgemm(m, m, m, 1.0, P[2], m, P[2], m, 0.0, P[4], m, st));
    CK(dgemm(m, m, m, 1.0, P[2], m, Q[2], m, 0.0, Q[4], m, st));
  }

  if (q == 13) {
    // W = Xa^6 (b13 Xa^6 + b11 Xa^4 + b9 Xa^2) + b7 Xa^6 + b5 Xa^4 + b3 Xa^2 + b1 I
    CK(dcombine(m, m, Tp, m, b[13], P[3], b[11], P[2], b[9], P[1], 0, nullptr, 0.0, m, st));
    CK(dcombine(m, m, Tq, m, b[13], Q[3], b[11], Q[2], b[9], Q[1], 0, nullptr, 0.0, m, st));
    CK(dcombine(m, m, Wp, m, b[7], P[3], b[5], P[2], b[3], P[1], 0, nullptr, b[1], m, st));
    CK(dcombine(m, m, Wq, m, b[7], Q[3], b[5], Q[2], b[3], Q[1], 0, nullptr, 0.0, m, st));
    CK(dgemm(m, m, m, 1.0, P[3], m, Tp, m, 1.0, Wp, m, st));
    CK(dgemm(m, m, m, 1.0, P[3], m, Tq, m, 1.0, Wq, m, st));
    // U = Xa W = [[X Wp, X Wq + b1 I], [0, 0]]
    CK(dgemm(m, m, m, 1.0, X, m, Wp, m, 0.0, Up, m, st));
    CK(dcombine(m, m, Uq, m, 0, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, b[1], m, st));
    CK(dgemm(m, m, m, 1.0, X, m, Wq, m, 1.0, Uq, m, st));
    // V = Xa^6 (b12 Xa^6 + b10 Xa^4 + b8 Xa^2) + b6 Xa^6 + b4 Xa^4 + b2 Xa^2 + b0 I
    CK(dcombine(m, m, Tp, m, b[12], P[3], b[10], P[2], b[8], P[1], 0, nullptr, 0.0, m, st));
    CK(dcombine(m, m, Tq, m, b[12], Q[3], b[10], Q[2], b[8], Q[1], 0, nullptr, 0.0, m, st));
    CK(dcombine(m, m, Vp, m, b[6], P[3], b[4], P[2], b[2], P[1], 0, nullptr, b[0], m, st));
    CK(dcombine(m, m, Vq, m, b[6], Q[3], b[4], Q[2], b[2], Q[1], 0, nullptr, 0.0, m, st));
    CK(dgemm(m, m, m, 1.0, P[3], m, Tp, m, 1.0, Vp, m, st));
    CK(dgemm(m, m, m, 1.0, P[3], m, Tq, m, 1.0, Vq, m, st));
  } else {
    // S = sum_{k odd} b_k Xa^{k-1} = [[Sp, Sq], [0, b1 I]];  U = Xa S = [[X Sp, X Sq + b1 I], [0, 0]]
    // V = sum_{k even} b_k Xa^k  = [[Vp, Vq], [0, b0 I]]
    const double* Pk[4] = {P[1], P[2], P[3], P[4]};
    const double* Qk[4] = {Q[1], Q[2], Q[3], Q[4]};
    double so[4] = {0, 0, 0, 0}, se[4] = {0, 0, 0, 0};
    for (int k = 1; k <= kmax; ++k) {
      so[k - 1] = b[2 * k + 1];
      se[k - 1] = b[2 * k];
    }
    auto Pn = [&](int i) { return i < kmax ? Pk[i] : nullptr; };
    auto Qn = [&](int i) { return i < kmax ? Qk[i] : nullptr; };
    CK(dcombine(m, m, Wp, m, so[0], Pn(0), so[1], Pn(1), so[2], Pn(2), so[3], Pn(3), b[1], m, st));
    CK(dcombine(m, m, Wq, m, so[0], Qn(0), so[1], Qn(1), so[2], Qn(2), so[3], Qn(3), 0.0, m, st));
    CK(dgemm(m, m, m, 1.0, X, m, Wp, m, 0.0, Up, m, st));
    CK(dcombine(m, m, Uq, m, 0, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, b[1], m, st));
    CK(dgemm(m, m, m, 1.0, X, m, Wq, m, 1.0, Uq, m, st));
    CK(dcombine(m, m, Vp, m, se[0], Pn(0), se[1], Pn(1), se[2], Pn(2), se[3], Pn(3), b[0], m, st));
    CK(dcombine(m, m, Vq, m, se[0], Qn(0), se[1], Qn(1), se[2], Qn(2), se[3], Qn(3), 0.0, m, st));
  }
  // (V - U) [E | F] = [Vp + Up | 2 Uq]
  CK(dcombine(m, m, LU, m, 1.0, Vp, -1.0, Up, 0, nullptr, 0, nullptr, 0.0, m, st));
  CK(dcombine(m, m, RHS, 2 * m, 1.0, Vp, 1.0, Up, 0, nullptr, 0, nullptr, 0.0, m, st));
  CK(dcombine(m, m, RHS + m, 2 * m, 2.0, Uq, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
  CK(dgetrf(m, LU, m, d_ipiv, nullptr, d_info, st));
  CK(dgetrs(m, 2 * m, LU, m, d_ipiv, RHS, 2 * m, st));
  // squaring phase on [E | F]: E at RHS[:, :m], F at RHS[:, m:] (leading dimension 2m);
  // ping-pong between (Ea, Fa) and (Eb, Fb) with leading dimension m.
  const double* F = RHS + m;
  int ldf = 2 * m;
  if (s > 0) {
    double* Ea = E2;
    double* Fa = F2;
    double* Eb = Tmp;
    double* Fb = work + mm * 23;
    CK(dcombine(m, m, Ea, m, 1.0, RHS, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, 2 * m, st));
    CK(dcombine(m, m, Fa, m, 1.0, RHS + m, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, 2 * m, st));
    for (int i = 0; i < s; ++i) {
      // F' = (E F + F)/2 ; E' = E E
      CK(dcombine(m, m, Fb, m, 0.5, Fa, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, m, st));
      CK(dgemm(m, m, m, 0.5, Ea, m, Fa, m, 1.0, Fb, m, st));
      CK(dgemm(m, m, m, 1.0, Ea, m, Ea, m, 0.0, Eb, m, st));
      std::swap(Ea, Eb);
      std::swap(Fa, Fb);
    }
    F = Fa;
    ldf = m;
  }
  // G = lambda phi1(X)
  CK(dcombine(m, m, d_G, m, lambda, F, 0, nullptr, 0, nullptr, 0, nullptr, 0.0, ldf, st));
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
