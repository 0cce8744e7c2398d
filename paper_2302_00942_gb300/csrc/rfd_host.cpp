// Step a1 of the RFD path on the host, in FP64 (Sec. 2.4): the random
// frequencies w_j ~ P and the importance weights r_j = tau(w_j)/p(w_j).
//
// P is a per-coordinate Gaussian N(0, sigma^2) truncated to [-R, R] (the
// "(truncated) Gaussian" of Sec. 2.4), sampled by rejection from the uniform
// distribution on [-R, R] with acceptance probability exp(-(w/sigma)^2/2):
// only +, *, / and one exp comparison per try, so two IEEE-754 implementations
// of this stream agree bit for bit except when u2 falls within an ulp of the
// acceptance threshold.
//
// tau is the Fourier transform of the eps-NN threshold function f with the
// 2 pi convention of Sec. 2.4 (f(z) = int exp(2 pi i w.z) tau(w) dw):
//  - the L-infinity cube 1[||z||_inf <= eps]:
//    tau(w) = prod_d sin(2 pi eps w_d) / (pi w_d), 2 eps at w_d = 0;
//  - the L2 ball 1[||z||_2 <= eps] (the Bessel-function case of Sec. 2.4):
//    tau(w) = int_{|z| <= eps} cos(2 pi w.z) dz = 4 pi (sin x - x cos x) / q^3,
//    q = 2 pi |w|, x = q eps (4 pi eps^3 / 3 at w = 0; a series below x = 0.1,
//    where sin x - x cos x cancels);
//  - the distance-weighted cube ||z||_1 1[||z||_inf <= eps]: the transform of
//    |z_d| 1[|z_d| <= eps] times the sincs of the other coordinates, summed
//    over d; int_{-eps}^{eps} |z| cos(2 pi w z) dz = 2 eps^2 (sin x / x +
//    (cos x - 1) / x^2), x = 2 pi eps w (a series below x = 0.1).
//
// This file must be compiled without floating-point contraction
// (-ffp-contract=off) so that R (2 u1 - 1) is two rounded operations.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include "rfd_internal.h"

namespace rfd {

namespace {

thread_local std::string g_last_error;

// SplitMix64 (Steele, Lea, Flood 2014): a Weyl sequence with increment
// 0x9E3779B97F4A7C15 followed by a 64-bit mixing finaliser.
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // 53 random bits centred in their cell: a double strictly inside (0, 1)
  double uniform() { return (static_cast<double>(next() >> 11) + 0.5) * 0x1.0p-53; }
};

constexpr int kMaxTries = 1 << 20;
constexpr double kPi = 3.14159265358979323846;

double sinc_cube(double w, double eps) {  // one coordinate of tau
  if (w == 0.0) return 2.0 * eps;
  return std::sin(2.0 * kPi * eps * w) / (kPi * w);
}

double abs_cube(double w, double eps) {  // int_{-eps}^{eps} |z| cos(2 pi w z) dz
  const double x = 2.0 * kPi * eps * w;
  double g;
  if (std::fabs(x) < 0.1) {
    // sum_n (-1)^n x^(2n) (2n + 1) / (2n + 2)!
    const double x2 = x * x;
    g = 0.5 - x2 * (1.0 / 8.0 - x2 * (1.0 / 144.0 - x2 * (1.0 / 5760.0 - x2 * (1.0 / 403200.0 - x2 / 43545600.0))));
  } else {
    g = std::sin(x) / x + (std::cos(x) - 1.0) / (x * x);
  }
  return 2.0 * eps * eps * g;
}

double tau_ball(const double (&w)[3], double eps) {
  const double q = 2.0 * kPi * std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  const double x = q * eps;
  if (x < 0.1) {
    // (sin x - x cos x) / x^3 = sum_k (-1)^k x^(2k) / ((2k+1)! (2k+3)) ... written out to x^10
    const double x2 = x * x;
    const double s = 1.0 / 3.0 - x2 * (1.0 / 30.0 - x2 * (1.0 / 840.0 - x2 * (1.0 / 45360.0 -
                     x2 * (1.0 / 3991680.0 - x2 / 518918400.0))));
    return 4.0 * kPi * eps * eps * eps * s;
  }
  return 4.0 * kPi * (std::sin(x) - x * std::cos(x)) / (q * q * q);
}

// f = 1[||z||_1 <= eps]: the octahedron is the union of the 8 simplices
// conv(0, s_1 eps e_1, s_2 eps e_2, s_3 eps e_3), s in {-1, 1}^3.  Over a simplex
// conv(0, v_1, v_2, v_3), the integral of exp(u . z) is 3! vol times the
// divided difference of exp at the nodes 0, u . v_1, u . v_2, u . v_3 (the
// exponential-simplex integral); here u = -2 pi i w (the transform's 2 pi
// convention) and each simplex has volume eps^3 / 6, and the 8 terms sum to a
// real number.  The divided difference of exp at y_0..y_3 is the top-right
// entry of exp(J), J the upper bidiagonal matrix with y on the diagonal and
// ones above it (Opitz 1964); exp(J) by scaling and squaring of its Taylor
// polynomial (degree 18 at norm <= 1), which stays accurate where the power
// series of the divided difference cancels (nodes of modulus up to tens).
using cplx = std::complex<double>;
struct Tri4 {
  cplx a[4][4];  // upper triangular
};
Tri4 mul(const Tri4& x, const Tri4& y) {
  Tri4 z{};
  for (int i = 0; i < 4; ++i)
    for (int j = i; j < 4; ++j) {
      cplx t = 0.0;
      for (int k = i; k <= j; ++k) t += x.a[i][k] * y.a[k][j];
      z.a[i][j] = t;
    }
  return z;
}
cplx divided_difference_exp(const cplx (&y)[4]) {
  double nrm = 1.0;  // the superdiagonal
  for (int i = 0; i < 4; ++i) nrm = std::max(nrm, std::abs(y[i]) + 1.0);
  int s = 0;
  while (nrm > 1.0) {
    nrm *= 0.5;
    ++s;
  }
  const double scale = std::ldexp(1.0, -s);
  Tri4 A{};
  for (int i = 0; i < 4; ++i) {
    A.a[i][i] = y[i] * scale;
    if (i < 3) A.a[i][i + 1] = scale;
  }
  Tri4 E{}, P{};
  for (int i = 0; i < 4; ++i) E.a[i][i] = P.a[i][i] = 1.0;
  for (int k = 1; k <= 18; ++k) {  // E = sum_k A^k / k!
    P = mul(P, A);
    for (int i = 0; i < 4; ++i)
      for (int j = i; j < 4; ++j) P.a[i][j] /= (double)k;
    for (int i = 0; i < 4; ++i)
      for (int j = i; j < 4; ++j) E.a[i][j] += P.a[i][j];
  }
  for (int k = 0; k < s; ++k) E = mul(E, E);
  return E.a[0][3];
}
double tau_l1_ball(const double (&w)[3], double eps) {
  double total = 0.0;
  for (int s = 0; s < 8; ++s) {
    cplx y[4];
    y[0] = 0.0;
    for (int d = 0; d < 3; ++d) y[d + 1] = cplx(0.0, ((s >> d) & 1 ? 2.0 : -2.0) * kPi * eps * w[d]);
    total += divided_difference_exp(y).real();
  }
  return eps * eps * eps * total;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
rfd_status fail(rfd_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
const char* last_error_cstr() { return g_last_error.c_str(); }

double default_sigma(double eps) { return 1.0 / (2.0 * eps); }
double default_radius(double eps) { return 1.0 / eps; }

rfd_status sample_frequencies_host(int m, double eps, uint64_t seed, double sigma,
                                   double radius, int kernel, double* omega, double* r) {
  if (m < 2 || (m & 1)) return fail(RFD_EINVAL, "m must be even and >= 2");
  if (kernel != RFD_KERNEL_CUBE && kernel != RFD_KERNEL_BALL && kernel != RFD_KERNEL_CUBE_L1 &&
      kernel != RFD_KERNEL_L1_BALL)
    return fail(RFD_EINVAL, "unknown kernel");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(RFD_EINVAL, "eps must be finite and > 0");
  if (sigma == 0.0) sigma = default_sigma(eps);
  if (radius == 0.0) radius = default_radius(eps);
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(RFD_EINVAL, "freq_sigma must be > 0");
  if (!(radius > 0.0) || !std::isfinite(radius)) return fail(RFD_EINVAL, "freq_radius must be > 0");
  const int h = m / 2;
  SplitMix64 rng(seed);
  // density normaliser per coordinate: sigma sqrt(2 pi) erf(R / (sigma sqrt 2))
  const double norm = sigma * std::sqrt(2.0 * kPi) * std::erf(radius / (sigma * std::sqrt(2.0)));
  for (int j = 0; j < h; ++j) {
    double w3[3];
    for (int d = 0; d < 3; ++d) {
      int t = 0;
      for (; t < kMaxTries; ++t) {
        const double u1 = rng.uniform();
        const double u2 = rng.uniform();
        const double w = radius * (2.0 * u1 - 1.0);
        const double a = w / sigma;
        if (u2 < std::exp(-0.5 * a * a)) {
          w3[d] = w;
          break;
        }
      }
      if (t == kMaxTries)
        return fail(RFD_EINVAL, "frequency sampler: acceptance rate too low (freq_radius >> freq_sigma)");
    }
    if (omega) std::memcpy(omega + 3 * j, w3, sizeof(w3));
    if (r) {
      double tau = 1.0, p = 1.0;
      for (int d = 0; d < 3; ++d) {
        if (kernel == RFD_KERNEL_CUBE) tau *= sinc_cube(w3[d], eps);
        const double a = w3[d] / sigma;
        p *= std::exp(-0.5 * a * a) / norm;
      }
      if (kernel == RFD_KERNEL_BALL) tau = tau_ball(w3, eps);
      if (kernel == RFD_KERNEL_L1_BALL) tau = tau_l1_ball(w3, eps);
      if (kernel == RFD_KERNEL_CUBE_L1) {
        const double s0 = sinc_cube(w3[0], eps), s1 = sinc_cube(w3[1], eps), s2 = sinc_cube(w3[2], eps);
        tau = abs_cube(w3[0], eps) * s1 * s2 + s0 * abs_cube(w3[1], eps) * s2 + s0 * s1 * abs_cube(w3[2], eps);
      }
      r[j] = tau / p;
    }
  }
  return RFD_OK;
}

}  // namespace rfd

extern "C" rfd_status rfd_sample_frequencies(int32_t m, double eps, uint64_t seed, double freq_sigma,
                                             double freq_radius, double* omega_out, double* r_out) {
  return rfd::sample_frequencies_host(m, eps, seed, freq_sigma, freq_radius, RFD_KERNEL_CUBE, omega_out, r_out);
}

extern "C" rfd_status rfd_sample_weights(int32_t m, double eps, uint64_t seed, double freq_sigma, double freq_radius,
                                         int32_t kernel, double* omega_out, double* r_out) {
  return rfd::sample_frequencies_host(m, eps, seed, freq_sigma, freq_radius, kernel, omega_out, r_out);
}
