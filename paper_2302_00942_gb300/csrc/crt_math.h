// Integer arithmetic of the modular (Chinese-remainder) FP64 emulation, shared
// by the device kernels (k_ozaki.cu) and usable from plain host C++: the
// moduli, the reconstruction constants, residues of the scaled integers, the
// signed 128-bit reconstruction and its correctly rounded conversion to FP64.
//
// The moduli are 16 pairwise coprime integers <= 256, so a residue in the
// symmetric range |r| <= 128 is an exact BF16 integer and the product of two
// is at most 2^14; their product P is about 2^125.19.
#pragma once
#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define RFD_HD __host__ __device__ __forceinline__
#else
#define RFD_HD inline
#endif

namespace rfd {
namespace crt {

constexpr int kNumMod = 16;
constexpr int kSegK = 1024;    // |sum| <= 1024 * 128^2 = 2^24: exact in FP32 accumulation
constexpr int kMaxKBits = 57;  // |X| < 2^57: three 19-bit limbs

RFD_HD constexpr uint32_t modulus(int j) {
  return j == 0 ? 256u : j == 1 ? 255u : j == 2 ? 253u : j == 3 ? 251u : j == 4 ? 247u : j == 5 ? 241u
       : j == 6 ? 239u : j == 7 ? 233u : j == 8 ? 229u : j == 9 ? 227u : j == 10 ? 223u : j == 11 ? 211u
       : j == 12 ? 199u : j == 13 ? 197u : j == 14 ? 193u : 191u;
}

// Reconstruction constants for the first nmod moduli (P = their product): with
// M_j = P / p_j and w_j = M_j^-1 mod p_j, W_j = M_j w_j < P satisfies
// W_j = 1 (mod p_j) and 0 (mod p_i, i != j), so C = sum_j r_j W_j (mod P); and
// sum_j r_j W_j / P = sum_j r_j w_j / p_j exactly.  Entries j >= nmod are zero,
// so a residue there contributes nothing.
struct Constants {
  int32_t nmod;            // moduli in use (the first nmod of modulus())
  int32_t pad_;
  uint32_t W[kNumMod][4];  // W_j, 32-bit words from the least significant
  uint32_t P[4];           // P, 32-bit words
  float c[kNumMod];        // w_j / p_j (rounded to FP32)
  float p[kNumMod];                  // p_j
  float inv_p[kNumMod];              // 1 / p_j (rounded to FP32)
};

// Computed once on the host (128-bit integer arithmetic).  Returns false if the
// moduli were not pairwise coprime (no inverse).
inline bool make_constants(Constants* out, int nmod = kNumMod) {
  *out = Constants{};
  out->nmod = nmod;
  unsigned __int128 P = 1;
  for (int j = 0; j < nmod; ++j) P *= modulus(j);
  for (int j = 0; j < nmod; ++j) {
    const uint32_t p = modulus(j);
    const unsigned __int128 Mj = P / p;
    const uint32_t mj = (uint32_t)(Mj % p);
    uint32_t w = 0;
    for (uint32_t t = 1; t < p; ++t)
      if ((uint64_t)mj * t % p == 1) {
        w = t;
        break;
      }
    if (w == 0) return false;
    const unsigned __int128 W = Mj * w;
    for (int k = 0; k < 4; ++k) out->W[j][k] = (uint32_t)(W >> (32 * k));
    out->c[j] = (float)((double)w / (double)p);
    out->p[j] = (float)p;
    out->inv_p[j] = 1.0f / (float)p;
  }
  for (int k = 0; k < 4; ++k) out->P[k] = (uint32_t)(P >> (32 * k));
  return true;
}

// Bits of the scaled integers for a contraction of length K over the first nmod
// moduli: the largest k <= 57 with K 2^(2k) <= P / 2, so that |C| < K 2^(2k)
// stays inside the symmetric range of the residues (all 16 moduli: k = 57 up to
// K = 1024, 56 up to K = 4096).  0 if none.
inline int kbits(int K, int nmod = kNumMod) {
  unsigned __int128 P = 1;
  for (int j = 0; j < nmod; ++j) P *= modulus(j);
  for (int k = kMaxKBits; k > 0; --k)
    if (((unsigned __int128)(uint64_t)K << (2 * k)) <= P / 2) return k;
  return 0;
}

// The integer X of an FP64 entry (bit pattern b) in a row or column whose
// largest biased exponent is emax: X = mant 2^(E - emax + sh0), truncated
// toward zero, so |X| < 2^(53 + sh0); the entry is X 2^(emax - 1075 - sh0)
// up to the dropped bits.  (Subnormals take E = 1 without the hidden bit.)
RFD_HD long long scaled_int(unsigned long long b, int emax, int sh0) {
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
  const int sh = (E ? E : 1) - emax + sh0;
  const unsigned long long F = (sh >= 0) ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
  return (b >> 63) ? -(long long)F : (long long)F;
}

// X (|X| < 2^60) as five signed 12-bit limbs in FP32: X = sum_i x[i] 2^(12 i).
struct Limbs {
  float x[5];
};
RFD_HD Limbs limbs_of(long long X) {
  const bool neg = X < 0;
  const unsigned long long a = neg ? (unsigned long long)(-X) : (unsigned long long)X;
  const float sg = neg ? -1.0f : 1.0f;
  Limbs L;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const uint32_t v = (uint32_t)(a >> (12 * i)) & 0xFFFu;
#if defined(__CUDA_ARCH__)
    const float f = __uint_as_float(0x4B000000u | v) - 8388608.0f;  // exact, no conversion unit
#else
    const float f = (float)v;
#endif
    L.x[i] = f * sg;
  }
  return L;
}

// The integer nearest to x (ties to even) for |x| < 2^22, by the FP32 add of
// 1.5 2^23 (whose unit in the last place is 1): no rounding or conversion unit.
RFD_HD float rint_small(float x) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
#else
  volatile float t = x + 12582912.0f;
  return t - 12582912.0f;
#endif
}

// X mod p_j in a symmetric range, |r| <= 128, as an FP32 integer.  For p < 256:
// s = sum_i x_i (2^(12 i) mod p) is exact in FP32 (|s| < 5 2^20) and
// r = s - p rint(s / p); the FP32 quotient errs by < 0.006, so a misrounded
// half gives |r| <= p / 2 + 0.006 p < 129.  For p = 256 (X mod 256 is the low
// byte) the integer form keeps r in [-128, 127].
template <int j>
RFD_HD float residue(const Limbs& L, long long X) {
  constexpr uint32_t p = modulus(j);
  if constexpr (p == 256) {
    const uint32_t u = (uint32_t)(((unsigned long long)X + 128ull) & 255ull);
#if defined(__CUDA_ARCH__)
    return __uint_as_float(0x4B000000u | u) - 8388736.0f;  // u - 128, exact
#else
    return (float)u - 128.0f;
#endif
  } else {
    constexpr float c1 = (float)((1ull << 12) % p), c2 = (float)((1ull << 24) % p), c3 = (float)((1ull << 36) % p),
                    c4 = (float)((1ull << 48) % p);
    constexpr float fp = (float)p, ip = 1.0f / (float)p;
    const float s = fmaf(L.x[4], c4, fmaf(L.x[3], c3, fmaf(L.x[2], c2, fmaf(L.x[1], c1, L.x[0]))));
    return fmaf(-fp, rint_small(s * ip), s);
  }
}

// a 128-bit integer from four 64-bit column sums t_k (each < 2^63) of 32-bit
// word products: sum_k t_k 2^(32 k) modulo 2^128, as low / high words
RFD_HD void fold_columns(unsigned long long t0, unsigned long long t1, unsigned long long t2, unsigned long long t3,
                         unsigned long long* lo, unsigned long long* hi) {
  const unsigned long long s1 = t1 << 32;
  *lo = t0 + s1;
  *hi = (t1 >> 32) + t2 + (t3 << 32) + (*lo < s1 ? 1ull : 0ull);
}

// S = sum_j r_j W_j modulo 2^128 (32-bit words: each column sum stays below
// 16 2^8 2^32 = 2^44) and q = the integer nearest to S / P; the signed result
// C = S - q P (mod 2^128) is exact whenever |C| < P / 2 (the FP32 sum for q
// errs by < 0.01, far inside the margin |C / P| <= 0.44).
template <int NM = kNumMod>
RFD_HD void reconstruct(const uint32_t (&r)[kNumMod], const Constants& cc, unsigned long long* lo_out,
                        unsigned long long* hi_out) {
  unsigned long long t0 = 0, t1 = 0, t2 = 0, t3 = 0;
  float qf = 0.f;
#pragma unroll
  for (int j = 0; j < NM; ++j) {  // the first NM moduli (cc.nmod == NM, or W_j = 0 beyond cc.nmod)
    const unsigned long long rj = r[j];
    t0 += rj * cc.W[j][0];
    t1 += rj * cc.W[j][1];
    t2 += rj * cc.W[j][2];
    t3 += rj * cc.W[j][3];
#if defined(__CUDA_ARCH__)
    const float rf = __uint_as_float(0x4B000000u | r[j]) - 8388608.0f;  // r < 2^23, exact, no conversion unit
#else
    const float rf = (float)r[j];
#endif
    qf = fmaf(rf, cc.c[j], qf);
  }
  const unsigned long long q = (unsigned long long)rintf(qf);
  unsigned long long lo, hi, ql, qh;
  fold_columns(t0, t1, t2, t3, &lo, &hi);
  fold_columns(q * cc.P[0], q * cc.P[1], q * cc.P[2], q * cc.P[3], &ql, &qh);
  *lo_out = lo - ql;
  *hi_out = hi - qh - (lo < ql ? 1ull : 0ull);
}

RFD_HD int clz64(unsigned long long x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

// Correctly rounded (to nearest, ties to even) FP64 value of the signed 128-bit
// integer hi:lo (two's complement) times 2^E, negated when flip.  Returns false
// when the result is not a normal double (the caller takes a plain FP64 route).
RFD_HD bool to_double(unsigned long long lo, unsigned long long hi, int E, bool flip, double* out) {
  bool neg = (long long)hi < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0 ? 1ull : 0ull);
  }
  if (hi == 0 && lo == 0) {
    *out = 0.0;
    return true;
  }
  neg = neg != flip;
  // normalise: the magnitude shifted left until its top bit is bit 127 of h:l
  const int z = hi ? clz64(hi) : 64 + clz64(lo);  // leading zeros, 0 .. 127
  unsigned long long h, l;
  if (z >= 64) {
    h = lo << (z - 64);
    l = 0;
  } else {
    h = z ? (hi << z) | (lo >> (64 - z)) : hi;
    l = lo << z;
  }
  int msb = 127 - z;
  // the top 53 bits, rounded to nearest even on the 75 below them (zeros for small values)
  unsigned long long mant = h >> 11;
  const unsigned long long rem = h & 0x7FFull;
  const bool half = (rem >> 10) != 0, sticky = ((rem & 0x3FFull) | l) != 0;
  mant += (half && (sticky || (mant & 1ull))) ? 1ull : 0ull;
  if (mant >> 53) {
    mant >>= 1;
    ++msb;
  }
  const int be = msb + E + 1023;
  if (be < 1 || be > 2046) return false;
  const unsigned long long bits =
      ((neg ? 1ull : 0ull) << 63) | ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1));
#if defined(__CUDA_ARCH__)
  *out = __longlong_as_double((long long)bits);
#else
  union {
    unsigned long long u;
    double d;
  } cv;
  cv.u = bits;
  *out = cv.d;
#endif
  return true;
}

// Plain FP64 value of hi:lo times 2^E (for results outside the normal range).
RFD_HD double to_double_plain(unsigned long long lo, unsigned long long hi, int E) {
  const bool neg = (long long)hi < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0 ? 1ull : 0ull);
  }
  const double v = ((double)hi * 18446744073709551616.0 + (double)lo);
#if defined(__CUDA_ARCH__)
  return neg ? -ldexp(v, E) : ldexp(v, E);
#else
  return neg ? -__builtin_ldexp(v, E) : __builtin_ldexp(v, E);
#endif
}

}  // namespace crt
}  // namespace rfd
