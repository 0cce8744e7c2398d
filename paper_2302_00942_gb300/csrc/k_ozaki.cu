// FP64-accurate GEMM on the BF16 tensor cores by error-free splitting
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)), used for the m x m products of
// step a4 (G = lambda phi1(lambda M)): GB300 runs native FP64 at ~1 TFLOP/s,
// the BF16 tensor cores at ~2 PFLOP/s.
//
// Splitting.  Row i of A is scaled by 2^-e_i (|A[i,:]| < 2^(e_i - 1)) so that
// a = A[i,k] 2^-e_i has |a| < 1/2, and the integer X = a 2^56 (exact up to the
// bits below 2^-56) is written in balanced base 128:
//     X = sum_{p=1..8} d_p 128^(8-p),   |d_p| <= 64,
// so A[i,k] = 2^e_i sum_p d_p 2^-7p + O(2^(e_i - 57)) with integers d_p,
// exact in BF16.  Columns of B are cut the same way (the kernel splits the
// rows of B^T).
//
// Products.  The slice products with p + q <= 9 (36 pairs; the rest lie below
// 2^-63 of |A||B|) are summed on the tensor cores per digit position
// t = p + q into one FP32 accumulator each: E_t = sum_{p+q=t} A_p B_q has
// |E_t| <= (t - 1) 64^2 K' <= 2^24 over K' <= 512 columns of K, so every
// partial sum is an integer the FP32 accumulation holds exactly.  After every
// 512 columns of K the eight accumulators are drained into exact int64 sums
//     T_A = sum_{t=2..5} E_t 2^(7 (5 - t)),   T_B = sum_{t=6..9} E_t 2^(7 (9 - t)),
// and C[i,j] = 2^(e_i+f_j) (T_A 2^-35 + T_B 2^-63): the only roundings are the
// two conversions to FP64 and their sum, so the result carries FP64 accuracy
// relative to |A||B|, for any K.
//
// Kernel layout: one CTA per 128 x 64 output tile.  Per 64-column chunk of K
// the 8 slices of the B tile stay resident as one set (64 KB, double-buffered)
// while the 8 slices of the A tile stream through a 4-deep ring (16 KB each,
// 128-byte swizzle); A slice p is multiplied with B slices q <= 9 - p, so each
// slice is read from L2 once per chunk and serves every pair it belongs to.
// Warp 0 issues the TMA loads, warp 1 the tcgen05.mma into the eight adjacent
// 64-column TMEM accumulators (A slice p against the concatenated B slices
// lands on accumulators p..7 at once: 12 wide MMAs per 16 of K), warps 2..9 drain them (two warps per TMEM
// lane quarter, 32 columns each) into exact integer sums and write the tile
// through shared memory with coalesced rows.  Waits are bounded (2 s) and
// record an error code instead of hanging.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include "kernels.h"
#include "tc_common.cuh"

namespace rfd {

namespace {

using namespace tc;

constexpr int kS = 8;             // slices per operand
constexpr int kBeta = 7;          // bits per slice
constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr int kATile = kBM * kBK * 2;          // 16 KB: one slice of the A tile (128-byte rows)
constexpr int kBTile = kBN * kBK * 2;          // 8 KB: one slice of the B tile
constexpr int kBSet = kS * kBTile;             // 64 KB: all slices of the B tile for one K chunk
constexpr int kBBufs = 2;                      // B sets in flight
constexpr int kARing = 4;                      // A slices in flight
constexpr int kPipeBytes = kBBufs * kBSet + kARing * kATile;  // 192 KB
constexpr int kDrainChunks = 512 / kBK;        // exactness bound of the FP32 accumulation: 512 of K
constexpr int kThreads = 320;                  // 10 warps
constexpr int kSmemBytes = kPipeBytes + 1024 + 256;
constexpr int kMaxK = 4096;
constexpr int kColSplitK = 256;                // K rows per block of the batched column split

// Row-wise split of a row-major FP64 matrix X (rows x cols, ld) into kS BF16
// slices [kS][rows_pad][cols_pad] (zero padded) and per-row exponents.
//
// Done on the bit pattern with integer operations (FP64 arithmetic is the
// slow pipe on this GPU): with E the biased exponent of an entry, Emax the
// largest in its row and mant its 53-bit significand, e = Emax - 1021 gives
// |a| = |x| 2^-e < 1/2 and X = a 2^56 = +-(mant << (E - Emax + 2)) (low bits
// dropped when the shift is negative).  The balanced base-128 digits come
// from the least significant end: d = ((X + 64) mod 128) - 64, X <- (X - d) / 128,
// the last quotient being the leading digit (|d_1| <= 64 since |X| < 2^55).
__device__ __forceinline__ void split_row(const double* __restrict__ X, int ld, int rows, int cols, int rows_pad,
                                          int cols_pad, __nv_bfloat16* __restrict__ slices, int* __restrict__ exps,
                                          int i, int lane) {
  int emax = 0;  // largest biased exponent in the row (0: all entries zero or subnormal)
  if (i < rows)
    for (int k = lane; k < cols; k += 32)
      emax = max(emax, (int)((__double_as_longlong(X[(size_t)i * ld + k]) >> 52) & 0x7FF));
  for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  if (emax == 0) emax = 1;  // subnormal-only rows: scale as the smallest normal binade
  if (lane == 0) exps[i] = emax - 1021;  // |X[i, :]| < 2^(emax - 1022) = 2^(e - 1)
  const size_t plane = (size_t)rows_pad * cols_pad;
  for (int k = lane; k < cols_pad; k += 32) {
    long long v = 0;
    if (i < rows && k < cols) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(X[(size_t)i * ld + k]);
      const int E = (int)((b >> 52) & 0x7FF);
      const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
      const int sh = (E ? E : 1) - emax + 2;
      const unsigned long long F = (sh >= 0) ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
      v = (b >> 63) ? -(long long)F : (long long)F;
    }
#pragma unroll
    for (int p = kS; p >= 2; --p) {
      const long long d = ((v + 64) & 127) - 64;
      slices[(p - 1) * plane + (size_t)i * cols_pad + k] = __int2bfloat16_rn((int)d);
      v = (v - d) >> kBeta;
    }
    slices[(size_t)i * cols_pad + k] = __int2bfloat16_rn((int)v);
  }
}

__global__ void split_rows_kernel(const double* __restrict__ X, int ld, int rows, int cols, int rows_pad,
                                  int cols_pad, __nv_bfloat16* __restrict__ slices, int* __restrict__ exps) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows_pad) return;
  split_row(X, ld, rows, cols, rows_pad, cols_pad, slices, exps, warp, lane);
}

__device__ __forceinline__ int find_job(const int* __restrict__ prefix, int count, int b) {
  int lo = 0, hi = count;  // prefix[lo] <= b < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double* pc_slot(const PhiCloud& pc, int slot) {
  return slot == kSlotM ? const_cast<double*>(pc.M) : (slot == kSlotG ? pc.G : pc.work + (size_t)slot * pc.m * pc.m);
}

// Batched row split of the A operand: one warp per padded row of every cloud
// (prefix over mpa rows): slot (m x m) -> sa [8][mpa][kp], ea.
__global__ void bsplit_rows_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix, int count,
                                   int slot, int mask_k) {
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wg >= __ldg(prefix + count)) return;
  const int j = find_job(prefix, count, wg);
  const PhiCloud pc = pcs[j];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  const int i = wg - prefix[j];
  split_row(pc_slot(pc, slot), pc.m, pc.m, pc.m, pc.mpa, pc.kp, reinterpret_cast<__nv_bfloat16*>(pc.sa), pc.ea, i,
            lane);
}

// Batched column split of B = slot (m x m, row-major) straight into the B^T
// slices sb [8][mpb][kp] and the column exponents eb: one block per strip of
// 32 columns and range of kColSplitK rows of K (prefix over strips x ranges
// per cloud).  Each block first takes its columns' largest exponents over the
// whole column (every range computes the same value; range 0 stores it), then
// stages 32 x 32 tiles of its K range in shared memory so that the digit
// planes are written along K (coalesced).  Digits as split_row.
__global__ void bsplit_cols_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix, int count,
                                   int slot, int mask_k) {
  const int jc = find_job(prefix, count, blockIdx.x);
  const PhiCloud pc = pcs[jc];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  const int m = pc.m;
  const int nranges = (pc.kp + kColSplitK - 1) / kColSplitK;
  const int local = blockIdx.x - prefix[jc];
  const int j0 = (local / nranges) * 32, kr = local % nranges;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const double* B = pc_slot(pc, slot);
  __shared__ double tile[32][33];
  __shared__ int red[8][32];
  __shared__ int emax_s[32];
  int e = 0;
  if (j0 + tx < m)
    for (int k = ty; k < m; k += 8) e = max(e, (int)((__double_as_longlong(B[(size_t)k * m + j0 + tx]) >> 52) & 0x7FF));
  red[ty][tx] = e;
  __syncthreads();
  if (ty == 0) {
    for (int y = 1; y < 8; ++y) e = max(e, red[y][tx]);
    if (e == 0) e = 1;
    emax_s[tx] = e;
    if (kr == 0) pc.eb[j0 + tx] = e - 1021;
  }
  __syncthreads();
  auto* sb = reinterpret_cast<__nv_bfloat16*>(pc.sb);
  const size_t plane = (size_t)pc.mpb * pc.kp;
  const int k_end = min(pc.kp, (kr + 1) * kColSplitK);
  for (int k0 = kr * kColSplitK; k0 < k_end; k0 += 32) {
    for (int y = ty; y < 32; y += 8) {
      const int k = k0 + y, j = j0 + tx;
      tile[y][tx] = (k < m && j < m) ? B[(size_t)k * m + j] : 0.0;
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {  // y: column offset (row of B^T), tx: K offset
      const int j = j0 + y, k = k0 + tx;
      const unsigned long long b = (unsigned long long)__double_as_longlong(tile[tx][y]);
      const int E = (int)((b >> 52) & 0x7FF);
      const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
      const int sh = (E ? E : 1) - emax_s[y] + 2;
      const unsigned long long F = (sh >= 0) ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
      long long v = (b >> 63) ? -(long long)F : (long long)F;
#pragma unroll
      for (int p = kS; p >= 2; --p) {
        const long long d = ((v + 64) & 127) - 64;
        sb[(p - 1) * plane + (size_t)j * pc.kp + k] = __int2bfloat16_rn((int)d);
        v = (v - d) >> kBeta;
      }
      sb[(size_t)j * pc.kp + k] = __int2bfloat16_rn((int)v);
    }
    __syncthreads();
  }
}

__global__ void transpose_kernel(const double* __restrict__ B, int ldb, int rows, int cols, double* __restrict__ Bt) {
  __shared__ double tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (r < rows && c < cols) ? B[(size_t)r * ldb + c] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (c < cols && r < rows) Bt[(size_t)c * rows + r] = tile[threadIdx.x][y];
  }
}

struct Smem {
  uint64_t bfull[kBBufs];
  uint64_t bempty[kBBufs];
  uint64_t afull[kARing];
  uint64_t aempty[kARing];
  uint64_t acc_full;
  uint64_t acc_empty;
  uint32_t tmem_base;
};

// Correctly rounded (to nearest, ties to even) double of S 2^E for the exact
// integer S = TA 2^28 + TB (|TA| < 2^46, |TB| < 2^50), in 64-bit integer
// arithmetic (the FP64 pipe is the slow one on this GPU).  S 2^(e-63) =
// T_A 2^(e-35) + T_B 2^(e-63), so this is the same single rounding as summing
// the two exact FP64 terms.  S = H 2^28 + r with 0 <= r < 2^28; |S| keeps that
// form with |H| and the complement of r.  Returns false when the result is not
// a normal double (the caller takes the FP64 route).
__device__ __forceinline__ bool exact_sum_to_double(long long TA, long long TB, int E, bool flip, double* out) {
  const long long H = TA + (TB >> 28);
  unsigned long long r = (unsigned long long)(TB & ((1ll << 28) - 1));
  unsigned long long Hm;
  if (H < 0) {
    if (r) {
      Hm = (unsigned long long)(-H - 1);
      r = (1ull << 28) - r;
    } else {
      Hm = (unsigned long long)(-H);
    }
  } else {
    Hm = (unsigned long long)H;
  }
  if (Hm == 0 && r == 0) {
    *out = 0.0;
    return true;
  }
  const bool neg = (H < 0) != flip;
  int msb;
  unsigned long long q;
  if (Hm == 0) {
    msb = 63 - __clzll((long long)r);
    q = r << (52 - msb);
  } else {
    const int mh = 63 - __clzll((long long)Hm);
    msb = mh + 28;
    if (msb <= 52) {
      q = ((Hm << 28) | r) << (52 - msb);
    } else {
      const int sh = msb - 52;  // 1 .. 27: the dropped bits all lie in r
      q = (Hm << (28 - sh)) + (r >> sh);
      const unsigned long long rem = r & ((1ull << sh) - 1), half = 1ull << (sh - 1);
      if (rem > half || (rem == half && (q & 1ull))) ++q;
      if (q >> 53) {
        q >>= 1;
        ++msb;
      }
    }
  }
  const int be = msb + E + 1023;
  if (be < 1 || be > 2046) return false;
  *out = __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) |
                                          (q & 0xFFFFFFFFFFFFFull)));
  return true;
}

// alpha = +-2^k: returns true with k and the sign, so the scaling is exact in the exponent.
__device__ __forceinline__ bool pow2_of(double alpha, int* k, bool* neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(alpha);
  const int E = (int)((b >> 52) & 0x7FF);
  if ((b & 0xFFFFFFFFFFFFFull) != 0 || E == 0 || E == 0x7FF) return false;
  *k = E - 1023;
  *neg = (b >> 63) != 0;
  return true;
}

// One 128 x 64 output tile (m0, n0) of C = alpha A B + beta C from the slice
// tensor maps (A: rows p M_pad + i, B^T: rows q N_pad + j; K_pad columns).
// D = alpha A B + beta C + diag I (C may be null when beta == 0; D may equal C).
__device__ __forceinline__ void ozaki_tile(const CUtensorMap* map_a_p, const CUtensorMap* map_b_p, int M, int N,
                                           int M_pad, int N_pad, int K_pad, const int* __restrict__ ea,
                                           const int* __restrict__ eb, double alpha, double beta, const double* C,
                                           double* D, int ldc, double diag, int m0, int n0, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const CUtensorMap& map_a = *map_a_p;
  const CUtensorMap& map_b = *map_b_p;
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  const uint32_t bbase = base, abase = base + kBBufs * kBSet;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + (base - raw_addr) + kPipeBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = K_pad / kBK;
  const int ndrain = (nkc + kDrainChunks - 1) / kDrainChunks;

  if (threadIdx.x == 0) {
    for (int b = 0; b < kBBufs; ++b) {
      mbar_init(smem_u32(&sm->bfull[b]), 1);
      mbar_init(smem_u32(&sm->bempty[b]), 1);
    }
    for (int a = 0; a < kARing; ++a) {
      mbar_init(smem_u32(&sm->afull[a]), 1);
      mbar_init(smem_u32(&sm->aempty[a]), 1);
    }
    mbar_init(smem_u32(&sm->acc_full), 1);
    mbar_init(smem_u32(&sm->acc_empty), 8);  // one arrive per epilogue warp
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(&sm->tmem_base), 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  // Per K chunk: the 8 B slices as one set (double-buffered), then the 8 A
  // slices one by one through a ring; A slice p meets B slices q <= 7 - p
  // (0-based), the pairs with p + q <= 9 (1-based).
  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      int issued_b = 0, issued_a = 0;
      for (int kc = 0; kc < nkc && ok; ++kc) {
        const int bs = kc % kBBufs;
        if (!mbar_wait(smem_u32(&sm->bempty[bs]), ((kc / kBBufs) & 1u) ^ 1u, err, 11)) { ok = false; break; }
        const uint32_t bf = smem_u32(&sm->bfull[bs]);
        mbar_arrive_expect_tx(bf, kBSet);
#pragma unroll
        for (int q = 0; q < kS; ++q) tma_load_2d(bbase + bs * kBSet + q * kBTile, &map_b, kc * kBK, q * N_pad + n0, bf);
        ++issued_b;
        for (int p = 0; p < kS; ++p) {
          const int it = kc * kS + p, as = it % kARing;
          if (!mbar_wait(smem_u32(&sm->aempty[as]), ((it / kARing) & 1u) ^ 1u, err, 12)) { ok = false; break; }
          const uint32_t af = smem_u32(&sm->afull[as]);
          mbar_arrive_expect_tx(af, kATile);
          tma_load_2d(abase + as * kATile, &map_a, kc * kBK, p * M_pad + m0, af);
          ++issued_a;
        }
      }
      // wait for the copies still in flight before the CTA may exit
      for (int u = (issued_b > kBBufs ? issued_b - kBBufs : 0); u < issued_b; ++u)
        mbar_wait(smem_u32(&sm->bfull[u % kBBufs]), (u / kBBufs) & 1u, err, 16);
      for (int u = (issued_a > kARing ? issued_a - kARing : 0); u < issued_a; ++u)
        mbar_wait(smem_u32(&sm->afull[u % kARing]), (u / kARing) & 1u, err, 17);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int kc = 0; kc < nkc && ok; ++kc) {
        const int drain = kc / kDrainChunks, in_drain = kc % kDrainChunks;
        if (in_drain == 0 && drain > 0) {  // the epilogue must have read the previous sums
          if (!mbar_wait(smem_u32(&sm->acc_empty), (drain - 1) & 1u, err, 13)) { ok = false; break; }
          fence_after();
        }
        const int bs = kc % kBBufs;
        if (!mbar_wait(smem_u32(&sm->bfull[bs]), (kc / kBBufs) & 1u, err, 14)) { ok = false; break; }
        fence_after();
        const uint32_t sb0 = bbase + bs * kBSet;
        for (int p = 0; p < kS && ok; ++p) {
          const int it = kc * kS + p, as = it % kARing;
          if (!mbar_wait(smem_u32(&sm->afull[as]), (it / kARing) & 1u, err, 18)) { ok = false; break; }
          fence_after();
          const uint32_t sa = abase + as * kATile;
          // A_p times the concatenated slices [B_0 .. B_(7-p)] (rows q*64 + j of the B set): column
          // block q of the product is pair (p, q), digit position t = p + q, whose accumulator sits at
          // TMEM columns t*64, so the whole product lands at columns p*64 .. 511 -- one or two wide
          // MMAs (N <= 256) instead of 8 - p narrow ones.
          const int ncols = (kS - p) * kBN;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint32_t acc = (in_drain > 0 || p > 0 || kk > 0) ? 1u : 0u;
            for (int c0 = 0; c0 < ncols; c0 += 256) {
              const int nc = min(256, ncols - c0);
              mma_bf16(tmem + (uint32_t)(p * kBN + c0), sdesc_sw128(sa + kk * 32),
                       sdesc_sw128(sb0 + (c0 / kBN) * kBTile + kk * 32), idesc_bf16(kBM, nc), acc);
            }
          }
          mma_commit(smem_u32(&sm->aempty[as]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&sm->bempty[bs]));
        if (in_drain == kDrainChunks - 1 || kc == nkc - 1) mma_commit(smem_u32(&sm->acc_full));
      }
    }
    __syncwarp();
  } else {
    // epilogue: two warps per TMEM lane quarter, 32 columns each
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int col0 = half * 32;
    const int gi = m0 + row;
    double* tile = reinterpret_cast<double*>(smem_raw + (base - raw_addr));  // kBM rows x (kBN + 1)
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)col0;
    int ak = 0;
    bool aneg = false;
    const bool ap2 = pow2_of(alpha, &ak, &aneg);
    const int eri = ea[gi < M_pad ? gi : 0];
    // alpha 2^e (T_A 2^-35 + T_B 2^-63), correctly rounded, into the shared-memory tile
    auto emit = [&](int c, long long ta, long long tb) {
      const int e = eri + eb[n0 + col0 + c];
      double v;
      if (!(ap2 && exact_sum_to_double(ta, tb, e - 63 + ak, aneg, &v)))
        v = alpha * (ldexp((double)ta, e - 35) + ldexp((double)tb, e - 63));
      tile[row * (kBN + 1) + col0 + c] = v;
    };
    bool ok = true;
    if (ndrain == 1) {
      // one drain (K <= 512): 8 columns at a time, the eight digit positions loaded under one wait
      ok = mbar_wait(smem_u32(&sm->acc_full), 0u, err, 15);
      if (ok) {
        fence_after();
#pragma unroll 1
        for (int g = 0; g < 32; g += 8) {
          uint32_t r[8][8];
#pragma unroll
          for (int t = 0; t < kS; ++t) tmem_ld8_nowait(taddr + (uint32_t)(t * kBN + g), r[t]);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            long long ta = 0, tb = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) ta += (long long)__float2int_rn(__uint_as_float(r[t][c])) << (kBeta * (3 - t));
#pragma unroll
            for (int t = 4; t < kS; ++t) tb += (long long)__float2int_rn(__uint_as_float(r[t][c])) << (kBeta * (7 - t));
            emit(g + c, ta, tb);
          }
        }
      }
    } else {
      long long TA[32], TB[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) { TA[c] = 0; TB[c] = 0; }
      for (int d = 0; d < ndrain && ok; ++d) {
        if (!mbar_wait(smem_u32(&sm->acc_full), d & 1u, err, 15)) { ok = false; break; }
        fence_after();
#pragma unroll 1
        for (int t = 2; t <= kS + 1; ++t) {
          float v[32];
          tmem_ld32(taddr + (uint32_t)((t - 2) * kBN), v);
          const int sh = (t <= 5) ? kBeta * (5 - t) : kBeta * (kS + 1 - t);
          if (t <= 5) {
#pragma unroll
            for (int c = 0; c < 32; ++c) TA[c] += (long long)__float2int_rn(v[c]) << sh;
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) TB[c] += (long long)__float2int_rn(v[c]) << sh;
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm->acc_empty));
      }
      if (ok) {
#pragma unroll
        for (int c = 0; c < 32; ++c) emit(c, TA[c], TB[c]);
      }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");  // the 8 epilogue warps
    // ... then out with coalesced rows: D = tile + beta C (+ diag on the diagonal)
    if (ok) {
      const int ew = warp - 2;
      for (int r = ew; r < kBM; r += 8) {
        const int i = m0 + r;
        if (i >= M) break;
        for (int jj = lane; jj < kBN; jj += 32) {
          const int j = n0 + jj;
          if (j >= N) continue;
          double v = tile[r * (kBN + 1) + jj];
          if (beta != 0.0) v = fma(beta, C[(size_t)i * ldc + j], v);
          if (i == j) v += diag;
          D[(size_t)i * ldc + j] = v;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

__global__ void __launch_bounds__(kThreads, 1)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M,
                  int N, int M_pad, int N_pad, int K_pad, const int* __restrict__ ea, const int* __restrict__ eb,
                  double alpha, double beta, double* C, int ldc, int* err) {
  ozaki_tile(&map_a, &map_b, M, N, M_pad, N_pad, K_pad, ea, eb, alpha, beta, C, C, ldc, 0.0, blockIdx.y * kBM,
             blockIdx.x * kBN, err);
}

// Batched: one CTA per OzTile of any cloud; D = alpha A B + beta C + diag I on
// the cloud's slots (c_slot kNoSlot: no C).  A cloud with s <= mask_k skips
// the product: its tile of D becomes a copy of C (if any).
__global__ void __launch_bounds__(kThreads, 1)
ozaki_gemm_batched_kernel(const CUtensorMap* __restrict__ maps, const OzTile* __restrict__ tiles,
                          const PhiCloud* __restrict__ pcs, int c_slot, int d_slot, double alpha, double beta,
                          double diag, int mask_k, int* err) {
  const OzTile t = tiles[blockIdx.x];
  const PhiCloud pc = pcs[t.cloud];
  const double* C = (c_slot == kNoSlot) ? nullptr : pc_slot(pc, c_slot);
  double* D = pc_slot(pc, d_slot);
  if (mask_k >= 0 && pc.s <= mask_k) {
    if (C && C != D)
      for (int e = threadIdx.x; e < kBM * kBN; e += blockDim.x) {
        const int i = t.m0 + e / kBN, j = t.n0 + e % kBN;
        if (i < pc.m && j < pc.m) D[(size_t)i * pc.m + j] = C[(size_t)i * pc.m + j];
      }
    return;
  }
  ozaki_tile(maps + pc.map_a, maps + pc.map_b, pc.m, pc.m, pc.mpa, pc.mpb, pc.kp, pc.ea, pc.eb, alpha, beta, C, D,
             pc.m, diag, t.m0, t.n0, err);
}

}  // namespace

bool make_ozaki_maps(void* map_a_host, void* map_b_host, const void* sa, const void* sb, int mpa, int mpb, int kp) {
  return tc::make_map_bf16(static_cast<CUtensorMap*>(map_a_host), sa, (uint64_t)kp, (uint64_t)kS * mpa, (uint64_t)kp,
                           kBM) &&
         tc::make_map_bf16(static_cast<CUtensorMap*>(map_b_host), sb, (uint64_t)kp, (uint64_t)kS * mpb, (uint64_t)kp,
                           kBN);
}

cudaError_t bgemm_prepare() {
  static const cudaError_t attr =  // once per process (thread-safe initialisation)
      cudaFuncSetAttribute(ozaki_gemm_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  return attr;
}

cudaError_t launch_bgemm(const PhiCloud* pc, int count, const int* row_prefix_a, int rows_a, const int* strip_prefix,
                         int col_strips, const OzTile* tiles, int num_tiles, const void* maps_dev, int a_slot,
                         int b_slot, int c_slot, int d_slot, double alpha, double beta, double diag, int mask_k,
                         bool split_a, bool split_b, int* err, cudaStream_t st) {
  const cudaError_t attr = bgemm_prepare();
  if (attr != cudaSuccess) return attr;
  if (split_a) {
    bsplit_rows_kernel<<<(rows_a * 32 + 255) / 256, 256, 0, st>>>(pc, row_prefix_a, count, a_slot, mask_k);
    count_launch();
  }
  if (split_b) {
    bsplit_cols_kernel<<<col_strips, dim3(32, 8), 0, st>>>(pc, strip_prefix, count, b_slot, mask_k);
    count_launch();
  }
  ozaki_gemm_batched_kernel<<<num_tiles, kThreads, kSmemBytes, st>>>(static_cast<const CUtensorMap*>(maps_dev), tiles,
                                                                     pc, c_slot, d_slot, alpha, beta, diag, mask_k,
                                                                     err);
  return launched();
}

int ozaki_col_split_blocks(int m) {
  const OzLayout L = ozaki_layout(m, m, m);
  return (L.np / 32) * ((L.kp + kColSplitK - 1) / kColSplitK);
}

OzLayout ozaki_layout(int M, int N, int K) {
  OzLayout L{};
  L.mp = (M + kBM - 1) / kBM * kBM;
  L.np = (N + kBN - 1) / kBN * kBN;
  L.kp = (K + kBK - 1) / kBK * kBK;
  auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  L.sa = 0;
  L.sb = a256(L.sa + (size_t)kS * L.mp * L.kp * 2);
  L.ea = a256(L.sb + (size_t)kS * L.np * L.kp * 2);
  L.eb = a256(L.ea + (size_t)L.mp * 4);
  L.bt = a256(L.eb + (size_t)L.np * 4);
  L.bytes = a256(L.bt + (size_t)N * K * 8);
  return L;
}

size_t ozaki_workspace_bytes(int M, int N, int K) { return ozaki_layout(M, N, K).bytes + 256; }

bool ozaki_supported(int K) { return K >= 1 && K <= kMaxK && tc::sm103_available(); }

cudaError_t dgemm_ozaki(int M, int N, int K, double alpha, const double* A, int lda, const double* B, int ldb,
                        double beta, double* C, int ldc, void* work, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 1 || K > kMaxK) return cudaErrorInvalidValue;
  const OzLayout L = ozaki_layout(M, N, K);
  const int mp = L.mp, np = L.np, kp = L.kp;
  uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
  auto* sa = reinterpret_cast<__nv_bfloat16*>(w + L.sa);
  auto* sb = reinterpret_cast<__nv_bfloat16*>(w + L.sb);
  int* ea = reinterpret_cast<int*>(w + L.ea);
  int* eb = reinterpret_cast<int*>(w + L.eb);
  double* bt = reinterpret_cast<double*>(w + L.bt);
  split_rows_kernel<<<(mp * 32 + 255) / 256, 256, 0, st>>>(A, lda, M, K, mp, kp, sa, ea);
  transpose_kernel<<<dim3((N + 31) / 32, (K + 31) / 32), dim3(32, 8), 0, st>>>(B, ldb, K, N, bt);
  split_rows_kernel<<<(np * 32 + 255) / 256, 256, 0, st>>>(bt, K, N, K, np, kp, sb, eb);
  count_launch(3);
  CUtensorMap ma, mb;
  if (!tc::make_map_bf16(&ma, sa, (uint64_t)kp, (uint64_t)kS * mp, (uint64_t)kp, kBM)) return cudaErrorInvalidValue;
  if (!tc::make_map_bf16(&mb, sb, (uint64_t)kp, (uint64_t)kS * np, (uint64_t)kp, kBN)) return cudaErrorInvalidValue;
  static const cudaError_t attr =  // once per process (thread-safe initialisation)
      cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (attr != cudaSuccess) return attr;
  ozaki_gemm_kernel<<<dim3(np / kBN, mp / kBM), kThreads, kSmemBytes, st>>>(ma, mb, M, N, mp, np, kp, ea, eb, alpha,
                                                                           beta, C, ldc, err);
  return launched();
}

}  // namespace rfd
