// FP64-accurate GEMM on the BF16 tensor cores by modular integer arithmetic,
// the Chinese-remainder form of the Ozaki scheme (Ozaki, Uchino, Imamura,
// "Ozaki Scheme II: a GEMM-oriented emulation of floating-point matrix
// multiplication using an integer modular technique", 2025), used for the
// m x m products of step a4 (G = lambda phi1(lambda M)): GB300 runs native
// FP64 at ~1 TFLOP/s, the BF16 tensor cores at ~2 PFLOP/s.
//
// Integers.  Row i of A is scaled by a power of two so that its largest entry
// becomes an integer of k bits (k = 57 for K <= 1024, 56 up to K = 4096, see
// crt::kbits); every entry becomes the integer X = trunc(A[i,l] 2^-ea_i),
// |X| < 2^k, exact except for bits below 2^-k of the row's largest entry.
// Columns of B likewise (exponents eb_j).  The product C' = X Y is then an
// exact integer with |C'| < K 2^2k <= P / 2, and C = 2^(ea_i + eb_j) C'.
//
// Residues.  For each of 16 pairwise coprime moduli p_j <= 256 (product
// P ~ 2^125.19) the residues X mod p_j, Y mod p_j in the symmetric range
// (|r| <= 128) are exact BF16 integers, and the BF16 product of the residue
// matrices accumulates exactly in FP32: a partial sum over 1024 of K is an
// integer of magnitude <= 1024 128^2 = 2^24.  Its value mod p_j is C' mod p_j
// (segments of 1024 of K add their residues mod p_j).
//
// Reconstruction.  C' = sum_j r_j W_j (mod P) with the constants W_j of
// crt_math.h, formed in 128-bit integer arithmetic and brought into (-P/2, P/2)
// by the nearest integer to S / P (an FP32 sum: its error is far inside the
// margin); the exact C' times 2^(ea_i + eb_j) is rounded once, to nearest
// even.  So the result carries FP64 accuracy relative to |A| |B| for any K.
//
// 16 BF16 products per FP64 product, where digit splitting needs 36 slice
// products (8 slices of 7 bits, pairs p + q <= 9) and eight TMEM accumulators.
//
// Kernel layout.  The residue GEMM: one CTA per (output tile, group of
// moduli): 128 or 256 rows (two M = 128 halves sharing the B rows) x up to 256
// columns x G moduli with halves x G x columns <= 512 TMEM columns.  The
// pipeline walks (64-wide K chunk, modulus) stages -- one or two 16 KB A boxes
// and N/64 8 KB B boxes, 128-byte swizzle, 3 stages of 64 KB.  Warp 0 issues
// the TMA loads, warp 1 one tcgen05.mma of 128 x N x 16 per half per 16 of K,
// warps 2..9 drain the FP32 sums into residues (FP32 floor arithmetic, exact
// below 2^24) and store them as bytes, planes [16][mp][np].  A second kernel
// reconstructs each entry and applies D = alpha A B + beta C + diag I.  Waits
// are bounded (2 s) and record an error code instead of hanging.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include <vector>
#include "crt_math.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace rfd {

namespace {

using namespace tc;
using crt::kNumMod;

constexpr int kBM = 128, kBK = 64, kBNMax = 256, kBBox = 64;
constexpr int kABytes = kBM * kBK * 2;                                 // 16 KB: 128 rows of 64 K
constexpr int kBBoxBytes = kBBox * kBK * 2;                            // 8 KB: 64 rows of 64 K
constexpr int kMaxStages = 8;
constexpr int kMaxBufs = 8;     // TMEM buffers (512 columns / the width of a unit)
constexpr int kThreads = 320;  // 10 warps
constexpr int kEpiWarps = 8;
constexpr int kSmemLimit = 232448;  // opt-in shared memory per CTA on sm_103
constexpr int kSmemExtra = 1024 + 512;  // alignment slack + barriers
constexpr int kMaxK = 4096;
constexpr int kColSplitK = 64;   // K rows per block of the column split
constexpr int kRowSeg = 256;     // columns per warp of the row split
constexpr int kChunksPerSeg = crt::kSegK / kBK;

// reconstruction constants for the first nmod moduli, nmod = 1..16
struct ConstantSets {
  crt::Constants c[kNumMod + 1];
};
const crt::Constants& constants(int nmod = kNumMod) {
  static const ConstantSets sets = [] {  // once per process (thread-safe initialisation)
    ConstantSets v{};
    for (int n = 1; n <= kNumMod; ++n) crt::make_constants(&v.c[n], n);
    return v;
  }();
  return sets.c[nmod < 1 ? 1 : (nmod > kNumMod ? kNumMod : nmod)];
}

// Residues of 8 consecutive integers X[e] (limbs L[e]) modulo p_j, j = J .. 15,
// as BF16 integers: plane j gets one 16-byte store at dst + j plane.  A residue
// is an FP32 integer with at most 8 significant bits, so its BF16 pattern is
// the upper half of its FP32 pattern.
__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
template <int J>
__device__ __forceinline__ void store_residues8(const crt::Limbs (&L)[8], const long long (&X)[8],
                                                __nv_bfloat16* dst, size_t plane, int nmod) {
  if (J >= nmod) return;  // planes of the moduli in use only
  uint4 w;
  w.x = bf16_pair(crt::residue<J>(L[0], X[0]), crt::residue<J>(L[1], X[1]));
  w.y = bf16_pair(crt::residue<J>(L[2], X[2]), crt::residue<J>(L[3], X[3]));
  w.z = bf16_pair(crt::residue<J>(L[4], X[4]), crt::residue<J>(L[5], X[5]));
  w.w = bf16_pair(crt::residue<J>(L[6], X[6]), crt::residue<J>(L[7], X[7]));
  *reinterpret_cast<uint4*>(dst + J * plane) = w;
  if constexpr (J + 1 < kNumMod) store_residues8<J + 1>(L, X, dst, plane, nmod);
}

// Row split of the row-major FP64 matrix X (rows x cols, ld) into the residue
// planes res [16][rows_pad][cols_pad] (zero padded, cols_pad a multiple of
// 64) and the row exponents exps (entry = int 2^exps[i]), integer operations
// only (the FP64 pipe is the slow one on this GPU).  L = 8, 16 or 32 lanes
// (cols_pad 64, 128, more) take a row, 8 consecutive columns each: a warp covers 32 / L rows, or
// one 256-column segment of a row (every segment takes the largest exponent
// over the whole row; segment 0 stores it).  Warp w of row_split_warps().
__host__ __device__ __forceinline__ int row_split_lanes(int cols_pad) {
  return cols_pad <= 64 ? 8 : (cols_pad <= 128 ? 16 : 32);  // a power of two (the shuffle reduction)
}
__host__ __device__ __forceinline__ int row_split_segs(int cols_pad) { return (cols_pad + kRowSeg - 1) / kRowSeg; }
// Largest biased exponent of row i (0: all entries zero or subnormal, or i >= rows)
// into eraw[i]; one warp, the row's loads issued back to back.
__device__ __forceinline__ void row_exponent_warp(const double* __restrict__ X, int ld, int rows, int cols,
                                                  int* __restrict__ eraw, int i, int lane) {
  int emax = 0;
  if (i < rows) {
    const double* row = X + (size_t)i * ld;
    int k = lane;
    for (; k + 7 * 32 < cols; k += 8 * 32) {
      unsigned long long b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = (unsigned long long)__double_as_longlong(row[k + q * 32]);
#pragma unroll
      for (int q = 0; q < 8; ++q) emax = max(emax, (int)((b[q] >> 52) & 0x7FF));
    }
    for (; k < cols; k += 32) emax = max(emax, (int)((__double_as_longlong(row[k]) >> 52) & 0x7FF));
  }
  for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  if (lane == 0) eraw[i] = emax;
}

// eraw: the rows' largest biased exponents from row_exponent_warp, or null (taken here)
__device__ __forceinline__ void split_rows_warp(const double* __restrict__ X, int ld, int rows, int cols,
                                                int rows_pad, int cols_pad, int sh0, int nmod,
                                                __nv_bfloat16* __restrict__ res, int* __restrict__ exps,
                                                const int* __restrict__ eraw, int w, int lane) {
  const int L = row_split_lanes(cols_pad), segs = row_split_segs(cols_pad);
  const int i = (w / segs) * (32 / L) + lane / L, seg = w % segs, sub = lane % L;
  int emax = 0;  // largest biased exponent in the row (0: all entries zero or subnormal)
  if (eraw) {
    if (i < rows) emax = eraw[i];
  } else {
    if (i < rows)
      for (int k = sub; k < cols; k += L) emax = max(emax, (int)((__double_as_longlong(X[(size_t)i * ld + k]) >> 52) & 0x7FF));
    for (int off = L / 2; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  }
  if (emax == 0) emax = 1;  // subnormal-only rows: scale as the smallest normal binade
  if (sub == 0 && seg == 0 && i < rows_pad) exps[i] = emax - 1075 - sh0;
  const int k0 = seg * kRowSeg + sub * 8;
  if (i >= rows_pad || k0 >= cols_pad) return;
  long long v[8];
  crt::Limbs limbs[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = k0 + e;
    v[e] = 0;
    if (i < rows && k < cols) v[e] = crt::scaled_int((unsigned long long)__double_as_longlong(X[(size_t)i * ld + k]), emax, sh0);
    limbs[e] = crt::limbs_of(v[e]);
  }
  store_residues8<0>(limbs, v, res + (size_t)i * cols_pad + k0, (size_t)rows_pad * cols_pad, nmod);
}
__host__ __device__ __forceinline__ int row_split_warps(int rows_pad, int cols_pad) {
  return rows_pad / (32 / row_split_lanes(cols_pad)) * row_split_segs(cols_pad);
}

// Largest biased exponents of columns j0 .. j0 + 31 of the row-major FP64
// matrix B (K x N, ld) over the K rows kr * 64 .. + 63, into
// part[kr * N_pad + j] (0: all zero or subnormal).  256 threads.
__device__ __forceinline__ void col_exponents(const double* __restrict__ B, int ld, int K, int N, int N_pad,
                                              int* __restrict__ part, int j0, int kr) {
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  __shared__ int red[8][32];
  int e = 0;
  if (j0 + tx < N)
#pragma unroll
    for (int q = 0; q < kColSplitK / 8; ++q) {
      const int k = kr * kColSplitK + ty + 8 * q;
      if (k < K) e = max(e, (int)((__double_as_longlong(B[(size_t)k * ld + j0 + tx]) >> 52) & 0x7FF));
    }
  red[ty][tx] = e;
  __syncthreads();
  if (ty == 0) {
    for (int y = 1; y < 8; ++y) e = max(e, red[y][tx]);
    part[(size_t)kr * N_pad + j0 + tx] = e;
  }
}

// Columns j0 .. j0 + 31 of the row-major FP64 matrix B (K x N, ld) over the
// K rows kr * 64 .. + 63 into the residue planes of B^T, res [16][N_pad][K_pad],
// and the column exponents exps (range 0 stores them), from the per-range
// exponents part of col_exponents.  The 64 x 32 tile is staged in shared
// memory; thread t takes column t / 8 and 8 consecutive rows of K, so every
// plane gets one 16-byte store per thread.  256 threads.
__device__ __forceinline__ void split_cols(const double* __restrict__ B, int ld, int K, int N, int K_pad, int N_pad,
                                           int sh0, int nmod, __nv_bfloat16* __restrict__ res, int* __restrict__ exps,
                                           const int* __restrict__ part, int j0, int kr) {
  const int t = threadIdx.x, tx = t & 31, ty = t >> 5;
  __shared__ double tile[kColSplitK][33];
  __shared__ int emax_s[32];
  if (ty == 0) {
    int e = 0;
    for (int r = 0; r < K_pad / kColSplitK; ++r) e = max(e, part[(size_t)r * N_pad + j0 + tx]);
    if (e == 0) e = 1;  // subnormal-only columns: scale as the smallest normal binade
    emax_s[tx] = e;
    if (kr == 0) exps[j0 + tx] = e - 1075 - sh0;
  }
  const size_t plane = (size_t)N_pad * K_pad;
  const int col = t >> 3, kg = (t & 7) * 8;
  {
    const int k0 = kr * kColSplitK;
    for (int y = ty; y < kColSplitK; y += 8) {
      const int k = k0 + y, j = j0 + tx;
      tile[y][tx] = (k < K && j < N) ? B[(size_t)k * ld + j] : 0.0;
    }
    __syncthreads();
    const int emax = emax_s[col];
    long long v[8];
    crt::Limbs limbs[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      v[q] = crt::scaled_int((unsigned long long)__double_as_longlong(tile[kg + q][col]), emax, sh0);
      limbs[q] = crt::limbs_of(v[q]);
    }
    store_residues8<0>(limbs, v, res + (size_t)(j0 + col) * K_pad + k0 + kg, plane, nmod);
    __syncthreads();
  }
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

struct Smem {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint32_t tmem_base;
};

// One work item of the residue GEMM: rows m0 .. m0 + 127 of the A residues against rows n0 .. n0 + nb of
// the B^T residues, for the moduli g0 .. g0 + G - 1 in turn, over kp of K;
// residues of the products into res planes [16][mp][np] (bytes in [0, p)).
struct Item {
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  uint8_t* res;
  int kp, mp, np, m0, n0, nb, g0, G;
  bool skip;  // the cloud skips this product
};

// The residue GEMM, persistent: CTA c takes items c, c + gridDim.x, ...  A
// unit is one modulus over one segment of at most 1024 of K (the FP32
// exactness bound); units alternate between two TMEM buffers of 256 columns,
// so the epilogue drains one unit while the MMAs of the next run.  Each CTA
// loads its own A rows and every B box of its item; stages (64 of K of one
// modulus) follow the units in order.
template <typename ItemFn>
__device__ __forceinline__ void residue_gemm_core(ItemFn item_of, int num_items, const crt::Constants& cc,
                                                  int stages, int stage_bytes, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + (base - raw_addr) + stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cid = (int)blockIdx.x, ncl = (int)gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&sm->full[s]), 1);
      mbar_init(smem_u32(&sm->empty[s]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&sm->acc_full[q]), 1);
      mbar_init(smem_u32(&sm->acc_empty[q]), kEpiWarps);
    }
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(&sm->tmem_base), 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int i = 0;
      bool ok = true;
      for (int it = cid; it < num_items && ok; it += ncl) {
        const Item I = item_of(it);
        if (I.skip) continue;
        const int nchunks = I.kp / kBK, nseg = (nchunks + kChunksPerSeg - 1) / kChunksPerSeg;
        const uint32_t tx = (uint32_t)(kBM + I.nb) * kBK * 2;  // A rows + every B box
        for (int u = 0; u < I.G * nseg && ok; ++u) {
          const int g = I.g0 + u / nseg, seg = u % nseg;
          const int c1 = min(nchunks, (seg + 1) * kChunksPerSeg);
          for (int c = seg * kChunksPerSeg; c < c1; ++c, ++i) {
            const int s = i % stages;
            if (!mbar_wait(smem_u32(&sm->empty[s]), ((uint32_t)(i / stages) & 1u) ^ 1u, err, 11)) {
              ok = false;
              break;
            }
            const uint32_t full = smem_u32(&sm->full[s]);
            mbar_arrive_expect_tx(full, tx);
            const uint32_t sa = base + s * stage_bytes, sb = sa + kABytes;
            tma_load_3d(sa, I.ma, c * kBK, I.m0, g, full);
            for (int q = 0; q < I.nb / kBBox; ++q)
              tma_load_3d(sb + q * kBBoxBytes, I.mb, c * kBK, I.n0 + q * kBBox, g, full);
          }
        }
      }
      // every stage this CTA filled has been released by its MMAs: no copy into this
      // CTA's shared memory is still in flight when it exits
      for (int t = (i > stages ? i - stages : 0); t < i; ++t)
        mbar_wait(smem_u32(&sm->empty[t % stages]), (uint32_t)(t / stages) & 1u, err, 12);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int i = 0, ug = 0;
      bool ok = true;
      for (int it = cid; it < num_items && ok; it += ncl) {
        const Item I = item_of(it);
        if (I.skip) continue;
        const uint32_t idesc = idesc_bf16(kBM, I.nb);
        const int nchunks = I.kp / kBK, nseg = (nchunks + kChunksPerSeg - 1) / kChunksPerSeg;
        for (int u = 0; u < I.G * nseg && ok; ++u, ++ug) {
          const int seg = u % nseg, q = ug & 1;
          // the buffer's previous unit must have been drained
          if (ug >= 2 && !mbar_wait(smem_u32(&sm->acc_empty[q]), (uint32_t)((ug >> 1) - 1) & 1u, err, 13)) {
            ok = false;
            break;
          }
          const int c0 = seg * kChunksPerSeg, c1 = min(nchunks, c0 + kChunksPerSeg);
          for (int c = c0; c < c1; ++c, ++i) {
            const int s = i % stages;
            if (!mbar_wait(smem_u32(&sm->full[s]), (uint32_t)(i / stages) & 1u, err, 14)) {
              ok = false;
              break;
            }
            fence_after();
            const uint32_t sa = base + s * stage_bytes, sb = sa + kABytes;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              mma_bf16(tmem + (uint32_t)(q * 256), sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                       (c > c0 || kk > 0) ? 1u : 0u);
            mma_commit(smem_u32(&sm->empty[s]));  // frees the stage when these MMAs finish
          }
          if (ok) mma_commit(smem_u32(&sm->acc_full[q]));  // the unit's sums are complete
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2..9, two per TMEM lane quarter) ----------------
    const int quarter = warp & 3, sub = (warp - 2) >> 2;
    int ug = 0;
    bool ok = true;
    for (int it = cid; it < num_items && ok; it += ncl) {
      const Item I = item_of(it);
      if (I.skip) continue;
      const int nchunks = I.kp / kBK, nseg = (nchunks + kChunksPerSeg - 1) / kChunksPerSeg;
      const size_t plane = (size_t)I.mp * I.np;
      const int row0 = I.m0;
      for (int u = 0; u < I.G * nseg; ++u, ++ug) {
        const int g = I.g0 + u / nseg, seg = u % nseg, q = ug & 1;
        if (!mbar_wait(smem_u32(&sm->acc_full[q]), (uint32_t)(ug >> 1) & 1u, err, 15)) {
          ok = false;
          break;
        }
        fence_after();
        const float p = cc.p[g], ip = cc.inv_p[g];
        const int row = row0 + quarter * 32 + lane;
        for (int cq = sub; cq < I.nb / 32; cq += 2) {
          const int c0 = cq * 32;
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(q * 256 + c0), v);
          uint8_t* dst = I.res + g * plane + (size_t)row * I.np + I.n0 + c0;
          uint32_t old[8] = {0, 0, 0, 0, 0, 0, 0, 0};
          if (seg > 0) {
            const uint4 a = reinterpret_cast<const uint4*>(dst)[0], b = reinterpret_cast<const uint4*>(dst)[1];
            old[0] = a.x; old[1] = a.y; old[2] = a.z; old[3] = a.w;
            old[4] = b.x; old[5] = b.y; old[6] = b.z; old[7] = b.w;
          }
          uint32_t w[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            uint32_t packed = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const float x = v[4 * e + b];  // an exact integer, |x| <= 2^24
              float r = fmaf(-crt::rint_small(x * ip), p, x);  // x - q p, exact, |r| <= p / 2 + 1
              if (r < 0.f) r += p;
              if (r >= p) r -= p;
              uint32_t t = (uint32_t)r;
              if (seg > 0) {
                t += (old[e] >> (8 * b)) & 0xFFu;
                if (t >= (uint32_t)p) t -= (uint32_t)p;
              }
              packed |= t << (8 * b);
            }
            w[e] = packed;
          }
          reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
          reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm->acc_empty[q]));
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

__device__ __forceinline__ bool pow2_of(double alpha, int* k, bool* neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(alpha);
  const int E = (int)((b >> 52) & 0x7FF);
  if ((b & 0xFFFFFFFFFFFFFull) != 0 || E == 0 || E == 0x7FF) return false;
  *k = E - 1023;
  *neg = (b >> 63) != 0;
  return true;
}

// alpha (A B)[i, j] from the residues r and the exponent e = ea_i + eb_j:
// correctly rounded when alpha is a power of two and the result is a normal
// double.
// alpha = (-1)^aneg 2^ak when ap2 (decoded once per thread by pow2_of)
template <int NM>
__device__ __forceinline__ double product_entry(const crt::Constants& cc, const uint32_t (&r)[kNumMod], int e,
                                                double alpha, bool ap2, int ak, bool aneg) {
  unsigned long long lo, hi;
  crt::reconstruct<NM>(r, cc, &lo, &hi);
  double v;
  if (ap2) {
    if (!crt::to_double(lo, hi, e + ak, aneg, &v)) v = alpha * crt::to_double_plain(lo, hi, e);
  } else {
    if (!crt::to_double(lo, hi, e, false, &v)) v = crt::to_double_plain(lo, hi, e);
    v *= alpha;
  }
  return v;
}

// D[i, j0 .. j0 + 3] (columns < ncols) = alpha (A B) + beta C + diag I from
// the residue planes (one 4-byte load per plane; res_row = row i of plane 0).
template <int NM>
__device__ __forceinline__ void combine4(const crt::Constants& cc, const uint8_t* __restrict__ res_row, size_t plane,
                                         int i, int j0, int ncols, int ea_i, const int* __restrict__ eb,
                                         double alpha, double beta, const double* C, double* D, double diag) {
  uint32_t w[kNumMod];
#pragma unroll
  for (int j = 0; j < kNumMod; ++j)  // the first NM moduli are in use (cc.nmod == NM)
    w[j] = j < NM ? __ldg(reinterpret_cast<const uint32_t*>(res_row + j * plane + j0)) : 0u;
  int ak = 0;
  bool aneg = false;
  const bool ap2 = pow2_of(alpha, &ak, &aneg);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = j0 + q;
    if (jj >= ncols) break;
    uint32_t r[kNumMod];
#pragma unroll
    for (int j = 0; j < kNumMod; ++j) r[j] = (w[j] >> (8 * q)) & 0xFFu;
    double v = product_entry<NM>(cc, r, ea_i + eb[jj], alpha, ap2, ak, aneg);
    if (beta != 0.0) v = fma(beta, C[jj], v);
    if (i == jj) v += diag;
    D[jj] = v;
  }
}

// ---- batched kernels (one table entry per cloud, slots resolved per call) ----

// Row split of the A operand, every cloud (warp prefix over ozaki_row_split_warps(m)),
// from the row exponents of the exponent pass.
__device__ __forceinline__ void bsplit_rows_warp(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix,
                                                 int count, int slot, int nmod, int mask_k, int wg, int lane) {
  if (wg >= __ldg(prefix + count)) return;
  const int j = find_job(prefix, count, wg);
  const PhiCloud pc = pcs[j];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  split_rows_warp(pc_slot(pc, slot), pc.m, pc.m, pc.m, pc.mpa, pc.kp, pc.kbits_n[nmod - 1] - 53, nmod,
                  reinterpret_cast<__nv_bfloat16*>(pc.sa), pc.ea, pc.eap, wg - prefix[j], lane);
}
// Row exponents of the A operand: one warp per padded row (block b: 8 rows; prefix over mpa / 8 blocks).
__device__ __forceinline__ void brow_exponents_block(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix,
                                                     int count, int slot, int mask_k, int b) {
  const int jc = find_job(prefix, count, b);
  const PhiCloud pc = pcs[jc];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  row_exponent_warp(pc_slot(pc, slot), pc.m, pc.m, pc.m, pc.eap, (b - prefix[jc]) * 8 + (threadIdx.x >> 5),
                    threadIdx.x & 31);
}
// Column exponents of the B operand: one block per strip of 32 columns and
// range of 64 rows of K (prefix over strips x ranges per cloud).
__device__ __forceinline__ void bcol_exponents_block(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix,
                                                     int count, int slot, int mask_k, int b) {
  const int jc = find_job(prefix, count, b);
  const PhiCloud pc = pcs[jc];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  const int nranges = pc.kp / kColSplitK, local = b - prefix[jc];
  col_exponents(pc_slot(pc, slot), pc.m, pc.m, pc.m, pc.mpb, pc.ebp, (local / nranges) * 32, local % nranges);
}
// The exponent pass of a product: blocks [0, row_blocks) take A's row exponents
// (a_slot >= 0 ... when split), the rest B's column exponents.  256 threads.
__global__ void bexponents_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ rexp_prefix,
                                  const int* __restrict__ strip_prefix, int count, int a_slot, int b_slot, int mask_k,
                                  int row_blocks) {
  if ((int)blockIdx.x < row_blocks)
    brow_exponents_block(pcs, rexp_prefix, count, a_slot, mask_k, blockIdx.x);
  else
    bcol_exponents_block(pcs, strip_prefix, count, b_slot, mask_k, blockIdx.x - row_blocks);
}
__device__ __forceinline__ void bsplit_cols_block(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix,
                                                  int count, int slot, int nmod, int mask_k, int b) {
  const int jc = find_job(prefix, count, b);
  const PhiCloud pc = pcs[jc];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  const int nranges = pc.kp / kColSplitK, local = b - prefix[jc];
  split_cols(pc_slot(pc, slot), pc.m, pc.m, pc.m, pc.kp, pc.mpb, pc.kbits_n[nmod - 1] - 53, nmod,
             reinterpret_cast<__nv_bfloat16*>(pc.sb), pc.eb, pc.ebp, (local / nranges) * 32, local % nranges);
}
// The split pass of a product: blocks [0, row_blocks) split A's rows (8 warps
// each), the rest B's columns.  256 threads.
__global__ void bsplit_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ row_prefix,
                              const int* __restrict__ strip_prefix, int count, int a_slot, int b_slot, int nmod,
                              int mask_k, int row_blocks) {
  if ((int)blockIdx.x < row_blocks)
    bsplit_rows_warp(pcs, row_prefix, count, a_slot, nmod, mask_k, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                     threadIdx.x & 31);
  else
    bsplit_cols_block(pcs, strip_prefix, count, b_slot, nmod, mask_k, blockIdx.x - row_blocks);
}

__global__ void __launch_bounds__(kThreads, 1)
bresidue_gemm_kernel(const CUtensorMap* __restrict__ maps, const OzTile* __restrict__ tiles, int num_tiles,
                     const PhiCloud* __restrict__ pcs, const __grid_constant__ crt::Constants cc, int stages,
                     int stage_bytes, int mask_k, int* err) {
  const int nmod = cc.nmod;
  // item a = (tile a / nmod, modulus a mod nmod): the moduli in use only, spread over the CTAs
  auto item_of = [&](int it) {
    const OzTile t = tiles[it / nmod];
    const PhiCloud& pc = pcs[t.cloud];
    Item I;
    I.ma = maps + pc.map_a;
    I.mb = maps + pc.map_b;
    I.res = pc.res;
    I.kp = pc.kp;
    I.mp = pc.mpa;
    I.np = pc.mpb;
    I.m0 = t.m0;
    I.n0 = t.n0;
    I.nb = t.nb;
    I.g0 = it % nmod;
    I.G = 1;
    I.skip = mask_k >= 0 && pc.s <= mask_k;
    return I;
  };
  residue_gemm_core(item_of, num_tiles * nmod, cc, stages, stage_bytes, err);
}

// D = alpha A B + beta C + diag I, one thread per 4 consecutive entries of a
// row (prefix over blocks of 256 such groups per cloud, m ceil(m / 4) groups).
// A cloud with s <= mask_k skipped the product: its D becomes a copy of C (if
// any).
template <int NM>
__global__ void bcombine_product_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix, int count,
                                        const __grid_constant__ crt::Constants cc, int c_slot, int d_slot,
                                        double alpha, double beta, double diag, int mask_k) {
  const int jc = find_job(prefix, count, blockIdx.x);
  const PhiCloud pc = pcs[jc];
  const int m = pc.m, gpr = (m + 3) / 4;
  const int64_t g = (int64_t)(blockIdx.x - prefix[jc]) * blockDim.x + threadIdx.x;
  if (g >= (int64_t)m * gpr) return;
  const int i = (int)(g / gpr), j0 = (int)(g % gpr) * 4;
  const double* C = (c_slot == kNoSlot) ? nullptr : pc_slot(pc, c_slot) + (size_t)i * m;
  double* D = pc_slot(pc, d_slot) + (size_t)i * m;
  if (mask_k >= 0 && pc.s <= mask_k) {
    if (C && C != D)
      for (int j = j0; j < min(m, j0 + 4); ++j) D[j] = C[j];
    return;
  }
  combine4<NM>(cc, pc.res + (size_t)i * pc.mpb, (size_t)pc.mpa * pc.mpb, i, j0, m, pc.ea[i], pc.eb, alpha, beta, C, D,
           diag);
}

// ---- single product (general M, N, K) ----

__global__ void split_rows_kernel(const double* __restrict__ X, int ld, int rows, int cols, int rows_pad,
                                  int cols_pad, int sh0, __nv_bfloat16* __restrict__ res, int* __restrict__ exps) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= row_split_warps(rows_pad, cols_pad)) return;
  split_rows_warp(X, ld, rows, cols, rows_pad, cols_pad, sh0, kNumMod, res, exps, nullptr, warp, lane);
}

__global__ void col_exponents_kernel(const double* __restrict__ B, int ld, int K, int N, int N_pad,
                                     int* __restrict__ part) {
  col_exponents(B, ld, K, N, N_pad, part, blockIdx.x * 32, blockIdx.y);
}
__global__ void split_cols_kernel(const double* __restrict__ B, int ld, int K, int N, int K_pad, int N_pad, int sh0,
                                  __nv_bfloat16* __restrict__ res, int* __restrict__ exps, const int* __restrict__ part) {
  split_cols(B, ld, K, N, K_pad, N_pad, sh0, kNumMod, res, exps, part, blockIdx.x * 32, blockIdx.y);
}

// items (row tile of 128, column tile of 256, modulus), one modulus each
__global__ void __launch_bounds__(kThreads, 1)
residue_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                    const __grid_constant__ crt::Constants cc, int K_pad, int mp, int np, uint8_t* res, int stages,
                    int stage_bytes, int* err) {
  const int ntn = (np + kBNMax - 1) / kBNMax, ntm = (mp + kBM - 1) / kBM;
  auto item_of = [&](int it) {
    Item I;
    I.ma = &map_a;
    I.mb = &map_b;
    I.res = res;
    I.kp = K_pad;
    I.mp = mp;
    I.np = np;
    I.g0 = it % kNumMod;
    I.G = 1;
    const int t = it / kNumMod;
    I.n0 = (t % ntn) * kBNMax;
    I.m0 = (t / ntn) * kBM;
    I.nb = min(kBNMax, np - I.n0);
    I.skip = false;
    return I;
  };
  residue_gemm_core(item_of, ntn * ntm * kNumMod, cc, stages, stage_bytes, err);
}

__global__ void combine_product_kernel(const __grid_constant__ crt::Constants cc, const uint8_t* __restrict__ res,
                                       const int* __restrict__ ea, const int* __restrict__ eb, int M, int N, int mp,
                                       int np, double alpha, double beta, double* C, int ldc) {
  const int gpr = (N + 3) / 4;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (int64_t)M * gpr) return;
  const int i = (int)(g / gpr), j0 = (int)(g % gpr) * 4;
  double* Ci = C + (size_t)i * ldc;
  combine4<kNumMod>(cc, res + (size_t)i * np, (size_t)mp * np, i, j0, N, ea[i], eb, alpha, beta, Ci, Ci, 0.0);
}

}  // namespace

bool make_ozaki_maps(void* map_a_host, void* map_b_host, const void* sa, const void* sb, int mpa, int mpb, int kp) {
  return tc::make_map_bf16_3d(static_cast<CUtensorMap*>(map_a_host), sa, (uint64_t)kp, (uint64_t)mpa, kNumMod, kBM) &&
         tc::make_map_bf16_3d(static_cast<CUtensorMap*>(map_b_host), sb, (uint64_t)kp, (uint64_t)mpb, kNumMod,
                              kBBox);
}

namespace {

// Co-resident CTAs of the residue GEMM (1 per SM, shared memory bound); the
// persistent grids use this count.
struct GemmSlots {
  cudaError_t status;
  int ctas;
};
const GemmSlots& gemm_slots() {
  static const GemmSlots g = [] {  // once per process (thread-safe initialisation)
    GemmSlots r{cudaSuccess, 0};
    constants();
    int dev = 0;
    r.status = cudaGetDevice(&dev);
    if (r.status == cudaSuccess) r.status = cudaDeviceGetAttribute(&r.ctas, cudaDevAttrMultiProcessorCount, dev);
    auto attr = [&](auto kern) {
      if (r.status == cudaSuccess)
        r.status = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    };
    attr(bresidue_gemm_kernel);
    attr(residue_gemm_kernel);
    return r;
  }();
  return g;
}

// stages of stage_bytes that fit the shared memory (2 .. kMaxStages), 0 if none
int stages_for(int stage_bytes) {
  const int s = (kSmemLimit - kSmemExtra) / stage_bytes;
  return s < 2 ? 0 : (s > kMaxStages ? kMaxStages : s);
}

// A persistent launch: one CTA per SM, at most one per item.
template <typename Kern, typename... Args>
cudaError_t launch_persistent(Kern kern, int items, int smem, cudaStream_t st, Args... args) {
  const GemmSlots& g = gemm_slots();
  if (g.status != cudaSuccess) return g.status;
  const int ctas = std::max(1, std::min(items, g.ctas));
  kern<<<ctas, kThreads, smem, st>>>(args...);
  return cudaGetLastError();
}

}  // namespace

cudaError_t bgemm_prepare() { return gemm_slots().status; }

void ozaki_batch_tiles(const std::vector<int>& ms, int sms, std::vector<OzTile>* out, int* stage_bytes) {
  (void)sms;
  out->clear();
  int nb_max = kBBox;
  for (int k = 0; k < (int)ms.size(); ++k) {
    const OzLayout L = ozaki_layout(ms[k], ms[k], ms[k]);
    for (int m0 = 0; m0 < L.mp; m0 += kBM)
      for (int n0 = 0; n0 < L.np; n0 += kBNMax) {
        const int nb = std::min(kBNMax, L.np - n0);
        nb_max = std::max(nb_max, nb);
        out->push_back(OzTile{k, m0, n0, nb, L.kp, 0, kNumMod, 0});
      }
  }
  // longest tiles first: the persistent CTAs take their (tile, modulus) items round robin
  std::stable_sort(out->begin(), out->end(),
                   [](const OzTile& a, const OzTile& b) { return (int64_t)a.nb * a.kp > (int64_t)b.nb * b.kp; });
  *stage_bytes = kABytes + nb_max * kBK * 2;
}

namespace {
// grid-stride launch of the batched residue GEMM over its items
cudaError_t launch_bresidue(const void* maps_dev, const OzTile* tiles, int num_tiles, const PhiCloud* pc,
                            int stage_bytes, int nmod, int mask_k, int* err, cudaStream_t st) {
  const int stages = stages_for(stage_bytes);
  if (stages == 0) return cudaErrorInvalidValue;
  const int smem = stages * stage_bytes + kSmemExtra;
  const auto* maps = static_cast<const CUtensorMap*>(maps_dev);
  return launch_persistent(bresidue_gemm_kernel, num_tiles * nmod, smem, st, maps, tiles, num_tiles, pc,
                           constants(nmod), stages, stage_bytes, mask_k, err);
}
}  // namespace

int ozaki_kbits(int K, int nmod) { return crt::kbits(K, nmod); }

int ozaki_moduli_for_bits(int K, int k) {
  for (int n = 1; n <= kNumMod; ++n)
    if (crt::kbits(K, n) >= k) return n;
  return kNumMod;
}

namespace {
// the reconstruction kernel specialised for the moduli count in use (1 .. 16)
template <int NM = 1, typename... Args>
void launch_bcombine_product(int nmod, int blocks, cudaStream_t st, Args... args) {
  if constexpr (NM < kNumMod) {
    if (nmod != NM) return launch_bcombine_product<NM + 1>(nmod, blocks, st, args...);
  }
  bcombine_product_kernel<NM><<<blocks, 256, 0, st>>>(args...);
}
}  // namespace

cudaError_t launch_bgemm(const PhiCloud* pc, int count, const int* row_prefix_a, int rows_a, const int* rexp_prefix,
                         int rexp_blocks, const int* strip_prefix,
                         int col_strips, const OzTile* tiles, int num_tiles, int stage_bytes,
                         const int* group_prefix, int group_blocks, int nmod,
                         const void* maps_dev, int a_slot, int b_slot, int c_slot, int d_slot, double alpha,
                         double beta, double diag, int mask_k, bool split_a, bool split_b, int* err, cudaStream_t st) {
  const cudaError_t attr = bgemm_prepare();
  if (attr != cudaSuccess) return attr;
  if (split_a || split_b) {
    // exponents of what changes, then its residues (row blocks first, column blocks after)
    const int reb = split_a ? rexp_blocks : 0, cb = split_b ? col_strips : 0;
    bexponents_kernel<<<reb + cb, 256, 0, st>>>(pc, rexp_prefix, strip_prefix, count, a_slot, b_slot, mask_k, reb);
    const int rsb = split_a ? (rows_a * 32 + 255) / 256 : 0;
    bsplit_kernel<<<rsb + cb, 256, 0, st>>>(pc, row_prefix_a, strip_prefix, count, a_slot, b_slot, nmod, mask_k, rsb);
    count_launch(2);
  }
  const cudaError_t e = launch_bresidue(maps_dev, tiles, num_tiles, pc, stage_bytes, nmod, mask_k, err, st);
  if (e != cudaSuccess) return e;
  count_launch();
  launch_bcombine_product(nmod, group_blocks, st, pc, group_prefix, count, constants(nmod), c_slot, d_slot, alpha,
                          beta, diag, mask_k);
  return launched();
}

int ozaki_combine_blocks(int m) { return (int)(((int64_t)m * ((m + 3) / 4) + 255) / 256); }

int ozaki_row_exponent_blocks(int m) { return ozaki_layout(m, m, m).mp / 8; }

int ozaki_row_split_warps(int m) {
  const OzLayout L = ozaki_layout(m, m, m);
  return row_split_warps(L.mp, L.kp);
}

int ozaki_col_split_blocks(int m) {
  const OzLayout L = ozaki_layout(m, m, m);
  return (L.np / 32) * ((L.kp + kColSplitK - 1) / kColSplitK);
}

OzLayout ozaki_layout(int M, int N, int K) {
  OzLayout L{};
  L.mp = (M + kBM - 1) / kBM * kBM;
  L.np = (N + kBBox - 1) / kBBox * kBBox;
  L.kp = (K + kBK - 1) / kBK * kBK;
  auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  L.sa = 0;
  L.sb = a256(L.sa + (size_t)kNumMod * L.mp * L.kp * 2);
  L.ea = a256(L.sb + (size_t)kNumMod * L.np * L.kp * 2);
  L.eb = a256(L.ea + (size_t)L.mp * 4);
  L.eap = a256(L.eb + (size_t)L.np * 4);
  L.ebp = a256(L.eap + (size_t)L.mp * 4);
  L.res = a256(L.ebp + (size_t)(L.kp / kColSplitK) * L.np * 4);
  L.bytes = a256(L.res + (size_t)kNumMod * L.mp * L.np);
  return L;
}

size_t ozaki_workspace_bytes(int M, int N, int K) { return ozaki_layout(M, N, K).bytes + 256; }

bool ozaki_supported(int K) { return K >= 1 && K <= kMaxK && tc::sm103_available(); }

cudaError_t dgemm_ozaki(int M, int N, int K, double alpha, const double* A, int lda, const double* B, int ldb,
                        double beta, double* C, int ldc, void* work, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 1 || K > kMaxK) return cudaErrorInvalidValue;
  const cudaError_t attr = bgemm_prepare();
  if (attr != cudaSuccess) return attr;
  const OzLayout L = ozaki_layout(M, N, K);
  const int mp = L.mp, np = L.np, kp = L.kp, sh0 = crt::kbits(K) - 53;
  uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
  auto* sa = reinterpret_cast<__nv_bfloat16*>(w + L.sa);
  auto* sb = reinterpret_cast<__nv_bfloat16*>(w + L.sb);
  int* ea = reinterpret_cast<int*>(w + L.ea);
  int* eb = reinterpret_cast<int*>(w + L.eb);
  int* ebp = reinterpret_cast<int*>(w + L.ebp);
  uint8_t* res = w + L.res;
  split_rows_kernel<<<(row_split_warps(mp, kp) * 32 + 255) / 256, 256, 0, st>>>(A, lda, M, K, mp, kp, sh0, sa, ea);
  const dim3 strips(np / 32, kp / kColSplitK);
  col_exponents_kernel<<<strips, 256, 0, st>>>(B, ldb, K, N, np, ebp);
  split_cols_kernel<<<strips, 256, 0, st>>>(B, ldb, K, N, kp, np, sh0, sb, eb, ebp);
  count_launch(3);
  CUtensorMap ma, mb;
  if (!make_ozaki_maps(&ma, &mb, sa, sb, mp, np, kp)) return cudaErrorInvalidValue;
  {
    const int stage_bytes = kABytes + kBNMax * kBK * 2, stages = stages_for(stage_bytes);
    const int smem = stages * stage_bytes + kSmemExtra, ntn = (np + kBNMax - 1) / kBNMax;
    const cudaError_t e = launch_persistent(residue_gemm_kernel, ntn * (mp / kBM) * kNumMod, smem, st, ma, mb,
                                            constants(), kp, mp, np, res, stages, stage_bytes, err);
    if (e != cudaSuccess) return e;
    count_launch();
  }
  const int64_t groups = (int64_t)M * ((N + 3) / 4);
  combine_product_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, st>>>(constants(), res, ea, eb, M, N, mp, np,
                                                                           alpha, beta, C, ldc);
  return launched();
}

}  // namespace rfd
