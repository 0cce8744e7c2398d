// FP64-accurate GEMM on the BF16 tensor cores by error-free splitting
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)), used for the m x m products of
// step a4 (G = lambda phi1(lambda M)): GB300 runs native FP64 at ~1 TFLOP/s,
// the BF16 tensor cores at ~2 PFLOP/s.
//
// Splitting.  Row i of A is scaled by 2^-e_i (|A[i,:]| < 2^e_i) and cut into
// S = 8 slices of 7 bits: a = A[i,k] 2^-e_i, and for p = 1..S
//     d_p = trunc(2^7 a),  a <- 2^7 a - d_p         (exact in FP64)
// so A[i,k] = 2^e_i sum_p d_p 2^-7p + O(2^(e_i - 56)) with integers
// |d_p| <= 127, exact in BF16.  Columns of B are cut the same way (the kernel
// splits the rows of B^T).
//
// Products.  D_pq = A_p B_q has integer entries bounded by 127^2 K < 2^24 for
// K <= 1024, so the tensor cores' FP32 accumulation is exact.  The pairs with
// p + q <= S + 1 (36 of them; the rest lie below 2^-63 of |A||B|) are drained
// from TMEM one by one and accumulated EXACTLY in integer registers:
//     E_t = sum_{p+q=t} D_pq        (int32, |E_t| < 2^27)
//     T_A = Horner_2^7 (E_2..E_5),  T_B = Horner_2^7 (E_6..E_9)  (int64, < 2^49)
//     C[i,j] = 2^(e_i+f_j) (T_A 2^-35 + T_B 2^-63),
// so the only roundings are the two conversions to FP64 and their sum: the
// result carries FP64 accuracy relative to |A||B|.
//
// Kernel layout: one CTA per 128 x 64 output tile; warp 0 issues TMA loads of
// the slice tiles (8-stage ring), warp 1 issues tcgen05.mma into one of eight
// 64-column TMEM accumulators (one per pair in flight), warps 2..9 drain the
// accumulators (two warps per TMEM lane quarter, 32 columns each).  Waits are
// bounded (2 s) and record an error code instead of hanging.
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
constexpr int kStages = 8;
constexpr int kABytes = kBM * kBK * 2;   // 16 KB
constexpr int kBBytes = kBN * kBK * 2;   // 8 KB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kBufs = 8;                 // TMEM accumulators (64 columns each)
constexpr int kThreads = 320;            // 10 warps
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr int kMaxK = 1024;              // exactness bound of one FP32 accumulation

// Row-wise split of a row-major FP64 matrix X (rows x cols, ld) into kS BF16
// slices [kS][rows_pad][cols_pad] (zero padded) and per-row exponents.
//
// Done on the bit pattern with integer operations (FP64 arithmetic is the
// slow pipe on this GPU): with E the biased exponent of an entry, Emax the
// largest in its row and mant its 53-bit significand, |a| = |x| 2^-e equals
// mant 2^(E - Emax - 53) (e = Emax - 1022), so F = floor(|a| 2^56) =
// mant << (E - Emax + 3) (or >> when negative) and the digits are the 7-bit
// fields d_p = (F >> (56 - 7p)) & 127 with the entry's sign: exactly the
// digits trunc(2^7 a), a <- 2^7 a - d_p produce.
__device__ __forceinline__ void split_row(const double* __restrict__ X, int ld, int rows, int cols, int rows_pad,
                                          int cols_pad, __nv_bfloat16* __restrict__ slices, int* __restrict__ exps,
                                          int i, int lane) {
  int emax = 0;  // largest biased exponent in the row (0: all entries zero or subnormal)
  if (i < rows)
    for (int k = lane; k < cols; k += 32)
      emax = max(emax, (int)((__double_as_longlong(X[(size_t)i * ld + k]) >> 52) & 0x7FF));
  for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  if (emax == 0) emax = 1;  // subnormal-only rows: scale as the smallest normal binade
  if (lane == 0) exps[i] = emax - 1022;  // |X[i, :]| < 2^(emax - 1022)
  const size_t plane = (size_t)rows_pad * cols_pad;
  for (int k = lane; k < cols_pad; k += 32) {
    unsigned long long F = 0;
    bool neg = false;
    if (i < rows && k < cols) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(X[(size_t)i * ld + k]);
      const int E = (int)((b >> 52) & 0x7FF);
      const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
      const int sh = (E ? E : 1) - emax + 3;
      F = (sh >= 0) ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
      neg = (b >> 63) != 0;
    }
#pragma unroll
    for (int p = 1; p <= kS; ++p) {
      const int d = (int)((F >> (56 - kBeta * p)) & 127ull);
      slices[(p - 1) * plane + (size_t)i * cols_pad + k] = __int2bfloat16_rn(neg ? -d : d);
    }
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

// Batched row split: one warp per padded row of every cloud (prefix over rows).
// operand 0: A = slot (rows/cols m, padded to mpa x kp) -> sa, ea;
// operand 1: B^T = bt (padded to mpb x kp) -> sb, eb.
__global__ void bsplit_rows_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix, int count,
                                   int operand, int slot, int mask_k) {
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wg >= __ldg(prefix + count)) return;
  const int j = find_job(prefix, count, wg);
  const PhiCloud pc = pcs[j];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  const int i = wg - prefix[j];
  if (operand == 0)
    split_row(pc_slot(pc, slot), pc.m, pc.m, pc.m, pc.mpa, pc.kp, reinterpret_cast<__nv_bfloat16*>(pc.sa), pc.ea, i,
              lane);
  else
    split_row(pc.bt, pc.m, pc.m, pc.m, pc.mpb, pc.kp, reinterpret_cast<__nv_bfloat16*>(pc.sb), pc.eb, i, lane);
}

// Batched transpose of slot -> bt (32 x 32 tiles; prefix over tiles per cloud).
__global__ void btranspose_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix, int count, int slot,
                                  int mask_k) {
  const int j = find_job(prefix, count, blockIdx.x);
  const PhiCloud pc = pcs[j];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  const int m = pc.m, nb = (m + 31) / 32;
  const int local = blockIdx.x - prefix[j];
  const int c0 = (local % nb) * 32, r0 = (local / nb) * 32;
  const double* B = pc_slot(pc, slot);
  __shared__ double tile[32][33];
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (r < m && c < m) ? B[(size_t)r * m + c] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;
    if (c < m && r < m) pc.bt[(size_t)c * m + r] = tile[threadIdx.x][y];
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
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[kBufs];
  uint64_t acc_empty[kBufs];
  uint32_t tmem_base;
};

// One 128 x 64 output tile (m0, n0) of C = alpha A B + beta C from the slice
// tensor maps (A: rows p M_pad + i, B^T: rows q N_pad + j; K_pad columns).
__device__ __forceinline__ void ozaki_tile(const CUtensorMap* map_a_p, const CUtensorMap* map_b_p, int M, int N,
                                           int M_pad, int N_pad, int K_pad, const int* __restrict__ ea,
                                           const int* __restrict__ eb, double alpha, double beta, double* C, int ldc,
                                           int m0, int n0, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const CUtensorMap& map_a = *map_a_p;
  const CUtensorMap& map_b = *map_b_p;
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + (base - raw_addr) + kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = K_pad / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&sm->full[s]), 1);
      mbar_init(smem_u32(&sm->empty[s]), 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(smem_u32(&sm->acc_full[b]), 1);
      mbar_init(smem_u32(&sm->acc_empty[b]), 8);  // one arrive per epilogue warp
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
      uint32_t it = 0;
      bool ok = true;
      for (int t = 2; t <= kS + 1 && ok; ++t)
        for (int p = max(1, t - kS); p <= min(kS, t - 1) && ok; ++p) {
          const int q = t - p;
          for (int kc = 0; kc < nkc; ++kc, ++it) {
            const int s = it % kStages;
            const uint32_t ph = (it / kStages) & 1u;
            if (!mbar_wait(smem_u32(&sm->empty[s]), ph ^ 1u, err, 11)) { ok = false; break; }
            const uint32_t full = smem_u32(&sm->full[s]);
            mbar_arrive_expect_tx(full, kStageBytes);
            const uint32_t sa = base + s * kStageBytes;
            tma_load_2d(sa, &map_a, kc * kBK, (p - 1) * M_pad + m0, full);
            tma_load_2d(sa + kABytes, &map_b, kc * kBK, (q - 1) * N_pad + n0, full);
          }
        }
      const uint32_t issued = it;
      for (uint32_t u = (issued > (uint32_t)kStages ? issued - kStages : 0); u < issued; ++u)
        mbar_wait(smem_u32(&sm->full[u % kStages]), (u / kStages) & 1u, err, 12);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kBM, kBN);
      uint32_t it = 0, pair = 0;
      bool ok = true;
      for (int t = 2; t <= kS + 1 && ok; ++t)
        for (int p = max(1, t - kS); p <= min(kS, t - 1) && ok; ++p, ++pair) {
          const int buf = pair % kBufs;
          const uint32_t use = pair / kBufs;
          if (!mbar_wait(smem_u32(&sm->acc_empty[buf]), (use & 1u) ^ 1u, err, 13)) { ok = false; break; }
          fence_after();
          const uint32_t d_tmem = tmem + (uint32_t)(buf * kBN);
          for (int kc = 0; kc < nkc; ++kc, ++it) {
            const int s = it % kStages;
            const uint32_t ph = (it / kStages) & 1u;
            if (!mbar_wait(smem_u32(&sm->full[s]), ph, err, 14)) { ok = false; break; }
            fence_after();
            const uint32_t sa = base + s * kStageBytes;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              mma_bf16(d_tmem, sdesc_sw128(sa + kk * 32), sdesc_sw128(sa + kABytes + kk * 32), idesc,
                       (kc > 0 || kk > 0) ? 1u : 0u);
            mma_commit(smem_u32(&sm->empty[s]));
          }
          if (!ok) break;
          mma_commit(smem_u32(&sm->acc_full[buf]));
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
    int32_t E[32];
    long long T[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) { E[c] = 0; T[c] = 0; }
    uint32_t pair = 0;
    bool ok = true;
    double* crow = C + (size_t)(gi < M ? gi : 0) * ldc;
    for (int t = 2; t <= kS + 1 && ok; ++t) {
      for (int p = max(1, t - kS); p <= min(kS, t - 1); ++p, ++pair) {
        const int buf = pair % kBufs;
        const uint32_t use = pair / kBufs;
        if (!mbar_wait(smem_u32(&sm->acc_full[buf]), use & 1u, err, 15)) { ok = false; break; }
        fence_after();
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kBN + col0), v);
#pragma unroll
        for (int c = 0; c < 32; ++c) E[c] += __float2int_rn(v[c]);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm->acc_empty[buf]));
      }
      if (!ok) break;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        T[c] = (T[c] << kBeta) + (long long)E[c];
        E[c] = 0;
      }
      if (t == 5 || t == kS + 1) {
        // T holds sum_{t' in group} E_t' 2^(7 (t - t')): value = 2^-7t T, exact in FP64 (< 2^49)
        if (gi < M) {
          const int eri = ea[gi];
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int gj = n0 + col0 + c;
            if (gj < N) {
              const double part = alpha * ldexp((double)T[c], eri + eb[gj] - kBeta * t);
              double* pc = crow + gj;
              if (t == 5)
                *pc = (beta == 0.0) ? part : fma(beta, *pc, part);
              else
                *pc += part;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 32; ++c) T[c] = 0;
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
  ozaki_tile(&map_a, &map_b, M, N, M_pad, N_pad, K_pad, ea, eb, alpha, beta, C, ldc, blockIdx.y * kBM,
             blockIdx.x * kBN, err);
}

// Batched: one CTA per OzTile of any cloud; C = slot c_slot of the cloud.
__global__ void __launch_bounds__(kThreads, 1)
ozaki_gemm_batched_kernel(const CUtensorMap* __restrict__ maps, const OzTile* __restrict__ tiles,
                          const PhiCloud* __restrict__ pcs, int c_slot, double alpha, double beta, int mask_k,
                          int* err) {
  const OzTile t = tiles[blockIdx.x];
  const PhiCloud pc = pcs[t.cloud];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  ozaki_tile(maps + pc.map_a, maps + pc.map_b, pc.m, pc.m, pc.mpa, pc.mpb, pc.kp, pc.ea, pc.eb, alpha, beta,
             pc_slot(pc, c_slot), pc.m, t.m0, t.n0, err);
}

}  // namespace

bool make_ozaki_maps(void* map_a_host, void* map_b_host, const void* sa, const void* sb, int mpa, int mpb, int kp) {
  return tc::make_map_bf16(static_cast<CUtensorMap*>(map_a_host), sa, (uint64_t)kp, (uint64_t)kS * mpa, (uint64_t)kp,
                           kBM) &&
         tc::make_map_bf16(static_cast<CUtensorMap*>(map_b_host), sb, (uint64_t)kp, (uint64_t)kS * mpb, (uint64_t)kp,
                           kBN);
}

cudaError_t launch_bgemm(const PhiCloud* pc, int count, const int* row_prefix_a, int rows_a, const int* row_prefix_b,
                         int rows_b, const int* t_prefix, int t_blocks, const OzTile* tiles, int num_tiles,
                         const void* maps_dev, int a_slot, int b_slot, int c_slot, double alpha, double beta,
                         int mask_k, int* err, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(ozaki_gemm_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  bsplit_rows_kernel<<<(rows_a * 32 + 255) / 256, 256, 0, st>>>(pc, row_prefix_a, count, 0, a_slot, mask_k);
  btranspose_kernel<<<t_blocks, dim3(32, 8), 0, st>>>(pc, t_prefix, count, b_slot, mask_k);
  bsplit_rows_kernel<<<(rows_b * 32 + 255) / 256, 256, 0, st>>>(pc, row_prefix_b, count, 1, 0, mask_k);
  count_launch(3);
  ozaki_gemm_batched_kernel<<<num_tiles, kThreads, kSmemBytes, st>>>(static_cast<const CUtensorMap*>(maps_dev), tiles,
                                                                     pc, c_slot, alpha, beta, mask_k, err);
  return launched();
}

size_t ozaki_workspace_bytes(int M, int N, int K) {
  const size_t mp = (size_t)((M + kBM - 1) / kBM) * kBM, np = (size_t)((N + kBN - 1) / kBN) * kBN;
  const size_t kp = (size_t)((K + kBK - 1) / kBK) * kBK;
  return kS * (mp + np) * kp * 2 + (mp + np) * 4 + (size_t)N * K * 8 + 4096;
}

bool ozaki_supported(int K) { return K >= 1 && K <= kMaxK && tc::sm103_available(); }

cudaError_t dgemm_ozaki(int M, int N, int K, double alpha, const double* A, int lda, const double* B, int ldb,
                        double beta, double* C, int ldc, void* work, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 1 || K > kMaxK) return cudaErrorInvalidValue;
  const int mp = (M + kBM - 1) / kBM * kBM, np = (N + kBN - 1) / kBN * kBN, kp = (K + kBK - 1) / kBK * kBK;
  uint8_t* w = static_cast<uint8_t*>(work);
  auto* sa = reinterpret_cast<__nv_bfloat16*>(w);
  w += (size_t)kS * mp * kp * 2;
  auto* sb = reinterpret_cast<__nv_bfloat16*>(w);
  w += (size_t)kS * np * kp * 2;
  int* ea = reinterpret_cast<int*>(w);
  w += (size_t)mp * 4;
  int* eb = reinterpret_cast<int*>(w);
  w += (size_t)np * 4;
  w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(w) + 255) & ~uintptr_t(255));
  double* bt = reinterpret_cast<double*>(w);
  split_rows_kernel<<<(mp * 32 + 255) / 256, 256, 0, st>>>(A, lda, M, K, mp, kp, sa, ea);
  transpose_kernel<<<dim3((N + 31) / 32, (K + 31) / 32), dim3(32, 8), 0, st>>>(B, ldb, K, N, bt);
  split_rows_kernel<<<(np * 32 + 255) / 256, 256, 0, st>>>(bt, K, N, K, np, kp, sb, eb);
  count_launch(3);
  CUtensorMap ma, mb;
  if (!tc::make_map_bf16(&ma, sa, (uint64_t)kp, (uint64_t)kS * mp, (uint64_t)kp, kBM)) return cudaErrorInvalidValue;
  if (!tc::make_map_bf16(&mb, sb, (uint64_t)kp, (uint64_t)kS * np, (uint64_t)kp, kBN)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  ozaki_gemm_kernel<<<dim3(np / kBN, mp / kBM), kThreads, kSmemBytes, st>>>(ma, mb, M, N, mp, np, kp, ea, eb, alpha,
                                                                           beta, C, ldc, err);
  return launched();
}

}  // namespace rfd
