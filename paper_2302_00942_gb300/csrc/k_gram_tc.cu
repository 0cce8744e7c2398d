// Step a3, BF16 tensor-core form: the reductions over N (Sec. 2.4:
// M = B^T A and Y = B^T F, "linear in N, cubic/quadratic in m") as
// BF16 x BF16 -> FP32 GEMMs on the 5th-generation tensor cores.
//
//   K[f, g]  = sum_n Psi[i0 + f][n] * Psi[j0 + g][n]     (Phi^T Phi, upper tiles)
//   Y'[f, c] = sum_n Psi[i0 + f][n] * Psi[m + c][n]      (Phi^T F)
//
// Psi (bf16, feature-major: n contiguous) makes both operands K-major.  Each
// work unit is a 128 x N tile (N <= 256) over a point range; TMA brings
// 128 x 64 (A) and N x 64 (B) slabs into shared memory with the 128-byte
// swizzle, one elected thread issues tcgen05.mma (M = 128, K = 16 per
// instruction, FP32 accumulators in TMEM), and four epilogue warps drain TMEM
// with tcgen05.ld into the unit's FP32 partial tile.
//
// Persistent CTAs (one per SM) walk the unit list round-robin.  Warp roles:
//   warp 0      TMA producer (one lane)
//   warp 1      TMEM allocator + MMA issuer (one lane)
//   warps 2..5  epilogue (TMEM lane quarter = warp % 4)
// Two 256-column TMEM accumulators let the epilogue of unit u overlap the
// MMAs of unit u + 1.  Every mbarrier wait is bounded by a %globaltimer
// limit; a wait that runs out records a code in *err and the CTA unwinds
// (waiting, again bounded, for its own TMA copies) instead of hanging.
#include <cuda_runtime.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdint>
#include "kernels.h"
#include "tc_common.cuh"

namespace rfd {

namespace {

constexpr int kStages = 4;
constexpr int kABytes = kTcBM * kTcBK * 2;          // 16 KB
constexpr int kBBytesMax = kTcBNMax * kTcBK * 2;    // 32 KB
constexpr int kStageBytes = kABytes + kBBytesMax;   // 48 KB
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;                 // 2 accumulators x 256 columns
using namespace tc;

struct Smem {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint32_t tmem_base;
};

__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap map_a,   // Phi rows, box 64 x 128
               const __grid_constant__ CUtensorMap map_b,   // Phi rows, box 64 x 256
               const __grid_constant__ CUtensorMap map_f,   // F rows,   box 64 x cpad
               const GramUnit* __restrict__ units, int num_units, int cpad, int a_rows_box,
               int b_rows_box, float* __restrict__ partials, int* err) {
  extern __shared__ uint8_t smem_raw[];
  // stage buffers 1024-aligned (the 128-byte swizzle atom); bookkeeping after them
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  uint8_t* base_ptr = smem_raw + (base - raw_addr);
  Smem* sm = reinterpret_cast<Smem*>(base_ptr + kStages * kStageBytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&sm->full[s]), 1);
      mbar_init(smem_u32(&sm->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sm->acc_full[b]), 1);
      mbar_init(smem_u32(&sm->acc_empty[b]), 4);  // one arrive per epilogue warp
    }
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(&sm->tmem_base), kTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;
  const int a_bytes = a_rows_box * kTcBK * 2;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      uint32_t kb = 0;  // global k-block counter (stage ring position)
      bool ok = true;
      for (int ui = blockIdx.x; ui < num_units && ok; ui += gridDim.x) {
        const GramUnit u = units[ui];
        const bool field = (u.kind == kTileField);
        const int b_bytes = (field ? cpad : b_rows_box) * kTcBK * 2;
        for (int64_t k = u.k0; k < u.k1; k += kTcBK, ++kb) {
          const int s = kb % kStages;
          const uint32_t ph = (kb / kStages) & 1u;
          if (!mbar_wait(smem_u32(&sm->empty[s]), ph ^ 1u, err, 1)) { ok = false; break; }
          const uint32_t full = smem_u32(&sm->full[s]);
          mbar_arrive_expect_tx(full, a_bytes + b_bytes);
          const uint32_t sa = base + s * kStageBytes;
          tma_load_2d(sa, &map_a, (int32_t)k, u.i0, full);
          if (field)
            tma_load_2d(sa + kABytes, &map_f, (int32_t)k, 0, full);  // the F map starts at Psi row m
          else
            tma_load_2d(sa + kABytes, &map_b, (int32_t)k, u.j0, full);
        }
      }
      // drain: our copies into the last stages must land before the CTA exits
      const uint32_t issued = kb;
      for (uint32_t t = (issued > (uint32_t)kStages ? issued - kStages : 0); t < issued; ++t)
        mbar_wait(smem_u32(&sm->full[t % kStages]), (t / kStages) & 1u, err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      uint32_t kb = 0;
      int local = 0;
      bool ok = true;
      for (int ui = blockIdx.x; ui < num_units && ok; ui += gridDim.x, ++local) {
        const GramUnit u = units[ui];
        const int buf = local & 1;
        const uint32_t use = (uint32_t)(local >> 1);
        if (!mbar_wait(smem_u32(&sm->acc_empty[buf]), (use & 1u) ^ 1u, err, 3)) { ok = false; break; }
        fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(buf * kTcBNMax);
        const uint32_t idesc = idesc_bf16(kTcBM, u.nj_mma);
        uint32_t accumulate = 0;
        for (int64_t k = u.k0; k < u.k1; k += kTcBK, ++kb) {
          const int s = kb % kStages;
          const uint32_t ph = (kb / kStages) & 1u;
          if (!mbar_wait(smem_u32(&sm->full[s]), ph, err, 4)) { ok = false; break; }
          fence_after();
          const uint32_t sa = base + s * kStageBytes;
#pragma unroll
          for (int kk = 0; kk < kTcBK / 16; ++kk) {
            const uint64_t da = sdesc_sw128(sa + kk * 32);
            const uint64_t db = sdesc_sw128(sa + kABytes + kk * 32);
            mma_bf16(d_tmem, da, db, idesc, accumulate);
            accumulate = 1;
          }
          mma_commit(smem_u32(&sm->empty[s]));  // frees the stage when these MMAs finish
        }
        if (!ok) break;
        mma_commit(smem_u32(&sm->acc_full[buf]));  // accumulator ready for the epilogue
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;           // TMEM lanes 32*quarter .. +31
    const int row = quarter * 32 + lane;    // tile row (feature f - i0)
    int local = 0;
    for (int ui = blockIdx.x; ui < num_units; ui += gridDim.x, ++local) {
      const GramUnit u = units[ui];
      const int buf = local & 1;
      const uint32_t use = (uint32_t)(local >> 1);
      if (!mbar_wait(smem_u32(&sm->acc_full[buf]), use & 1u, err, 5)) break;
      fence_after();
      float* out = partials + u.out + (size_t)row * kTcBNMax;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kTcBNMax);
      for (int c0 = 0; c0 < u.nj_mma; c0 += 32) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)c0, v);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(out + c0 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sm->acc_empty[buf]));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

bool make_map(CUtensorMap* map, const void* base, uint64_t n_pad, uint64_t rows, uint32_t box_rows) {
  return make_map_bf16(map, base, n_pad, rows, n_pad, box_rows);
}

}  // namespace

bool tc_gram_supported() { return tc::sm103_available(); }

cudaError_t launch_gram_tc(const TcGramArgs& a, int grid, cudaStream_t st) {
  if (a.num_units <= 0) return cudaSuccess;
  if (a.cpad < 16 || a.cpad > 256 || (a.cpad % 16) || (a.n_pad % kTcBK)) return cudaErrorInvalidValue;
  CUtensorMap ma, mb, mf;
  const uint32_t a_rows = (uint32_t)(a.m < kTcBM ? a.m : kTcBM);
  const uint32_t b_rows = (uint32_t)(a.m < kTcBNMax ? a.m : kTcBNMax);
  const auto* psi = static_cast<const uint16_t*>(a.psi);
  if (!make_map(&ma, psi, (uint64_t)a.n_pad, (uint64_t)a.m, a_rows)) return cudaErrorInvalidValue;
  if (!make_map(&mb, psi, (uint64_t)a.n_pad, (uint64_t)a.m, b_rows)) return cudaErrorInvalidValue;
  if (!make_map(&mf, psi + (size_t)a.m * a.n_pad, (uint64_t)a.n_pad, (uint64_t)a.cpad, (uint32_t)a.cpad))
    return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (grid > a.num_units) grid = a.num_units;
  gram_tc_kernel<<<grid, kThreads, kSmemBytes, st>>>(ma, mb, mf, a.units, a.num_units, a.cpad, (int)a_rows,
                                                     (int)b_rows, a.partials, a.err);
  return launched();
}

}  // namespace rfd
