// Step a3, BF16 tensor-core form: the reductions over N (Sec. 2.4:
// M = B^T A and Y = B^T F, "linear in N, cubic/quadratic in m") as
// BF16 x BF16 -> FP32 GEMMs on the 5th-generation tensor cores.
//
//   K[f, g]  = sum_n Psi[i0 + f][n] * Psi[j0 + g][n]     (Phi^T Phi, upper tiles)
//   Y'[f, c] = sum_n Psi[i0 + f][n] * Psi[m + c][n]      (Phi^T F)
//
// Psi (bf16, blocked: 64-point blocks holding all rows, 128 B per row per
// block, see psi_index) makes both operands K-major, and a 64-point slab of
// any rows is one contiguous span (a 3-D TMA box), whatever N.  Each
// CTA (a TcUnit) owns a pair of 128-row tiles of one cloud -- feature rows
// i0.. and i0+128.. against the same up to 256 rows of B: Gram rows j0.. and,
// on the last tile of each row block, the cpad field rows right after them in
// shared memory -- and one "lane" of that cloud's point axis: the 64-point
// blocks kb = lane, lane + L, lane + 2L, ...  Sharing the B rows between two
// 128-row halves cuts the L2->SM bytes per point by about a fifth against
// 128-row tiles, and those bytes, not the tensor pipe, set the pace.  The
// lanes of a cloud run in the same wave and walk its point axis together,
// so each 64-point slab of Psi is fetched from HBM once and served from L2 to
// every tile that needs it.  One MMA per half (N = Gram rows + field rows)
// per 16 points covers K and Y' of the tile, so B^T F costs neither an extra
// pass over Psi nor extra MMA instructions (each costs ~100 cycles to issue).
// Tensor maps live in global memory (four per cloud), so one launch can serve
// many clouds.
//
// Warp roles: warp 0 TMA producer (one lane), warp 1 TMEM allocator + MMA
// issuer (one lane), warps 2..9 epilogue (half (warp - 2) / 4, TMEM lane
// quarter warp % 4).
// Every mbarrier wait is bounded by a %globaltimer limit; a wait that runs
// out records a code in *err and the CTA unwinds (waiting, again bounded, for
// its own TMA copies) instead of hanging.
#include <cuda_runtime.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdint>
#include "kernels.h"
#include "tc_common.cuh"

namespace rfd {

namespace {

using namespace tc;

constexpr int kMaxStages = 8;
constexpr int kABytes = kTcBM * kTcBK * 2;          // 16 KB per 128-row A box
constexpr int kBBytes = kTcBNMax * kTcBK * 2;       // 32 KB: Gram rows then field rows, <= 256 in all
constexpr int kThreads = 320;                       // producer, MMA, 8 epilogue warps (4 per half)
constexpr uint32_t kTmemCols = 512;  // half 0 at columns [0, 256), half 1 at [256, 512); in each, the
                                     // Gram part first and the field part right after it
constexpr int kSmemLimit = 232448;                  // opt-in shared memory per CTA on sm_103
constexpr int kSmemExtra = 1024 + 256;              // alignment slack + barriers

struct Smem {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t acc_full;
  uint32_t tmem_base;
};

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// v[0..n) -> out[0..n) (n = 16 or 32), added to what is there when accumulate
template <int n>
__device__ __forceinline__ void store_cols(float* out, const float* v, bool accumulate) {
#pragma unroll
  for (int q = 0; q < n / 4; ++q) {
    float4* o = reinterpret_cast<float4*>(out + 4 * q);
    float4 w = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    if (accumulate) {
      const float4 old = *o;
      w.x += old.x;
      w.y += old.y;
      w.z += old.z;
      w.w += old.w;
    }
    *o = w;
  }
}

__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(const CUtensorMap* __restrict__ maps, const TcUnit* __restrict__ units, int stages, int stage_bytes,
               int b_off, int kb0, int kb_len, int* err, unsigned long long* prof) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + (base - raw_addr) + stages * stage_bytes);
  const TcUnit u = units[blockIdx.x];
  const CUtensorMap* map_a = maps + u.map;
  const CUtensorMap* map_b = maps + u.map + 1;    // 64-row box
  const CUtensorMap* map_f = maps + u.map + 2;
  const CUtensorMap* map_b16 = maps + u.map + 5;  // 16-row box
  const bool has_f = u.has_f != 0;
  const bool two = u.out1 != nullptr;  // rows i0 + 128 .. i0 + 255 as well
  // this launch's phase of the point axis: blocks kb in [kb0, kb1) with kb = lane (mod nlanes)
  const int kb1 = min(kb0 + kb_len, u.kb_total);
  const int kb_first = kb0 + ((u.lane - kb0 % u.nlanes) + u.nlanes) % u.nlanes;
  const int count = (kb_first < kb1) ? (kb1 - kb_first + u.nlanes - 1) / u.nlanes : 0;
  const bool accumulate = kb0 > 0;  // later phases add to the lane's partial

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&sm->full[s]), 1);
      mbar_init(smem_u32(&sm->empty[s]), 1);
    }
    mbar_init(smem_u32(&sm->acc_full), 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(&sm->tmem_base), kTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;
  const unsigned long long t_start = (prof && threadIdx.x == 0) ? globaltimer() : 0ull;
  // B rows: 64-row boxes while they fit (m >= 64), then 16-row boxes (min(16, m) rows each)
  const int b64 = (u.b_rows >= 64) ? u.nj_mma / 64 : 0;
  const int b16_rows = u.b_rows < 16 ? u.b_rows : 16;
  const int b16 = (u.nj_mma - b64 * 64) / 16;
  const int fw = has_f ? u.cpad : 0;
  const int n0 = u.nj_mma + fw;             // half 0: one MMA covers the Gram and field rows
  const int n1 = two ? n0 - u.skip1 : 0;    // half 1 starts skip1 rows into B
  const uint32_t tx_bytes = ((two ? 2 : 1) * u.a_rows + b64 * 64 + b16 * b16_rows + fw) * kTcBK * 2;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int i = 0;
      for (; i < count; ++i) {
        const int s = i % stages;
        const uint32_t ph = (uint32_t)(i / stages) & 1u;
        if (!mbar_wait(smem_u32(&sm->empty[s]), ph ^ 1u, err, 1)) break;
        const uint32_t full = smem_u32(&sm->full[s]);
        mbar_arrive_expect_tx(full, tx_bytes);
        const uint32_t sa = base + s * stage_bytes;
        const int32_t kb = kb_first + i * u.nlanes;  // 64-point block of the blocked Psi
        tma_load_3d(sa, map_a, 0, u.i0, kb, full);
        if (two) tma_load_3d(sa + kABytes, map_a, 0, u.i0 + kTcBM, kb, full);
        const uint32_t sb = sa + b_off;
        for (int q = 0; q < b64; ++q) tma_load_3d(sb + q * 64 * 128, map_b, 0, u.j0 + q * 64, kb, full);
        for (int q = 0; q < b16; ++q)
          tma_load_3d(sb + (b64 * 64 + q * 16) * 128, map_b16, 0, u.j0 + b64 * 64 + q * 16, kb, full);
        if (has_f) tma_load_3d(sb + u.nj_mma * 128, map_f, 0, 0, kb, full);  // the F map starts at Psi row m
      }
      // drain: our copies into the last stages must land before the CTA exits
      for (int t = (i > stages ? i - stages : 0); t < i; ++t)
        mbar_wait(smem_u32(&sm->full[t % stages]), (uint32_t)(t / stages) & 1u, err, 2);
    }
  } else if (warp == 1) {
    if (lane == 0 && count > 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc0 = idesc_bf16(kTcBM, n0);
      const uint32_t idesc1 = idesc_bf16(kTcBM, n1 > 0 ? n1 : 16);
      bool ok = true;
      for (int i = 0; i < count; ++i) {
        const int s = i % stages;
        const uint32_t ph = (uint32_t)(i / stages) & 1u;
        if (!mbar_wait(smem_u32(&sm->full[s]), ph, err, 4)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t sa = base + s * stage_bytes, sb = sa + b_off;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 16; ++kk) {
          const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
          mma_bf16(tmem, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc0, acc);
          if (n1 > 0)
            mma_bf16(tmem + kTcBNMax, sdesc_sw128(sa + kABytes + kk * 32),
                     sdesc_sw128(sb + u.skip1 * 128 + kk * 32), idesc1, acc);
        }
        mma_commit(smem_u32(&sm->empty[s]));  // frees the stage when these MMAs finish
      }
      if (ok) mma_commit(smem_u32(&sm->acc_full));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2..9: half = (warp - 2) / 4) ----------------
    const int quarter = warp & 3;         // TMEM lanes 32*quarter .. +31
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;  // tile row (feature f - i0 - 128 * half)
    const int nh = half ? n1 : n0;
    if (half == 0 || n1 > 0) {
      float* out = (half ? u.out1 : u.out) + (size_t)row * kTcLd;
      const bool ready = (count > 0) && mbar_wait(smem_u32(&sm->acc_full), 0u, err, 5);
      if (ready) fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * kTcBNMax);
      auto drain = [&](int tcol0, int col0, int ncols) {  // TMEM columns tcol0.. -> partial columns col0..
        if (!ready && accumulate) return;  // nothing in this phase: the partial stands
        for (int c0 = 0; c0 < ncols; c0 += 32) {
          float v[32];
          const bool wide = c0 + 32 <= ncols;  // ncols is a multiple of 16
          if (ready) {
            if (wide)
              tmem_ld32(taddr + (uint32_t)(tcol0 + c0), v);
            else
              tmem_ld16(taddr + (uint32_t)(tcol0 + c0), v);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = 0.f;  // no point blocks in this lane: a zero partial
          }
          if (wide)
            store_cols<32>(out + col0 + c0, v, accumulate);
          else
            store_cols<16>(out + col0 + c0, v, accumulate);
        }
      };
      const int ng = nh - fw;  // Gram columns of this half
      if (ng > 0) drain(0, 0, ng);
      if (has_f) drain(ng, kTcBNMax, fw);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (prof && threadIdx.x == 0) {
    prof[2 * blockIdx.x] = t_start;
    prof[2 * blockIdx.x + 1] = globaltimer();
  }
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

bool tc_gram_supported() { return tc::sm103_available(); }

bool make_gram_maps(void* maps_host3, void* map_b16, void* maps_pair2, const void* psi, int64_t n_pad, int m,
                    int cpad, int rows_alloc) {
  auto* maps = static_cast<CUtensorMap*>(maps_host3);
  const uint32_t a_rows = (uint32_t)(m < kTcBM ? m : kTcBM);
  const uint32_t b_rows = (uint32_t)(m < 64 ? m : 64);
  const uint32_t b16_rows = (uint32_t)(m < 16 ? m : 16);
  const auto* p = static_cast<const uint16_t*>(psi);
  const uint64_t nb = (uint64_t)(n_pad / 64), ra = (uint64_t)rows_alloc;
  return make_map_bf16_blocked(&maps[0], p, (uint64_t)m, ra, nb, a_rows) &&
         make_map_bf16_blocked(&maps[1], p, (uint64_t)m, ra, nb, b_rows) &&
         make_map_bf16_blocked(&maps[2], p + (size_t)m * 64, (uint64_t)cpad, ra, nb, (uint32_t)cpad) &&
         make_map_bf16_blocked(static_cast<CUtensorMap*>(map_b16), p, (uint64_t)m, ra, nb, b16_rows) &&
         make_map_bf16_blocked(static_cast<CUtensorMap*>(maps_pair2), p, (uint64_t)m, ra, nb, m < 8 ? m : 8) &&
         make_map_bf16_blocked(static_cast<CUtensorMap*>(maps_pair2) + 1, p + (size_t)m * 64, (uint64_t)cpad, ra, nb,
                               (uint32_t)(cpad / 2));
}

cudaError_t gram_tc_prepare() {
  static const cudaError_t attr =  // once per process (thread-safe initialisation)
      cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
  return attr;
}

cudaError_t launch_gram_tc_phase(const void* maps_dev, const TcUnit* units, int num_units, int a_boxes, int kb0,
                                 int phase_blocks, int* err, cudaStream_t st, unsigned long long* prof) {
  if (num_units <= 0) return cudaSuccess;
  if (a_boxes < 1 || a_boxes > 2 || phase_blocks < 1) return cudaErrorInvalidValue;
  const int b_off = a_boxes * kABytes;
  const int stage_bytes = b_off + kBBytes;  // multiples of 1024 (the 128-byte swizzle's atom)
  int stages = (kSmemLimit - kSmemExtra) / stage_bytes;
  if (stages > kMaxStages) stages = kMaxStages;
  if (stages < 2) return cudaErrorInvalidValue;
  const int smem = stages * stage_bytes + kSmemExtra;
  const cudaError_t attr = gram_tc_prepare();
  if (attr != cudaSuccess) return attr;
  gram_tc_kernel<<<num_units, kThreads, smem, st>>>(static_cast<const CUtensorMap*>(maps_dev), units, stages,
                                                    stage_bytes, b_off, kb0, phase_blocks, err, prof);
  return launched();
}

cudaError_t launch_gram_tc(const void* maps_dev, const TcUnit* units, int num_units, int a_boxes, int max_kb,
                           int phase_blocks, int* err, cudaStream_t st) {
  if (num_units <= 0) return cudaSuccess;
  // the point axis in phases of phase_blocks 64-point blocks, one launch each, so that the
  // lanes of a tile restart in step (and the slab they share stays in L2) every phase
  if (phase_blocks < 1) phase_blocks = kGramPhaseBlocks;
  const int phases = max_kb > 0 ? (max_kb + phase_blocks - 1) / phase_blocks : 1;
  for (int ph = 0; ph < phases; ++ph) {
    const cudaError_t e = launch_gram_tc_phase(maps_dev, units, num_units, a_boxes, ph * phase_blocks, phase_blocks,
                                               err, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace rfd
