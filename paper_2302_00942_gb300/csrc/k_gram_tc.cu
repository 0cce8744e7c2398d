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
// CTA (a TcUnit) owns one tile of one cloud -- 128 feature rows against up to
// 256 rows of B: Gram rows j0.. and, on the last tile of each row block, the
// cpad field rows right after them in shared memory -- and one "lane" of that
// cloud's point axis: the 64-point blocks kb = lane, lane + L, lane + 2L, ...
// The lanes of a cloud run in the same wave and walk its point axis together,
// so each 64-point slab of Psi is fetched from HBM once and served from L2 to
// every tile that needs it.  One MMA (N = Gram rows + field rows) per 16
// points covers K and Y' of the tile, so B^T F costs neither an extra pass
// over Psi nor extra MMA instructions (each costs ~100 cycles to issue).
// Tensor maps live in global memory (four per cloud), so one launch can serve
// many clouds.
//
// Warp roles: warp 0 TMA producer (one lane), warp 1 TMEM allocator + MMA
// issuer (one lane), warps 2..5 epilogue (TMEM lane quarter = warp % 4).
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
constexpr int kABytes = kTcBM * kTcBK * 2;          // 16 KB
constexpr int kBBytes = kTcBNMax * kTcBK * 2;       // 32 KB: Gram rows then field rows, <= 256 in all
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;  // Gram part [0, nj_mma), field part [nj_mma, nj_mma + cpad); the
                                     // epilogue reads whole 32-column chunks, past column 256
constexpr int kSmemLimit = 232448;                  // opt-in shared memory per CTA on sm_103
constexpr int kSmemExtra = 1024 + 256;              // alignment slack + barriers

struct Smem {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t acc_full;
  uint32_t tmem_base;
};

__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(const CUtensorMap* __restrict__ maps, const TcUnit* __restrict__ units, int stages, int stage_bytes,
               int kb0, int kb_len, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + (base - raw_addr) + stages * stage_bytes);
  const TcUnit u = units[blockIdx.x];
  const CUtensorMap* map_a = maps + u.map;
  const CUtensorMap* map_b = maps + u.map + 1;    // 64-row box
  const CUtensorMap* map_f = maps + u.map + 2;
  const CUtensorMap* map_b16 = maps + u.map + 5;  // 16-row box
  const bool has_g = u.nj_mma > 0, has_f = u.has_f != 0;
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
  // B rows: 64-row boxes while they fit (m >= 64), then 16-row boxes (min(16, m) rows each)
  const int b64 = (u.b_rows >= 64) ? u.nj_mma / 64 : 0;
  const int b16_rows = u.b_rows < 16 ? u.b_rows : 16;
  const int b16 = (u.nj_mma - b64 * 64) / 16;
  const int n_mma = u.nj_mma + (has_f ? u.cpad : 0);  // one MMA covers the Gram and field rows
  const uint32_t tx_bytes = (u.a_rows + b64 * 64 + b16 * b16_rows + (has_f ? u.cpad : 0)) * kTcBK * 2;

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
        const uint32_t sb = sa + kABytes;
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
      const uint32_t idesc = idesc_bf16(kTcBM, n_mma);
      bool ok = true;
      for (int i = 0; i < count; ++i) {
        const int s = i % stages;
        const uint32_t ph = (uint32_t)(i / stages) & 1u;
        if (!mbar_wait(smem_u32(&sm->full[s]), ph, err, 4)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t sa = base + s * stage_bytes;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 16; ++kk)
          mma_bf16(tmem, sdesc_sw128(sa + kk * 32), sdesc_sw128(sa + kABytes + kk * 32), idesc,
                   (i > 0 || kk > 0) ? 1u : 0u);
        mma_commit(smem_u32(&sm->empty[s]));  // frees the stage when these MMAs finish
      }
      if (ok) mma_commit(smem_u32(&sm->acc_full));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quarter = warp & 3;         // TMEM lanes 32*quarter .. +31
    const int row = quarter * 32 + lane;  // tile row (feature f - i0)
    float* out = u.out + (size_t)row * kTcLd;
    const bool ready = (count > 0) && mbar_wait(smem_u32(&sm->acc_full), 0u, err, 5);
    if (ready) fence_after();
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
    auto drain = [&](int tcol0, int col0, int ncols) {  // TMEM columns tcol0.. -> partial columns col0..
      if (!ready && accumulate) return;  // nothing in this phase: the partial stands
      for (int c0 = 0; c0 < ncols; c0 += 32) {
        float v[32];
        if (ready) {
          tmem_ld32(taddr + (uint32_t)(tcol0 + c0), v);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0.f;  // no point blocks in this lane: a zero partial
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4* o = reinterpret_cast<float4*>(out + col0 + c0 + 4 * q);
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
    };
    if (has_g) drain(0, 0, u.nj_mma);
    if (has_f) drain(u.nj_mma, kTcBNMax, u.cpad);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

int stage_bytes_for(int) { return (kABytes + kBBytes + 1023) / 1024 * 1024; }

}  // namespace

bool tc_gram_supported() { return tc::sm103_available(); }

bool make_gram_maps(void* maps_host3, void* map_b16, const void* psi, int64_t n_pad, int m, int cpad,
                    int rows_alloc) {
  auto* maps = static_cast<CUtensorMap*>(maps_host3);
  const uint32_t a_rows = (uint32_t)(m < kTcBM ? m : kTcBM);
  const uint32_t b_rows = (uint32_t)(m < 64 ? m : 64);
  const uint32_t b16_rows = (uint32_t)(m < 16 ? m : 16);
  const auto* p = static_cast<const uint16_t*>(psi);
  const uint64_t nb = (uint64_t)(n_pad / 64), ra = (uint64_t)rows_alloc;
  return make_map_bf16_blocked(&maps[0], p, (uint64_t)m, ra, nb, a_rows) &&
         make_map_bf16_blocked(&maps[1], p, (uint64_t)m, ra, nb, b_rows) &&
         make_map_bf16_blocked(&maps[2], p + (size_t)m * 64, (uint64_t)cpad, ra, nb, (uint32_t)cpad) &&
         make_map_bf16_blocked(static_cast<CUtensorMap*>(map_b16), p, (uint64_t)m, ra, nb, b16_rows);
}

cudaError_t gram_tc_prepare() {
  static const cudaError_t attr =  // once per process (thread-safe initialisation)
      cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
  return attr;
}

cudaError_t launch_gram_tc(const void* maps_dev, const TcUnit* units, int num_units, int max_cpad, int max_kb,
                           int phase_blocks, int* err, cudaStream_t st) {
  if (num_units <= 0) return cudaSuccess;
  if (max_cpad < 16 || max_cpad > 256) return cudaErrorInvalidValue;
  const int stage_bytes = stage_bytes_for(max_cpad);
  int stages = (kSmemLimit - kSmemExtra) / stage_bytes;
  if (stages > kMaxStages) stages = kMaxStages;
  if (stages < 2) return cudaErrorInvalidValue;
  const int smem = stages * stage_bytes + kSmemExtra;
  const cudaError_t attr = gram_tc_prepare();
  if (attr != cudaSuccess) return attr;
  // the point axis in phases of phase_blocks 64-point blocks, one launch each, so that the
  // lanes of a tile restart in step (and the slab they share stays in L2) every phase
  if (phase_blocks < 1) phase_blocks = kGramPhaseBlocks;
  const int phases = max_kb > 0 ? (max_kb + phase_blocks - 1) / phase_blocks : 1;
  for (int ph = 0; ph < phases; ++ph) {
    gram_tc_kernel<<<num_units, kThreads, smem, st>>>(static_cast<const CUtensorMap*>(maps_dev), units, stages,
                                                      stage_bytes, ph * phase_blocks, phase_blocks, err);
    const cudaError_t e = launched();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace rfd
