// Step a3, BF16 tensor-core form on CTA pairs (m >= 512): the reductions over
// N (Sec. 2.4: M = B^T A and Y = B^T F, "linear in N, cubic/quadratic in m")
// with the 2-SM MMA, tcgen05.mma.cta_group::2.
//
//   K[f, g]  = sum_n Psi[f][n] Psi[g][n]        (Phi^T Phi, upper tiles)
//   Y'[f, c] = sum_n Psi[f][n] Psi[m + c][n]    (Phi^T F)
//
// A pair tile covers 512 feature rows r0 .. r0 + 511 (two row blocks S0 =
// r0 .., S1 = r0 + 256 ..) against nc <= 256 columns c0 .. c0 + nc - 1 of the
// upper triangle.  The even CTA of the pair issues, per 16 points, one M = 256
// MMA for S0 (its rows r0 .. +127 and the odd CTA's r0 + 128 .. +255) and one
// for S1, both against the same nc columns of B, half of which (nc / 2 rows)
// each CTA loads.  Per SM and 64-point block that is 256 A rows + nc / 2 B
// rows for 256 x nc outputs, where one CTA computing 256 x nc alone loads
// 256 + nc rows: at nc = 256, a quarter fewer bytes per MMA, and the load of
// a stage, not the tensor pipe, is what sets the pace of these reductions.
// The first column tile of each 512-row block (c0 = r0) has no S1 part (it
// lies below the diagonal); its TMEM columns 256.. take the field MMAs instead:
// S0 x F and S1 x F (N = cpad, half of the field rows from each CTA).
//
// Lanes, phases and partials work as in the one-SM kernel (k_gram_tc.cu): a
// pair unit owns one lane of the point axis (64-point blocks kb = lane,
// lane + L, ...) within the launch's phase; each CTA writes the 128-row
// logical halves it holds in TMEM (S0 and S1 rows 128 rank ..) to its lane's
// FP32 partials, adding to them in later phases.
//
// Warp roles: warp 0 TMA producer (one lane, each CTA loads its own halves);
// warp 1 of the even CTA issues the MMAs; warps 2..9 epilogue (TMEM lane
// quarter warp % 4; warps 2..5 the columns 0.., warps 6..9 the columns
// 256..).  The CTAs meet on barriers without a forwarding thread:
//   full[s]  (even CTA) expects both CTAs' bytes of stage s: the even CTA's
//            loads complete on it locally, the odd CTA's loads (the
//            cta_group::2 form of the TMA load) complete on it remotely;
//   empty[s] (each CTA) gets one commit of the even CTA's MMAs of stage s,
//            one commit per CTA (a plain commit to each address, no multicast);
//   acc_full (each CTA) likewise, after the last stage.
// Every wait is bounded by a %globaltimer limit; a wait that runs out records
// a code in *err and the CTA unwinds; both CTAs meet at a cluster barrier
// before the pair frees its TMEM, so no CTA leaves while its peer may still
// address it.
#include <cuda_runtime.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdint>
#include "kernels.h"
#include "tc_common.cuh"

namespace rfd {

namespace {

using namespace tc;

constexpr int kThreads = 320;
constexpr int kMaxStages = 6;
constexpr int kABox = kTcBM * kTcBK * 2;  // 16 KB: 128 rows of 64 points
constexpr int kSmemLimit = 232448;        // opt-in shared memory per CTA on sm_103
constexpr int kSmemExtra = 1024 + 512;    // alignment slack + barriers
constexpr uint32_t kTmemCols = 512;

struct Smem {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t acc_full;
  uint32_t tmem_base;
};

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
gram_pair_kernel(const CUtensorMap* __restrict__ maps, const PairUnit* __restrict__ units, int stages,
                 int stage_bytes, int kb0, int kb_len, int* err, unsigned long long* prof) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;  // the same offset in both CTAs of the pair
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + (base - raw_addr) + stages * stage_bytes);
  const uint32_t rank = cluster_ctarank();
  const PairUnit u = units[blockIdx.x >> 1];
  const CUtensorMap* map_a = maps + u.map;        // 128-row box
  const CUtensorMap* map_b64 = maps + u.map + 1;  // 64-row box
  const CUtensorMap* map_b16 = maps + u.map + 5;  // 16-row box
  const CUtensorMap* map_b8 = maps + u.map + 6;   // 8-row box
  const CUtensorMap* map_fh = maps + u.map + 7;   // the field rows, box cpad / 2 rows
  const bool has_f = u.has_f != 0, g2 = u.g2 != 0, a1 = u.a1 != 0;
  const int nh = u.nc / 2, fh = has_f ? u.cpad / 2 : 0;  // B and F rows this CTA loads
  // this CTA's A rows: S0 at r0 + 128 rank, S1 at r0 + 256 + 128 rank (loads of rows >= m are skipped:
  // those TMEM lanes then hold rows the reduction never reads)
  const int ra0 = u.r0 + kTcBM * (int)rank, ra1 = ra0 + 2 * kTcBM;
  const bool load_a0 = ra0 < u.m, load_a1 = a1 && ra1 < u.m;
  const uint32_t off_a1 = kABox, off_b = a1 ? 2 * kABox : kABox, off_f = off_b + (uint32_t)nh * 128;
  // bytes of a stage, both CTAs (the even CTA's full barrier expects them all)
  auto rows_of = [&](int rk) {
    const int r0a = u.r0 + kTcBM * rk, r1a = r0a + 2 * kTcBM;
    return (r0a < u.m ? kTcBM : 0) + ((a1 && r1a < u.m) ? kTcBM : 0) + nh + fh;
  };
  const uint32_t tx_pair = (uint32_t)(rows_of(0) + rows_of(1)) * kTcBK * 2;
  // this launch's phase of the point axis: blocks kb in [kb0, kb1) with kb = lane (mod nlanes)
  const int kb1 = min(kb0 + kb_len, u.kb_total);
  const int kb_first = kb0 + ((u.lane - kb0 % u.nlanes) + u.nlanes) % u.nlanes;
  const int count = (kb_first < kb1) ? (kb1 - kb_first + u.nlanes - 1) / u.nlanes : 0;
  const bool accumulate = kb0 > 0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&sm->full[s]), 1);
      mbar_init(smem_u32(&sm->empty[s]), 1);
    }
    mbar_init(smem_u32(&sm->acc_full), 1);
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc_pair(smem_u32(&sm->tmem_base), kTmemCols);
  fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers exist and the pair's TMEM is allocated before any remote arrival
  fence_after();
  const uint32_t tmem = sm->tmem_base;
  const unsigned long long t_start = (prof && threadIdx.x == 0) ? globaltimer() : 0ull;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (each CTA its own halves) ----------------
      int i = 0;
      for (; i < count; ++i) {
        const int s = i % stages;
        const uint32_t ph = (uint32_t)(i / stages) & 1u;
        if (!mbar_wait_cluster(smem_u32(&sm->empty[s]), ph ^ 1u, err, 41)) break;
        // every load of the stage completes on the even CTA's full[s]
        const uint32_t full = rank == 0 ? smem_u32(&sm->full[s]) : mapa_shared(smem_u32(&sm->full[s]), 0);
        if (rank == 0) mbar_arrive_expect_tx(full, tx_pair);
        const uint32_t sa = base + s * stage_bytes;
        const int32_t kb = kb_first + i * u.nlanes;
        if (load_a0) tma_load_3d_pair(sa, map_a, 0, ra0, kb, full);
        if (load_a1) tma_load_3d_pair(sa + off_a1, map_a, 0, ra1, kb, full);
        const uint32_t sb = sa + off_b;
        const int b0 = u.c0 + (int)rank * nh;
        int r = 0;
        for (; r + 64 <= nh; r += 64) tma_load_3d_pair(sb + r * 128, map_b64, 0, b0 + r, kb, full);
        for (; r + 16 <= nh; r += 16) tma_load_3d_pair(sb + r * 128, map_b16, 0, b0 + r, kb, full);
        for (; r + 8 <= nh; r += 8) tma_load_3d_pair(sb + r * 128, map_b8, 0, b0 + r, kb, full);
        if (has_f) tma_load_3d_pair(sa + off_f, map_fh, 0, (int)rank * fh, kb, full);
      }
      // drain: the copies into the last stages land (both CTAs' bytes count on the even
      // CTA's full barriers) before the even CTA can leave; the odd CTA waits for its
      // stages to be released, which needs its copies
      for (int t = (i > stages ? i - stages : 0); t < i; ++t) {
        const uint32_t pt = (uint32_t)(t / stages) & 1u;
        if (rank == 0)
          mbar_wait_cluster(smem_u32(&sm->full[t % stages]), pt, err, 42);
        else
          mbar_wait_cluster(smem_u32(&sm->empty[t % stages]), pt, err, 46);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && count > 0 && rank == 0) {
      // ---------------- MMA issuer (even CTA) ----------------
      const uint32_t idesc_g = idesc_bf16(2 * kTcBM, u.nc);
      const uint32_t idesc_f = idesc_bf16(2 * kTcBM, has_f ? u.cpad : 16);
      bool ok = true;
      for (int i = 0; i < count; ++i) {
        const int s = i % stages;
        const uint32_t ph = (uint32_t)(i / stages) & 1u;
        if (!mbar_wait_cluster(smem_u32(&sm->full[s]), ph, err, 43)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t sa = base + s * stage_bytes;
#pragma unroll
        for (int kk = 0; kk < kTcBK / 16; ++kk) {
          const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
          const uint64_t da0 = sdesc_sw128(sa + kk * 32), da1 = sdesc_sw128(sa + off_a1 + kk * 32);
          mma_bf16_pair(tmem, da0, sdesc_sw128(sa + off_b + kk * 32), idesc_g, acc);
          if (g2) mma_bf16_pair(tmem + 256, da1, sdesc_sw128(sa + off_b + kk * 32), idesc_g, acc);
          if (has_f) {
            const uint64_t df = sdesc_sw128(sa + off_f + kk * 32);
            mma_bf16_pair(tmem + 256, da0, df, idesc_f, acc);
            if (a1) mma_bf16_pair(tmem + 256 + (uint32_t)u.cpad, da1, df, idesc_f, acc);
          }
        }
        // stage s is free in both CTAs once these MMAs finish
        mma_commit_pair(smem_u32(&sm->empty[s]));
        mma_commit_pair(mapa_shared(smem_u32(&sm->empty[s]), 1));
      }
      if (ok) {
        mma_commit_pair(smem_u32(&sm->acc_full));
        mma_commit_pair(mapa_shared(smem_u32(&sm->acc_full), 1));
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int quarter = warp & 3;         // TMEM lanes 32 quarter .. + 31
    const int grp = (warp - 2) >> 2;      // 0: TMEM columns 0.. (S0 x B); 1: columns 256.. (S1 x B, or the field)
    const int row = quarter * 32 + lane;  // row of this CTA's logical halves
    const bool ready = (count > 0) && mbar_wait_cluster(smem_u32(&sm->acc_full), 0u, err, 45);
    if (ready) fence_after();
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16);
    // TMEM columns tcol0 .. tcol0 + ncols - 1 -> partial columns of out (ncols a multiple of 16)
    auto drain = [&](float* out, int tcol0, int ncols) {
      if (!out || (!ready && accumulate)) return;  // nothing in this phase: the partial stands
      out += (size_t)row * kTcLd;
      for (int c0 = 0; c0 < ncols; c0 += 16) {
        float v[16];
        if (ready) {
          tmem_ld16(tbase + (uint32_t)(tcol0 + c0), v);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = 0.f;  // no point blocks in this lane: a zero partial
        }
        store_cols<16>(out + c0, v, accumulate);
      }
    };
    float* out0 = u.out0[rank];
    float* out1 = u.out1[rank];
    if (grp == 0) {
      drain(out0, 0, u.nc);
    } else if (g2) {
      drain(out1, 256, u.nc);
    } else if (has_f) {
      drain(out0 ? out0 + kTcBNMax : nullptr, 256, u.cpad);
      if (a1) drain(out1 ? out1 + kTcBNMax : nullptr, 256 + u.cpad, u.cpad);
    }
  }
  fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs are done with TMEM and with each other's barriers
  fence_after();
  if (prof && threadIdx.x == 0) {
    prof[2 * blockIdx.x] = t_start;
    prof[2 * blockIdx.x + 1] = globaltimer();
  }
  if (warp == 1) tmem_dealloc_pair(tmem, kTmemCols);
}

}  // namespace

cudaError_t gram_pair_prepare() {
  static const cudaError_t attr =  // once per process (thread-safe initialisation)
      cudaFuncSetAttribute(gram_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
  return attr;
}

int gram_pair_max_clusters() {
  // co-resident CTA pairs at the largest stage size (two pairs never share an SM): the
  // pairs of a launch beyond this count would wait for a second wave
  static const int n = [] {  // once per process (thread-safe initialisation)
    if (gram_pair_prepare() != cudaSuccess) return 0;
    const int stage = gram_pair_stage_bytes(kTcBNMax, 128);
    int stages = (kSmemLimit - kSmemExtra) / stage;
    if (stages > kMaxStages) stages = kMaxStages;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeClusterDimension;
    la[0].val.clusterDim.x = 2;
    la[0].val.clusterDim.y = 1;
    la[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = stages * stage + kSmemExtra;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, gram_pair_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return c;
  }();
  return n;
}

int gram_pair_stage_bytes(int max_nc, int max_cpad) {
  return 2 * kABox + (max_nc / 2) * 128 + (max_cpad / 2) * 128;
}

cudaError_t launch_gram_pair_phase(const void* maps_dev, const PairUnit* units, int num_units, int stage_bytes,
                                   int kb0, int phase_blocks, int* err, cudaStream_t st,
                                   unsigned long long* prof) {
  if (num_units <= 0) return cudaSuccess;
  if (phase_blocks < 1 || stage_bytes % 1024) return cudaErrorInvalidValue;
  int stages = (kSmemLimit - kSmemExtra) / stage_bytes;
  if (stages > kMaxStages) stages = kMaxStages;
  if (stages < 2) return cudaErrorInvalidValue;
  const cudaError_t attr = gram_pair_prepare();
  if (attr != cudaSuccess) return attr;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute la[1];
  la[0].id = cudaLaunchAttributeClusterDimension;
  la[0].val.clusterDim.x = 2;
  la[0].val.clusterDim.y = 1;
  la[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * num_units);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = stages * stage_bytes + kSmemExtra;
  cfg.stream = st;
  cfg.attrs = la;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, gram_pair_kernel, static_cast<const CUtensorMap*>(maps_dev), units,
                                           stages, stage_bytes, kb0, phase_blocks, err, prof);
  if (e != cudaSuccess) return e;
  return launched();
}

}  // namespace rfd
