// Step a6, out = F + Phi Z (Sec. 2.4: the apply A (G (B^T F)) of the low-rank
// factors, "linear in N"), on the 5th-generation tensor cores for fields of
// 5..64 channels.  Phi is not read back from the BF16 feature matrix: producer
// warps recompute each point's features in FP32 (the SIMT apply's phase and
// MUFU sin/cos, bit for bit), split each value v into BF16 hi = bf16(v) and
// lo = bf16(v - hi), and write both into shared memory in the MMA's operand
// layout; Z is split the same way.  Per 16 features one MMA forms
//   D[:, 0:2cp]  += Phi_hi [Z_hi | Z_lo]      (N = 2 cp)
// and a second adds Phi_lo Z_hi into the Z_lo columns D[:, cp:2cp], so that
// D[:, ch] + D[:, cp + ch] = (Phi Z)[:, ch] up to the dropped Phi_lo Z_lo and
// the 16-bit splits: a relative error of about 2^-16 per term, against 2^-8 for
// one BF16 product.  The FP32 accumulators stay in TMEM for all of K.
//
// A tile is 256 points (two M = 128 halves); K runs over chunks of 64
// features, the cos then the sin of 32 frequencies (Z's rows are permuted to
// match by apply_prep).  Two producer threads share a point, one for each half
// of the chunk's frequencies, and each writes four 16-byte pieces of the
// point's 128-byte row in each operand.  The CTAs are persistent, one per SM,
// walking the tiles of all clouds of the batch.
//
// Warp roles: warps 0..15 produce the A operand, warp 16 allocates TMEM and
// issues the MMAs (one lane), warp 17 copies each chunk's Z image and its 32
// frequencies 2 pi w into shared memory with the bulk copy engine (one lane;
// the producers read w there, a broadcast, instead of through the L1 cache
// that the epilogue's stream of F evicts), warps 18..21 drain the
// accumulators (TMEM lane quarter warp % 4) and write out = F + D.  Two A
// stages, four B stages and two accumulator buffers (2 x 256 TMEM columns)
// let the epilogue of one tile run beside the MMAs of the next.  Every
// mbarrier wait is bounded by a %globaltimer limit; a wait that runs out
// records a code in *err and the role stops, waiting (again bounded) for its
// own copies and MMAs before the CTA frees its TMEM and exits.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include "kernels.h"
#include "tc_common.cuh"

namespace rfd {

namespace {

using namespace tc;

constexpr int kAtHalf = 128 * 128;            // one M = 128 half of one split: 128 rows x 128 B
constexpr int kAtAStage = 4 * kAtHalf;        // hi (half 0, half 1), then lo (half 0, half 1)
constexpr int kAtZBytes = 128 * 128;          // the Z image: 2 cp <= 128 rows of 128 B
constexpr int kAtBStage = kAtZBytes + 1024;   // then the chunk's 32 frequencies 2 pi w (512 B)
constexpr int kAtAStages = 2, kAtBStages = 4;
constexpr int kAtProducers = 512;             // two per point: frequencies 0..15 / 16..31 of each chunk
constexpr int kMmaWarp = kAtProducers / 32, kLoadWarp = kMmaWarp + 1;
constexpr int kAtThreads = kAtProducers + 32 + 32 + 128;
constexpr uint32_t kAtTmemCols = 512;  // buffer b at columns [256 b, 256 b + 256): half h at + 128 h
constexpr int kAtSmem = 1024 + kAtAStages * kAtAStage + kAtBStages * kAtBStage + 256;

struct AtSmem {
  uint64_t afull[kAtAStages], aempty[kAtAStages];
  uint64_t bfull[kAtBStages], bempty[kAtBStages];
  uint64_t accf[2], acce[2];
  uint64_t done;
  uint32_t tmem_base;
};

__device__ __forceinline__ int find_job_at(const int* __restrict__ prefix, int count, int b) {
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

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
// (a, b) -> BF16 pairs hi = (bf16(a), bf16(b)) and lo = (bf16(a - hi.x), bf16(b - hi.y)),
// the first value in the low half (the lower address)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
// 16 consecutive FP32 columns of this thread's TMEM lane, without waiting
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__global__ void __launch_bounds__(kAtThreads, 1)
apply_tc_kernel(const ApplyTcJob* __restrict__ jobs, const int* __restrict__ prefix, int count, int total_tiles,
                const CloudCall* __restrict__ calls, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  const uint32_t sA = base, sB = base + kAtAStages * kAtAStage;
  AtSmem* sm = reinterpret_cast<AtSmem*>(smem_raw + (base - raw_addr) + kAtAStages * kAtAStage +
                                         kAtBStages * kAtBStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kAtAStages; ++s) {
      mbar_init(smem_u32(&sm->afull[s]), kAtProducers);
      mbar_init(smem_u32(&sm->aempty[s]), 1);
    }
    for (int s = 0; s < kAtBStages; ++s) {
      mbar_init(smem_u32(&sm->bfull[s]), 1);
      mbar_init(smem_u32(&sm->bempty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sm->accf[b]), 1);
      mbar_init(smem_u32(&sm->acce[b]), 128);
    }
    mbar_init(smem_u32(&sm->done), 1);
    fence_mbar_init();
  }
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&sm->tmem_base), kAtTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp < kMmaWarp) {
    // ---------------- A producers: two threads per point ----------------
    const int pt = threadIdx.x & 255, fh = threadIdx.x >> 8;  // point of the tile, half of the chunk's frequencies
    const int half = pt >> 7, r = pt & 127, r7 = r & 7;
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
      const int j = find_job_at(prefix, count, t);
      const int64_t p = (int64_t)(t - prefix[j]) * 256 + pt;
      const int64_t n = jobs[j].n;
      const float* __restrict__ xyz = jobs[j].xyz;
      const int kchunks = jobs[j].kchunks;
      const float x0 = p < n ? xyz[p * 3] : 0.f, x1 = p < n ? xyz[p * 3 + 1] : 0.f, x2 = p < n ? xyz[p * 3 + 2] : 0.f;
      for (int kc = 0; kc < kchunks; ++kc, ++it) {
        const int s = it & 1, u = it >> 1, bs = it & 3;
        if ((u > 0 && !mbar_wait(smem_u32(&sm->aempty[s]), (uint32_t)(u - 1) & 1u, err, 21)) ||
            !mbar_wait(smem_u32(&sm->bfull[bs]), (uint32_t)(it >> 2) & 1u, err, 29)) {
          ok = false;
          break;
        }
        const uint32_t rowhi = sA + s * kAtAStage + half * kAtHalf + r * 128;
        const uint32_t rowlo = rowhi + 2 * kAtHalf;
        // the chunk's 2 pi w, copied in beside its Z image
        const float4* wk = reinterpret_cast<const float4*>(smem_raw + (sB - raw_addr) + bs * kAtBStage + kAtZBytes);
#pragma unroll
        for (int gg = 0; gg < 2; ++gg) {  // frequencies 8 g .. 8 g + 7: pieces g (cos) and 4 + g (sin)
          const int g = 2 * fh + gg;
          uint32_t ch[4], cl[4], sh[4], sl[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float4 wa = wk[8 * g + 2 * e], wb = wk[8 * g + 2 * e + 1];
            const float ta = fmaf(wa.x, x0, fmaf(wa.y, x1, wa.z * x2));
            const float tb = fmaf(wb.x, x0, fmaf(wb.y, x1, wb.z * x2));
            split2(__cosf(ta), __cosf(tb), ch[e], cl[e]);
            split2(__sinf(ta), __sinf(tb), sh[e], sl[e]);
          }
          const uint32_t oc = (uint32_t)((g ^ r7) << 4), os = (uint32_t)(((4 + g) ^ r7) << 4);
          st_shared_v4(rowhi + oc, ch[0], ch[1], ch[2], ch[3]);
          st_shared_v4(rowhi + os, sh[0], sh[1], sh[2], sh[3]);
          st_shared_v4(rowlo + oc, cl[0], cl[1], cl[2], cl[3]);
          st_shared_v4(rowlo + os, sl[0], sl[1], sl[2], sl[3]);
        }
        fence_proxy_async();  // the generic-proxy stores, before the MMAs read them
        mbar_arrive(smem_u32(&sm->afull[s]));
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int it = 0, tc = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x, ++tc) {
        const int j = find_job_at(prefix, count, t);
        const int kchunks = jobs[j].kchunks;
        const int cp = apply_tc_cpad(calls[jobs[j].cloud].c);
        const uint32_t id_hi = idesc_bf16(128, 2 * cp), id_lo = idesc_bf16(128, cp);
        const int buf = tc & 1, ub = tc >> 1;
        if (ub > 0 && !mbar_wait(smem_u32(&sm->acce[buf]), (uint32_t)(ub - 1) & 1u, err, 22)) break;
        fence_after();
        const uint32_t d0 = tmem + (uint32_t)(buf * 256);
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int s = it & 1, bs = it & 3;
          if (!mbar_wait(smem_u32(&sm->afull[s]), (uint32_t)(it >> 1) & 1u, err, 23) ||
              !mbar_wait(smem_u32(&sm->bfull[bs]), (uint32_t)(it >> 2) & 1u, err, 24)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t a = sA + s * kAtAStage, b = sB + bs * kAtBStage;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint32_t d = d0 + (uint32_t)(h * 128);
              const uint64_t bd = sdesc_sw128(b + kk * 32);
              mma_bf16(d, sdesc_sw128(a + h * kAtHalf + kk * 32), bd, id_hi, (kc > 0 || kk > 0) ? 1u : 0u);
              mma_bf16(d + (uint32_t)cp, sdesc_sw128(a + (2 + h) * kAtHalf + kk * 32), bd, id_lo, 1u);
            }
          }
          mma_commit(smem_u32(&sm->aempty[s]));  // frees the stages when these MMAs finish
          mma_commit(smem_u32(&sm->bempty[bs]));
        }
        if (ok) mma_commit(smem_u32(&sm->accf[buf]));
      }
      // every MMA issued has finished before the TMEM is freed
      mma_commit(smem_u32(&sm->done));
      mbar_wait(smem_u32(&sm->done), 0u, err, 25);
    }
    __syncwarp();
  } else if (warp == kLoadWarp) {
    // ---------------- Z images: bulk copies ----------------
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
        const int j = find_job_at(prefix, count, t);
        const int kchunks = jobs[j].kchunks;
        const uint8_t* zimg = jobs[j].zimg;
        const float4* w2 = jobs[j].w2pi;
        const uint32_t zbytes = (uint32_t)(2 * apply_tc_cpad(calls[jobs[j].cloud].c) * 128);
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int bs = it & 3, bu = it >> 2;
          if (bu > 0 && !mbar_wait(smem_u32(&sm->bempty[bs]), (uint32_t)(bu - 1) & 1u, err, 26)) {
            ok = false;
            break;
          }
          const uint32_t full = smem_u32(&sm->bfull[bs]);
          mbar_arrive_expect_tx(full, zbytes + 512u);
          bulk_load(sB + bs * kAtBStage, zimg + (size_t)kc * zbytes, zbytes, full);
          bulk_load(sB + bs * kAtBStage + kAtZBytes, w2 + kc * 32, 512u, full);
        }
      }
      // drain: our copies into the last stages must land before the CTA exits
      for (int q = (it > kAtBStages ? it - kAtBStages : 0); q < it; ++q)
        mbar_wait(smem_u32(&sm->bfull[q & 3]), (uint32_t)(q >> 2) & 1u, err, 27);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: out = F + D_hi + D_lo ----------------
    const int quarter = warp & 3;  // TMEM lanes 32 quarter .. + 31
    const int r = quarter * 32 + lane;
    int tc = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++tc) {
      const int j = find_job_at(prefix, count, t);
      const int64_t n = jobs[j].n;
      const CloudCall cc = calls[jobs[j].cloud];
      const int c = cc.c, cp = apply_tc_cpad(c);
      const int buf = tc & 1;
      if (!mbar_wait(smem_u32(&sm->accf[buf]), (uint32_t)(tc >> 1) & 1u, err, 28)) break;
      fence_after();
      const bool vec = ((cc.ldF | cc.ldOut) & 3) == 0 &&
                       ((reinterpret_cast<uintptr_t>(cc.F) | reinterpret_cast<uintptr_t>(cc.out)) & 15) == 0;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int64_t p = (int64_t)(t - prefix[j]) * 256 + h * 128 + r;
        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 256 + h * 128);
#pragma unroll 1
        for (int c0 = 0; c0 < cp; c0 += 16) {
          uint32_t hi[16], lo[16];
          tmem_ld16_nowait(ta + (uint32_t)c0, hi);
          tmem_ld16_nowait(ta + (uint32_t)(cp + c0), lo);
          tmem_wait_ld();
          if (p < n) {
            const float* f = cc.F + p * cc.ldF + c0;
            float* o = cc.out + p * cc.ldOut + c0;
            if (vec && c0 + 16 <= c) {
              float4 fv[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) fv[q] = reinterpret_cast<const float4*>(f)[q];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                float4 v = fv[q];
                v.x += __uint_as_float(hi[4 * q]) + __uint_as_float(lo[4 * q]);
                v.y += __uint_as_float(hi[4 * q + 1]) + __uint_as_float(lo[4 * q + 1]);
                v.z += __uint_as_float(hi[4 * q + 2]) + __uint_as_float(lo[4 * q + 2]);
                v.w += __uint_as_float(hi[4 * q + 3]) + __uint_as_float(lo[4 * q + 3]);
                reinterpret_cast<float4*>(o)[q] = v;
              }
            } else {
              const int nq = min(16, c - c0);
              float fv[16];
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (q < nq) fv[q] = f[q];
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (q < nq) o[q] = fv[q] + (__uint_as_float(hi[q]) + __uint_as_float(lo[q]));
            }
          }
        }
      }
      fence_before();
      mbar_arrive(smem_u32(&sm->acce[buf]));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, kAtTmemCols);
}

// Z (m x c FP32, rows f < h the cos features, h + f the sin ones) as the MMA's
// B operand: per chunk kc of 64 features, 2 cp rows of 128 B (rows ch < cp the
// hi parts of channel ch, rows cp + ch the lo parts), each row eight 16-byte
// pieces -- piece q holds features 8 q .. 8 q + 7 of the chunk (q < 4: the cos
// of frequencies 32 kc + 8 q + e; q >= 4: their sin) -- stored at position
// q ^ (row mod 8), the 128-byte swizzle; and 2 pi w per frequency, zero past h.
__global__ void __launch_bounds__(256) apply_prep_kernel(const ApplyTcJob* __restrict__ jobs,
                                                         const int* __restrict__ prefix, int count,
                                                         const CloudCall* __restrict__ calls) {
  const int j = find_job_at(prefix, count, blockIdx.x);
  const ApplyTcJob jb = jobs[j];
  const int c = calls[jb.cloud].c, cp = apply_tc_cpad(c), rows = 2 * cp;
  const int idx = (blockIdx.x - prefix[j]) * 256 + threadIdx.x;
  if (idx < 32 * jb.kchunks) {
    const float two_pi = 6.283185307179586f;
    const float* w = jb.omega_hi + (size_t)idx * 3;
    jb.w2pi[idx] = idx < jb.h ? make_float4(two_pi * w[0], two_pi * w[1], two_pi * w[2], 0.f)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (idx >= jb.kchunks * rows * 8) return;
  const int q = idx & 7, row = (idx >> 3) % rows, kc = (idx >> 3) / rows;
  const bool lo = row >= cp;
  const int ch = lo ? row - cp : row;
  uint32_t packed[4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    float v[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int k = 8 * q + e + t;        // feature of the chunk
      const int f = 32 * kc + (k & 31);   // its frequency
      const int zr = k < 32 ? f : jb.h + f;
      const float z = (ch < c && f < jb.h) ? jb.Z[(size_t)zr * c + ch] : 0.f;
      const float hz = __bfloat162float(__float2bfloat16_rn(z));
      v[t] = lo ? z - hz : z;
    }
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[0], v[1]);
    packed[e / 2] = *reinterpret_cast<const uint32_t*>(&b2);
  }
  uint4* dst = reinterpret_cast<uint4*>(jb.zimg + (size_t)kc * rows * 128 + (size_t)row * 128 +
                                        (size_t)((q ^ (row & 7)) << 4));
  *dst = make_uint4(packed[0], packed[1], packed[2], packed[3]);
}

}  // namespace

bool apply_tc_supported() { return tc::sm103_available(); }

cudaError_t apply_tc_prepare() {
  static cudaError_t once = cudaFuncSetAttribute(apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAtSmem);
  return once;
}

cudaError_t launch_apply_prep(const ApplyTcJob* jobs, const int* prefix, int count, int total_blocks,
                              const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  apply_prep_kernel<<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls);
  return launched();
}

cudaError_t launch_apply_tc(const ApplyTcJob* jobs, const int* tile_prefix, int count, int total_tiles, int grid,
                            const CloudCall* calls, int* err, cudaStream_t st) {
  if (total_tiles <= 0) return cudaSuccess;
  apply_tc_kernel<<<grid, kAtThreads, kAtSmem, st>>>(jobs, tile_prefix, count, total_tiles, calls, err);
  return launched();
}

}  // namespace rfd
