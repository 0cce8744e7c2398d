// Step a6, out = F + Phi Z (Sec. 2.4: the apply A (G (B^T F)) of the low-rank
// factors, "linear in N"), on the 5th-generation tensor cores for fields of
// up to 64 channels.  Phi is not read back from the BF16 feature matrix:
// producer warps recompute each point's features in FP32 (the SIMT apply's
// phase and MUFU sin/cos, bit for bit) and split each value v into BF16
// hi = bf16(v) and lo = bf16(v - hi); Z is split the same way (apply_prep).
// The MMAs form the transpose, D = Z^T Phi^T: M = 128 rows of Z's image, N =
// the 256 points of a tile, so that one MMA per 16 features and product
// covers the whole tile (each MMA costs ~100 cycles to issue, and one of
// N = 256 keeps the tensor pipe busy for about as long).  In shared memory
// Z's image of a chunk is cp rows of Z_hi^T then cp rows of Z_lo^T (cp =
// channels rounded up to 16), right after cp rows of zeros; two 128-row
// windows of it are the A operands:
//   rows [2cp - 128, 2cp) of the image:  D += [.. | Z_hi | Z_lo]^T Phi_hi
//   rows [cp - 128, cp) of the image:    D += [.. | 0    | Z_hi]^T Phi_lo
// so that TMEM lane 128 - cp + ch accumulates Z_lo Phi_hi + Z_hi Phi_lo and
// lane 128 - 2cp + ch accumulates Z_hi Phi_hi for channel ch, and their sum is
// (Phi Z)[:, ch] up to the dropped Phi_lo Z_lo and the 16-bit splits: a
// relative error of about 2^-16 per term, against 2^-8 for one BF16 product.
// (The lanes below 128 - 2cp read whatever lies before the zeros and are never
// used.)  The FP32 accumulators stay in TMEM for all of K.
//
// A tile is 256 points; K runs over chunks of 64 features, the cos then the
// sin of 32 frequencies (Z's rows are permuted to match by apply_prep).  A
// producer thread takes two points (rows r and r + 128 of the tile) and a
// quarter of the chunk's frequencies, so each broadcast load of w serves two
// points, and writes two 16-byte pieces of each point's 128-byte row of
// Phi_hi and of Phi_lo (the shared-memory port, not the arithmetic, sets this
// kernel's pace: Phi's stores and the MMAs' operand reads share it).  The CTAs are persistent, one per SM, walking
// the tiles of all clouds of the batch.
//
// Warp roles: warps 0..15 produce Phi, warp 16 allocates TMEM and issues the
// MMAs (one lane), warp 17 copies each chunk's Z image and its 32 frequencies
// 2 pi w into shared memory with the bulk copy engine (one lane; the
// producers read w there, a broadcast), warps 18..21 drain the accumulators:
// 32 points at a time, each warp moves its TMEM lane quarter to shared memory,
// and the four warps then write out = F + D_x + D_y with lanes along the
// channels (coalesced rows of out).  Two Phi stages, three Z stages and two
// accumulator buffers (2 x 256 TMEM columns) let the epilogue of one tile run
// beside the MMAs of the next.  Every mbarrier wait is bounded by a
// %globaltimer limit; a wait that runs out records a code in *err and the
// role stops, waiting (again bounded) for its own copies and MMAs before the
// CTA frees its TMEM and exits.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include "kernels.h"
#include "tc_common.cuh"

namespace rfd {

namespace {

using namespace tc;

constexpr int kAtPhi = 256 * 128;             // one split of Phi: 256 point rows x 128 B
constexpr int kAtAStage = 2 * kAtPhi;         // Phi_hi, then Phi_lo
constexpr int kAtAStages = 2;
constexpr int kAtZeros = 64 * 128;            // zero rows before each Z image (cp <= 64 of them are read)
constexpr int kAtZData = 128 * 128;           // the Z image: 2 cp <= 128 rows of 128 B
constexpr int kAtBStage = kAtZeros + kAtZData;
constexpr int kAtBStages = 3;
constexpr int kAtEPitch = 33;                 // epilogue exchange: 128 lanes x 32 points, padded
constexpr int kAtProducers = 512;             // two points x 8 of each chunk's 32 frequencies per thread
constexpr int kMmaWarp = kAtProducers / 32, kLoadWarp = kMmaWarp + 1, kEpiWarp0 = kLoadWarp + 1;
constexpr int kAtThreads = kAtProducers + 32 + 32 + 128;
constexpr uint32_t kAtTmemCols = 512;  // accumulator buffer b at columns [256 b, 256 b + 256)
// layout after the 1024-aligned base: Phi stages, Z stages (zeros then image), the chunks' 2 pi w,
// the epilogue exchange, the barriers
constexpr int kAtOffB = kAtAStages * kAtAStage;
constexpr int kAtOffW = kAtOffB + kAtBStages * kAtBStage;
constexpr int kAtOffE = kAtOffW + kAtBStages * 512;
constexpr int kAtOffBar = kAtOffE + 128 * kAtEPitch * 4;
constexpr int kAtSmem = 1024 + kAtOffBar + 256;

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
// the four epilogue warps: barrier 1, and the AND of a predicate over them (so that they
// leave the tile loop together and never strand one another at the barrier)
__device__ __forceinline__ float4 ld_shared_f4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, 128, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
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

__global__ void __launch_bounds__(kAtThreads, 1)
apply_tc_kernel(const ApplyTcJob* __restrict__ jobs, const int* __restrict__ prefix, int count, int total_tiles,
                const CloudCall* __restrict__ calls, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw_addr);
  const uint32_t sA = base, sB = base + kAtOffB;
  AtSmem* sm = reinterpret_cast<AtSmem*>(gbase + kAtOffBar);
  float* E = reinterpret_cast<float*>(gbase + kAtOffE);
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
  // the zero rows before each Z image (never written again)
  for (int i = threadIdx.x; i < kAtBStages * (kAtZeros / 16); i += kAtThreads) {
    const int s = i / (kAtZeros / 16), q = i % (kAtZeros / 16);
    st_shared_v4(sB + s * kAtBStage + q * 16, 0u, 0u, 0u, 0u);
  }
  fence_proxy_async();  // before the MMAs read them
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&sm->tmem_base), kAtTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp < kMmaWarp) {
    // ---------------- Phi producers: two points and 8 frequencies per thread ----------------
    const int pr = threadIdx.x & 127, fq = threadIdx.x >> 7;  // points pr and pr + 128; frequencies 8 fq .. + 7
    const int r7 = pr & 7;                                     // (pr + 128) mod 8 as well
    const uint32_t oc = (uint32_t)((fq ^ r7) << 4), os = (uint32_t)(((4 + fq) ^ r7) << 4);
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
      const int j = find_job_at(prefix, count, t);
      const int64_t pa = (int64_t)(t - prefix[j]) * 256 + pr, pb = pa + 128;
      const int64_t n = jobs[j].n;
      const float* __restrict__ xyz = jobs[j].xyz;
      const int kchunks = jobs[j].kchunks;
      float xa[3], xb[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        xa[d] = pa < n ? xyz[pa * 3 + d] : 0.f;
        xb[d] = pb < n ? xyz[pb * 3 + d] : 0.f;
      }
      for (int kc = 0; kc < kchunks; ++kc, ++it) {
        const int s = it & 1, u = it >> 1, bs = it % kAtBStages;
        if ((u > 0 && !mbar_wait(smem_u32(&sm->aempty[s]), (uint32_t)(u - 1) & 1u, err, 21)) ||
            !mbar_wait(smem_u32(&sm->bfull[bs]), (uint32_t)(it / kAtBStages) & 1u, err, 29)) {
          ok = false;
          break;
        }
        // the chunk's 2 pi w, copied in beside its Z image: one broadcast 16-byte load per frequency
        const uint32_t wk = base + kAtOffW + bs * 512 + fq * 8 * 16;
        uint32_t cha[4], cla[4], sha[4], sla[4], chb[4], clb[4], shb[4], slb[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4 wa = ld_shared_f4(wk + (2 * e) * 16), wb = ld_shared_f4(wk + (2 * e + 1) * 16);
          const float t0 = fmaf(wa.x, xa[0], fmaf(wa.y, xa[1], wa.z * xa[2]));
          const float t1 = fmaf(wb.x, xa[0], fmaf(wb.y, xa[1], wb.z * xa[2]));
          const float t2 = fmaf(wa.x, xb[0], fmaf(wa.y, xb[1], wa.z * xb[2]));
          const float t3 = fmaf(wb.x, xb[0], fmaf(wb.y, xb[1], wb.z * xb[2]));
          split2(__cosf(t0), __cosf(t1), cha[e], cla[e]);
          split2(__sinf(t0), __sinf(t1), sha[e], sla[e]);
          split2(__cosf(t2), __cosf(t3), chb[e], clb[e]);
          split2(__sinf(t2), __sinf(t3), shb[e], slb[e]);
        }
        const uint32_t ra = sA + s * kAtAStage + pr * 128, rb = ra + 128 * 128;  // rows pr, pr + 128 of Phi_hi
        st_shared_v4(ra + oc, cha[0], cha[1], cha[2], cha[3]);
        st_shared_v4(ra + os, sha[0], sha[1], sha[2], sha[3]);
        st_shared_v4(ra + kAtPhi + oc, cla[0], cla[1], cla[2], cla[3]);
        st_shared_v4(ra + kAtPhi + os, sla[0], sla[1], sla[2], sla[3]);
        st_shared_v4(rb + oc, chb[0], chb[1], chb[2], chb[3]);
        st_shared_v4(rb + os, shb[0], shb[1], shb[2], shb[3]);
        st_shared_v4(rb + kAtPhi + oc, clb[0], clb[1], clb[2], clb[3]);
        st_shared_v4(rb + kAtPhi + os, slb[0], slb[1], slb[2], slb[3]);
        fence_proxy_async();  // the generic-proxy stores, before the MMAs read them
        mbar_arrive(smem_u32(&sm->afull[s]));
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int it = 0, tc = 0;
      bool ok = true;
      const uint32_t idesc = idesc_bf16(128, 256);
      for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x, ++tc) {
        const int j = find_job_at(prefix, count, t);
        const int kchunks = jobs[j].kchunks;
        const int cp = apply_tc_cpad(calls[jobs[j].cloud].c);
        const int buf = tc & 1, ub = tc >> 1;
        if (ub > 0 && !mbar_wait(smem_u32(&sm->acce[buf]), (uint32_t)(ub - 1) & 1u, err, 22)) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 256);
        for (int kc = 0; kc < kchunks; ++kc, ++it) {
          const int s = it & 1, bs = it % kAtBStages;
          if (!mbar_wait(smem_u32(&sm->afull[s]), (uint32_t)(it >> 1) & 1u, err, 23) ||
              !mbar_wait(smem_u32(&sm->bfull[bs]), (uint32_t)(it / kAtBStages) & 1u, err, 24)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t phi = sA + s * kAtAStage;
          const uint32_t zimg = sB + bs * kAtBStage + kAtZeros;  // the image's row 0
          const uint32_t a1 = zimg - (uint32_t)((128 - 2 * cp) * 128), a2 = zimg - (uint32_t)((128 - cp) * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma_bf16(d, sdesc_sw128(a1 + kk * 32), sdesc_sw128(phi + kk * 32), idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, sdesc_sw128(a2 + kk * 32), sdesc_sw128(phi + kAtPhi + kk * 32), idesc, 1u);
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
    // ---------------- Z images and 2 pi w: bulk copies ----------------
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
          const int bs = it % kAtBStages, bu = it / kAtBStages;
          if (bu > 0 && !mbar_wait(smem_u32(&sm->bempty[bs]), (uint32_t)(bu - 1) & 1u, err, 26)) {
            ok = false;
            break;
          }
          const uint32_t full = smem_u32(&sm->bfull[bs]);
          mbar_arrive_expect_tx(full, zbytes + 512u);
          bulk_load(sB + bs * kAtBStage + kAtZeros, zimg + (size_t)kc * zbytes, zbytes, full);
          bulk_load(base + kAtOffW + bs * 512, w2 + kc * 32, 512u, full);
        }
      }
      // drain: our copies into the last stages must land before the CTA exits
      for (int q = (it > kAtBStages ? it - kAtBStages : 0); q < it; ++q)
        mbar_wait(smem_u32(&sm->bfull[q % kAtBStages]), (uint32_t)(q / kAtBStages) & 1u, err, 27);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: out = F + D_x + D_y ----------------
    const int quarter = warp & 3;                 // TMEM lanes 32 quarter .. + 31
    const int et = threadIdx.x - kEpiWarp0 * 32;  // 0..127
    const int ch = et & 63, pofs = et >> 6;       // output channel, point parity
    int tc = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++tc) {
      const int j = find_job_at(prefix, count, t);
      const int64_t n = jobs[j].n;
      const CloudCall cc = calls[jobs[j].cloud];
      const int c = cc.c, cp = apply_tc_cpad(c);
      const int lx = 128 - cp + ch, ly = 128 - 2 * cp + ch;  // the TMEM lanes of channel ch
      const int buf = tc & 1;
      const int64_t p0 = (int64_t)(t - prefix[j]) * 256;
      // F of 32 points is loaded one round ahead of its use -- the first round's before the
      // wait for the accumulators -- so its latency overlaps the wait, the TMEM reads and the
      // barriers (a thread's loads of a point precede its store: out may be F itself)
      float f[16], fn[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int64_t p = p0 + 2 * k + pofs;
        f[k] = (ch < c && p < n) ? cc.F[p * cc.ldF + ch] : 0.f;
      }
      if (!epi_all(mbar_wait(smem_u32(&sm->accf[buf]), (uint32_t)(tc >> 1) & 1u, err, 28))) break;
      fence_after();
#pragma unroll 1
      for (int col0 = 0; col0 < 256; col0 += 32) {  // 32 points of the tile
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int64_t p = p0 + col0 + 32 + 2 * k + pofs;
          fn[k] = (ch < c && col0 + 32 < 256 && p < n) ? cc.F[p * cc.ldF + ch] : 0.f;
        }
        float* er = E + (quarter * 32 + lane) * kAtEPitch;
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          uint32_t v[8];
          tmem_ld8_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 256 + col0 + 8 * hh), v);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 8; ++q) er[8 * hh + q] = __uint_as_float(v[q]);
        }
        epi_sync();
        if (ch < c) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int q = 2 * k + pofs;
            const int64_t p = p0 + col0 + q;
            if (p < n) cc.out[p * cc.ldOut + ch] = f[k] + (E[lx * kAtEPitch + q] + E[ly * kAtEPitch + q]);
          }
        }
        epi_sync();
#pragma unroll
        for (int k = 0; k < 16; ++k) f[k] = fn[k];
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

// Z (m x c FP32, rows f < h the cos features, h + f the sin ones) as rows of
// the MMA's A operand (Z^T, K-major): per chunk kc of 64 features, 2 cp rows of
// 128 B (rows ch < cp the hi parts of channel ch, rows cp + ch the lo parts), each row eight 16-byte
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

// Y' = Phi^T F from the points on the tensor cores (compact plans, fields of
// more than 16 channels, or more than 8 with m >= 512): the apply's machinery
// with K running over the points instead of the features.  A work item is one
// chunk of the cloud's points (the FieldPtsJob's chunks) and one tile of 128
// frequencies (256 features: their cos, then their sin); per step of 64 points
//   D += [.. | F_hi | F_lo]^T Phi_hi^T  and  D += [.. | 0 | F_hi]^T Phi_lo^T
// (M = 128 rows of F's image, N = the 256 features, K = 16 points per MMA), so
// that TMEM lane 128 - cp + ch gathers F_lo Phi_hi + F_hi Phi_lo and lane
// 128 - 2cp + ch gathers F_hi Phi_hi.  The producers write both operands each
// step: Phi^T (a thread per frequency and 16 points: the phase and MUFU sin/cos
// of the SIMT fieldpts kernel, split into BF16 hi / lo) and F's image (a thread
// per channel and 8 points, F split the same way; zero for points >= N).  The
// points of each step come in by bulk copy (a ring of four).  The epilogue
// writes the item's FP32 partial part[chunk][f][ch] = lane x + lane y, which
// fieldpts_reduce sums over the chunks as it does the SIMT kernel's.
constexpr int kFtPhi = 256 * 128;           // Phi^T split: 256 feature rows x 64 points (128 B)
constexpr int kFtZeros = 64 * 128;          // zero rows before F's image
constexpr int kFtImg = 128 * 128;           // F's image: 2 cp <= 128 channel rows x 64 points
constexpr int kFtStage = 2 * kFtPhi + kFtZeros + kFtImg;
constexpr int kFtStages = 2;
constexpr int kFtXSlots = 4;                // points ring: 64 points x 12 B each
constexpr int kFtOffX = kFtStages * kFtStage;
constexpr int kFtOffE = kFtOffX + kFtXSlots * 768;
constexpr int kFtOffBar = kFtOffE + 128 * kAtEPitch * 4;
constexpr int kFtSmem = 1024 + kFtOffBar + 256;

struct FtSmem {
  uint64_t afull[kFtStages], aempty[kFtStages];
  uint64_t xfull[kFtXSlots], xempty[kFtXSlots];
  uint64_t accf[2], acce[2];
  uint64_t done;
  uint32_t tmem_base;
};

// the item's chunk and frequency tile, and its points [p_begin, p_end)
struct FtItem {
  int j, chunk, ft, steps;
  int64_t p_begin, p_end;
};
__device__ __forceinline__ FtItem ft_item(const FieldPtsJob* __restrict__ jobs, const int* __restrict__ prefix,
                                          int count, int t) {
  FtItem r;
  r.j = find_job_at(prefix, count, t);
  const FieldPtsJob& jb = jobs[r.j];
  const int ftiles = (jb.h + 127) / 128;
  const int local = t - prefix[r.j];
  r.chunk = local / ftiles;
  r.ft = local % ftiles;
  r.p_begin = (int64_t)r.chunk * jb.pts;
  r.p_end = min(jb.n, r.p_begin + jb.pts);
  r.steps = r.p_end > r.p_begin ? (int)((r.p_end - r.p_begin + 63) / 64) : 0;
  return r;
}

__global__ void __launch_bounds__(kAtThreads, 1)
fieldpts_tc_kernel(const FieldPtsJob* __restrict__ jobs, const int* __restrict__ prefix, int count, int total_items,
                   const CloudCall* __restrict__ calls, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_u32(smem_raw);
  const uint32_t base = (raw_addr + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw_addr);
  FtSmem* sm = reinterpret_cast<FtSmem*>(gbase + kFtOffBar);
  float* E = reinterpret_cast<float*>(gbase + kFtOffE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kFtStages; ++s) {
      mbar_init(smem_u32(&sm->afull[s]), kAtProducers);
      mbar_init(smem_u32(&sm->aempty[s]), 1);
    }
    for (int s = 0; s < kFtXSlots; ++s) {
      mbar_init(smem_u32(&sm->xfull[s]), 1);
      mbar_init(smem_u32(&sm->xempty[s]), kAtProducers);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sm->accf[b]), 1);
      mbar_init(smem_u32(&sm->acce[b]), 128);
    }
    mbar_init(smem_u32(&sm->done), 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < kFtStages * (kFtZeros / 16); i += kAtThreads) {
    const int s = i / (kFtZeros / 16), q = i % (kFtZeros / 16);
    st_shared_v4(base + s * kFtStage + 2 * kFtPhi + q * 16, 0u, 0u, 0u, 0u);
  }
  fence_proxy_async();
  if (warp == kMmaWarp) tmem_alloc(smem_u32(&sm->tmem_base), kAtTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp < kMmaWarp) {
    // ---------------- producers: Phi^T (a frequency x 16 points) and F's image (a channel x 8 points) ----
    const int fj = threadIdx.x & 127, pq = threadIdx.x >> 7;  // frequency of the tile, 16-point quarter
    const int fch = threadIdx.x & 63, pg = threadIdx.x >> 6;  // channel, 8-point group
    const int r7 = fj & 7, c7 = fch & 7;
    const float two_pi = 6.283185307179586f;
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total_items && ok; t += gridDim.x) {
      const FtItem im = ft_item(jobs, prefix, count, t);
      const FieldPtsJob& jb = jobs[im.j];
      const CloudCall cc = calls[jb.cloud];
      const int c = cc.c, cp = apply_tc_cpad(c);
      const int fidx = im.ft * 128 + fj;
      float w[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) w[d] = fidx < jb.h ? two_pi * jb.omega_hi[(size_t)fidx * 3 + d] : 0.f;
      // F of the first step (then of the next, loaded one step ahead)
      float fv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t p = im.p_begin + pg * 8 + e;
        fv[e] = (fch < c && p < im.p_end) ? cc.F[p * cc.ldF + fch] : 0.f;
      }
      for (int k = 0; k < im.steps; ++k, ++it) {
        const int s = it & 1, u = it >> 1, xs = it % kFtXSlots;
        const int64_t p0 = im.p_begin + (int64_t)k * 64;
        const int np = (int)min((int64_t)64, im.p_end - p0);
        if ((u > 0 && !mbar_wait(smem_u32(&sm->aempty[s]), (uint32_t)(u - 1) & 1u, err, 31)) ||
            !mbar_wait(smem_u32(&sm->xfull[xs]), (uint32_t)(it / kFtXSlots) & 1u, err, 32)) {
          ok = false;
          break;
        }
        const uint32_t st0 = base + s * kFtStage;
        // Phi^T rows fj (cos) and 128 + fj (sin): pieces 2 pq and 2 pq + 1 (points 16 pq ..)
        const float* xsm = reinterpret_cast<const float*>(gbase + kFtOffX + xs * 768);
        uint32_t chv[8], clv[8], shv[8], slv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int pa = pq * 16 + 2 * e, pb = pa + 1;
          const float ax = pa < np ? xsm[pa * 3] : 0.f, ay = pa < np ? xsm[pa * 3 + 1] : 0.f,
                      az = pa < np ? xsm[pa * 3 + 2] : 0.f;
          const float bx = pb < np ? xsm[pb * 3] : 0.f, by = pb < np ? xsm[pb * 3 + 1] : 0.f,
                      bz = pb < np ? xsm[pb * 3 + 2] : 0.f;
          const float ta = fmaf(w[0], ax, fmaf(w[1], ay, w[2] * az));
          const float tb = fmaf(w[0], bx, fmaf(w[1], by, w[2] * bz));
          split2(__cosf(ta), __cosf(tb), chv[e], clv[e]);
          split2(__sinf(ta), __sinf(tb), shv[e], slv[e]);
        }
        mbar_arrive(smem_u32(&sm->xempty[xs]));  // done with this step's points
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const uint32_t off = (uint32_t)(((2 * pq + h2) ^ r7) << 4);
          const uint32_t rc = st0 + fj * 128 + off, rs = st0 + (128 + fj) * 128 + off;
          st_shared_v4(rc, chv[4 * h2], chv[4 * h2 + 1], chv[4 * h2 + 2], chv[4 * h2 + 3]);
          st_shared_v4(rs, shv[4 * h2], shv[4 * h2 + 1], shv[4 * h2 + 2], shv[4 * h2 + 3]);
          st_shared_v4(rc + kFtPhi, clv[4 * h2], clv[4 * h2 + 1], clv[4 * h2 + 2], clv[4 * h2 + 3]);
          st_shared_v4(rs + kFtPhi, slv[4 * h2], slv[4 * h2 + 1], slv[4 * h2 + 2], slv[4 * h2 + 3]);
        }
        // F's image: rows fch (hi) and cp + fch (lo), piece pg (points 8 pg ..)
        if (fch < cp) {
          uint32_t hv[4], lv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split2(fv[2 * e], fv[2 * e + 1], hv[e], lv[e]);
          const uint32_t img = st0 + 2 * kFtPhi + kFtZeros;
          st_shared_v4(img + fch * 128 + (uint32_t)((pg ^ c7) << 4), hv[0], hv[1], hv[2], hv[3]);
          const int rl = cp + fch;
          st_shared_v4(img + rl * 128 + (uint32_t)((pg ^ (rl & 7)) << 4), lv[0], lv[1], lv[2], lv[3]);
        }
        // the next step's F
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int64_t p = p0 + 64 + pg * 8 + e;
          fv[e] = (fch < c && p < im.p_end) ? cc.F[p * cc.ldF + fch] : 0.f;
        }
        fence_proxy_async();
        mbar_arrive(smem_u32(&sm->afull[s]));
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int it = 0, tc = 0;
      bool ok = true;
      const uint32_t idesc = idesc_bf16(128, 256);
      for (int t = blockIdx.x; t < total_items && ok; t += gridDim.x, ++tc) {
        const FtItem im = ft_item(jobs, prefix, count, t);
        const int cp = apply_tc_cpad(calls[jobs[im.j].cloud].c);
        const int buf = tc & 1, ub = tc >> 1;
        if (ub > 0 && !mbar_wait(smem_u32(&sm->acce[buf]), (uint32_t)(ub - 1) & 1u, err, 33)) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * 256);
        for (int k = 0; k < im.steps; ++k, ++it) {
          const int s = it & 1;
          if (!mbar_wait(smem_u32(&sm->afull[s]), (uint32_t)(it >> 1) & 1u, err, 34)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t st0 = base + s * kFtStage, img = st0 + 2 * kFtPhi + kFtZeros;
          const uint32_t a1 = img - (uint32_t)((128 - 2 * cp) * 128), a2 = img - (uint32_t)((128 - cp) * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma_bf16(d, sdesc_sw128(a1 + kk * 32), sdesc_sw128(st0 + kk * 32), idesc, (k > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, sdesc_sw128(a2 + kk * 32), sdesc_sw128(st0 + kFtPhi + kk * 32), idesc, 1u);
          }
          mma_commit(smem_u32(&sm->aempty[s]));
        }
        if (ok) mma_commit(smem_u32(&sm->accf[buf]));
      }
      mma_commit(smem_u32(&sm->done));
      mbar_wait(smem_u32(&sm->done), 0u, err, 35);
    }
    __syncwarp();
  } else if (warp == kLoadWarp) {
    // ---------------- the points of each step: bulk copies ----------------
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total_items && ok; t += gridDim.x) {
        const FtItem im = ft_item(jobs, prefix, count, t);
        const float* xyz = jobs[im.j].xyz;
        for (int k = 0; k < im.steps; ++k, ++it) {
          const int xs = it % kFtXSlots, xu = it / kFtXSlots;
          if (xu > 0 && !mbar_wait(smem_u32(&sm->xempty[xs]), (uint32_t)(xu - 1) & 1u, err, 36)) {
            ok = false;
            break;
          }
          const int64_t p0 = im.p_begin + (int64_t)k * 64;
          const int np = (int)min((int64_t)64, im.p_end - p0);
          // np x 12 bytes, rounded up to 16: within the points' allocation (rounded up to 256 B)
          const uint32_t bytes = (uint32_t)((np * 12 + 15) & ~15);
          const uint32_t full = smem_u32(&sm->xfull[xs]);
          mbar_arrive_expect_tx(full, bytes);
          bulk_load(base + kFtOffX + xs * 768, xyz + p0 * 3, bytes, full);
        }
      }
      for (int q = (it > kFtXSlots ? it - kFtXSlots : 0); q < it; ++q)
        mbar_wait(smem_u32(&sm->xfull[q % kFtXSlots]), (uint32_t)(q / kFtXSlots) & 1u, err, 37);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: part[chunk][f][ch] = D_x + D_y ----------------
    const int quarter = warp & 3;
    const int et = threadIdx.x - kEpiWarp0 * 32;
    const int ch = et & 63, pofs = et >> 6;
    int tc = 0;
    for (int t = blockIdx.x; t < total_items; t += gridDim.x, ++tc) {
      const FtItem im = ft_item(jobs, prefix, count, t);
      const FieldPtsJob& jb = jobs[im.j];
      const int c = calls[jb.cloud].c, cp = apply_tc_cpad(c);
      const int lx = 128 - cp + ch, ly = 128 - 2 * cp + ch;
      const int buf = tc & 1;
      if (!epi_all(mbar_wait(smem_u32(&sm->accf[buf]), (uint32_t)(tc >> 1) & 1u, err, 38))) break;
      fence_after();
      float* part = jb.part + (size_t)im.chunk * jb.m * jb.ld;
#pragma unroll 1
      for (int col0 = 0; col0 < 256; col0 += 32) {
        float* er = E + (quarter * 32 + lane) * kAtEPitch;
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          uint32_t v[8];
          tmem_ld8_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 256 + col0 + 8 * hh), v);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 8; ++q) er[8 * hh + q] = __uint_as_float(v[q]);
        }
        epi_sync();
        if (ch < c) {
#pragma unroll 4
          for (int k = 0; k < 16; ++k) {
            const int col = col0 + 2 * k + pofs;  // feature column of the tile
            const int fr = im.ft * 128 + (col & 127);
            if (fr < jb.h) {
              const int f = (col < 128 ? 0 : jb.h) + fr;
              part[(size_t)f * jb.ld + ch] =
                  im.steps ? E[lx * kAtEPitch + 2 * k + pofs] + E[ly * kAtEPitch + 2 * k + pofs] : 0.f;
            }
          }
        }
        epi_sync();
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

}  // namespace

bool apply_tc_supported() { return tc::sm103_available(); }

cudaError_t apply_tc_prepare() {
  static cudaError_t once = [] {
    cudaError_t e = cudaFuncSetAttribute(apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAtSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fieldpts_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFtSmem);
    return e;
  }();
  return once;
}

cudaError_t launch_fieldpts_tc(const FieldPtsJob* jobs, const int* item_prefix, int count, int total_items, int grid,
                               const CloudCall* calls, int* err, cudaStream_t st) {
  if (total_items <= 0) return cudaSuccess;
  fieldpts_tc_kernel<<<grid, kAtThreads, kFtSmem, st>>>(jobs, item_prefix, count, total_items, calls, err);
  return launched();
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
