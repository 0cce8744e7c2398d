// Batched forms of the RFD steps (Sec. 2.4) around the tensor-core kernels:
// one launch serves every cloud of a batch (a single cloud is a batch of one).
// Jobs with a per-cloud number of blocks find their cloud by binary search over
// a prefix array of block counts (prefix[count] = total blocks).
//   a2  features_batched:  Phi[n, j] = cos 2 pi w_j^T x_n, Phi[n, h+j] = sin ..., bf16, blocked layout
//                          (64-point blocks of all rows, psi_index)
//       fill_batched:      F^T into rows m.. of the same buffer (bf16)
//   a3  reduce_batched:    fixed-order sum of the split-K partials, column scales applied
//   a5  small_batched:     Z = diag(s sgn r) G Y
//   a6  apply_batched:     out = F + Phi Z (F read before out is written: in place is fine)
//   a4  bcombine / bnorm1 / bfinite: element-wise pieces of the phi1 evaluation
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include "kernels.h"

namespace rfd {

namespace {

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

constexpr int kFeatThreads = 256;
constexpr int kFeatPts = 512;   // 8 warps x one 64-point block
constexpr int kFeatFreq = 32;

// A warp takes one 64-point block of Psi and 32 frequencies: lane = 8 g + pl
// handles points 8 pl .. 8 pl + 7 of the block and the frequencies
// j0 + 4 t + g (t = 0..7), so each store instruction writes rows
// j0 + 4t .. j0 + 4t + 3 of the block -- 4 adjacent rows of 128 bytes, one
// contiguous 512-byte span -- with 16-byte stores.
// blk_n > 0: a single cloud (job 0), only its 512-point blocks blk0 .. blk0 + blk_n - 1
// (the grid is blk_n x frequency groups); blk_n = 0: every block of every job.
__global__ void __launch_bounds__(kFeatThreads)
features_batched_kernel(const FeatJob* __restrict__ jobs, const int* __restrict__ prefix, int count,
                        const CloudCall* __restrict__ calls, int blk0, int blk_n) {
  int j = 0, bxi, byi;
  if (blk_n > 0) {
    bxi = blk0 + (int)(blockIdx.x % blk_n);
    byi = (int)(blockIdx.x / blk_n);
  } else {
    j = find_job(prefix, count, blockIdx.x);
    const int local = blockIdx.x - prefix[j];
    bxi = local % jobs[j].bx;
    byi = local / jobs[j].bx;
  }
  const FeatJob jb = jobs[j];
  const float* __restrict__ pts = calls[jb.cloud].pts;
  if (!pts) return;  // a call table without this cloud's points: nothing to read
  __shared__ float w_s[kFeatFreq][3];  // 2 pi w: the phase in radians
  const int j0 = byi * kFeatFreq;
  const int jn = min(kFeatFreq, jb.h - j0);
  if (threadIdx.x < jn * 3)
    w_s[threadIdx.x / 3][threadIdx.x % 3] = 6.283185307179586f * jb.omega[(size_t)j0 * 3 + threadIdx.x];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, pl = lane & 7, g = lane >> 3;
  const int64_t p0 = (int64_t)bxi * kFeatPts + warp * 64 + pl * 8;  // first of this lane's 8 points
  if (p0 >= jb.n_pad) return;  // whole 64-point blocks: the warp exits together
  float x[8][3];
  bool valid[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    valid[q] = (p0 + q) < jb.n;
#pragma unroll
    for (int d = 0; d < 3; ++d) x[q][d] = valid[q] ? pts[(p0 + q) * 3 + d] : 0.f;
  }
  if (byi == 0 && g == 0)  // the cloud's own copy of its points, for the apply
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (valid[q])
#pragma unroll
        for (int d = 0; d < 3; ++d) jb.xyz[(p0 + q) * 3 + d] = x[q][d];
  auto* psi = reinterpret_cast<uint4*>(jb.psi);
  for (int t = 0; t < kFeatFreq / 4; ++t) {
    const int jj = 4 * t + g;
    if (jj >= jn) break;
    const float w0 = w_s[jj][0], w1 = w_s[jj][1], w2 = w_s[jj][2];
    uint32_t c2[4], s2[4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      float c[2], sn[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        // the phase straight into MUFU sin/cos: ~|ang| 2^-23 of error (1.4e-4 at 1000 rad), far
        // below the BF16 rounding of the stored features; reducing it first cost 4 instructions
        // of ~13 in this issue-bound loop
        const float ang = fmaf(w0, x[q + u][0], fmaf(w1, x[q + u][1], w2 * x[q + u][2]));
        c[u] = valid[q + u] ? __cosf(ang) : 0.f;
        sn[u] = valid[q + u] ? __sinf(ang) : 0.f;
      }
      const __nv_bfloat162 cb = __floats2bfloat162_rn(c[0], c[1]), sb = __floats2bfloat162_rn(sn[0], sn[1]);
      c2[q / 2] = *reinterpret_cast<const uint32_t*>(&cb);
      s2[q / 2] = *reinterpret_cast<const uint32_t*>(&sb);
    }
    const int jg = j0 + jj;
    // 8 bf16 of row jg (and row h + jg) at points 8 pl .. of the block: one 16-byte store each
    psi[psi_index(p0, jg, jb.rows_alloc) / 8] = make_uint4(c2[0], c2[1], c2[2], c2[3]);
    psi[psi_index(p0, jb.h + jg, jb.rows_alloc) / 8] = make_uint4(s2[0], s2[1], s2[2], s2[3]);
  }
}

// F^T rows of the feature buffer, for fields of up to 8 channels: one point
// per thread, every row of the point written by it (coalesced along the
// points); points >= N and rows beyond the channels get zeros.
__global__ void __launch_bounds__(256)
fill_batched_kernel(const FillJob* __restrict__ jobs, const int* __restrict__ prefix, int count,
                    const CloudCall* __restrict__ calls) {
  const int j = find_job(prefix, count, blockIdx.x);
  const FillJob jb = jobs[j];
  const CloudCall cc = calls[jb.cloud];
  const int64_t p = (int64_t)(blockIdx.x - prefix[j]) * 256 + threadIdx.x;
  if (p >= jb.n_pad) return;
  auto* psi = reinterpret_cast<__nv_bfloat16*>(jb.psi);
  const int c = cc.c, r0 = jb.row0, ra = jb.rows_alloc;
  const bool valid = p < jb.n;
  const float* f = cc.F + (valid ? p * cc.ldF : 0);
  for (int ch = 0; ch < c; ++ch) {
    const float v = valid ? f[ch] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    psi[psi_index(p, r0 + ch, ra)] = hi;
    // row c + ch: the lo part of channel ch (fsplit)
    if (jb.fsplit) psi[psi_index(p, r0 + c + ch, ra)] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int row = jb.fsplit ? 2 * c : c; row < jb.cpad; ++row) psi[psi_index(p, r0 + row, ra)] = zero;
}

// The same for wider fields: a block per 64-point block of Psi and group of 32
// channels; each warp takes 8 points, each lane one channel: 8 loads of F (a
// warp's loads are 128 contiguous bytes when ldF = c), then the 8 points' hi
// and lo parts as one 16-byte store each into the channel's rows.  The first
// channel group's block also zeroes the rows beyond the channels.
__global__ void __launch_bounds__(256)
fill_wide_batched_kernel(const FillJob* __restrict__ jobs, const int* __restrict__ prefix, int count,
                         const CloudCall* __restrict__ calls) {
  const int j = find_job(prefix, count, blockIdx.x);
  const FillJob jb = jobs[j];
  const CloudCall cc = calls[jb.cloud];
  const int local = blockIdx.x - prefix[j];
  const int pb = local % jb.bxw, cgi = local / jb.bxw;
  const int c = cc.c, r0 = jb.row0, ra = jb.rows_alloc;
  const int lane = threadIdx.x & 31;
  const int64_t p0 = (int64_t)pb * 64 + (threadIdx.x >> 5) * 8;
  auto* psi = reinterpret_cast<uint4*>(jb.psi);  // 8 points of row r: psi_index(p0, r, ra) / 8
  const int ch = cgi * 32 + lane;
  if (ch < c) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (p0 + e < jb.n) ? cc.F[(p0 + e) * cc.ldF + ch] : 0.f;
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
      hi[e] = *reinterpret_cast<const uint32_t*>(&h);
      lo[e] = *reinterpret_cast<const uint32_t*>(&l);
    }
    psi[psi_index(p0, r0 + ch, ra) / 8] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    // row c + ch: the lo part of channel ch (fsplit)
    if (jb.fsplit) psi[psi_index(p0, r0 + c + ch, ra) / 8] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
  if (cgi == 0)
    for (int rr = (jb.fsplit ? 2 * c : c) + lane; rr < jb.cpad; rr += 32)
      psi[psi_index(p0, r0 + rr, ra) / 8] = make_uint4(0u, 0u, 0u, 0u);
}

// One thread per tile element; lanes summed in order (deterministic),
// compensated FP32; the compensated sum scaled by the column scales in FP64
// (step a4's input).
__global__ void reduce_batched_kernel(const RedTile* __restrict__ tiles, const CloudCall* __restrict__ calls) {
  const RedTile t = tiles[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = e / kTcBNMax, col = e % kTcBNMax;
  if (r >= t.ni || col >= t.nj) return;
  const float* p = t.part + (int64_t)r * t.ld + t.col_off + col;
  Fp32Sum acc;
  int u = 0;
  for (; u + 4 <= t.count; u += 4) {  // four loads in flight, summed in lane order
    const float a0 = p[(int64_t)u * t.slot_elems], a1 = p[(int64_t)(u + 1) * t.slot_elems];
    const float a2 = p[(int64_t)(u + 2) * t.slot_elems], a3 = p[(int64_t)(u + 3) * t.slot_elems];
    acc.add(a0);
    acc.add(a1);
    acc.add(a2);
    acc.add(a3);
  }
  for (; u < t.count; ++u) acc.add(p[(int64_t)u * t.slot_elems]);
  const int f = t.i0 + r;
  if (t.kind == kTileGram) {
    const int g = t.j0 + col;
    if (f > g) return;  // the mirrored entry (g, f) is covered as (row g, column f)
    // M = diag(s) K diag(s sgn r) with the commutative product s_f s_g, so that
    // M diag(sgn r) is exactly symmetric
    const double v = acc.wide() * (t.ob[f] * t.ob[g]);
    t.M[(size_t)f * t.m + g] = t.oa[g] < 0.0 ? -v : v;
    if (f != g) t.M[(size_t)g * t.m + f] = t.oa[f] < 0.0 ? -v : v;
  } else {
    const int c = calls[t.cloud].c;
    if (col < c) {
      if (t.fsplit) {  // add the lo column of the same channel
        const float* q = t.part + (int64_t)r * t.ld + t.col_off + c + col;
        for (int u = 0; u < t.count; ++u) acc.add(q[(int64_t)u * t.slot_elems]);
      }
      t.Y[(size_t)f * c + col] = t.ob[f] * acc.wide();
    }
  }
}

// Z[f, ch] = oa[f] sum_g G[f, g] Y[g, ch]: a block of 256 threads per row f,
// the threads over g, channels in groups of 8.  FP32 products; each thread's
// terms, the warp sums and the 8 warps' sums are compensated FP32 sums (Z is
// stored in FP32 and enters out = F + Phi Z, an increment on F).
__global__ void __launch_bounds__(256) small_batched_kernel(const ApplyJob* __restrict__ jobs,
                                                            const int* __restrict__ prefix, int count,
                                                            const CloudCall* __restrict__ calls) {
  constexpr int kCC = 8;
  const int j = find_job(prefix, count, blockIdx.x);
  const ApplyJob jb = jobs[j];
  const int f = blockIdx.x - prefix[j];
  const int c = calls[jb.cloud].c, m = jb.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ float red[8][kCC][2];
  const double* grow = jb.G + (size_t)f * m;
  for (int ch0 = 0; ch0 < c; ch0 += kCC) {
    const int nc = min(kCC, c - ch0);
    Fp32Sum acc[kCC];
    for (int g = threadIdx.x; g < m; g += 256) {
      const float gv = (float)grow[g];
      const double* yrow = jb.Y + (size_t)g * c + ch0;
#pragma unroll
      for (int q = 0; q < kCC; ++q)
        if (q < nc) acc[q].add(gv * (float)yrow[q]);
    }
#pragma unroll
    for (int q = 0; q < kCC; ++q) {
      if (q >= nc) break;  // the group's channels only (nc is uniform across the block)
      // warp sum of the (sum, compensation) pairs: each butterfly step adds a pair as two terms
      Fp32Sum v = acc[q];
      for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, v.s, o), oc = __shfl_xor_sync(0xffffffffu, v.c, o);
        v.add(os);
        v.c += oc;
      }
      if (lane == 0) {
        red[warp][q][0] = v.s;
        red[warp][q][1] = v.c;
      }
    }
    __syncthreads();
    if (threadIdx.x < nc) {
      Fp32Sum tot;
      for (int w = 0; w < 8; ++w) {
        tot.add(red[w][threadIdx.x][0]);
        tot.add(red[w][threadIdx.x][1]);
      }
      jb.Z[(size_t)f * c + ch0 + threadIdx.x] = (float)jb.oa[f] * tot.value();
    }
    __syncthreads();
  }
}

// Z for wide fields (more than 16 channels): a block per 8 rows f and 64
// channels; each thread one channel, all 8 rows (8 independent sums) and a
// quarter of g.  G's rows pass through shared memory (as FP32) 512 columns at
// a time, Y is read along the channels.  Each thread's terms are compensated
// FP32 sums in g order, and the four quarters' (sum, compensation) pairs are
// added in quarter order (Z is stored in FP32).  Blocks of channels >= c
// return at once (the prefix counts the plan's max_channels).
__global__ void __launch_bounds__(256) small_wide_batched_kernel(const ApplyJob* __restrict__ jobs,
                                                                 const int* __restrict__ prefix, int count,
                                                                 const CloudCall* __restrict__ calls) {
  constexpr int kG = 512;
  const int j = find_job(prefix, count, blockIdx.x);
  const ApplyJob jb = jobs[j];
  const int c = calls[jb.cloud].c, m = jb.m;
  const int local = blockIdx.x - prefix[j];
  const int nrb = (m + 7) / 8;
  const int f0 = (local % nrb) * 8, ch0 = (local / nrb) * 64;
  if (ch0 >= c) return;
  const int cl = threadIdx.x & 63, qt = threadIdx.x >> 6, ch = ch0 + cl;
  __shared__ float gs[8][kG];
  __shared__ float red[4][8][64][2];
  Fp32Sum a[8];
  for (int g0 = 0; g0 < m; g0 += kG) {
    const int gn = min(kG, m - g0);
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * kG; i += 256) {
      const int r = i / kG, gi = i % kG;
      gs[r][gi] = (f0 + r < m && gi < gn) ? (float)jb.G[(size_t)(f0 + r) * m + g0 + gi] : 0.f;
    }
    __syncthreads();
    const int qn = (gn + 3) / 4, gb = qt * qn, ge = min(gn, gb + qn);
    if (ch < c)
      for (int gi = gb; gi < ge; ++gi) {
        const float y = (float)jb.Y[(size_t)(g0 + gi) * c + ch];
#pragma unroll
        for (int r = 0; r < 8; ++r) a[r].add(gs[r][gi] * y);
      }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    red[qt][r][cl][0] = a[r].s;
    red[qt][r][cl][1] = a[r].c;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r = qt * 2 + k, f = f0 + r;
    if (ch < c && f < m) {
      Fp32Sum tot;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        tot.add(red[q][r][cl][0]);
        tot.add(red[q][r][cl][1]);
      }
      jb.Z[(size_t)f * c + ch] = (float)jb.oa[f] * tot.value();
    }
  }
}

// out[n, ch] = F[n, ch] + sum_j (cos(2 pi w_j^T x_n) Z[j, ch] + sin(2 pi w_j^T x_n) Z[h + j, ch]):
// the features are recomputed in FP32 from the cloud's copy of its points
// instead of read back from the BF16 Psi, so the apply carries no BF16
// rounding and reads only points, F and out.  The phase in radians is the
// FP32 t = (2 pi w)^T x (absolute error ~|t| 2^-24), given to MUFU sin/cos
// as it is: their own handling of a large argument adds about |t| 2^-23
// (measured on this GPU: 1.4e-4 at |t| = 1000), far below the BF16 rounding
// of Phi in the B^T F of the form this kernel serves.  Reducing t to one
// period first (4 of the ~19 instructions per point and frequency) made this
// issue-bound kernel 11 % slower.  A block of 256 threads covers 512 points,
// two per thread (p and p + 256), which share each frequency's shared-memory
// loads (its w and Z rows); four points per thread cut the instructions by
// 14 % but halved the resident warps and left a 1.6-wave tail at N = 10^6,
// and ran 10 % slower.  CG channels per thread.  F[n] is read before out[n]
// is written by the same thread.
template <int CG>
__global__ void __launch_bounds__(kApplyPts / 2)
apply_batched_kernel(const ApplyJob* __restrict__ jobs, const int* __restrict__ prefix, int count,
                     const CloudCall* __restrict__ calls) {
  constexpr int kChunk = 64;
  constexpr int UP = 2;  // points per thread
  constexpr int kThreads = kApplyPts / UP;
  constexpr int CW = (CG + 3) / 4;  // float4 per row of Z in shared memory (CG channels used)
  __shared__ float4 w_s[kChunk];
  __shared__ float4 zc[kChunk][CW], zsn[kChunk][CW];
  const int j = find_job(prefix, count, blockIdx.x);
  const ApplyJob jb = jobs[j];
  const CloudCall cc = calls[jb.cloud];
  const int local = blockIdx.x - prefix[j];
  const int bxi = local % jb.bx, cgi = local / jb.bx;
  const int h = jb.m / 2;
  int64_t p[UP];
  bool valid[UP];
  float x[UP][3];
#pragma unroll
  for (int u = 0; u < UP; ++u) {
    p[u] = (int64_t)bxi * kApplyPts + u * kThreads + threadIdx.x;
    valid[u] = p[u] < jb.n;
#pragma unroll
    for (int d = 0; d < 3; ++d) x[u][d] = valid[u] ? jb.xyz[p[u] * 3 + d] : 0.f;
  }
  const int ch0 = cgi * CG;
  const int cg = min(CG, cc.c - ch0);
  float acc[UP][CG];
#pragma unroll
  for (int u = 0; u < UP; ++u)
#pragma unroll
    for (int q = 0; q < CG; ++q) acc[u][q] = 0.f;
  const float two_pi = 6.283185307179586f;
  for (int f0 = 0; f0 < h; f0 += kChunk) {
    const int fn = min(kChunk, h - f0);
    __syncthreads();
    for (int i = threadIdx.x; i < kChunk; i += kThreads) {  // 2 pi w: the phase in radians
      const float* w = jb.omega_hi + (size_t)(f0 + i) * 3;
      w_s[i] = i < fn ? make_float4(two_pi * w[0], two_pi * w[1], two_pi * w[2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = threadIdx.x; i < kChunk * CW * 4; i += kThreads) {
      const int fr = i / (CW * 4), q = i % (CW * 4);
      const bool ok = fr < fn && q < cg;
      reinterpret_cast<float*>(zc[fr])[q] = ok ? jb.Z[(size_t)(f0 + fr) * cc.c + ch0 + q] : 0.f;
      reinterpret_cast<float*>(zsn[fr])[q] = ok ? jb.Z[(size_t)(h + f0 + fr) * cc.c + ch0 + q] : 0.f;
    }
    __syncthreads();
    for (int fr = 0; fr < fn; ++fr) {
      const float4 w = w_s[fr];
      float cs[UP], sn[UP];
#pragma unroll
      for (int u = 0; u < UP; ++u) {
        const float ang = fmaf(w.x, x[u][0], fmaf(w.y, x[u][1], w.z * x[u][2]));
        cs[u] = __cosf(ang);
        sn[u] = __sinf(ang);
      }
#pragma unroll
      for (int q4 = 0; q4 < CW; ++q4) {
        const float4 a4 = zc[fr][q4], b4 = zsn[fr][q4];
        const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (4 * q4 + e < CG)  // compile-time: the channels of the group only
#pragma unroll
            for (int u = 0; u < UP; ++u)
              acc[u][4 * q4 + e] = fmaf(cs[u], a[e], fmaf(sn[u], b[e], acc[u][4 * q4 + e]));
      }
    }
  }
#pragma unroll
  for (int u = 0; u < UP; ++u)
    if (valid[u])
      for (int q = 0; q < cg; ++q) {
        const float fv = cc.F[p[u] * cc.ldF + ch0 + q];
        cc.out[p[u] * cc.ldOut + ch0 + q] = fv + acc[u][q];
      }
}

// Y' partials from the points (compact plans, see FieldPtsJob): 256 threads,
// each with FPT frequencies (fieldpts_fpt: 2 for up to 8 channels per block,
// else 1), one chunk of points and CG channels per block.  The points (as
// float4) and the block's F columns (float4 groups) pass through shared memory
// 128 points at a time; every thread reads the same point, so each point costs
// one 16-byte broadcast load plus one per 4 channels, shared by the thread's
// frequencies.  Phi(n, f) is the apply's FP32 feature (the phase in radians,
// unreduced, into MUFU sin / cos); plain FP32 sums over the chunk's points.
template <int CG>
__global__ void __launch_bounds__(256)
fieldpts_batched_kernel(const FieldPtsJob* __restrict__ jobs, const int* __restrict__ prefix, int count,
                        const CloudCall* __restrict__ calls) {
  constexpr int kTile = 128;
  constexpr int FPT = fieldpts_fpt(CG);
  constexpr int CW = (CG + 3) / 4;
  __shared__ float4 xs[kTile];
  __shared__ float4 fs[kTile][CW];
  const int j = find_job(prefix, count, blockIdx.x);
  const FieldPtsJob jb = jobs[j];
  const CloudCall cc = calls[jb.cloud];
  const int fgroups = (jb.h + 256 * FPT - 1) / (256 * FPT);
  const int local = blockIdx.x - prefix[j];
  const int chunk = local % jb.chunks, rest = local / jb.chunks;
  const int fg = rest % fgroups, cgi = rest / fgroups;
  const int ch0 = cgi * CG, cg = min(CG, cc.c - ch0);
  const float two_pi = 6.283185307179586f;
  int fi[FPT];
  float w[FPT][3];  // 2 pi w: the phase in radians
#pragma unroll
  for (int u = 0; u < FPT; ++u) {
    fi[u] = (fg * FPT + u) * 256 + threadIdx.x;
#pragma unroll
    for (int d = 0; d < 3; ++d) w[u][d] = fi[u] < jb.h ? two_pi * jb.omega_hi[(size_t)fi[u] * 3 + d] : 0.f;
  }
  float acc_c[FPT][CG], acc_s[FPT][CG];
#pragma unroll
  for (int u = 0; u < FPT; ++u)
#pragma unroll
    for (int q = 0; q < CG; ++q) acc_c[u][q] = acc_s[u][q] = 0.f;
  const int64_t p_begin = (int64_t)chunk * jb.pts, p_end = min(jb.n, p_begin + jb.pts);
  for (int64_t p0 = p_begin; p0 < p_end; p0 += kTile) {
    const int np = (int)min((int64_t)kTile, p_end - p0);
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      const float* x = jb.xyz + (p0 + i) * 3;
      xs[i] = make_float4(x[0], x[1], x[2], 0.f);
    }
    for (int i = threadIdx.x; i < np * CW * 4; i += blockDim.x) {
      const int pp = i / (CW * 4), q = i % (CW * 4);
      reinterpret_cast<float*>(fs[pp])[q] = q < cg ? cc.F[(p0 + pp) * cc.ldF + ch0 + q] : 0.f;
    }
    __syncthreads();
    for (int pp = 0; pp < np; ++pp) {
      const float4 x = xs[pp];
      float fv[CW * 4];
#pragma unroll
      for (int q4 = 0; q4 < CW; ++q4) {
        const float4 v = fs[pp][q4];
        fv[4 * q4] = v.x;
        fv[4 * q4 + 1] = v.y;
        fv[4 * q4 + 2] = v.z;
        fv[4 * q4 + 3] = v.w;
      }
#pragma unroll
      for (int u = 0; u < FPT; ++u) {
        const float ang = fmaf(w[u][0], x.x, fmaf(w[u][1], x.y, w[u][2] * x.z));
        const float cs = __cosf(ang), sn = __sinf(ang);
#pragma unroll
        for (int q = 0; q < CG; ++q) {
          acc_c[u][q] = fmaf(cs, fv[q], acc_c[u][q]);
          acc_s[u][q] = fmaf(sn, fv[q], acc_s[u][q]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < FPT; ++u) {
    if (fi[u] >= jb.h) continue;
    float* pc = jb.part + ((size_t)chunk * jb.m + fi[u]) * jb.ld + ch0;
    float* ps = jb.part + ((size_t)chunk * jb.m + jb.h + fi[u]) * jb.ld + ch0;
#pragma unroll
    for (int q = 0; q < CG; ++q)
      if (q < cg) {
        pc[q] = acc_c[u][q];
        ps[q] = acc_s[u][q];
      }
  }
}

// Y[f, ch] = ob[f] sum over the chunks of the fieldpts partials (compact plans):
// one warp per feature row f and group of 4 channels; lane l sums the chunks
// l, l + 32, ... (one 16-byte load each) in compensated FP32, the lanes'
// (sum, carry) pairs meet in a fixed butterfly order (deterministic), and the
// pair is scaled in FP64.  The loads of a warp go to 32 chunks at once.
__global__ void __launch_bounds__(256) fieldpts_reduce_kernel(const FieldPtsJob* __restrict__ jobs,
                                                              const int* __restrict__ prefix, int count,
                                                              const CloudCall* __restrict__ calls) {
  const int j = find_job(prefix, count, blockIdx.x);
  const FieldPtsJob jb = jobs[j];
  const int c = calls[jb.cloud].c, cq = (c + 3) / 4;
  const int w = (blockIdx.x - prefix[j]) * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= jb.m * cq) return;  // w is uniform across the warp
  const int f = w / cq, q0 = (w % cq) * 4;
  const float* base = jb.part + (size_t)f * jb.ld + q0;
  const size_t chunk_stride = (size_t)jb.m * jb.ld;
  Fp32Sum acc[4];
  for (int u = lane; u < jb.chunks; u += 32) {
    const float4 v = *reinterpret_cast<const float4*>(base + (size_t)u * chunk_stride);
    acc[0].add(v.x);
    acc[1].add(v.y);
    acc[2].add(v.z);
    acc[3].add(v.w);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    Fp32Sum v = acc[q];
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, v.s, o), oc = __shfl_xor_sync(0xffffffffu, v.c, o);
      v.add(os);
      v.add(oc);
    }
    if (lane == 0 && q0 + q < c) jb.Y[(size_t)f * c + q0 + q] = jb.ob[f] * v.wide();
  }
}

__device__ __forceinline__ const double* slot_ptr(const PhiCloud& pc, int slot) {
  return slot == kSlotM ? pc.M : (slot == kSlotG ? pc.G : pc.work + (size_t)slot * pc.m * pc.m);
}

struct Comb {
  int src[4];
  double a[4];
};

__global__ void bcombine_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix, int count, int dst,
                                Comb cb, double diag, int kmode, int mask_k) {
  const int j = find_job(prefix, count, blockIdx.x);
  const PhiCloud pc = pcs[j];
  if (mask_k >= 0 && pc.s <= mask_k) return;
  const int64_t e = (int64_t)(blockIdx.x - prefix[j]) * blockDim.x + threadIdx.x;
  const int m = pc.m;
  if (e >= (int64_t)m * m) return;
  const int r = (int)(e / m), c = (int)(e % m);
  const double k = (kmode == 1) ? pc.lambda : (kmode == 2 ? pc.scale : 1.0);
  double v = (r == c) ? diag : 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (cb.src[i] != 0x7fffffff) v += cb.a[i] * slot_ptr(pc, cb.src[i])[e];
  const_cast<double*>(slot_ptr(pc, dst))[e] = k * v;
}

// Max column abs-sum per cloud: block (32 columns x 32 row lanes), atomicMax on the bits.
__global__ void bnorm1_kernel(const PhiCloud* __restrict__ pcs, int slot, unsigned long long* norms) {
  const PhiCloud pc = pcs[blockIdx.y];
  const int m = pc.m;
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (blockIdx.x * 32 >= m) return;
  const double* X = slot_ptr(pc, slot);
  __shared__ double part[32][33];
  double s = 0.0;
  if (col < m)
    for (int i = threadIdx.y; i < m; i += 32) s += fabs(X[(size_t)i * m + col]);
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && col < m) {
    double t = 0.0;
    for (int y = 0; y < 32; ++y) t += part[y][threadIdx.x];
    if (!(t == t)) t = __longlong_as_double(0x7FF0000000000000ll);
    atomicMax(norms + blockIdx.y, (unsigned long long)__double_as_longlong(t));
  }
}

// Squarings of each cloud (degree-5 rule): s = 0 when ||X||_1 <= theta, else the
// least s with 2^-s ||X||_1 <= theta, found exactly from the binary exponent of
// ||X||_1 / theta.  Writes s and 2^-s into the cloud table, s into sv[k] and
// the largest s into sv[count].  A cloud whose norm is not finite or needs more
// than max_s squarings is flagged (and runs with s = 0: its G is not used).
__global__ void bselect_kernel(PhiCloud* __restrict__ pcs, int count, const double* __restrict__ norms,
                               double theta, int max_s, int* __restrict__ sv) {
  __shared__ int smax;
  if (threadIdx.x == 0) smax = 0;
  __syncthreads();
  int mx = 0;
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    const double nrm = norms[k];
    bool bad = !isfinite(nrm);
    int s = 0;
    if (!bad && nrm > theta) {
      int e = 0;
      const double f = frexp(nrm / theta, &e);  // nrm / theta = f 2^e, f in [1/2, 1)
      s = (f == 0.5) ? e - 1 : e;
      bad = s > max_s;
    }
    if (bad) {
      s = 0;
      atomicExch(pcs[k].flag, 1);
    }
    pcs[k].s = s;
    pcs[k].scale = ldexp(1.0, -s);
    sv[k] = s;
    mx = max(mx, s);
  }
  atomicMax(&smax, mx);
  __syncthreads();
  if (threadIdx.x == 0) sv[count] = smax;
}

__global__ void bfinite_kernel(const PhiCloud* __restrict__ pcs, const int* __restrict__ prefix, int count, int slot) {
  const int j = find_job(prefix, count, blockIdx.x);
  const PhiCloud pc = pcs[j];
  const int64_t e = (int64_t)(blockIdx.x - prefix[j]) * blockDim.x + threadIdx.x;
  if (e >= (int64_t)pc.m * pc.m) return;
  if (!isfinite(slot_ptr(pc, slot)[e])) atomicExch(pc.flag, 1);
}

}  // namespace

cudaError_t launch_features_batched(const FeatJob* jobs, const int* prefix, int count, int total_blocks,
                                    const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  features_batched_kernel<<<total_blocks, kFeatThreads, 0, st>>>(jobs, prefix, count, calls, 0, 0);
  return launched();
}

cudaError_t launch_features_range(const FeatJob* jobs, const CloudCall* calls, int h, int blk0, int blk_n,
                                  cudaStream_t st) {
  if (blk_n <= 0) return cudaSuccess;
  const int groups = (h + kFeatFreq - 1) / kFeatFreq;
  features_batched_kernel<<<blk_n * groups, kFeatThreads, 0, st>>>(jobs, nullptr, 1, calls, blk0, blk_n);
  return launched();
}

cudaError_t launch_fill_batched(const FillJob* jobs, const int* prefix, int count, int total_blocks,
                                const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  fill_batched_kernel<<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls);
  return launched();
}

cudaError_t launch_fill_wide_batched(const FillJob* jobs, const int* prefix, int count, int total_blocks,
                                     const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  fill_wide_batched_kernel<<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls);
  return launched();
}

cudaError_t launch_reduce_batched(const RedTile* tiles, int num_tiles, const CloudCall* calls, cudaStream_t st) {
  if (num_tiles <= 0) return cudaSuccess;
  dim3 grid((unsigned)((kTcBM * kTcBNMax + 255) / 256), (unsigned)num_tiles);
  reduce_batched_kernel<<<grid, 256, 0, st>>>(tiles, calls);
  return launched();
}

cudaError_t launch_small_batched(const ApplyJob* jobs, const int* prefix, int count, int total_rows,
                                 const CloudCall* calls, cudaStream_t st) {
  if (total_rows <= 0) return cudaSuccess;
  small_batched_kernel<<<total_rows, 256, 0, st>>>(jobs, prefix, count, calls);
  return launched();
}

cudaError_t launch_small_wide_batched(const ApplyJob* jobs, const int* prefix, int count, int total_blocks,
                                      const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  small_wide_batched_kernel<<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls);
  return launched();
}

cudaError_t launch_apply_batched(const ApplyJob* jobs, const int* prefix, int count, int total_blocks, int cg,
                                 const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  switch (cg) {
    case 3: apply_batched_kernel<3><<<total_blocks, kApplyPts / 2, 0, st>>>(jobs, prefix, count, calls); break;
    case 4: apply_batched_kernel<4><<<total_blocks, kApplyPts / 2, 0, st>>>(jobs, prefix, count, calls); break;
    case 8: apply_batched_kernel<8><<<total_blocks, kApplyPts / 2, 0, st>>>(jobs, prefix, count, calls); break;
    case 16: apply_batched_kernel<16><<<total_blocks, kApplyPts / 2, 0, st>>>(jobs, prefix, count, calls); break;
    case 32: apply_batched_kernel<32><<<total_blocks, kApplyPts / 2, 0, st>>>(jobs, prefix, count, calls); break;
    default: return cudaErrorInvalidValue;
  }
  return launched();
}

cudaError_t launch_fieldpts_batched(const FieldPtsJob* jobs, const int* prefix, int count, int total_blocks, int cg,
                                    const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  switch (cg) {
    case 3: fieldpts_batched_kernel<3><<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls); break;
    case 4: fieldpts_batched_kernel<4><<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls); break;
    case 8: fieldpts_batched_kernel<8><<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls); break;
    case 16: fieldpts_batched_kernel<16><<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls); break;
    case 32: fieldpts_batched_kernel<32><<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls); break;
    default: return cudaErrorInvalidValue;
  }
  return launched();
}

cudaError_t launch_fieldpts_reduce(const FieldPtsJob* jobs, const int* prefix, int count, int total_blocks,
                                   const CloudCall* calls, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  fieldpts_reduce_kernel<<<total_blocks, 256, 0, st>>>(jobs, prefix, count, calls);
  return launched();
}

cudaError_t launch_bcombine(const PhiCloud* pc, const int* prefix, int count, int total_blocks, int dst,
                            const int* src4, const double* a4, double diag, int kmode, int mask_k, cudaStream_t st) {
  Comb cb;
  for (int i = 0; i < 4; ++i) {
    cb.src[i] = src4 ? src4[i] : 0x7fffffff;
    cb.a[i] = a4 ? a4[i] : 0.0;
  }
  bcombine_kernel<<<total_blocks, 256, 0, st>>>(pc, prefix, count, dst, cb, diag, kmode, mask_k);
  return launched();
}

cudaError_t launch_bnorm1(const PhiCloud* pc, int count, int max_m, int slot, double* norms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(norms, 0, (size_t)count * sizeof(double), st);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((max_m + 31) / 32), (unsigned)count);
  bnorm1_kernel<<<grid, dim3(32, 32), 0, st>>>(pc, slot, reinterpret_cast<unsigned long long*>(norms));
  return launched();
}

cudaError_t launch_bselect(PhiCloud* pc, int count, const double* norms, double theta, int max_s, int* sv,
                           cudaStream_t st) {
  bselect_kernel<<<1, 256, 0, st>>>(pc, count, norms, theta, max_s, sv);
  return launched();
}

cudaError_t launch_bfinite(const PhiCloud* pc, const int* prefix, int count, int total_blocks, int slot,
                           cudaStream_t st) {
  bfinite_kernel<<<total_blocks, 256, 0, st>>>(pc, prefix, count, slot);
  return launched();
}

}  // namespace rfd
