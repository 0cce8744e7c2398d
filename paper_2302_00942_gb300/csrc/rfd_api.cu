// C ABI of the RFD integrator: plan management and the entry points that run
// steps a2..a6 (Sec. 2.4) on the plan's CUDA stream.  See include/rfd.h for
// the contract of every function.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "kernels.h"
#include "rfd_internal.h"
#include "rfd_phi1.h"

namespace rfd {
const char* last_error_cstr();
thread_local long long t_kernel_launches = 0;
}

using namespace rfd;

namespace {

constexpr int kMaxM = 4096;
constexpr int kMaxChannels = 256;

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Allocation hook: every device allocation of a plan goes through here, so a
// test can make the n-th allocation fail (RFD_ENOMEM path) without a GPU fault.
int g_fail_alloc_after = -1;  // -1: never; k >= 0: the allocation after k more succeeds fails

cudaError_t dev_alloc(void** p, size_t bytes) {
  if (g_fail_alloc_after == 0) {
    g_fail_alloc_after = -1;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (g_fail_alloc_after > 0) --g_fail_alloc_after;
  return cudaMalloc(p, bytes);
}

struct TileSet {
  std::vector<GramTile> tiles;
  std::vector<GramUnit> units;
  GramTile* d_tiles = nullptr;
  GramUnit* d_units = nullptr;
  int slots = 0;  // partial slots used
};

}  // namespace

struct rfd_plan_s {
  rfd_params p{};
  cudaStream_t stream = nullptr;
  int m = 0, h = 0, cpad = 0, sms = 0;
  int64_t n = 0, n_pad = 0;
  int rows_alloc = 0;
  bool bf16 = false;
  std::vector<double> omega, r, oa, ob;
  // device
  float* d_omega_hi = nullptr;
  float* d_omega_lo = nullptr;
  double* d_oa = nullptr;
  double* d_ob = nullptr;
  void* d_psi = nullptr;
  float* d_part = nullptr;
  int64_t slot_elems = 0;
  double* d_M = nullptr;
  double* d_Y = nullptr;
  double* d_G = nullptr;
  float* d_Z = nullptr;
  double* d_work = nullptr;
  int* d_ipiv = nullptr;
  int* d_ints = nullptr;      // [0] error word, [1] LU info, [2] finite flag
  double* d_scalar = nullptr;
  TileSet gram_only, field_only, both;
  bool have_G = false;
  rfd_stats stats{};
  std::vector<void*> allocs;
  // step timing (RFD_FLAG_TIMING): a ring of per-call event sets, folded into
  // the sums when the stream is synchronised by rfd_plan_stats
  struct Slot {
    cudaEvent_t ev[2 * RFD_NUM_STEPS];
    bool used[RFD_NUM_STEPS];
  };
  bool timing = false;
  std::vector<Slot> ring;
  int ring_head = 0, ring_pending = 0;
  Slot* cur = nullptr;
  double step_sum[RFD_NUM_STEPS] = {};
  long long timed_calls = 0;
  long long launches = 0;
  long long launch_mark = 0;
};

namespace {

constexpr int kRing = 64;

void fold_timings(rfd_plan_s* pl) {
  if (!pl->timing || pl->ring_pending == 0) return;
  cudaStreamSynchronize(pl->stream);
  for (int k = pl->ring_pending; k > 0; --k) {
    auto& s = pl->ring[(pl->ring_head - k + kRing) % kRing];
    for (int i = 0; i < RFD_NUM_STEPS; ++i) {
      if (!s.used[i]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s.ev[2 * i], s.ev[2 * i + 1]) == cudaSuccess) pl->step_sum[i] += ms;
    }
    ++pl->timed_calls;
  }
  pl->ring_pending = 0;
}

// Brackets one entry-point call: picks a timing slot and snapshots the launch counter.
struct CallScope {
  rfd_plan_s* pl;
  explicit CallScope(rfd_plan_s* p) : pl(p) {
    pl->launch_mark = t_kernel_launches;
    if (!pl->timing) return;
    if (pl->ring_pending == kRing) fold_timings(pl);
    pl->cur = &pl->ring[pl->ring_head];
    for (bool& u : pl->cur->used) u = false;
  }
  ~CallScope() {
    pl->launches += t_kernel_launches - pl->launch_mark;
    if (!pl->timing) return;
    pl->cur = nullptr;
    pl->ring_head = (pl->ring_head + 1) % kRing;
    ++pl->ring_pending;
  }
};

// Records CUDA events around one step of the path on the plan's stream.
struct StepScope {
  rfd_plan_s* pl;
  int step;
  StepScope(rfd_plan_s* p, int s) : pl(p), step(s) {
    if (pl->cur) cudaEventRecord(pl->cur->ev[2 * step], pl->stream);
  }
  ~StepScope() {
    if (pl->cur) {
      cudaEventRecord(pl->cur->ev[2 * step + 1], pl->stream);
      pl->cur->used[step] = true;
    }
  }
};

rfd_status cuda_fail(const char* what, cudaError_t e) {
  return fail(RFD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RFD_CUDA(call)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(#call, e_); \
  } while (0)

template <typename T>
rfd_status plan_alloc(rfd_plan_s* pl, T** p, size_t count) {
  void* raw = nullptr;
  cudaError_t e = dev_alloc(&raw, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return fail(RFD_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  pl->allocs.push_back(raw);
  *p = static_cast<T*>(raw);
  return RFD_OK;
}

void plan_free(rfd_plan_s* pl) {
  for (void* p : pl->allocs) cudaFree(p);
  pl->allocs.clear();
}

// Split-K schedule.  Each tile gets a number of point-range pieces in
// proportion to its cost so that all pieces cost about the same; pieces are
// ordered split-major (all tiles' first pieces, then the second ones, ...) so
// that CTAs running at the same time read the same point range of Psi and the
// L2 serves it to all of them.  Depends only on (N, m, channel capacity, SM
// count): the result of a cloud never depends on other work.
void schedule(TileSet& ts, int64_t n_pad, int kstep, int target_units, const std::vector<double>& cost,
              int tile_rows, int ld) {
  const int64_t ksteps = n_pad / kstep;
  double total = 0;
  for (double c : cost) total += c;
  int slot = 0;
  std::vector<int> splits(ts.tiles.size());
  for (size_t t = 0; t < ts.tiles.size(); ++t) {
    int64_t s = (int64_t)std::llround(cost[t] / total * target_units);
    s = std::max<int64_t>(1, std::min<int64_t>(s, ksteps));
    splits[t] = (int)s;
    ts.tiles[t].unit_first = slot;
    ts.tiles[t].unit_count = (int)s;
    ts.tiles[t].ld = ld;
    slot += (int)s;
  }
  ts.slots = slot;
  const int smax = *std::max_element(splits.begin(), splits.end());
  for (int s = 0; s < smax; ++s)
    for (size_t t = 0; t < ts.tiles.size(); ++t) {
      if (s >= splits[t]) continue;
      const GramTile& T = ts.tiles[t];
      GramUnit u{};
      u.tile = (int)t;
      u.kind = T.kind;
      u.i0 = T.i0;
      u.j0 = T.j0;
      u.nj_mma = (int)round_up(T.nj, 16);
      const int64_t a = ksteps * s / splits[t], b = ksteps * (s + 1) / splits[t];
      u.k0 = a * kstep;
      u.k1 = b * kstep;
      u.out = (int64_t)(T.unit_first + s) * tile_rows * ld;
      ts.units.push_back(u);
    }
  (void)tile_rows;
}

void build_tiles(rfd_plan_s* pl, bool with_gram, bool with_field, TileSet& ts) {
  const int m = pl->m;
  std::vector<double> cost;
  if (pl->bf16) {
    // Compute tiles: 128 feature rows x up to 256 Gram rows on the upper
    // triangle of Phi^T Phi; the row block's field part (Phi^T F, cpad columns)
    // rides on the tile whose Gram block holds the row block's diagonal (or on
    // a field-only tile when there is no Gram work).  Each tile gets L lanes of
    // the point axis, L = SMs / tiles, all CTAs in one wave (lockstep in kb).
    struct CT { int i0, j0, ni, nj; bool f; };
    std::vector<CT> ct;
    for (int i0 = 0; i0 < m; i0 += kTcBM) {
      const int ni = std::min(kTcBM, m - i0);
      if (!with_gram) {
        ct.push_back(CT{i0, -1, ni, 0, true});
        continue;
      }
      for (int j0 = 0; j0 < m; j0 += kTcBNMax) {
        const int nj = std::min(kTcBNMax, m - j0);
        if (j0 + nj - 1 < i0) continue;  // entirely below the diagonal
        ct.push_back(CT{i0, j0, ni, nj, with_field && j0 == (i0 / kTcBNMax) * kTcBNMax});
      }
    }
    const int64_t kb_total = pl->n_pad / kTcBK;
    const int T = (int)ct.size();
    const int L = (int)std::max<int64_t>(1, std::min<int64_t>(kb_total, pl->sms / std::max(T, 1)));
    for (int t = 0; t < T; ++t) {
      const CT& c = ct[t];
      if (c.nj > 0)
        ts.tiles.push_back(GramTile{c.i0, c.j0, c.ni, c.nj, kTileGram, t * L, L, kTcLd, 0, 0});
      if (c.f) ts.tiles.push_back(GramTile{c.i0, m, c.ni, pl->cpad, kTileField, t * L, L, kTcLd, kTcBNMax, 0});
      for (int l = 0; l < L; ++l) {
        GramUnit u{};
        u.tile = t;
        u.kind = c.nj > 0 ? kTileGram : kTileField;
        u.i0 = c.i0;
        u.j0 = c.j0;
        u.nj_mma = c.nj > 0 ? (int)round_up(c.nj, 16) : 0;
        u.has_f = c.f ? 1 : 0;
        u.lane = l;
        u.nlanes = L;
        u.out = (int64_t)(t * L + l) * kTcBM * kTcLd;
        ts.units.push_back(u);
      }
    }
    ts.slots = T * L;
  } else {
    for (int i0 = 0; i0 < m && with_gram; i0 += kSimtTile)
      for (int j0 = i0; j0 < m; j0 += kSimtTile) {
        ts.tiles.push_back(
            GramTile{i0, j0, std::min(kSimtTile, m - i0), std::min(kSimtTile, m - j0), kTileGram, 0, 0, 0, 0, 0});
        cost.push_back(1.0);
      }
    for (int i0 = 0; i0 < m && with_field; i0 += kSimtTile)
      for (int c0 = 0; c0 < pl->cpad; c0 += kSimtTile) {
        ts.tiles.push_back(GramTile{i0, m + c0, std::min(kSimtTile, m - i0), std::min(kSimtTile, pl->cpad - c0),
                                    kTileField, 0, 0, 0, 0, 0});
        cost.push_back(1.0);
      }
    schedule(ts, pl->n_pad, kSimtK, 2 * pl->sms, cost, kSimtTile, kSimtTile);
  }
}

rfd_status upload_tiles(rfd_plan_s* pl, TileSet& ts) {
  rfd_status s = plan_alloc(pl, &ts.d_tiles, ts.tiles.size());
  if (s != RFD_OK) return s;
  s = plan_alloc(pl, &ts.d_units, ts.units.size());
  if (s != RFD_OK) return s;
  RFD_CUDA(cudaMemcpy(ts.d_tiles, ts.tiles.data(), ts.tiles.size() * sizeof(GramTile), cudaMemcpyHostToDevice));
  RFD_CUDA(cudaMemcpy(ts.d_units, ts.units.data(), ts.units.size() * sizeof(GramUnit), cudaMemcpyHostToDevice));
  return RFD_OK;
}

// Step a3 for one tile set: reductions over N, then the fixed-order reduce.
rfd_status run_reductions(rfd_plan_s* pl, const TileSet& ts, int c) {
  cudaStream_t st = pl->stream;
  if (pl->bf16) {
    TcGramArgs a{};
    a.psi = pl->d_psi;
    a.n_pad = pl->n_pad;
    a.m = pl->m;
    a.cpad = pl->cpad;
    a.units = ts.d_units;
    a.num_units = (int)ts.units.size();
    a.partials = pl->d_part;
    a.err = pl->d_ints;
    {
      StepScope t(pl, RFD_STEP_GRAM);
      RFD_CUDA(launch_gram_tc(a, pl->sms, st));
    }
    StepScope t(pl, RFD_STEP_REDUCE);
    RFD_CUDA(launch_reduce(ts.d_tiles, (int)ts.tiles.size(), pl->d_part, pl->slot_elems, pl->d_oa, pl->d_ob, pl->m, c,
                           pl->d_M, pl->d_Y, kTcBM, kTcBNMax, st));
  } else {  // (the tile columns above bound both parts: Gram nj <= 256, field cpad <= 256)
    {
      StepScope t(pl, RFD_STEP_GRAM);
      RFD_CUDA(launch_gram_simt(static_cast<const float*>(pl->d_psi), pl->n_pad, ts.d_units, (int)ts.units.size(),
                                pl->d_part, st));
    }
    StepScope t(pl, RFD_STEP_REDUCE);
    RFD_CUDA(launch_reduce(ts.d_tiles, (int)ts.tiles.size(), pl->d_part, pl->slot_elems, pl->d_oa, pl->d_ob, pl->m, c,
                           pl->d_M, pl->d_Y, kSimtTile, kSimtTile, st));
  }
  return RFD_OK;
}

rfd_status check_device_error(rfd_plan_s* pl) {
  int err = 0;
  RFD_CUDA(cudaMemcpyAsync(&err, pl->d_ints, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  if (err) {
    cudaMemsetAsync(pl->d_ints, 0, sizeof(int), pl->stream);
    return fail(RFD_ETIMEDOUT, "a device-side wait ran out (code " + std::to_string(err) + ")");
  }
  return RFD_OK;
}

rfd_status run_phi1(rfd_plan_s* pl) {
  Phi1Info info{};
  rfd_status s;
  StepScope t(pl, RFD_STEP_PHI1);
  s = phi1_fp64(pl->m, pl->p.lambda, pl->d_M, pl->d_G, pl->d_work, pl->d_ipiv, pl->d_ints + 1, pl->d_scalar,
                pl->d_ints + 2, pl->d_ints, (pl->p.flags & RFD_FLAG_NATIVE_FP64) == 0, pl->stream, &info);
  pl->stats.phi1_emulated = info.emulated;
  pl->stats.phi1_gemms = info.gemms;
  pl->stats.norm1 = info.norm1;
  pl->stats.pade_degree = info.degree;
  pl->stats.squarings = info.squarings;
  pl->stats.nonfinite = info.nonfinite;
  if (s == RFD_ECUDA) return fail(s, std::string("phi1: ") + cudaGetErrorString(cudaGetLastError()));
  if (s == RFD_ENUMERIC) return fail(s, "G = lambda phi1(lambda M) is not finite (||lambda M||_1 = " +
                                            std::to_string(info.norm1) + ")");
  if (s != RFD_OK) return s;
  rfd_status e = check_device_error(pl);
  if (e != RFD_OK) return e;
  pl->have_G = true;
  return RFD_OK;
}

rfd_status check_field_args(rfd_plan_s* pl, const float* F, int c, int64_t ldF, const float* out, int64_t ldOut) {
  if (!F || !out) return fail(RFD_EINVAL, "null field or output pointer");
  if (c < 1 || c > pl->p.max_channels) return fail(RFD_EINVAL, "c must be in [1, max_channels]");
  if (ldF < c || ldOut < c) return fail(RFD_EINVAL, "leading dimensions must be >= c");
  if (F == out && ldF != ldOut) return fail(RFD_EINVAL, "in-place integration needs ldOut == ldF");
  return RFD_OK;
}

rfd_status apply_step(rfd_plan_s* pl, const float* F, int c, int64_t ldF, float* out, int64_t ldOut) {
  {
    StepScope t(pl, RFD_STEP_SMALL);
    RFD_CUDA(launch_small_product(pl->d_G, pl->d_Y, pl->d_oa, pl->m, c, pl->d_Z, pl->stream));
  }
  StepScope t(pl, RFD_STEP_APPLY);
  RFD_CUDA(launch_apply_simt(pl->d_psi, pl->bf16, pl->n, pl->n_pad, pl->m, pl->d_Z, c, F, ldF, out, ldOut,
                             pl->stream));
  return RFD_OK;
}

}  // namespace

extern "C" {

const char* rfd_last_error(void) { return rfd::last_error_cstr(); }
const char* rfd_version(void) { return "rfd-gb300 0.1 (sm_103a)"; }

rfd_status rfd_plan(const rfd_params* params, void* cuda_stream, rfd_plan_t* out) {
  if (!params || !out) return fail(RFD_EINVAL, "null params or output pointer");
  *out = nullptr;
  const rfd_params& p = *params;
  if (p.n < 1) return fail(RFD_EINVAL, "n must be >= 1");
  if (p.m < 2 || p.m > kMaxM || (p.m & 1)) return fail(RFD_EINVAL, "m must be even, 2 <= m <= 4096");
  if (p.max_channels < 1 || p.max_channels > kMaxChannels) return fail(RFD_EINVAL, "max_channels must be in [1, 256]");
  if (!std::isfinite(p.lambda)) return fail(RFD_EINVAL, "lambda must be finite");
  if (p.precision != RFD_FP32_PLAIN && p.precision != RFD_BF16_TC) return fail(RFD_EINVAL, "unknown precision");
  if (p.flags & ~(RFD_FLAG_TIMING | RFD_FLAG_NATIVE_FP64)) return fail(RFD_EINVAL, "unknown bits in flags");
  if (p.n > (int64_t)1 << 31) return fail(RFD_EINVAL, "n must be < 2^31");
  auto* pl = new (std::nothrow) rfd_plan_s();
  if (!pl) return fail(RFD_ENOMEM, "host allocation failed");
  pl->p = p;
  pl->stream = static_cast<cudaStream_t>(cuda_stream);
  pl->m = p.m;
  pl->h = p.m / 2;
  pl->n = p.n;
  pl->n_pad = round_up(p.n, 128);
  pl->cpad = (int)round_up(p.max_channels, 16);
  pl->bf16 = (p.precision == RFD_BF16_TC);
  pl->timing = (p.flags & RFD_FLAG_TIMING) != 0;
  pl->omega.resize((size_t)pl->h * 3);
  pl->r.resize(pl->h);
  rfd_status st = rfd::sample_frequencies_host(p.m, p.eps, p.seed, p.freq_sigma, p.freq_radius, pl->omega.data(),
                                               pl->r.data());
  if (st != RFD_OK) {
    delete pl;
    return st;
  }
  // column scales: s = sqrt(2|r|/m); Omega_a = s sgn r, Omega_b = s (cos half, then sin half)
  pl->oa.resize(p.m);
  pl->ob.resize(p.m);
  for (int j = 0; j < pl->h; ++j) {
    const double s = std::sqrt(2.0 * std::fabs(pl->r[j]) / p.m);
    const double sa = (pl->r[j] < 0) ? -s : s;
    pl->oa[j] = pl->oa[pl->h + j] = sa;
    pl->ob[j] = pl->ob[pl->h + j] = s;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce != cudaSuccess) {
    delete pl;
    return cuda_fail("device query", ce);
  }
  if (pl->bf16 && !tc_gram_supported()) {
    delete pl;
    return fail(RFD_ENOTSUP, "the BF16 tensor-core form needs an sm_103 GPU (tcgen05) and cuTensorMapEncodeTiled");
  }
  auto bail = [&](rfd_status s) {
    plan_free(pl);
    delete pl;
    return s;
  };
  // host tables
  build_tiles(pl, true, false, pl->gram_only);
  build_tiles(pl, false, true, pl->field_only);
  build_tiles(pl, true, true, pl->both);
  const int slots = std::max({pl->gram_only.slots, pl->field_only.slots, pl->both.slots});
  pl->slot_elems = pl->bf16 ? (int64_t)kTcBM * kTcLd : (int64_t)kSimtTile * kSimtTile;
  pl->rows_alloc = (int)std::max<int64_t>(round_up(p.m, 128), p.m + round_up(pl->cpad, 128));
  const size_t esz = pl->bf16 ? 2 : 4;
  // device buffers
  std::vector<float> whi(pl->omega.size()), wlo(pl->omega.size());
  for (size_t i = 0; i < pl->omega.size(); ++i) {
    whi[i] = (float)pl->omega[i];
    wlo[i] = (float)(pl->omega[i] - (double)whi[i]);
  }
  if ((st = plan_alloc(pl, &pl->d_omega_hi, whi.size())) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_omega_lo, wlo.size())) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_oa, (size_t)p.m)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_ob, (size_t)p.m)) != RFD_OK) return bail(st);
  void* psi = nullptr;
  if ((st = plan_alloc(pl, reinterpret_cast<uint8_t**>(&psi), (size_t)pl->rows_alloc * pl->n_pad * esz)) != RFD_OK)
    return bail(st);
  pl->d_psi = psi;
  if ((st = plan_alloc(pl, &pl->d_part, (size_t)slots * pl->slot_elems)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_M, (size_t)p.m * p.m)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_Y, (size_t)p.m * p.max_channels)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_G, (size_t)p.m * p.m)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_Z, (size_t)p.m * p.max_channels)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_work, phi1_workspace_doubles(p.m))) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_ipiv, (size_t)p.m)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_ints, 4)) != RFD_OK) return bail(st);
  if ((st = plan_alloc(pl, &pl->d_scalar, 2)) != RFD_OK) return bail(st);
  if ((st = upload_tiles(pl, pl->gram_only)) != RFD_OK) return bail(st);
  if ((st = upload_tiles(pl, pl->field_only)) != RFD_OK) return bail(st);
  if ((st = upload_tiles(pl, pl->both)) != RFD_OK) return bail(st);
  auto up = [&](void* dst, const void* src, size_t bytes) { return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice); };
  if ((ce = up(pl->d_omega_hi, whi.data(), whi.size() * 4)) != cudaSuccess ||
      (ce = up(pl->d_omega_lo, wlo.data(), wlo.size() * 4)) != cudaSuccess ||
      (ce = up(pl->d_oa, pl->oa.data(), pl->oa.size() * 8)) != cudaSuccess ||
      (ce = up(pl->d_ob, pl->ob.data(), pl->ob.size() * 8)) != cudaSuccess ||
      (ce = cudaMemset(pl->d_psi, 0, (size_t)pl->rows_alloc * pl->n_pad * esz)) != cudaSuccess ||
      (ce = cudaMemset(pl->d_ints, 0, 4 * sizeof(int))) != cudaSuccess) {
    cuda_fail("plan upload", ce);
    return bail(RFD_ECUDA);
  }
  pl->stats.splits = pl->both.units.empty() ? 0 : (int)(pl->both.units.size() / pl->both.tiles.size());
  if (pl->timing) {
    pl->ring.resize(kRing);
    for (auto& s : pl->ring)
      for (cudaEvent_t& e : s.ev) e = nullptr;
    for (auto& s : pl->ring)
      for (cudaEvent_t& e : s.ev)
        if ((ce = cudaEventCreate(&e)) != cudaSuccess) {
          for (auto& s2 : pl->ring)
            for (cudaEvent_t e2 : s2.ev)
              if (e2) cudaEventDestroy(e2);
          cuda_fail("event creation", ce);
          return bail(RFD_ECUDA);
        }
  }
  *out = pl;
  return RFD_OK;
}

rfd_status rfd_plan_destroy(rfd_plan_t plan) {
  if (!plan) return RFD_OK;
  cudaStreamSynchronize(plan->stream);
  for (auto& s : plan->ring)
    for (cudaEvent_t e : s.ev) cudaEventDestroy(e);
  plan_free(plan);
  delete plan;
  return RFD_OK;
}

static rfd_status features_step(rfd_plan_t pl, const float* d_points) {
  StepScope t(pl, RFD_STEP_FEATURES);
  RFD_CUDA(launch_features(d_points, pl->n, pl->n_pad, pl->d_omega_hi, pl->d_omega_lo, pl->h, pl->bf16, pl->d_psi,
                           pl->stream));
  return RFD_OK;
}

static rfd_status field_step(rfd_plan_t pl, const float* d_F, int c, int64_t ldF) {
  StepScope t(pl, RFD_STEP_FIELD);
  void* rows = static_cast<uint8_t*>(pl->d_psi) + (size_t)pl->m * pl->n_pad * (pl->bf16 ? 2 : 4);
  RFD_CUDA(launch_fill_field_rows(d_F, ldF, c, pl->n, pl->n_pad, pl->cpad, pl->bf16, rows, pl->stream));
  return RFD_OK;
}

rfd_status rfd_features(rfd_plan_t pl, const float* d_points) {
  if (!pl || !d_points) return fail(RFD_EINVAL, "null plan or points");
  CallScope call(pl);
  pl->have_G = false;
  rfd_status s = features_step(pl, d_points);
  if (s == RFD_OK) s = run_reductions(pl, pl->gram_only, 1);
  if (s == RFD_OK) s = run_phi1(pl);
  return s;
}

rfd_status rfd_integrate(rfd_plan_t pl, const float* d_F, int32_t c, int64_t ldF, float* d_out, int64_t ldOut) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  rfd_status s = check_field_args(pl, d_F, c, ldF, d_out, ldOut);
  if (s != RFD_OK) return s;
  if (!pl->have_G) return fail(RFD_EINVAL, "rfd_features (or rfd_gfi) must run before rfd_integrate");
  CallScope call(pl);
  s = field_step(pl, d_F, c, ldF);
  if (s == RFD_OK) s = run_reductions(pl, pl->field_only, c);
  if (s == RFD_OK) s = apply_step(pl, d_F, c, ldF, d_out, ldOut);
  return s;
}

rfd_status rfd_gfi(rfd_plan_t pl, const float* d_points, const float* d_F, int32_t c, int64_t ldF, float* d_out,
                   int64_t ldOut) {
  if (!pl || !d_points) return fail(RFD_EINVAL, "null plan or points");
  rfd_status s = check_field_args(pl, d_F, c, ldF, d_out, ldOut);
  if (s != RFD_OK) return s;
  CallScope call(pl);
  pl->have_G = false;
  s = features_step(pl, d_points);
  if (s == RFD_OK) s = field_step(pl, d_F, c, ldF);
  if (s == RFD_OK) s = run_reductions(pl, pl->both, c);
  if (s == RFD_OK) s = run_phi1(pl);
  if (s == RFD_OK) s = apply_step(pl, d_F, c, ldF, d_out, ldOut);
  return s;
}

rfd_status rfd_phi1(int32_t m, double lambda, const double* d_M, double* d_G, int32_t flags, void* cuda_stream,
                    rfd_stats* stats_out) {
  if (m < 1 || m > kMaxM) return fail(RFD_EINVAL, "m must be in [1, 4096]");
  if (!d_M || !d_G || d_M == d_G) return fail(RFD_EINVAL, "null or aliased M / G");
  if (!std::isfinite(lambda)) return fail(RFD_EINVAL, "lambda must be finite");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rfd_plan_s tmp;  // only used as an allocation owner
  double* work = nullptr;
  int* ints = nullptr;
  int* ipiv = nullptr;
  double* scalar = nullptr;
  rfd_status s;
  if ((s = plan_alloc(&tmp, &work, phi1_workspace_doubles(m))) != RFD_OK ||
      (s = plan_alloc(&tmp, &ipiv, (size_t)m)) != RFD_OK || (s = plan_alloc(&tmp, &ints, 4)) != RFD_OK ||
      (s = plan_alloc(&tmp, &scalar, 2)) != RFD_OK) {
    plan_free(&tmp);
    return s;
  }
  Phi1Info info{};
  s = phi1_fp64(m, lambda, d_M, d_G, work, ipiv, ints + 1, scalar, ints + 2, ints, (flags & RFD_FLAG_NATIVE_FP64) == 0,
                st, &info);
  cudaStreamSynchronize(st);
  int err = 0;
  cudaMemcpy(&err, ints, sizeof(int), cudaMemcpyDeviceToHost);
  if (s == RFD_OK && err) s = fail(RFD_ETIMEDOUT, "a device-side wait ran out in phi1 (code " + std::to_string(err) + ")");
  plan_free(&tmp);
  if (stats_out) {
    *stats_out = rfd_stats{};
    stats_out->norm1 = info.norm1;
    stats_out->pade_degree = info.degree;
    stats_out->squarings = info.squarings;
    stats_out->nonfinite = info.nonfinite;
    stats_out->phi1_emulated = info.emulated;
    stats_out->phi1_gemms = info.gemms;
  }
  if (s == RFD_ECUDA) return fail(s, std::string("phi1: ") + cudaGetErrorString(cudaGetLastError()));
  if (s == RFD_ENUMERIC) return fail(s, "G is not finite");
  return s;
}

rfd_status rfd_sync(rfd_plan_t pl) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  return check_device_error(pl);
}

rfd_status rfd_plan_export(rfd_plan_t pl, double* omega, double* r, double* G) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  if (omega) std::memcpy(omega, pl->omega.data(), pl->omega.size() * sizeof(double));
  if (r) std::memcpy(r, pl->r.data(), pl->r.size() * sizeof(double));
  if (G) {
    if (!pl->have_G) return fail(RFD_EINVAL, "G has not been computed");
    RFD_CUDA(cudaMemcpyAsync(G, pl->d_G, (size_t)pl->m * pl->m * sizeof(double), cudaMemcpyDeviceToHost, pl->stream));
    RFD_CUDA(cudaStreamSynchronize(pl->stream));
  }
  return RFD_OK;
}

rfd_status rfd_plan_stats(rfd_plan_t pl, rfd_stats* out) {
  if (!pl || !out) return fail(RFD_EINVAL, "null plan or output");
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  fold_timings(pl);
  *out = pl->stats;
  for (int i = 0; i < RFD_NUM_STEPS; ++i)
    out->step_ms[i] = pl->timed_calls ? pl->step_sum[i] / (double)pl->timed_calls : 0.0;
  out->timed_calls = pl->timed_calls;
  out->kernel_launches = pl->launches;
  return RFD_OK;
}

rfd_status rfd_plan_stats_reset(rfd_plan_t pl) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  fold_timings(pl);
  for (double& v : pl->step_sum) v = 0.0;
  pl->timed_calls = 0;
  pl->launches = 0;
  return RFD_OK;
}

// Test hook (host-side fault injection): the k-th device allocation from now
// on fails with RFD_ENOMEM (k = 0: the next one); k < 0 disables.
void rfd_debug_fail_alloc_after(int32_t k) { g_fail_alloc_after = k; }

rfd_status rfd_debug_dgemm(int32_t method, int32_t M, int32_t N, int32_t K, double alpha, const double* A, int32_t lda,
                           const double* B, int32_t ldb, double beta, double* C, int32_t ldc, void* cuda_stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || lda < K || ldb < N || ldc < N)
    return fail(RFD_EINVAL, "invalid GEMM arguments");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (method == 0) {
    RFD_CUDA(dgemm(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st));
    RFD_CUDA(cudaStreamSynchronize(st));
    return RFD_OK;
  }
  if (method != 1) return fail(RFD_EINVAL, "method must be 0 or 1");
  if (!ozaki_supported(K)) return fail(RFD_ENOTSUP, "emulated FP64 GEMM needs K <= 1024 on sm_103");
  rfd_plan_s tmp;
  uint8_t* work = nullptr;
  int* err = nullptr;
  rfd_status s;
  if ((s = plan_alloc(&tmp, &work, ozaki_workspace_bytes(M, N, K))) != RFD_OK ||
      (s = plan_alloc(&tmp, &err, 1)) != RFD_OK) {
    plan_free(&tmp);
    return s;
  }
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = dgemm_ozaki(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, work, err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
  plan_free(&tmp);
  if (e != cudaSuccess) return cuda_fail("emulated dgemm", e);
  if (h_err) return fail(RFD_ETIMEDOUT, "a device-side wait ran out (code " + std::to_string(h_err) + ")");
  return RFD_OK;
}

}  // extern "C"
