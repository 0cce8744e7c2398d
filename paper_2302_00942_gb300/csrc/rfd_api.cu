// C ABI of the RFD integrator: plan management and the entry points that run
// steps a2..a6 (Sec. 2.4) on the plan's CUDA stream.  See include/rfd.h for
// the contract of every function.
//
// BF16 tensor-core plans run through the batched path (rfd_batch.cu) as a
// batch of one; rfd_batch_* run many plans with shared launches.  FP32 plain
// plans run the SIMT reductions and the native-FP64 step a4.
#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <vector>
#include "kernels.h"
#include "rfd_internal.h"
#include "rfd_phi1.h"
#include "rfd_plan.h"

namespace rfd {
const char* last_error_cstr();
thread_local long long t_kernel_launches = 0;
// the points-based Phi^T F of a full BF16 plan, with the Gram partials as its scratch
void set_points_field_job(rfd_plan_s* pl);
}  // namespace rfd

using namespace rfd;

struct rfd_batch_s {
  BatchImpl* impl = nullptr;
  std::vector<rfd_plan_t> plans;
  Timing timing;
  cudaStream_t stream = nullptr;
  int options = 0;
  GramTuning tune;
  bool autotune = false, tuned = false;
};

namespace {

constexpr int kMaxM = 4096;
constexpr int kMaxChannels = 256;

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Allocation hook: every device allocation of a plan goes through here, so a
// test can make the n-th allocation fail (RFD_ENOMEM path) without a GPU fault.
int g_fail_alloc_after = -1;

cudaError_t dev_alloc(void** p, size_t bytes) {
  if (g_fail_alloc_after == 0) {
    g_fail_alloc_after = -1;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (g_fail_alloc_after > 0) --g_fail_alloc_after;
  return cudaMalloc(p, bytes);
}

struct CudaMem final : MemSource {
  void* dev(size_t bytes) override {
    void* p = nullptr;
    if (dev_alloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void dev_free(void* p) override { cudaFree(p); }
  void* pinned(size_t bytes) override {
    void* p = nullptr;
    if (g_fail_alloc_after == 0) {
      g_fail_alloc_after = -1;
      return nullptr;
    }
    if (g_fail_alloc_after > 0) --g_fail_alloc_after;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void pinned_free(void* p) override { cudaFreeHost(p); }
};

rfd_status cuda_fail(const char* what, cudaError_t e) {
  return fail(RFD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RFD_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(#call, e_); \
  } while (0)

template <typename T>
rfd_status plan_alloc(rfd_plan_s* pl, T** p, size_t count) {
  void* raw = nullptr;
  cudaError_t e = dev_alloc(&raw, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
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

// ---- FP32 plain form: SIMT split-K schedule --------------------------------
// Each tile gets point-range pieces in proportion to its cost; pieces are
// ordered split-major so concurrently running CTAs read the same point range.
// Depends only on (N, m, channel capacity, SM count).
// The tiles of one launch (narrow == the narrow-kernel field tiles, or the rest) get
// point-range pieces in proportion to their cost: one piece per tile, then the rest of
// the target one at a time to the tile with the most cost per piece, so the pieces never
// exceed the target (one wave) and their costs even out.
void split_simt(const TileSet& ts, const std::vector<double>& cost, const std::vector<bool>& narrow, bool which,
                int64_t ksteps, int target_units, std::vector<int>& splits) {
  const int T = (int)ts.tiles.size();
  int n = 0;
  for (int t = 0; t < T; ++t) n += narrow[t] == which ? 1 : 0;
  for (int left = target_units - n; left > 0; --left) {
    int best = -1;
    for (int t = 0; t < T; ++t)
      if (narrow[t] == which && splits[t] < ksteps && (best < 0 || cost[t] / splits[t] > cost[best] / splits[best]))
        best = t;
    if (best < 0) break;
    ++splits[best];
  }
}

// FP32 plain form: split-K schedule of the square tiles (target_units pieces, one wave)
// and, in a launch of their own, the narrow field tiles (target_narrow pieces); pieces
// are ordered split-major within each launch so that concurrently running CTAs read the
// same point range.  Depends only on (N, m, channel capacity, SM count).
void schedule_simt(TileSet& ts, int64_t n_pad, int target_units, int target_narrow, const std::vector<double>& cost,
                   const std::vector<bool>& narrow) {
  const int64_t ksteps = n_pad / kSimtK;
  const int T = (int)ts.tiles.size();
  std::vector<int> splits(T, 1);
  split_simt(ts, cost, narrow, false, ksteps, target_units, splits);
  split_simt(ts, cost, narrow, true, ksteps, target_narrow, splits);
  int slot = 0;
  for (int t = 0; t < T; ++t) {
    ts.tiles[t].unit_first = slot;
    ts.tiles[t].unit_count = splits[t];
    ts.tiles[t].ld = kSimtTile;
    slot += splits[t];
  }
  ts.slots = slot;
  ts.n_narrow = 0;
  const int smax = T ? *std::max_element(splits.begin(), splits.end()) : 0;
  for (bool which : {false, true})
    for (int s = 0; s < smax; ++s)
      for (int t = 0; t < T; ++t) {
        if (narrow[t] != which || s >= splits[t]) continue;
        const GramTile& Tt = ts.tiles[t];
        GramUnit u{};
        u.tile = t;
        u.kind = Tt.kind;
        u.i0 = Tt.i0;
        u.j0 = Tt.j0;
        const int64_t a = ksteps * s / splits[t], b = ksteps * (s + 1) / splits[t];
        u.k0 = a * kSimtK;
        u.k1 = b * kSimtK;
        u.out = (int64_t)(Tt.unit_first + s) * kSimtTile * kSimtTile;
        ts.units.push_back(u);
        if (which) ++ts.n_narrow;
      }
}

void build_tiles_simt(rfd_plan_s* pl, bool with_gram, bool with_field, TileSet& ts) {
  const int m = pl->m;
  std::vector<double> cost;
  for (int i0 = 0; i0 < m && with_gram; i0 += kSimtTile)
    for (int j0 = i0; j0 < m; j0 += kSimtTile) {
      ts.tiles.push_back(
          GramTile{i0, j0, std::min(kSimtTile, m - i0), std::min(kSimtTile, m - j0), kTileGram, 0, 0, 0, 0, 0});
      cost.push_back(1.0);
    }
  std::vector<bool> narrow(cost.size(), false);
  for (int i0 = 0; i0 < m && with_field; i0 += kSimtTile)
    for (int c0 = 0; c0 < pl->cpad; c0 += kSimtTile) {
      const int nj = std::min(kSimtTile, pl->cpad - c0);
      ts.tiles.push_back(GramTile{i0, m + c0, std::min(kSimtTile, m - i0), nj, kTileField, 0, 0, 0, 0, 0});
      cost.push_back(1.0);
      narrow.push_back(nj <= kSimtNarrow);  // 128 x 16 tiles in a launch of their own
    }
  // one wave each: two square-kernel CTAs per SM, four narrow-kernel CTAs per SM
  schedule_simt(ts, pl->n_pad, 2 * pl->sms, 4 * pl->sms, cost, narrow);
}

// ---- BF16 tensor-core form: the plan's batched-path descriptors -------------
// Compute tiles of one mode.  For each block of 256 feature rows i0.. (two
// halves of 128 rows that share their B rows), the Gram columns [i0, m) (the
// upper triangle and the diagonal blocks) and, when the mode has a field, the
// cpad field columns are cut into tiles of at most 256 columns (multiples of
// 16, as even as possible); the field rides on the last tile, whose B operand
// is its Gram rows followed by the F rows, so one MMA per half covers both (a
// separate field-only tile if it does not fit).  Half 1 (rows i0+128..) skips
// the first min(128, width) columns of the block's first tile, which lie below
// the diagonal.  Without Gram work (integrate) every row block gets a
// field-only tile.
struct GramCT {
  int i0, j0, ni, nj, nj_mma;  // half 0: nj real Gram columns, nj_mma padded width (multiple of 16)
  bool f;
  int ni1, nj1, skip1;  // half 1 (rows i0 + 128 ..; ni1 = 0: absent): Gram columns j0 + skip1 .., nj1 real
};

std::vector<GramCT> gram_tiles(int m, int cpad, int mode) {
  const bool with_gram = mode != kModeIntegrate, with_field = mode != kModeFeatures;
  std::vector<GramCT> ct;
  for (int i0 = 0; i0 < m; i0 += 2 * kTcBM) {
    const int ni = std::min(kTcBM, m - i0);
    const int ni1 = std::max(0, std::min(kTcBM, m - i0 - kTcBM));
    if (!with_gram) {
      ct.push_back(GramCT{i0, -1, ni, 0, 0, true, ni1, 0, 0});
      continue;
    }
    const int Gp = (int)round_up(m - i0, 16), Fw = with_field ? cpad : 0;
    int units = (Gp + Fw) / 16, k = (units * 16 + kTcBNMax - 1) / kTcBNMax;
    bool field_here = Fw > 0;
    if (field_here && (units / k) * 16 < Fw) {  // the field does not fit the last tile: a tile of its own
      field_here = false;
      units = Gp / 16;
      k = (Gp + kTcBNMax - 1) / kTcBNMax;
    }
    int col = i0;
    for (int t = 0; t < k; ++t) {
      const int w = (units / k + (t < units % k ? 1 : 0)) * 16;
      const bool f = field_here && t == k - 1;
      const int gw = f ? w - Fw : w;
      GramCT c{i0, col, ni, std::max(0, std::min(gw, m - col)), gw, f, 0, 0, 0};
      if (ni1 > 0) {
        c.skip1 = (col == i0) ? std::min(kTcBM, gw) : 0;
        c.nj1 = std::max(0, std::min(gw - c.skip1, m - col - c.skip1));
        if (gw - c.skip1 > 0 || f) c.ni1 = ni1;
      }
      ct.push_back(c);
      col += gw;
    }
    if (Fw > 0 && !field_here) ct.push_back(GramCT{i0, -1, ni, 0, 0, true, ni1, 0, 0});
  }
  return ct;
}

// Logical 128-row tiles (halves) of a mode: each has its own partial slots.
int gram_halves(const std::vector<GramCT>& ct) {
  int h = 0;
  for (const GramCT& c : ct) h += c.ni1 > 0 ? 2 : 1;
  return h;
}

// Cost of one 64-point block for a compute tile's CTA, in SM clocks: the
// larger of its MMA time (2 clocks per MMA column per 128-row half at the
// BF16 rate) and the time its TMA loads take to arrive (~2.6 clocks per
// 128-byte row of A and B, the L2 -> SM rate measured for this kernel).
int gram_tile_cost(const GramCT& c, int cpad) {
  const int n0 = c.nj_mma + (c.f ? cpad : 0);
  const int n1 = c.ni1 > 0 ? n0 - c.skip1 : 0;
  const int a_rows = c.ni1 > 0 ? 2 * kTcBM : kTcBM;
  return std::max(2 * (n0 + n1), (26 * (a_rows + n0)) / 10);
}

// Lanes of the point axis per compute tile.  The tiles' CTAs fill lanes_pct %
// of the SMs (at least one lane each, at most one per 64-point block), and the
// lanes go to the tiles in proportion to their cost (greedily to the tile with
// the most work per lane), so that every CTA has about the same work and the
// tiles' lanes sweep the point axis at the same pace (their slabs of Psi are
// then shared in L2).
// meas: the tiles' measured per-block costs (any unit), in place of the model.
std::vector<int> gram_tile_lanes(const std::vector<GramCT>& ct, int cpad, int64_t kb_total, int sms, int lanes_pct,
                                 const std::vector<double>* meas = nullptr) {
  const int T = (int)ct.size();
  std::vector<int> L(T, 1);
  if (T == 0) return L;
  std::vector<double> w(T);
  for (int t = 0; t < T; ++t)
    w[t] = (meas && (int)meas->size() == T) ? (*meas)[t] : (double)gram_tile_cost(ct[t], cpad);
  int budget = std::max(T, sms * lanes_pct / 100) - T;
  while (budget-- > 0) {
    int best = -1;
    for (int t = 0; t < T; ++t)
      if (L[t] < kb_total && (best < 0 || w[t] / L[t] > w[best] / L[best])) best = t;
    if (best < 0) break;
    ++L[best];
  }
  return L;
}

constexpr int kTuneLanesMax = 200;  // the largest lanes_pct the autotuner tries

// ---- the 2-SM (CTA pair) form of the Gram modes, m >= 512 ----------------------
// Pair tiles: for each block of 512 feature rows r0.. (S0 = r0.., S1 = r0 + 256..),
// the column tiles c0 = r0, r0 + 256, ... of at most 256 columns; S1 x B where
// some column lies right of S1's first row (g2); the field on the first column
// tile (c0 = r0, whose S1 part lies below the diagonal).
struct PairCT {
  int r0, c0, nc;
  bool g2, f, a1;
};
std::atomic<int> g_gram_pairs{0};  // test hook: the Gram form new plans start with (1: CTA pairs)
bool pair_eligible(const rfd_plan_s* pl) {
  return pl->bf16 && pl->m >= 512 && pl->m % 16 == 0 && pl->cpad <= 128 && tc_gram_supported();
}
std::vector<PairCT> pair_tiles(int m, int mode) {
  std::vector<PairCT> ct;
  if (mode == kModeIntegrate) return ct;
  for (int r0 = 0; r0 < m; r0 += 4 * kTcBM) {
    const bool s1 = r0 + 2 * kTcBM < m;
    for (int c0 = r0; c0 < m; c0 += kTcBNMax) {
      PairCT t{r0, c0, std::min(kTcBNMax, m - c0), false, false, false};
      t.g2 = s1 && c0 + t.nc > r0 + 2 * kTcBM;
      t.f = mode != kModeFeatures && c0 == r0;
      t.a1 = t.g2 || (t.f && s1);
      ct.push_back(t);
    }
  }
  return ct;
}
// per-block cost of a pair tile (SM clocks, as gram_tile_cost): the larger of the MMA
// columns of the pair's M = 256 MMAs (2 clocks each) and the 128-byte rows one CTA loads
// (~2.6 clocks each).  Measured: weighting by the MMA columns alone gives the diagonal
// tiles (half the MMAs, about the same loads) too few lanes, and they finish last.
int pair_tile_cost(const PairCT& t, int cpad) {
  const int mma_cols = t.nc * (t.g2 ? 2 : 1) + (t.f ? cpad * (t.a1 ? 2 : 1) : 0);
  const int rows = kTcBM * (t.a1 ? 2 : 1) + t.nc / 2 + (t.f ? cpad / 2 : 0);
  return std::max(2 * mma_cols, (26 * rows) / 10);
}
// lanes per pair tile: lanes_pct % of the SM pairs, by cost (greedy, as gram_tile_lanes)
std::vector<int> pair_tile_lanes(const std::vector<PairCT>& ct, int cpad, int64_t kb_total, int sms, int lanes_pct,
                                 const std::vector<double>* meas = nullptr) {
  const int T = (int)ct.size();
  std::vector<int> L(T, 1);
  std::vector<double> w(T);
  for (int t = 0; t < T; ++t)
    w[t] = (meas && (int)meas->size() == T) ? (*meas)[t] : (double)pair_tile_cost(ct[t], cpad);
  // a wave is the co-resident pairs (clusters need both SMs in one GPU processing cluster,
  // so fewer than sms / 2 may fit at once)
  const int fit = gram_pair_max_clusters();
  const int wave = fit > 0 ? std::min(sms / 2, fit) : sms / 2;
  int budget = std::max(T, wave * lanes_pct / 100) - T;
  while (budget-- > 0) {
    int best = -1;
    for (int t = 0; t < T; ++t)
      if (L[t] < kb_total && (best < 0 || w[t] / L[t] > w[best] / L[best])) best = t;
    if (best < 0) break;
    ++L[best];
  }
  return L;
}
int pair_partial_slots(int m, int64_t n_pad, int cpad, int sms, int lanes_pct) {
  int slots = 0;
  for (int mode = 0; mode < 3; ++mode) {
    const std::vector<PairCT> ct = pair_tiles(m, mode);
    const std::vector<int> L = pair_tile_lanes(ct, cpad, n_pad / kTcBK, sms, lanes_pct);
    int sum = 0;
    for (size_t t = 0; t < ct.size(); ++t) sum += (ct[t].a1 ? 4 : 2) * L[t];
    slots = std::max(slots, sum);
  }
  return slots;
}

// The pair units and reduce tiles of the Gram modes (partial slots: each logical 128-row
// half of a pair tile takes L_t consecutive slots, one per lane).
rfd_status build_pair_desc(rfd_plan_s* pl) {
  PlanDesc& d = pl->desc;
  const int m = pl->m, cpad = pl->cpad;
  const int64_t kb_total = pl->n_pad / kTcBK;
  int max_nc = 16;
  for (int mode = 0; mode < 3; ++mode) {
    d.pair_units[mode].clear();
    d.pair_red[mode].clear();
    if (!pair_eligible(pl)) continue;
    const std::vector<PairCT> ct = pair_tiles(m, mode);
    std::vector<int> Ls = pair_tile_lanes(ct, cpad, kb_total, pl->sms, pl->tune.lanes_pct, &pl->tile_cost[1][mode]);
    {  // measured lanes whose partial slots would not fit the allocation: the model's
      int64_t need = 0;
      for (size_t t = 0; t < ct.size(); ++t) need += (int64_t)(ct[t].a1 ? 4 : 2) * Ls[t];
      if (need > pl->part_slots) Ls = pair_tile_lanes(ct, cpad, kb_total, pl->sms, pl->tune.lanes_pct);
    }
    int64_t base = 0;
    for (size_t t = 0; t < ct.size(); ++t) {
      const PairCT& c = ct[t];
      const int L = Ls[t];
      max_nc = std::max(max_nc, c.nc);
      auto slot = [&](int half, int l) { return pl->d_part + (base + (int64_t)half * L + l) * pl->slot_elems; };
      for (int l = 0; l < L; ++l) {
        PairUnit u{};
        u.out0[0] = slot(0, l);
        u.out0[1] = slot(1, l);
        u.out1[0] = c.a1 ? slot(2, l) : nullptr;
        u.out1[1] = c.a1 ? slot(3, l) : nullptr;
        u.map = 0;
        u.r0 = c.r0;
        u.c0 = c.c0;
        u.nc = c.nc;
        u.cpad = cpad;
        u.m = m;
        u.g2 = c.g2 ? 1 : 0;
        u.has_f = c.f ? 1 : 0;
        u.a1 = c.a1 ? 1 : 0;
        u.lane = l;
        u.nlanes = L;
        u.kb_total = (int)kb_total;
        u.work = pair_tile_cost(c, cpad);
        d.pair_units[mode].push_back(u);
      }
      for (int half = 0; half < (c.a1 ? 4 : 2); ++half) {
        const int row0 = c.r0 + (half < 2 ? 0 : 2 * kTcBM) + kTcBM * (half & 1);
        if (row0 >= m) continue;
        RedTile r{};
        r.part = slot(half, 0);
        r.M = pl->d_M;
        r.Y = pl->d_Y;
        r.oa = pl->d_oa;
        r.ob = pl->d_ob;
        r.slot_elems = pl->slot_elems;
        r.i0 = row0;
        r.ni = std::min(kTcBM, m - row0);
        r.count = L;
        r.ld = kTcLd;
        r.m = m;
        r.cloud = 0;
        if (half < 2 || c.g2) {
          r.j0 = c.c0;
          r.nj = c.nc;
          r.kind = kTileGram;
          r.col_off = 0;
          d.pair_red[mode].push_back(r);
        }
        if (c.f) {
          r.j0 = m;
          r.nj = cpad;
          r.fsplit = pl->fsplit ? 1 : 0;
          r.kind = kTileField;
          r.col_off = kTcBNMax;
          d.pair_red[mode].push_back(r);
        }
      }
      base += (int64_t)(c.a1 ? 4 : 2) * L;
    }
    if (base > pl->part_slots) return fail(RFD_ECUDA, "internal: pair partial slots exceed their allocation");
  }
  d.pair_stage_bytes = gram_pair_stage_bytes(max_nc, cpad);
  return RFD_OK;
}

// split-K lanes per compute tile, rounded mean over the tiles (0 without units)
int mean_lanes(const std::vector<TcUnit>& units) {
  int tiles = 0;
  for (const TcUnit& u : units) tiles += u.lane == 0 ? 1 : 0;
  return tiles ? (int)((units.size() + tiles / 2) / tiles) : 0;
}

int tc_partial_slots(int m, int cpad, int64_t n_pad, int sms, int lanes_pct) {
  int slots = 1;
  for (int mode = 0; mode < 3; ++mode) {
    const std::vector<GramCT> ct = gram_tiles(m, cpad, mode);
    const std::vector<int> L = gram_tile_lanes(ct, cpad, n_pad / kTcBK, sms, lanes_pct);
    int sum = 0;
    for (size_t t = 0; t < ct.size(); ++t) sum += (ct[t].ni1 > 0 ? 2 : 1) * L[t];
    slots = std::max(slots, sum);
  }
  return slots;
}

// The tensor-core apply's job of a BF16 plan (k_apply_tc.cu)
ApplyTcJob apply_tc_job(const rfd_plan_s* pl) {
  return ApplyTcJob{pl->d_xyz, pl->d_omega_hi, pl->d_Z, pl->d_w2pi, pl->d_zimg, pl->n, pl->h, (pl->h + 31) / 32, 0,
                    (int)((pl->n + 255) / 256)};
}

// Each compute tile t gets L_t lanes of the point axis (gram_tile_lanes), so a
// lone cloud fills the GPU in one wave (lanes_pct 100).  The partial slots of
// the logical 128-row halves follow each other: half s (of tile t) takes L_t
// consecutive slots, one per lane.  TcUnit.slot is the logical half index of
// half 0, TcUnit.work the tile's cost (a batch rescales the lanes with it).
rfd_status build_desc(rfd_plan_s* pl) {
  PlanDesc& d = pl->desc;
  for (int mode = 0; mode < 3; ++mode) {
    d.units[mode].clear();
    d.red[mode].clear();
  }
  const int m = pl->m;
  const int64_t kb_total = pl->n_pad / kTcBK;
  const int a_rows = std::min(kTcBM, m);
  for (int mode = 0; mode < 3; ++mode) {
    const std::vector<GramCT> ct = gram_tiles(m, pl->cpad, mode);
    const int T = (int)ct.size();
    std::vector<int> Ls = gram_tile_lanes(ct, pl->cpad, kb_total, pl->sms, pl->tune.lanes_pct, &pl->tile_cost[0][mode]);
    {  // measured lanes whose partial slots would not fit the allocation: the model's
      int64_t need = 0;
      for (int t = 0; t < T; ++t) need += (int64_t)(ct[t].ni1 > 0 ? 2 : 1) * Ls[t];
      if (need > pl->part_slots) Ls = gram_tile_lanes(ct, pl->cpad, kb_total, pl->sms, pl->tune.lanes_pct);
    }
    int slot = 0;
    int64_t base = 0;  // first partial slot of the current logical half
    for (int t = 0; t < T; ++t) {
      const GramCT& c = ct[t];
      const bool two = c.ni1 > 0;
      const int L = Ls[t];
      for (int l = 0; l < L; ++l) {
        TcUnit u{};
        u.out = pl->d_part + (base + l) * pl->slot_elems;
        u.out1 = two ? pl->d_part + (base + L + l) * pl->slot_elems : nullptr;
        u.map = 0;
        u.i0 = c.i0;
        u.j0 = c.j0;
        u.nj_mma = c.nj_mma;
        u.has_f = c.f ? 1 : 0;
        u.cpad = pl->cpad;
        u.lane = l;
        u.nlanes = L;
        u.kb_total = (int)kb_total;
        u.a_rows = a_rows;
        u.b_rows = m;
        u.slot = slot;
        u.skip1 = c.skip1;
        u.work = gram_tile_cost(c, pl->cpad);
        d.units[mode].push_back(u);
      }
      // reduce tiles: .count holds the logical half index until a batch assigns lanes
      for (int h = 0; h < (two ? 2 : 1); ++h) {
        RedTile r{};
        r.M = pl->d_M;
        r.Y = pl->d_Y;
        r.oa = pl->d_oa;
        r.ob = pl->d_ob;
        r.slot_elems = pl->slot_elems;
        r.i0 = c.i0 + h * kTcBM;
        r.ni = h ? c.ni1 : c.ni;
        r.count = slot + h;
        r.ld = kTcLd;
        r.m = m;
        const int nj = h ? c.nj1 : c.nj;
        if (nj > 0) {
          r.j0 = c.j0 + (h ? c.skip1 : 0);
          r.nj = nj;
          r.kind = kTileGram;
          r.col_off = 0;
          d.red[mode].push_back(r);
        }
        if (c.f) {
          r.j0 = m;
          r.nj = pl->cpad;
          r.fsplit = pl->fsplit ? 1 : 0;
          r.kind = kTileField;
          r.col_off = kTcBNMax;
          d.red[mode].push_back(r);
        }
      }
      slot += two ? 2 : 1;
      base += (two ? 2 : 1) * (int64_t)L;
    }
    if (base > pl->part_slots) return fail(RFD_ECUDA, "internal: Gram partial slots exceed their allocation");
  }
  if (rfd_status ps = build_pair_desc(pl); ps != RFD_OK) return ps;
  set_points_field_job(pl);
  auto* psi = static_cast<__nv_bfloat16_raw*>(pl->d_psi);
  d.feat = FeatJob{pl->n, pl->n_pad, pl->d_omega_hi, psi, pl->d_xyz, pl->h, (int)((pl->n_pad + 511) / 512), 0,
                   pl->rows_alloc};
  d.fill = FillJob{pl->n, pl->n_pad, psi, pl->cpad, (int)((pl->n_pad + 255) / 256), 0, pl->fsplit ? 1 : 0, m,
                   pl->rows_alloc, (int)(pl->n_pad / 64), (pl->p.max_channels + 31) / 32};
  d.apply = ApplyJob{pl->d_xyz,  pl->d_omega_hi, pl->d_omega_lo, pl->d_G, pl->d_Y, pl->d_oa, pl->d_Z,
                     pl->n,      pl->n_pad,      m, 0, (int)((pl->n + kApplyPts - 1) / kApplyPts), 0};
  d.apply_tc = apply_tc_job(pl);
  // step a4 on the emulated path: slots in the FP64 workspace, the residue buffers after them
  PhiCloud& pc = d.phi;
  pc = PhiCloud{};
  pc.work = pl->d_work;
  pc.M = pl->d_M;
  pc.G = pl->d_G;
  pc.m = m;
  const OzLayout L = ozaki_layout(m, m, m);
  pc.mpa = L.mp;
  pc.mpb = L.np;
  pc.kp = L.kp;
  auto* oz0 = reinterpret_cast<unsigned char*>(pl->d_work + (size_t)m * m * 18);
  auto* oz = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(oz0) + 255) & ~uintptr_t(255));
  if ((size_t)(oz - oz0) + L.bytes > ozaki_workspace_bytes(m, m, m))
    return fail(RFD_ECUDA, "internal: phi1 workspace layout exceeds its allocation");
  pc.sa = reinterpret_cast<__nv_bfloat16_raw*>(oz + L.sa);
  pc.sb = reinterpret_cast<__nv_bfloat16_raw*>(oz + L.sb);
  pc.ea = reinterpret_cast<int*>(oz + L.ea);
  pc.eb = reinterpret_cast<int*>(oz + L.eb);
  pc.ebp = reinterpret_cast<int*>(oz + L.ebp);
  pc.eap = reinterpret_cast<int*>(oz + L.eap);
  pc.res = oz + L.res;
  for (int nm = 1; nm <= 16; ++nm) pc.kbits_n[nm - 1] = (int8_t)ozaki_kbits(m, nm);
  pc.lambda = pl->p.lambda;
  pc.scale = 1.0;
  pc.map_a = 3;
  pc.map_b = 4;
  if (!make_gram_maps(d.maps[0], d.maps[5], d.maps[6], pl->d_psi, pl->n_pad, m, pl->cpad, pl->rows_alloc))
    return fail(RFD_ECUDA, "tensor-map encoding of the feature matrix failed");
  if (!make_ozaki_maps(d.maps[3], d.maps[4], pc.sa, pc.sb, pc.mpa, pc.mpb, pc.kp))
    return fail(RFD_ECUDA, "tensor-map encoding of the FP64-emulation residues failed");
  return RFD_OK;
}

// ---- FP32 plain form steps ---------------------------------------------------
rfd_status run_reductions_simt(rfd_plan_s* pl, const TileSet& ts, int c) {
  cudaStream_t st = pl->stream;
  {
    StepScope t(&pl->timing, st, RFD_STEP_GRAM);
    const int nfull = (int)ts.units.size() - ts.n_narrow;
    RFD_CUDA(launch_gram_simt(static_cast<const float*>(pl->d_psi), pl->n_pad, ts.d_units, nfull, pl->d_part, st));
    RFD_CUDA(launch_gram_simt_narrow(static_cast<const float*>(pl->d_psi), pl->n_pad, ts.d_units + nfull,
                                     ts.n_narrow, pl->d_part, st));
  }
  StepScope t(&pl->timing, st, RFD_STEP_REDUCE);
  RFD_CUDA(launch_reduce(ts.d_tiles, (int)ts.tiles.size(), pl->d_part, pl->slot_elems, pl->d_oa, pl->d_ob, pl->m, c,
                         pl->d_M, pl->d_Y, kSimtTile, kSimtTile, st));
  return RFD_OK;
}

rfd_status check_device_error(rfd_plan_s* pl) {
  if (pl->bf16) return batch_check_error(pl->self);
  int err = 0;
  RFD_CUDA(cudaMemcpyAsync(&err, pl->d_ints, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  if (err) {
    cudaMemsetAsync(pl->d_ints, 0, sizeof(int), pl->stream);
    return fail(RFD_ETIMEDOUT, "a device-side wait ran out (code " + std::to_string(err) + ")");
  }
  return RFD_OK;
}

rfd_status run_phi1_simt(rfd_plan_s* pl) {
  Phi1Info info{};
  rfd_status s;
  {
    StepScope t(&pl->timing, pl->stream, RFD_STEP_PHI1);
    s = phi1_fp64(pl->m, pl->p.lambda, pl->d_M, pl->d_G, pl->d_work, pl->d_ipiv, pl->d_ints + 1, pl->d_scalar,
                  pl->d_ints + 2, pl->d_ints, (pl->p.flags & RFD_FLAG_NATIVE_FP64) == 0, pl->stream, &info);
  }
  pl->stats.phi1_emulated = info.emulated;
  pl->stats.phi1_gemms = info.gemms;
  pl->stats.norm1 = info.norm1;
  pl->stats.pade_degree = info.degree;
  pl->stats.squarings = info.squarings;
  pl->stats.nonfinite = info.nonfinite;
  if (s == RFD_ECUDA) return fail(s, std::string("phi1: ") + cudaGetErrorString(cudaGetLastError()));
  if (s == RFD_ENUMERIC)
    return fail(s, "G = lambda phi1(lambda M) is not finite (||lambda M||_1 = " + std::to_string(info.norm1) + ")");
  if (s != RFD_OK) return s;
  rfd_status e = check_device_error(pl);
  if (e != RFD_OK) return e;
  pl->have_G = true;
  return RFD_OK;
}

rfd_status apply_simt(rfd_plan_s* pl, const float* F, int c, int64_t ldF, float* out, int64_t ldOut) {
  {
    StepScope t(&pl->timing, pl->stream, RFD_STEP_SMALL);
    RFD_CUDA(launch_small_product(pl->d_G, pl->d_Y, pl->d_oa, pl->m, c, pl->d_Z, pl->stream));
  }
  StepScope t(&pl->timing, pl->stream, RFD_STEP_APPLY);
  RFD_CUDA(launch_apply_simt(pl->d_psi, false, pl->n, pl->n_pad, pl->m, pl->d_Z, c, F, ldF, out, ldOut, pl->stream));
  return RFD_OK;
}

rfd_status check_field_args(rfd_plan_s* pl, const float* F, int c, int64_t ldF, const float* out, int64_t ldOut) {
  if (!F || !out) return fail(RFD_EINVAL, "null field or output pointer");
  if (c < 1 || c > pl->p.max_channels) return fail(RFD_EINVAL, "c must be in [1, max_channels]");
  if (ldF < c || ldOut < c) return fail(RFD_EINVAL, "leading dimensions must be >= c");
  if (F == out && ldF != ldOut) return fail(RFD_EINVAL, "in-place integration needs ldOut == ldF");
  return RFD_OK;
}

// Brackets one entry-point call for the timing ring and the launch count.
struct CallScope {
  Timing* t;
  cudaStream_t st;
  CallScope(Timing* tt, cudaStream_t s) : t(tt), st(s) { t->begin_call(st); }
  ~CallScope() { t->end_call(); }
};

// ---- autotuner -------------------------------------------------------------
// Picks the launch parameters of the tensor-core reductions by timing them on
// the cloud's own features after its first features pass: split-K lanes of a
// lone cloud (50 / 100 / 200 % of SMs per tile) or the waves a batch plans
// for (2 / 4 / 8), times the phase length of the point axis (1024 / 2048 /
// 4096 / 8192 blocks of 64 points; for a lone cloud with several phases the
// features run beside the Gram, phase by phase, and are timed with it), and
// for a lone cloud with m >= 512 both forms of the Gram (one SM per tile, or
// CTA pairs).  Choices are kept per bucket -- (m, log2 of the
// point blocks, field width) for plans, (clouds, log2 of the work) for batches
// -- and reused without timing by later plans / batches of the same bucket.
std::mutex g_tune_mu;
struct PlanTuneEntry {
  GramTuning t;
  std::vector<double> cost[2][3];  // the measured tile costs (rfd_plan_s::tile_cost)
  double form_ms[2] = {0.0, 0.0};
};
std::map<std::tuple<int, int, int>, PlanTuneEntry> g_plan_tune;
std::map<std::pair<int, int>, GramTuning> g_batch_tune;
constexpr int kTunePhases[5] = {1024, 2048, 4096, 8192, 16384};

int ilog2(double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); }

// Options of a plan's batch of one: CUDA graphs when the plan asks for them.
int self_options(const rfd_plan_s* pl) { return (pl->p.flags & RFD_FLAG_GRAPH) ? kBatchGraphs : 0; }

// Rebuilds the plan's descriptors and its batch of one for pl->tune.
rfd_status rebuild_self(rfd_plan_s* pl) {
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  rfd_status s = build_desc(pl);
  if (s != RFD_OK) return s;
  BatchImpl* nb = nullptr;
  rfd_plan_s* self = pl;
  if ((s = batch_build(&self, 1, pl->stream, pl->mem, self_options(pl), pl->tune, &nb)) != RFD_OK) return s;
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  batch_free(pl->self);
  pl->self = nb;
  pl->stats.splits = mean_lanes(pl->desc.units[kModeGfi]);
  return RFD_OK;
}

// Measures every compute tile's cost per 64-point block (ns for one lane) in one launch over
// the whole point axis with the plan's current lanes of form `form` (0: one SM per tile, 1: CTA
// pairs), into pl->tile_cost[form][mode].  The units of a tile are consecutive, lane 0 first.
rfd_status measure_tile_costs(rfd_plan_s* pl, int form, int mode, const CloudCall* cc) {
  pl->tune.pairs = form;
  rfd_status s = build_desc(pl);
  BatchImpl* tb = nullptr;
  rfd_plan_s* self = pl;
  if (s == RFD_OK) s = batch_build(&self, 1, pl->stream, cuda_mem(), 0, pl->tune, &tb);
  if (s != RFD_OK) return s;
  const int64_t kb_total = pl->n_pad / kTcBK;
  const int n_units = form ? (int)pl->desc.pair_units[mode].size() : (int)pl->desc.units[mode].size();
  const int ctas = form ? 2 * n_units : n_units;
  std::vector<unsigned long long> h(2 * (size_t)ctas, 0ull);
  unsigned long long* d = nullptr;
  cudaError_t e = cudaSuccess;
  if (ctas > 0) {
    e = cudaMalloc(reinterpret_cast<void**>(&d), h.size() * sizeof(unsigned long long));
    if (e == cudaSuccess) {
      batch_set_phase(tb, (int)std::min<int64_t>(kb_total, 1 << 30));
      batch_set_profile(tb, d);
      float ms = 0.f;
      s = batch_time_gram(tb, mode, 1, &ms, cc);
      batch_set_profile(tb, nullptr);
      if (s == RFD_OK) e = cudaMemcpy(h.data(), d, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
      cudaFree(d);
    }
  }
  cudaStreamSynchronize(pl->stream);
  batch_free(tb);
  if (s != RFD_OK) return s;
  if (e != cudaSuccess) return cuda_fail("tile timing", e);
  std::vector<double> cost;
  double sum = 0.0;
  int nl = 0;
  for (int i = 0; i < n_units; ++i) {
    int lane, nlanes;
    unsigned long long t0, t1;
    if (form) {
      const PairUnit& u = pl->desc.pair_units[mode][i];
      lane = u.lane;
      nlanes = u.nlanes;
      t0 = std::min(h[4 * i], h[4 * i + 2]);
      t1 = std::max(h[4 * i + 1], h[4 * i + 3]);
    } else {
      const TcUnit& u = pl->desc.units[mode][i];
      lane = u.lane;
      nlanes = u.nlanes;
      t0 = h[2 * i];
      t1 = h[2 * i + 1];
    }
    if (lane == 0 && i > 0) {  // the previous tile is complete
      cost.push_back(nl > 0 ? sum / nl : -1.0);
      sum = 0.0;
      nl = 0;
    }
    const int64_t blocks = nlanes > 0 ? (kb_total - lane + nlanes - 1) / nlanes : 0;
    if (blocks > 0 && t1 > t0) {
      sum += (double)(t1 - t0) / (double)blocks;
      ++nl;
    }
  }
  if (n_units > 0) cost.push_back(nl > 0 ? sum / nl : -1.0);
  bool all = true;
  for (double c : cost) all = all && c > 0.0;
  pl->tile_cost[form][mode] = all ? cost : std::vector<double>();  // a tile without a measure: the model
  return RFD_OK;
}

rfd_status tune_plan(rfd_plan_s* pl, int mode, const CloudCall* cc) {
  const auto key = std::make_tuple(pl->m, ilog2((double)(pl->n_pad / kTcBK)), pl->cpad);
  pl->tuned = true;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_plan_tune.find(key);
    if (it != g_plan_tune.end()) {
      pl->tune = it->second.t;
      for (int f = 0; f < 2; ++f) {
        for (int md = 0; md < 3; ++md) pl->tile_cost[f][md] = it->second.cost[f][md];
        pl->tune_form_ms[f] = it->second.form_ms[f];
      }
      return rebuild_self(pl);
    }
  }
  RFD_CUDA(cudaStreamSynchronize(pl->stream));  // the features of the first pass are in place
  float best = 1e30f;
  GramTuning best_t = pl->tune;
  for (int form = 0; form < (pair_eligible(pl) ? 2 : 1); ++form) {
    // the tiles' lanes from their measured pace: two rounds (measure with the model's lanes,
    // then with the measured ones), so that every tile sweeps the point axis at one pace and
    // the slabs of Psi the tiles share are read from HBM once
    pl->tune.pairs = form;
    pl->tune.lanes_pct = 100;
    pl->tile_cost[form][mode].clear();
    pl->tune_form_ms[form] = 0.0;
    for (int round = 0; round < 2; ++round)
      if (rfd_status s = measure_tile_costs(pl, form, mode, cc); s != RFD_OK) return s;
    for (int lp : {50, 100, kTuneLanesMax}) {
      pl->tune.lanes_pct = lp;
      pl->tune.pairs = form;
      rfd_status s = build_desc(pl);
      BatchImpl* tb = nullptr;
      rfd_plan_s* self = pl;
      if (s == RFD_OK) s = batch_build(&self, 1, pl->stream, cuda_mem(), 0, pl->tune, &tb);
      if (s != RFD_OK) return s;
      for (int ph : kTunePhases) {
        batch_set_phase(tb, ph);
        // the serial schedule only: the features beside the Gram (batch_set_overlap) gained
        // 1.5 - 2 % of the step at N = 10^6, m = 1024, but the two kernels then share the SMs,
        // so the Gram's own time is no longer measurable, and the tuner's isolated timings of
        // the two schedules were within its run-to-run noise (it flipped between them)
        batch_set_overlap(tb, false);
        float ms = 0.f;
        s = batch_time_gram(tb, mode, 3, &ms, cc);
        if (s != RFD_OK) break;
        if (pl->tune_form_ms[form] == 0.0 || ms < pl->tune_form_ms[form]) pl->tune_form_ms[form] = ms;
        if (ms < best) {
          best = ms;
          best_t = pl->tune;
          best_t.phase_blocks = ph;
          best_t.overlap = 0;
        }
      }
      cudaStreamSynchronize(pl->stream);
      batch_free(tb);
      if (s != RFD_OK) return s;
    }
  }
  pl->tune = best_t;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    PlanTuneEntry& en = g_plan_tune[key];
    en.t = best_t;
    for (int f = 0; f < 2; ++f) {
      for (int md = 0; md < 3; ++md) en.cost[f][md] = pl->tile_cost[f][md];
      en.form_ms[f] = pl->tune_form_ms[f];
    }
  }
  return rebuild_self(pl);
}

rfd_status run_plan(rfd_plan_s* pl, int mode, const float* pts, const float* F, int c, int64_t ldF, float* out,
                    int64_t ldOut) {
  CallScope call(&pl->timing, pl->stream);
  if (pl->bf16) {
    CloudCall cc{pts, F, out, ldF, ldOut, c, 0};
    rfd_status s = batch_run(pl->self, mode, &cc, &pl->timing);
    if (s == RFD_OK && pl->autotune && !pl->tuned && mode != kModeIntegrate) s = tune_plan(pl, mode, &cc);
    return s;
  }
  cudaStream_t st = pl->stream;
  void* rows = static_cast<uint8_t*>(pl->d_psi) + (size_t)pl->m * pl->n_pad * 4;
  if (mode != kModeIntegrate) {
    pl->have_G = false;
    StepScope t(&pl->timing, st, RFD_STEP_FEATURES);
    RFD_CUDA(launch_features(pts, pl->n, pl->n_pad, pl->d_omega_hi, pl->d_omega_lo, pl->h, false, pl->d_psi, st));
  }
  if (mode != kModeFeatures) {
    StepScope t(&pl->timing, st, RFD_STEP_FIELD);
    RFD_CUDA(launch_fill_field_rows(F, ldF, c, pl->n, pl->n_pad, pl->cpad, false, rows, st));
  }
  const TileSet& ts = mode == kModeFeatures ? pl->gram_only : (mode == kModeIntegrate ? pl->field_only : pl->both);
  rfd_status s = run_reductions_simt(pl, ts, mode == kModeFeatures ? 1 : c);
  if (s == RFD_OK && mode != kModeIntegrate) s = run_phi1_simt(pl);
  if (s == RFD_OK && mode != kModeFeatures) s = apply_simt(pl, F, c, ldF, out, ldOut);
  return s;
}

void fill_stats(const Timing& tm, rfd_stats* out) {
  for (int i = 0; i < RFD_NUM_STEPS; ++i) out->step_ms[i] = tm.calls ? tm.sum[i] / (double)tm.calls : 0.0;
  out->timed_calls = tm.calls;
  out->kernel_launches = tm.launches;
}

}  // namespace

// ---- plan construction (shared by rfd_plan and the server) ------------------
namespace rfd {

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The plan's device buffers, carved from one chunk in a fixed order.
struct PlanCarve {
  size_t total = 0;
  std::vector<std::pair<void**, size_t>> items;
  void bytes(void** p, size_t n) {
    items.push_back({p, align256(std::max<size_t>(n, 1))});
    total += items.back().second;
  }
  template <typename T>
  void add(T** p, size_t count) {
    bytes(reinterpret_cast<void**>(p), count * sizeof(T));
  }
  void assign(void* base) {
    size_t off = 0;
    for (auto& it : items) {
      *it.first = static_cast<unsigned char*>(base) + off;
      off += it.second;
    }
  }
};

void plan_carve(rfd_plan_s* pl, PlanCarve& c) {
  const int m = pl->m;
  c.add(&pl->d_omega_hi, (size_t)pl->h * 3);
  c.add(&pl->d_omega_lo, (size_t)pl->h * 3);
  c.add(&pl->d_oa, (size_t)m);
  c.add(&pl->d_ob, (size_t)m);
  if (pl->bf16) c.add(&pl->d_xyz, (size_t)pl->n * 3);
  c.bytes(&pl->d_psi, (size_t)pl->rows_alloc * pl->n_pad * (pl->bf16 ? 2 : 4));
  c.add(&pl->d_part, (size_t)pl->part_slots * pl->slot_elems);
  c.add(&pl->d_M, (size_t)m * m);
  c.add(&pl->d_Y, (size_t)m * pl->p.max_channels);
  c.add(&pl->d_G, (size_t)m * m);
  c.add(&pl->d_Z, (size_t)m * pl->p.max_channels);
  if (pl->bf16) {
    c.add(&pl->d_w2pi, (size_t)32 * ((pl->h + 31) / 32));
    c.bytes(reinterpret_cast<void**>(&pl->d_zimg), apply_tc_zimg_bytes(pl->h, pl->p.max_channels));
  }
  c.add(&pl->d_work, phi1_workspace_doubles(m));
  c.add(&pl->d_ipiv, (size_t)m);
  c.add(&pl->d_ints, 4);
  c.add(&pl->d_scalar, 2);
  if (!pl->bf16)
    for (TileSet* ts : {&pl->gram_only, &pl->field_only, &pl->both}) {
      c.add(&ts->d_tiles, ts->tiles.size());
      c.add(&ts->d_units, ts->units.size());
    }
}

// Chunks of the points-based Phi^T F of a compact plan: enough for ~6 blocks of 256 threads
// per SM (at 512 frequencies per block), of at least 1024 points each, with partials
// ([chunks][m][ld] floats, ld = channels padded to 4) no larger than the points' own
// 12 N bytes (4 MB at least) and, where given, no larger than max_floats.
void fieldpts_shape(const rfd_plan_s* pl, int* chunks, int64_t* pts, int* ld, int64_t max_floats = 0) {
  *ld = (int)round_up(pl->p.max_channels, 4);
  const int64_t fgroups = (pl->h + 511) / 512;
  const int64_t want = std::max<int64_t>(1, (6ll * std::max(pl->sms, 1) + fgroups - 1) / fgroups);
  int64_t cap = std::max<int64_t>(4ll << 20, 12 * pl->n) / ((int64_t)pl->m * *ld * 4);
  if (max_floats > 0) cap = std::min<int64_t>(cap, max_floats / ((int64_t)pl->m * *ld));
  cap = std::max<int64_t>(1, cap);
  int64_t ch = std::min<int64_t>({want, cap, std::max<int64_t>(1, (pl->n + 1023) / 1024)});
  *pts = (pl->n + ch - 1) / ch;
  *chunks = (int)((pl->n + *pts - 1) / *pts);
}

void plan_carve_compact(rfd_plan_s* pl, PlanCarve& c) {
  const int m = pl->m;
  int chunks, ld;
  int64_t pts;
  fieldpts_shape(pl, &chunks, &pts, &ld);
  c.add(&pl->d_omega_hi, (size_t)pl->h * 3);
  c.add(&pl->d_omega_lo, (size_t)pl->h * 3);
  c.add(&pl->d_oa, (size_t)m);
  c.add(&pl->d_ob, (size_t)m);
  c.add(&pl->d_xyz, (size_t)pl->n * 3);
  c.add(&pl->d_M, (size_t)m * m);
  c.add(&pl->d_Y, (size_t)m * pl->p.max_channels);
  c.add(&pl->d_G, (size_t)m * m);
  c.add(&pl->d_Z, (size_t)m * pl->p.max_channels);
  c.add(&pl->d_w2pi, (size_t)32 * ((pl->h + 31) / 32));
  c.bytes(reinterpret_cast<void**>(&pl->d_zimg), apply_tc_zimg_bytes(pl->h, pl->p.max_channels));
  c.add(&pl->d_ints, 4);
  c.add(&pl->d_scalar, 2);
  c.add(&pl->d_fpart, (size_t)chunks * m * ld);
}

// The compact plan's descriptors: the points-based Phi^T F (with its sum over the chunks)
// and the apply (as the full plan's).
void build_compact_desc(rfd_plan_s* pl) {
  PlanDesc& d = pl->desc;
  for (int mode = 0; mode < 3; ++mode) {
    d.units[mode].clear();
    d.red[mode].clear();
    d.pair_units[mode].clear();
    d.pair_red[mode].clear();
  }
  int chunks, ld;
  int64_t pts;
  fieldpts_shape(pl, &chunks, &pts, &ld);
  d.fpts = FieldPtsJob{pl->d_xyz, pl->d_omega_hi, pl->d_fpart, pl->n, pts, pl->h, pl->m, chunks, ld, 0, 0,
                       pl->d_Y,   pl->d_ob};
  d.apply = ApplyJob{pl->d_xyz, pl->d_omega_hi, pl->d_omega_lo, pl->d_G, pl->d_Y, pl->d_oa, pl->d_Z,
                     pl->n,     pl->n_pad,      pl->m, 0, (int)((pl->n + kApplyPts - 1) / kApplyPts), 0};
  d.apply_tc = apply_tc_job(pl);
}

}  // namespace

void set_points_field_job(rfd_plan_s* pl) {
  if (pl->compact) return;  // a compact plan's job (build_compact_desc) stays
  pl->desc.fpts = FieldPtsJob{};
  if (!pl->bf16 || !pl->d_part || pl->part_slots < 1) return;
  int chunks, ld;
  int64_t pts;
  fieldpts_shape(pl, &chunks, &pts, &ld, (int64_t)pl->part_slots * pl->slot_elems);
  pl->desc.fpts = FieldPtsJob{pl->d_xyz, pl->d_omega_hi, pl->d_part, pl->n, pts, pl->h, pl->m, chunks, ld, 0, 0,
                              pl->d_Y,   pl->d_ob};
}

size_t plan_compact_bytes(const rfd_plan_s* pl) {
  rfd_plan_s tmp;  // the carve only reads the sizes
  tmp.p = pl->p;
  tmp.sms = pl->sms;
  tmp.m = pl->m;
  tmp.h = pl->h;
  tmp.n = pl->n;
  PlanCarve c;
  plan_carve_compact(&tmp, c);
  return c.total;
}

rfd_status plan_compact(rfd_plan_s* pl, bool self_batch) {
  if (!pl->bf16) return fail(RFD_EINVAL, "only BF16 tensor-core plans have a compact form");
  if (pl->compact) return RFD_OK;
  if (!pl->have_G) return fail(RFD_EINVAL, "rfd_features (or rfd_gfi) must run before the plan is compacted");
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  // the buffers that stay, and where they are now
  struct Keep {
    void** field;
    void* old;
    size_t bytes;
  };
  const int m = pl->m;
  std::vector<Keep> keep = {
      {reinterpret_cast<void**>(&pl->d_omega_hi), pl->d_omega_hi, (size_t)pl->h * 3 * 4},
      {reinterpret_cast<void**>(&pl->d_omega_lo), pl->d_omega_lo, (size_t)pl->h * 3 * 4},
      {reinterpret_cast<void**>(&pl->d_oa), pl->d_oa, (size_t)m * 8},
      {reinterpret_cast<void**>(&pl->d_ob), pl->d_ob, (size_t)m * 8},
      {reinterpret_cast<void**>(&pl->d_xyz), pl->d_xyz, (size_t)pl->n * 12},
      {reinterpret_cast<void**>(&pl->d_M), pl->d_M, (size_t)m * m * 8},
      {reinterpret_cast<void**>(&pl->d_Y), pl->d_Y, (size_t)m * pl->p.max_channels * 8},
      {reinterpret_cast<void**>(&pl->d_G), pl->d_G, (size_t)m * m * 8},
      {reinterpret_cast<void**>(&pl->d_Z), pl->d_Z, (size_t)m * pl->p.max_channels * 4},
      {reinterpret_cast<void**>(&pl->d_ints), pl->d_ints, 4 * 4},
      {reinterpret_cast<void**>(&pl->d_scalar), pl->d_scalar, 2 * 8}};
  const size_t bytes = plan_compact_bytes(pl);
  void* chunk = pl->mem->dev(bytes);
  if (!chunk) return fail(RFD_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes (compact plan) failed");
  PlanCarve c;
  plan_carve_compact(pl, c);  // points the plan's fields into the new chunk
  c.assign(chunk);
  cudaError_t e = cudaSuccess;
  for (const Keep& k : keep)
    if (e == cudaSuccess) e = cudaMemcpyAsync(*k.field, k.old, k.bytes, cudaMemcpyDeviceToDevice, pl->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
  if (e != cudaSuccess) {  // back to the full chunk, which still holds everything
    for (const Keep& k : keep) *k.field = k.old;
    pl->mem->dev_free(chunk);
    return cuda_fail("plan compaction", e);
  }
  if (pl->self) batch_free(pl->self);
  pl->self = nullptr;
  pl->mem->dev_free(pl->chunk);
  pl->chunk = chunk;
  pl->chunk_bytes = bytes;
  pl->d_psi = nullptr;
  pl->d_part = nullptr;
  pl->d_work = nullptr;
  pl->d_ipiv = nullptr;
  pl->compact = true;
  build_compact_desc(pl);
  if (self_batch) {
    rfd_plan_s* self = pl;
    rfd_status s = batch_build(&self, 1, pl->stream, pl->mem, 0, pl->tune, &pl->self);
    if (s != RFD_OK) return s;
    RFD_CUDA(cudaStreamSynchronize(pl->stream));
  }
  return RFD_OK;
}

MemSource* cuda_mem() {
  static CudaMem m;
  return &m;
}

rfd_status plan_prepare(const rfd_params& p, cudaStream_t stream, rfd_plan_s** out) {
  *out = nullptr;
  if (p.n < 1) return fail(RFD_EINVAL, "n must be >= 1");
  if (p.m < 2 || p.m > kMaxM || (p.m & 1)) return fail(RFD_EINVAL, "m must be even, 2 <= m <= 4096");
  if (p.max_channels < 1 || p.max_channels > kMaxChannels) return fail(RFD_EINVAL, "max_channels must be in [1, 256]");
  if (!std::isfinite(p.lambda)) return fail(RFD_EINVAL, "lambda must be finite");
  if (p.precision != RFD_FP32_PLAIN && p.precision != RFD_BF16_TC) return fail(RFD_EINVAL, "unknown precision");
  if (p.flags & ~(RFD_FLAG_TIMING | RFD_FLAG_NATIVE_FP64 | RFD_FLAG_AUTOTUNE | RFD_FLAG_GRAPH))
    return fail(RFD_EINVAL, "unknown bits in flags");
  if (p.n > (int64_t)1 << 31) return fail(RFD_EINVAL, "n must be < 2^31");
  if (p.kernel != RFD_KERNEL_CUBE && p.kernel != RFD_KERNEL_BALL && p.kernel != RFD_KERNEL_CUBE_L1 &&
      p.kernel != RFD_KERNEL_L1_BALL)
    return fail(RFD_EINVAL, "unknown kernel");
  if (p.reserved_ != 0) return fail(RFD_EINVAL, "rfd_params.reserved_ must be 0");
  auto* pl = new (std::nothrow) rfd_plan_s();
  if (!pl) return fail(RFD_ENOMEM, "host allocation failed");
  pl->p = p;
  pl->stream = stream;
  pl->m = p.m;
  pl->h = p.m / 2;
  pl->n = p.n;
  pl->n_pad = round_up(p.n, 128);
  pl->bf16 = (p.precision == RFD_BF16_TC);
  // BF16 form: F enters as hi + lo rows (2c) while that fits the field part of the Gram tiles
  pl->fsplit = pl->bf16 && 2 * p.max_channels <= 256;
  pl->cpad = (int)round_up(pl->fsplit ? 2 * p.max_channels : p.max_channels, 16);
  pl->omega.resize((size_t)pl->h * 3);
  pl->r.resize(pl->h);
  rfd_status st = sample_frequencies_host(p.m, p.eps, p.seed, p.freq_sigma, p.freq_radius, p.kernel, pl->omega.data(),
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
  pl->omega_hi_h.resize(pl->omega.size());
  pl->omega_lo_h.resize(pl->omega.size());
  for (size_t i = 0; i < pl->omega.size(); ++i) {
    pl->omega_hi_h[i] = (float)pl->omega[i];
    pl->omega_lo_h[i] = (float)(pl->omega[i] - (double)pl->omega_hi_h[i]);
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
  // partial slots: SIMT tiles, or the tensor-core tiles x lanes
  if (!pl->bf16) {
    build_tiles_simt(pl, true, false, pl->gram_only);
    build_tiles_simt(pl, false, true, pl->field_only);
    build_tiles_simt(pl, true, true, pl->both);
  }
  pl->autotune = pl->bf16 && (p.flags & RFD_FLAG_AUTOTUNE);
  pl->tune.pairs = g_gram_pairs.load() && pair_eligible(pl) ? 1 : 0;
  pl->part_slots = pl->bf16 ? std::max(tc_partial_slots(pl->m, pl->cpad, pl->n_pad, pl->sms,
                                                         pl->autotune ? kTuneLanesMax : 100),
                                        pair_eligible(pl) ? pair_partial_slots(pl->m, pl->n_pad, pl->cpad, pl->sms,
                                                                               pl->autotune ? kTuneLanesMax : 100)
                                                          : 0)
                            : std::max({pl->gram_only.slots, pl->field_only.slots, pl->both.slots});
  pl->slot_elems = pl->bf16 ? (int64_t)kTcBM * kTcLd : (int64_t)kSimtTile * kSimtTile;
  pl->rows_alloc = (int)std::max<int64_t>(round_up(p.m, 128), p.m + round_up(pl->cpad, 128));
  *out = pl;
  return RFD_OK;
}

size_t plan_device_bytes(rfd_plan_s* pl) {
  PlanCarve c;
  plan_carve(pl, c);
  return c.total;
}

void plan_destroy(rfd_plan_s* pl) {
  if (!pl) return;
  if (pl->self) batch_free(pl->self);
  pl->timing.destroy();
  if (pl->chunk) pl->mem->dev_free(pl->chunk);
  plan_free(pl);
  delete pl;
}

rfd_status plan_materialize(rfd_plan_s* pl, MemSource* mem, bool self_batch, bool sync_init) {
  auto bail = [&](rfd_status s) {
    if (sync_init || pl->self) cudaStreamSynchronize(pl->stream);
    plan_destroy(pl);
    return s;
  };
  pl->mem = mem;
  PlanCarve c;
  plan_carve(pl, c);
  if (!pl->chunk) pl->chunk = mem->dev(c.total);  // a caller may have reserved it
  if (!pl->chunk) {
    fail(RFD_ENOMEM, "device allocation of " + std::to_string(c.total) + " bytes failed");
    return bail(RFD_ENOMEM);
  }
  pl->chunk_bytes = c.total;
  c.assign(pl->chunk);
  cudaStream_t st = pl->stream;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  cudaError_t ce = up(pl->d_omega_hi, pl->omega_hi_h.data(), pl->omega_hi_h.size() * 4);
  if (ce == cudaSuccess) ce = up(pl->d_omega_lo, pl->omega_lo_h.data(), pl->omega_lo_h.size() * 4);
  if (ce == cudaSuccess) ce = up(pl->d_oa, pl->oa.data(), pl->oa.size() * 8);
  if (ce == cudaSuccess) ce = up(pl->d_ob, pl->ob.data(), pl->ob.size() * 8);
  if (ce == cudaSuccess)
    ce = cudaMemsetAsync(pl->d_psi, 0, (size_t)pl->rows_alloc * pl->n_pad * (pl->bf16 ? 2 : 4), st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(pl->d_ints, 0, 4 * sizeof(int), st);
  if (!pl->bf16)
    for (TileSet* ts : {&pl->gram_only, &pl->field_only, &pl->both}) {
      if (ce == cudaSuccess) ce = up(ts->d_tiles, ts->tiles.data(), ts->tiles.size() * sizeof(GramTile));
      if (ce == cudaSuccess) ce = up(ts->d_units, ts->units.data(), ts->units.size() * sizeof(GramUnit));
    }
  if (ce != cudaSuccess) {
    cuda_fail("plan upload", ce);
    return bail(RFD_ECUDA);
  }
  rfd_status st2;
  if (pl->bf16) {
    if ((st2 = build_desc(pl)) != RFD_OK) return bail(st2);
    if (self_batch) {
      rfd_plan_s* self = pl;
      if ((st2 = batch_build(&self, 1, st, mem, self_options(pl), pl->tune, &pl->self)) != RFD_OK) return bail(st2);
    }
    pl->stats.splits = mean_lanes(pl->desc.units[kModeGfi]);
  } else {
    pl->stats.splits = pl->both.units.empty() ? 0 : (int)(pl->both.units.size() / pl->both.tiles.size());
  }
  if (pl->p.flags & RFD_FLAG_TIMING) {
    if ((ce = pl->timing.init()) != cudaSuccess) {
      cuda_fail("event creation", ce);
      return bail(RFD_ECUDA);
    }
  }
  if (sync_init && (ce = cudaStreamSynchronize(st)) != cudaSuccess) {
    cuda_fail("plan upload", ce);
    return bail(RFD_ECUDA);
  }
  return RFD_OK;
}

}  // namespace rfd

extern "C" {

const char* rfd_last_error(void) { return rfd::last_error_cstr(); }
const char* rfd_version(void) { return "rfd-gb300 0.3 (sm_103a)"; }

rfd_status rfd_plan(const rfd_params* params, void* cuda_stream, rfd_plan_t* out) {
  if (!params || !out) return fail(RFD_EINVAL, "null params or output pointer");
  *out = nullptr;
  rfd_plan_s* pl = nullptr;
  rfd_status st = plan_prepare(*params, static_cast<cudaStream_t>(cuda_stream), &pl);
  if (st != RFD_OK) return st;
  if ((st = plan_materialize(pl, cuda_mem(), true, true)) != RFD_OK) return st;
  *out = pl;
  return RFD_OK;
}

rfd_status rfd_plan_destroy(rfd_plan_t plan) {
  if (!plan) return RFD_OK;
  cudaStreamSynchronize(plan->stream);
  plan_destroy(plan);
  return RFD_OK;
}

rfd_status rfd_features(rfd_plan_t pl, const float* d_points) {
  if (!pl || !d_points) return fail(RFD_EINVAL, "null plan or points");
  if (pl->compact) return fail(RFD_EINVAL, "a compact plan has no feature matrix: create a new plan");
  return run_plan(pl, kModeFeatures, d_points, nullptr, 1, 1, nullptr, 1);
}

rfd_status rfd_integrate(rfd_plan_t pl, const float* d_F, int32_t c, int64_t ldF, float* d_out, int64_t ldOut) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  rfd_status s = check_field_args(pl, d_F, c, ldF, d_out, ldOut);
  if (s != RFD_OK) return s;
  if (!pl->have_G) return fail(RFD_EINVAL, "rfd_features (or rfd_gfi) must run before rfd_integrate");
  return run_plan(pl, kModeIntegrate, nullptr, d_F, c, ldF, d_out, ldOut);
}

rfd_status rfd_gfi(rfd_plan_t pl, const float* d_points, const float* d_F, int32_t c, int64_t ldF, float* d_out,
                   int64_t ldOut) {
  if (!pl || !d_points) return fail(RFD_EINVAL, "null plan or points");
  if (pl->compact) return fail(RFD_EINVAL, "a compact plan has no feature matrix: create a new plan");
  rfd_status s = check_field_args(pl, d_F, c, ldF, d_out, ldOut);
  if (s != RFD_OK) return s;
  return run_plan(pl, kModeGfi, d_points, d_F, c, ldF, d_out, ldOut);
}

rfd_status rfd_plan_compact(rfd_plan_t pl) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  return plan_compact(pl, true);
}

rfd_status rfd_plan_device_bytes(rfd_plan_t pl, int64_t* out) {
  if (!pl || !out) return fail(RFD_EINVAL, "null plan or output");
  *out = (int64_t)pl->chunk_bytes;
  return RFD_OK;
}

rfd_status rfd_phi1(int32_t m, double lambda, const double* d_M, double* d_G, int32_t flags, void* cuda_stream,
                    rfd_stats* stats_out) {
  if (m < 1 || m > kMaxM) return fail(RFD_EINVAL, "m must be in [1, 4096]");
  if (!d_M || !d_G || d_M == d_G) return fail(RFD_EINVAL, "null or aliased M / G");
  if (!std::isfinite(lambda)) return fail(RFD_EINVAL, "lambda must be finite");
  if (flags & ~RFD_FLAG_NATIVE_FP64) return fail(RFD_EINVAL, "unknown bits in flags");
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
  cudaMemsetAsync(ints, 0, 4 * sizeof(int), st);
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
  pl->timing.fold(pl->stream);
  *out = pl->stats;
  fill_stats(pl->timing, out);
  out->tune_lanes_pct = pl->tune.lanes_pct;
  out->tune_waves = pl->tune.waves;
  out->tune_phase_blocks = pl->tune.phase_blocks;
  out->tune_pair_gram = pl->tune.pairs;
  out->tune_overlap = pl->tune.overlap;
  for (int f = 0; f < 2; ++f) out->tune_form_ms[f] = pl->tune_form_ms[f];
  out->tuned = pl->tuned ? 1 : 0;
  return RFD_OK;
}

rfd_status rfd_plan_stats_reset(rfd_plan_t pl) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  pl->timing.reset(pl->stream);
  return RFD_OK;
}

// ---- batches -------------------------------------------------------------------
rfd_status rfd_batch_create(const rfd_plan_t* plans, int32_t count, int32_t flags, void* cuda_stream,
                            rfd_batch_t* out) {
  if (!plans || !out || count < 1) return fail(RFD_EINVAL, "null plans / output or count < 1");
  if (flags & ~(RFD_FLAG_TIMING | RFD_FLAG_GRAPH | RFD_FLAG_AUTOTUNE)) return fail(RFD_EINVAL, "unknown bits in flags");
  *out = nullptr;
  std::vector<rfd_plan_s*> v(plans, plans + count);
  for (int i = 0; i < count; ++i) {
    if (!v[i]) return fail(RFD_EINVAL, "null plan in batch");
    if (!v[i]->bf16) return fail(RFD_EINVAL, "batches run the BF16 tensor-core form: plan " + std::to_string(i));
    for (int j = 0; j < i; ++j)
      if (v[j] == v[i]) return fail(RFD_EINVAL, "a plan appears twice in the batch");
  }
  auto* b = new (std::nothrow) rfd_batch_s();
  if (!b) return fail(RFD_ENOMEM, "host allocation failed");
  b->plans = v;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->options = (flags & RFD_FLAG_GRAPH) ? kBatchGraphs : 0;
  b->autotune = (flags & RFD_FLAG_AUTOTUNE) != 0;
  rfd_status s = batch_build(v.data(), count, b->stream, cuda_mem(), b->options, b->tune, &b->impl);
  if (s == RFD_OK && (flags & RFD_FLAG_TIMING)) {
    cudaError_t ce = b->timing.init();
    if (ce != cudaSuccess) s = cuda_fail("event creation", ce);
  }
  if (s != RFD_OK) {
    cudaStreamSynchronize(b->stream);
    if (b->impl) batch_free(b->impl);
    b->timing.destroy();
    delete b;
    return s;
  }
  *out = b;
  return RFD_OK;
}

rfd_status rfd_batch_destroy(rfd_batch_t b) {
  if (!b) return RFD_OK;
  cudaStreamSynchronize(b->stream);
  batch_free(b->impl);
  b->timing.destroy();
  delete b;
  return RFD_OK;
}

// Batch autotuning (see tune_plan): waves x phase length, timed on the batch's own features.
static rfd_status tune_batch(rfd_batch_t b, int mode, const CloudCall* calls) {
  b->tuned = true;
  double work = 0.0;
  for (rfd_plan_s* pl : b->plans) work += (double)pl->desc.units[kModeGfi].size() * (double)(pl->n_pad / kTcBK);
  const auto key = std::make_pair((int)b->plans.size(), ilog2(work));
  GramTuning best_t = b->tune;
  bool cached = false;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_batch_tune.find(key);
    if (it != g_batch_tune.end()) {
      best_t = it->second;
      cached = true;
    }
  }
  RFD_CUDA(cudaStreamSynchronize(b->stream));
  if (!cached) {
    float best = 1e30f;
    for (int waves : {2, 4, 8}) {
      GramTuning t = b->tune;
      t.waves = waves;
      BatchImpl* tb = nullptr;
      rfd_status s = batch_build(b->plans.data(), (int)b->plans.size(), b->stream, cuda_mem(), 0, t, &tb);
      if (s != RFD_OK) return s;
      for (int ph : kTunePhases) {
        batch_set_phase(tb, ph);
        float ms = 0.f;
        s = batch_time_gram(tb, mode, 2, &ms, calls);
        if (s != RFD_OK) break;
        if (ms < best) {
          best = ms;
          best_t = t;
          best_t.phase_blocks = ph;
        }
      }
      cudaStreamSynchronize(b->stream);
      batch_free(tb);
      if (s != RFD_OK) return s;
    }
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_batch_tune[key] = best_t;
  }
  b->tune = best_t;
  BatchImpl* nb = nullptr;
  rfd_status s = batch_build(b->plans.data(), (int)b->plans.size(), b->stream, cuda_mem(), b->options, b->tune, &nb);
  if (s != RFD_OK) return s;
  RFD_CUDA(cudaStreamSynchronize(b->stream));
  batch_free(b->impl);
  b->impl = nb;
  return RFD_OK;
}

static rfd_status batch_call(rfd_batch_t b, int mode, const rfd_batch_item* items) {
  if (!b || !items) return fail(RFD_EINVAL, "null batch or items");
  std::vector<CloudCall> calls(b->plans.size());
  for (size_t k = 0; k < b->plans.size(); ++k) {
    rfd_plan_s* pl = b->plans[k];
    const rfd_batch_item& it = items[k];
    if (mode != kModeIntegrate && !it.d_points) return fail(RFD_EINVAL, "null points for item " + std::to_string(k));
    int c = 1;
    if (mode != kModeFeatures) {
      rfd_status s = check_field_args(pl, it.d_F, it.c, it.ldF, it.d_out, it.ldOut);
      if (s != RFD_OK) return fail(s, "item " + std::to_string(k) + ": " + rfd_last_error());
      if (mode == kModeIntegrate && !pl->have_G)
        return fail(RFD_EINVAL, "item " + std::to_string(k) + ": features not computed");
      c = it.c;
    }
    calls[k] = CloudCall{it.d_points, it.d_F, it.d_out, it.ldF, it.ldOut, c, 0};
  }
  CallScope call(&b->timing, b->stream);
  rfd_status s = batch_run(b->impl, mode, calls.data(), &b->timing);
  if (s == RFD_OK && b->autotune && !b->tuned && mode != kModeIntegrate) s = tune_batch(b, mode, calls.data());
  return s;
}

rfd_status rfd_batch_features(rfd_batch_t b, const rfd_batch_item* items) { return batch_call(b, kModeFeatures, items); }
rfd_status rfd_batch_integrate(rfd_batch_t b, const rfd_batch_item* items) {
  return batch_call(b, kModeIntegrate, items);
}
rfd_status rfd_batch_gfi(rfd_batch_t b, const rfd_batch_item* items) { return batch_call(b, kModeGfi, items); }

rfd_status rfd_batch_eigenvalues(rfd_batch_t b, const rfd_batch_item* items, int32_t k, int32_t largest,
                                 float* d_out) {
  if (!b || !items || !d_out) return fail(RFD_EINVAL, "null batch, items or output");
  if (largest != 0 && largest != 1) return fail(RFD_EINVAL, "largest must be 0 or 1");
  const int n = (int)b->plans.size();
  rfd_status s = check_eigen_args(b->plans.data(), n, k);
  if (s != RFD_OK) return s;
  std::vector<CloudCall> calls((size_t)n);
  for (int i = 0; i < n; ++i) {
    if (!items[i].d_points) return fail(RFD_EINVAL, "null points for item " + std::to_string(i));
    calls[i] = CloudCall{items[i].d_points, nullptr, nullptr, 0, 0, 1, 0};
  }
  CallScope call(&b->timing, b->stream);
  s = batch_run(b->impl, kModeGram, calls.data(), &b->timing);
  if (s == RFD_OK) s = batch_eigenvalues(b->plans.data(), n, k, largest, d_out, b->stream, &b->timing);
  return s;
}

rfd_status rfd_batch_sync(rfd_batch_t b) {
  if (!b) return fail(RFD_EINVAL, "null batch");
  RFD_CUDA(cudaStreamSynchronize(b->stream));
  return batch_check_error(b->impl);
}

rfd_status rfd_batch_stats(rfd_batch_t b, rfd_stats* out) {
  if (!b || !out) return fail(RFD_EINVAL, "null batch or output");
  RFD_CUDA(cudaStreamSynchronize(b->stream));
  b->timing.fold(b->stream);
  *out = rfd_stats{};
  fill_stats(b->timing, out);
  out->tune_lanes_pct = b->tune.lanes_pct;
  out->tune_waves = b->tune.waves;
  out->tune_phase_blocks = b->tune.phase_blocks;
  out->tuned = b->tuned ? 1 : 0;
  return RFD_OK;
}

rfd_status rfd_batch_stats_reset(rfd_batch_t b) {
  if (!b) return fail(RFD_EINVAL, "null batch");
  RFD_CUDA(cudaStreamSynchronize(b->stream));
  b->timing.reset(b->stream);
  return RFD_OK;
}

// Test hook (host-side fault injection): the k-th device allocation from now
// on fails with RFD_ENOMEM (k = 0: the next one); k < 0 disables.
void rfd_debug_fail_alloc_after(int32_t k) { g_fail_alloc_after = k; }

rfd_status rfd_debug_plan_phi1(rfd_plan_t pl, const double* d_M) {
  if (!pl || !d_M) return fail(RFD_EINVAL, "null plan or M");
  if (!pl->bf16 || !pl->self) return fail(RFD_EINVAL, "the batched step a4 runs for BF16 plans");
  RFD_CUDA(cudaMemcpyAsync(pl->d_M, d_M, (size_t)pl->m * pl->m * sizeof(double), cudaMemcpyDeviceToDevice,
                           pl->stream));
  rfd_status s = batch_phi1_only(pl->self);
  if (s != RFD_OK) return s;
  RFD_CUDA(cudaStreamSynchronize(pl->stream));
  return check_device_error(pl);
}

void rfd_debug_gram_pairs(int32_t enable) { g_gram_pairs.store(enable ? 1 : 0); }

rfd_status rfd_debug_plan_set_phase(rfd_plan_t pl, int32_t phase_blocks) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  if (!pl->bf16 || !pl->self) return fail(RFD_EINVAL, "the phase length belongs to the tensor-core reductions");
  if (pl->p.flags & (RFD_FLAG_GRAPH | RFD_FLAG_AUTOTUNE))
    return fail(RFD_EINVAL, "not for plans with RFD_FLAG_GRAPH or RFD_FLAG_AUTOTUNE");
  if (phase_blocks < 1) return fail(RFD_EINVAL, "phase_blocks must be >= 1");
  pl->tune.phase_blocks = phase_blocks;
  batch_set_phase(pl->self, phase_blocks);
  return RFD_OK;
}

rfd_status rfd_debug_plan_set_overlap(rfd_plan_t pl, int32_t enable) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  if (!pl->bf16 || !pl->self) return fail(RFD_EINVAL, "the schedule belongs to the tensor-core reductions");
  if (pl->p.flags & (RFD_FLAG_GRAPH | RFD_FLAG_AUTOTUNE))
    return fail(RFD_EINVAL, "not for plans with RFD_FLAG_GRAPH or RFD_FLAG_AUTOTUNE");
  if (!batch_set_overlap(pl->self, enable != 0) && enable) {
    batch_set_overlap(pl->self, false);
    pl->tune.overlap = 0;
    return fail(RFD_EINVAL, "features beside the Gram need several phases of a multiple of 8 blocks");
  }
  pl->tune.overlap = enable ? 1 : 0;
  return RFD_OK;
}

rfd_status rfd_debug_plan_set_apply_tc(rfd_plan_t pl, int32_t enable) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  if (!pl->bf16 || !pl->self) return fail(RFD_EINVAL, "the tensor-core apply belongs to the BF16 form");
  if (pl->p.flags & RFD_FLAG_GRAPH) return fail(RFD_EINVAL, "not for plans with RFD_FLAG_GRAPH");
  if (enable < 0 || enable > 2) return fail(RFD_EINVAL, "enable must be 0, 1 or 2");
  if (!batch_set_apply_tc(pl->self, enable) && enable == 2) return fail(RFD_ENOTSUP, "the tensor-core apply needs sm_103");
  return RFD_OK;
}

rfd_status rfd_debug_plan_wait_timeout(rfd_plan_t pl, int32_t limit_us) {
  if (!pl) return fail(RFD_EINVAL, "null plan");
  if (limit_us < 1 || limit_us > 1000000) return fail(RFD_EINVAL, "limit_us must be in [1, 1000000]");
  if (!tc_gram_supported()) return fail(RFD_ENOTSUP, "the probe uses tcgen05 (sm_103 only)");
  int* err = pl->bf16 ? batch_error_word(pl->self) : pl->d_ints;
  cudaStream_t st = pl->bf16 ? batch_stream(pl->self) : pl->stream;
  RFD_CUDA(launch_wait_probe((unsigned long long)limit_us * 1000ull, err, st));
  return RFD_OK;
}

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
  if (!ozaki_supported(K)) return fail(RFD_ENOTSUP, "emulated FP64 GEMM needs K <= 4096 on sm_103");
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
