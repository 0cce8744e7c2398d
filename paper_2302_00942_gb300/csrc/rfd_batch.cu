// Batched execution of the BF16 tensor-core path: one launch per step serves
// every cloud of a batch (Sec. 2.4 steps a2..a6 for many point clouds of uneven
// N and m); a single cloud runs as a batch of one.
//
// Step a4 runs on the FP64-accurate tensor-core GEMM for all clouds at once:
// the degree-16 Taylor polynomial of phi1 at 2^-s_c lambda M, evaluated by
// Paterson-Stockmeyer (X^2, X^3, X^4, then three Horner steps in X^4: six
// products), and per-cloud squarings s_c chosen on the device from
// ||lambda M||_1 so that ||2^-s_c lambda M||_1 <= theta_16 (clouds with
// s_c <= k skip squaring step k).  The host waits once per call, for the largest s_c, which sets the
// number of squaring launches.  Non-finite results and device-side timeouts
// are recorded in sticky device words that batch_check_error reads.
//
// A batch's tables live in one device block and one pinned host block from its
// memory source.  With kBatchGraphs the launches of a call are captured once per
// shape (mode, largest s_c, apply grid) into CUDA graphs and replayed.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>
#include "kernels.h"
#include "rfd_phi1.h"
#include "rfd_plan.h"

namespace rfd {

namespace {

// theta_16: the largest ||X||_1 with sum_{k > 16} ||X||_1^k / (k+1)! <= 2^-53, the tail
// of the Taylor series of phi1 after degree 16 (0.97709 by bisection; rounded down)
constexpr double kThetaT16 = 0.977;
constexpr int kTaylorDegree = 16;
constexpr int kMaxSquarings = 60;                 // beyond this exp(lambda M) overflows anyway
constexpr int kPtsMaxChannels = 4;  // integrate calls of full plans up to this c take Phi^T F from the points
// matrix slots of the phi1 evaluation (see kernels.h: slot k = work + k m^2)
enum : int { sX = 0, sX2, sX3, sX4, sB, sF, sFb, sE, sT1 };

std::vector<int> prefix_of(const std::vector<int>& counts) {
  std::vector<int> p(counts.size() + 1, 0);
  for (size_t i = 0; i < counts.size(); ++i) p[i + 1] = p[i] + counts[i];
  return p;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Lays out sections in one block: add() returns each section's offset.
struct Layout {
  size_t total = 0;
  size_t add(size_t bytes) {
    const size_t off = total;
    total += align256(std::max<size_t>(bytes, 1));
    return off;
  }
};

}  // namespace

struct BatchImpl {
  std::vector<rfd_plan_s*> plans;
  int count = 0;
  cudaStream_t st = nullptr;
  MemSource* mem = nullptr;
  int options = 0;
  unsigned char* dblob = nullptr;  // device tables + per-call device words
  size_t dbytes = 0;
  unsigned char* hblob = nullptr;  // pinned: table image, call staging ring, read-back words
  // device tables
  void* d_maps = nullptr;
  TcUnit* d_units[3] = {};
  int n_units[3] = {};
  bool compact = false;      // every plan compact: integrate computes Phi^T F from the points
  bool pts_ok = false;       // every plan has a points-based Phi^T F (compact, or a full BF16 plan)
  FieldPtsJob* d_fpts = nullptr;
  std::vector<FieldPtsJob> fpts_h;  // host copies (block counts per call)
  // the same on the tensor cores (wide fields): chunks of a multiple of 64 points, as many as
  // fill the GPU with their 128-frequency tiles, and the work items' prefix
  FieldPtsJob* d_fpts_tc = nullptr;
  int* d_item_prefix = nullptr;
  int fpts_items = 0;
  int64_t total_n = 0;  // the points of all clouds
  PairUnit* d_pair[3] = {};  // a lone cloud with m >= 512: the 2-SM form of the Gram modes
  int n_pair[3] = {};
  int pair_stage_bytes = 0;
  RedTile* d_red[3] = {};
  int n_red[3] = {};
  FeatJob* d_feat = nullptr;
  int* d_feat_prefix = nullptr;
  int feat_blocks = 0;
  FillJob* d_fill = nullptr;
  int* d_fill_prefix = nullptr;
  int fill_blocks = 0;
  int* d_fillw_prefix = nullptr;  // the wide form (fields of more than 8 channels)
  int fillw_blocks = 0;
  ApplyJob* d_apply = nullptr;
  std::vector<int> apply_bx;
  // the tensor-core apply (k_apply_tc.cu): jobs, their 256-point tiles, whether every plan
  // has its buffers (apply_tc_ok), and when the form is taken (apply_tc_mode)
  ApplyTcJob* d_apply_tc = nullptr;
  std::vector<ApplyTcJob> apply_tc_h;
  int* d_tile_prefix = nullptr;
  int apply_tiles = 0;
  int max_channels = 0;  // the smallest max_channels of the plans (their Z images' capacity)
  int min_m = 0;         // the smallest m of the plans
  bool apply_tc_ok = false;
  int apply_tc_mode = 1;  // 0: SIMT always, 1: by the channel count and m, 2: tensor cores where they can
  int sms = 0;
  int* d_small_prefix = nullptr;
  int small_rows = 0;
  int* d_wide_prefix = nullptr;  // step a5 for wide fields (small_wide_blocks per cloud)
  int wide_blocks = 0;
  PhiCloud* d_phi = nullptr;
  int* d_elem_prefix = nullptr;
  int elem_blocks = 0;
  int* d_rexp_prefix = nullptr;  // blocks of the row-exponent pass (8 rows each)
  int rexp_blocks = 0;
  int* d_grp_prefix = nullptr;  // blocks of the product reconstruction (8 entries per thread)
  int grp_blocks = 0;
  int* d_rowa_prefix = nullptr;
  int rows_a = 0;
  int* d_strip_prefix = nullptr;  // blocks of the B operand's column split
  int col_strips = 0;
  OzTile* d_oz = nullptr;
  int oz_stage_bytes = 0;  // pipeline stage of the residue GEMM
  int n_oz = 0;
  int max_m = 0, max_cpad = 16, max_kb = 0;
  int a_boxes = 1;  // 2 when some Gram unit has a second 128-row half
  int phase_blocks = kGramPhaseBlocks;
  bool overlap = false;     // features phase by phase beside the Gram (a lone cloud, tuned)
  unsigned long long* prof = nullptr;  // the autotuner's per-CTA times of the Gram launches (or null)
  bool phi_batched = true;  // all clouds on the emulated path (no native-FP64 flag)
  // per-call device words
  CloudCall* d_calls = nullptr;  // followed by four block prefixes (count + 1 ints each)
  double* d_norms = nullptr;
  int* d_sv = nullptr;     // squarings per cloud, then their maximum
  int* d_flags = nullptr;  // sticky: G of cloud k not finite
  int* d_err = nullptr;    // sticky: a bounded device-side wait ran out
  // pinned
  static constexpr int kStageRing = 4;  // per-call staging buffers, reused round-robin
  unsigned char* h_stage[kStageRing] = {};
  cudaEvent_t stage_done[kStageRing] = {};
  int stage_next = 0;
  size_t stage_bytes = 0;
  double* h_norms = nullptr;
  int* h_sv = nullptr;
  int* h_flags = nullptr;  // followed by the error word
  cudaEvent_t ev_mid = nullptr;
  // features beside the Gram (a lone cloud with several point-axis phases): a side
  // stream runs the features of phase p + 1 while the main stream runs the Gram of phase p
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_phase;  // features of phase p done
  // CUDA graphs (kBatchGraphs)
  cudaStream_t cap = nullptr;  // capture-only stream (the caller's stream may be the legacy one)
  struct Graph {
    int key[4];
    cudaGraphExec_t exec;
    long long launches;
  };
  std::vector<Graph> graphs;
};

cudaStream_t batch_stream(BatchImpl* b) { return b->st; }
size_t batch_device_bytes(BatchImpl* b) { return b ? b->dbytes : 0; }

void batch_free(BatchImpl* b) {
  if (!b) return;
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int i = 0; i < BatchImpl::kStageRing; ++i)
    if (b->stage_done[i]) cudaEventDestroy(b->stage_done[i]);
  if (b->ev_mid) cudaEventDestroy(b->ev_mid);
  for (cudaEvent_t e : b->ev_phase) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->dblob) b->mem->dev_free(b->dblob);
  if (b->hblob) b->mem->pinned_free(b->hblob);
  delete b;
}

rfd_status batch_build(rfd_plan_s* const* plans, int count, cudaStream_t st, MemSource* mem, int options,
                       const GramTuning& tune, BatchImpl** out) {
  *out = nullptr;
  auto* b = new (std::nothrow) BatchImpl();
  if (!b) return fail(RFD_ENOMEM, "host allocation failed");
  b->plans.assign(plans, plans + count);
  b->count = count;
  b->st = st;
  b->mem = mem;
  b->options = options;
  b->phase_blocks = tune.phase_blocks;
  b->overlap = tune.overlap != 0;
  auto bail = [&](rfd_status s, const std::string& msg) {
    batch_free(b);
    return fail(s, msg);
  };
  const int sms = plans[0]->sms;
  // --- Gram lanes: every tile's lanes share the batch's CTAs in proportion to its cost
  double work = 0.0;  // SM clocks of all tiles over all their 64-point blocks
  for (int k = 0; k < count; ++k)
    for (const TcUnit& u : plans[k]->desc.units[kModeGfi])
      if (u.lane == 0) work += (double)u.work * (double)(plans[k]->n_pad / kTcBK);
  const double target = (count == 1) ? 1e300 : std::max(1.0, work / (tune.waves * (double)sms));  // clocks per CTA
  std::vector<TcUnit> units[3];
  std::vector<PairUnit> pairs[3];
  std::vector<RedTile> red[3];
  std::vector<unsigned char> maps((size_t)count * kMapsPerCloud * kTensorMapBytes);
  std::vector<FeatJob> feat;
  std::vector<FieldPtsJob> fpts;
  int n_compact = 0;
  for (int k = 0; k < count; ++k) n_compact += plans[k]->compact ? 1 : 0;
  if (n_compact && n_compact != count) return bail(RFD_EINVAL, "a batch cannot mix compact and full plans");
  b->compact = n_compact == count;
  b->pts_ok = true;
  for (int k = 0; k < count; ++k) b->pts_ok = b->pts_ok && plans[k]->desc.fpts.part != nullptr;
  if (b->pts_ok)
    for (int k = 0; k < count; ++k) {
      b->fpts_h.push_back(plans[k]->desc.fpts);
      b->fpts_h.back().cloud = k;
    }
  std::vector<FillJob> fill;
  std::vector<ApplyJob> apply;
  std::vector<int> tiles_n, wide_n, fillw_n, items_n;
  std::vector<FieldPtsJob> fpts_tc;
  b->apply_tc_ok = apply_tc_supported();
  b->max_channels = plans[0]->p.max_channels;
  b->sms = sms;
  std::vector<PhiCloud> phi;
  std::vector<int> feat_n, fill_n, small_n, elem_n, grp_n, rowa_n, rexp_n, strip_n;
  std::vector<OzTile> oz;
  for (int k = 0; k < count; ++k) {
    rfd_plan_s* pl = plans[k];
    const PlanDesc& d = pl->desc;
    b->max_m = std::max(b->max_m, pl->m);
    b->max_cpad = std::max(b->max_cpad, pl->cpad);
    b->max_kb = std::max<int>(b->max_kb, (int)(pl->n_pad / kTcBK));
    if (!ozaki_supported(pl->m) || (pl->p.flags & RFD_FLAG_NATIVE_FP64)) b->phi_batched = false;
    std::memcpy(maps.data() + (size_t)k * kMapsPerCloud * kTensorMapBytes, d.maps, sizeof(d.maps));
    const int64_t kb = pl->n_pad / kTcBK;
    if (b->pts_ok) {  // integrate from the points (always for compact plans)
      FieldPtsJob fj = d.fpts;
      fj.cloud = k;
      fpts.push_back(fj);
      // the tensor-core form: chunks of a multiple of 64 points, no more than the partials hold;
      // a lone cloud takes as many as fill whole waves of SMs with its frequency tiles
      const int ftiles = (fj.h + 127) / 128;
      int want = fj.chunks;
      if (count == 1 && fj.chunks * ftiles > sms)
        want = std::max(1, (std::max(1, fj.chunks * ftiles / sms) * sms) / ftiles);
      want = std::min(want, fj.chunks);
      FieldPtsJob tj = fj;
      tj.pts = std::max<int64_t>(64, (fj.n + want - 1) / want + 63) / 64 * 64;
      tj.chunks = (int)((fj.n + tj.pts - 1) / tj.pts);
      fpts_tc.push_back(tj);
      items_n.push_back(fieldpts_tc_items(tj));
    }
    for (int mode = 0; mode < 3 && !b->compact; ++mode) {
      if (count == 1 && tune.pairs && !d.pair_units[mode].empty()) {  // a lone cloud: the plan's pair units
        pairs[mode] = d.pair_units[mode];
        red[mode] = d.pair_red[mode];
        b->pair_stage_bytes = d.pair_stage_bytes;
        continue;
      }
      // the plan's own units give each tile L_plan lanes; a batch may give it fewer
      const std::vector<TcUnit>& pu = d.units[mode];
      if (pu.empty()) continue;
      std::vector<int64_t> half_base;  // first partial slot of each logical half
      std::vector<int> half_lanes;
      int64_t base = 0;
      for (size_t i = 0; i < pu.size(); i += pu[i].nlanes) {
        const TcUnit& u0 = pu[i];
        const int L_plan = u0.nlanes;
        int L = L_plan;
        if (count > 1)
          L = (int)std::max<int64_t>(1, std::min<int64_t>(L_plan, (int64_t)std::ceil((double)kb * u0.work / target)));
        const int halves = u0.out1 ? 2 : 1;
        half_base.resize(u0.slot + halves);
        half_lanes.resize(u0.slot + halves);
        for (int h = 0; h < halves; ++h) {
          half_base[u0.slot + h] = base + (int64_t)h * L;
          half_lanes[u0.slot + h] = L;
        }
        for (int l = 0; l < L; ++l) {
          TcUnit u = u0;
          u.lane = l;
          u.nlanes = L;
          u.map += k * kMapsPerCloud;
          u.out = pl->d_part + (base + l) * pl->slot_elems;
          if (u.out1) u.out1 = pl->d_part + (base + L + l) * pl->slot_elems;
          if (u.out1) b->a_boxes = 2;
          units[mode].push_back(u);
        }
        base += (int64_t)halves * L;
      }
      for (RedTile r : d.red[mode]) {
        // red tiles of the plan name their logical half in .count: point them at its lanes' partials
        const int s = r.count;
        r.part = pl->d_part + half_base[s] * pl->slot_elems;
        r.count = half_lanes[s];
        r.cloud = k;
        red[mode].push_back(r);
      }
    }
    FeatJob fj = d.feat;
    fj.cloud = k;
    feat.push_back(fj);
    feat_n.push_back(fj.bx * ((fj.h + 31) / 32));
    FillJob fl = d.fill;
    fl.cloud = k;
    fill.push_back(fl);
    fill_n.push_back(fl.bx);
    fillw_n.push_back(fl.bxw * fl.cgw);
    ApplyJob aj = d.apply;
    aj.cloud = k;
    apply.push_back(aj);
    b->apply_bx.push_back(aj.bx);
    ApplyTcJob tj = d.apply_tc;
    tj.cloud = k;
    b->apply_tc_h.push_back(tj);
    tiles_n.push_back(tj.tiles);
    b->apply_tc_ok = b->apply_tc_ok && tj.zimg != nullptr && tj.w2pi != nullptr;
    b->max_channels = std::min(b->max_channels, pl->p.max_channels);
    b->min_m = (k == 0) ? pl->m : std::min(b->min_m, pl->m);
    b->total_n += pl->n;
    small_n.push_back(pl->m);
    wide_n.push_back(small_wide_blocks(pl->m, pl->p.max_channels));
    PhiCloud pc = d.phi;
    pc.map_a += k * kMapsPerCloud;
    pc.map_b += k * kMapsPerCloud;
    pc.s = 0;
    pc.scale = 1.0;
    phi.push_back(pc);
    elem_n.push_back((int)(((int64_t)pl->m * pl->m + 255) / 256));
    grp_n.push_back(ozaki_combine_blocks(pl->m));
    rowa_n.push_back(ozaki_row_split_warps(pl->m));
    rexp_n.push_back(ozaki_row_exponent_blocks(pl->m));
    strip_n.push_back(ozaki_col_split_blocks(pl->m));
  }
  const std::vector<int> pre_tiles = prefix_of(tiles_n), pre_wide = prefix_of(wide_n), pre_fillw = prefix_of(fillw_n),
                         pre_items = prefix_of(items_n);
  b->fpts_items = pre_items.back();
  b->fillw_blocks = pre_fillw.back();
  b->apply_tiles = pre_tiles.back();
  b->wide_blocks = pre_wide.back();
  const std::vector<int> pre_feat = prefix_of(feat_n), pre_fill = prefix_of(fill_n), pre_small = prefix_of(small_n),
                         pre_elem = prefix_of(elem_n), pre_grp = prefix_of(grp_n), pre_rexp = prefix_of(rexp_n), pre_rowa = prefix_of(rowa_n), pre_strip = prefix_of(strip_n);
  b->feat_blocks = pre_feat.back();
  b->fill_blocks = pre_fill.back();
  b->small_rows = pre_small.back();
  b->elem_blocks = pre_elem.back();
  b->grp_blocks = pre_grp.back();
  b->rexp_blocks = pre_rexp.back();
  b->rows_a = pre_rowa.back();
  b->col_strips = pre_strip.back();
  {
    std::vector<int> ms;
    for (int k = 0; k < count; ++k) ms.push_back(plans[k]->m);
    ozaki_batch_tiles(ms, sms, &oz, &b->oz_stage_bytes);
  }
  b->n_oz = (int)oz.size();
  // --- one device block: the tables, then the per-call words
  struct Sec {
    size_t off;
    const void* src;
    size_t bytes;
  };
  std::vector<Sec> secs;
  Layout L;
  auto table = [&](const void* src, size_t bytes) {
    secs.push_back(Sec{L.add(bytes), src, bytes});
    return secs.back().off;
  };
  auto vtable = [&](const auto& v) { return table(v.data(), v.size() * sizeof(v[0])); };
  const size_t o_maps = vtable(maps);
  size_t o_units[3], o_pair[3], o_red[3];
  for (int mode = 0; mode < 3; ++mode) {
    o_units[mode] = vtable(units[mode]);
    o_pair[mode] = vtable(pairs[mode]);
    o_red[mode] = vtable(red[mode]);
    b->n_units[mode] = (int)units[mode].size();
    b->n_pair[mode] = (int)pairs[mode].size();
    b->n_red[mode] = (int)red[mode].size();
  }
  const size_t o_feat = vtable(feat), o_feat_pre = vtable(pre_feat), o_fill = vtable(fill),
               o_fill_pre = vtable(pre_fill), o_apply = vtable(apply), o_small_pre = vtable(pre_small),
               o_phi = vtable(phi), o_elem_pre = vtable(pre_elem), o_grp_pre = vtable(pre_grp), o_rexp_pre = vtable(pre_rexp), o_rowa_pre = vtable(pre_rowa),
               o_strip_pre = vtable(pre_strip), o_oz = vtable(oz), o_fpts = vtable(fpts),
               o_apply_tc = vtable(b->apply_tc_h), o_tile_pre = vtable(pre_tiles), o_wide_pre = vtable(pre_wide),
               o_fillw_pre = vtable(pre_fillw), o_fpts_tc = vtable(fpts_tc), o_items_pre = vtable(pre_items);
  const size_t table_bytes = L.total;
  // per call: the CloudCalls, then the block prefixes of the apply, the points-based Phi^T F,
  // its sum over the chunks and the tensor-core apply's Z images
  b->stage_bytes = (size_t)count * sizeof(CloudCall) + 4 * (size_t)(count + 1) * sizeof(int);
  const size_t o_calls = L.add(b->stage_bytes);
  const size_t o_norms = L.add((size_t)count * sizeof(double));
  const size_t o_sv = L.add((size_t)(count + 1) * sizeof(int));
  const size_t o_flags = L.add((size_t)(count + 1) * sizeof(int));  // flags, then the error word
  b->dbytes = L.total;
  // --- one pinned block: the table image (same offsets), the staging ring, read-back words
  Layout H;
  H.add(table_bytes);
  size_t o_stage[BatchImpl::kStageRing];
  for (size_t& o : o_stage) o = H.add(b->stage_bytes);
  const size_t o_hn = H.add((size_t)count * sizeof(double));
  const size_t o_hsv = H.add((size_t)(count + 1) * sizeof(int));
  const size_t o_hf = H.add((size_t)(count + 1) * sizeof(int));
  b->dblob = static_cast<unsigned char*>(mem->dev(b->dbytes));
  if (!b->dblob) return bail(RFD_ENOMEM, "device allocation of " + std::to_string(b->dbytes) + " bytes (batch tables) failed");
  b->hblob = static_cast<unsigned char*>(mem->pinned(H.total));
  if (!b->hblob) return bail(RFD_ENOMEM, "pinned allocation of " + std::to_string(H.total) + " bytes failed");
  unsigned char* D = b->dblob;
  b->d_maps = D + o_maps;
  for (int mode = 0; mode < 3; ++mode) {
    b->d_units[mode] = reinterpret_cast<TcUnit*>(D + o_units[mode]);
    b->d_pair[mode] = reinterpret_cast<PairUnit*>(D + o_pair[mode]);
    b->d_fpts = reinterpret_cast<FieldPtsJob*>(D + o_fpts);
    b->d_red[mode] = reinterpret_cast<RedTile*>(D + o_red[mode]);
  }
  b->d_feat = reinterpret_cast<FeatJob*>(D + o_feat);
  b->d_feat_prefix = reinterpret_cast<int*>(D + o_feat_pre);
  b->d_fill = reinterpret_cast<FillJob*>(D + o_fill);
  b->d_fill_prefix = reinterpret_cast<int*>(D + o_fill_pre);
  b->d_apply = reinterpret_cast<ApplyJob*>(D + o_apply);
  b->d_apply_tc = reinterpret_cast<ApplyTcJob*>(D + o_apply_tc);
  b->d_tile_prefix = reinterpret_cast<int*>(D + o_tile_pre);
  b->d_wide_prefix = reinterpret_cast<int*>(D + o_wide_pre);
  b->d_fillw_prefix = reinterpret_cast<int*>(D + o_fillw_pre);
  b->d_fpts_tc = reinterpret_cast<FieldPtsJob*>(D + o_fpts_tc);
  b->d_item_prefix = reinterpret_cast<int*>(D + o_items_pre);
  b->d_small_prefix = reinterpret_cast<int*>(D + o_small_pre);
  b->d_phi = reinterpret_cast<PhiCloud*>(D + o_phi);
  b->d_elem_prefix = reinterpret_cast<int*>(D + o_elem_pre);
  b->d_grp_prefix = reinterpret_cast<int*>(D + o_grp_pre);
  b->d_rexp_prefix = reinterpret_cast<int*>(D + o_rexp_pre);
  b->d_rowa_prefix = reinterpret_cast<int*>(D + o_rowa_pre);
  b->d_strip_prefix = reinterpret_cast<int*>(D + o_strip_pre);
  b->d_oz = reinterpret_cast<OzTile*>(D + o_oz);
  b->d_calls = reinterpret_cast<CloudCall*>(D + o_calls);
  b->d_norms = reinterpret_cast<double*>(D + o_norms);
  b->d_sv = reinterpret_cast<int*>(D + o_sv);
  b->d_flags = reinterpret_cast<int*>(D + o_flags);
  b->d_err = b->d_flags + count;
  for (int k = 0; k < count; ++k) phi[k].flag = b->d_flags + k;
  for (const Sec& s : secs)
    if (s.bytes) std::memcpy(b->hblob + s.off, s.src, s.bytes);
  for (int i = 0; i < BatchImpl::kStageRing; ++i) b->h_stage[i] = b->hblob + o_stage[i];
  b->h_norms = reinterpret_cast<double*>(b->hblob + o_hn);
  b->h_sv = reinterpret_cast<int*>(b->hblob + o_hsv);
  b->h_flags = reinterpret_cast<int*>(b->hblob + o_hf);
  cudaError_t e = cudaMemcpyAsync(b->dblob, b->hblob, table_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dblob + table_bytes, 0, b->dbytes - table_bytes, st);
  for (int i = 0; i < BatchImpl::kStageRing && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&b->stage_done[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_mid, cudaEventDisableTiming);
  if (e == cudaSuccess && count == 1) {
    e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  }
  if (e == cudaSuccess && (options & kBatchGraphs)) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = gram_tc_prepare();
  if (e == cudaSuccess && b->n_pair[0] + b->n_pair[1] + b->n_pair[2] > 0) e = gram_pair_prepare();
  if (e == cudaSuccess) e = bgemm_prepare();
  if (e == cudaSuccess && b->apply_tc_ok) e = apply_tc_prepare();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(RFD_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
  }
  *out = b;
  return RFD_OK;
}

namespace {

rfd_status cuda_fail2(const char* what, cudaError_t e) {
  return fail(RFD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BCK(call)                                        \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail2(#call, e_); \
  } while (0)

// Step a4, first part, for every cloud: X = lambda M, ||X||_1, and the
// squarings s_c (device); the s_c and norms are copied to pinned memory.
rfd_status phi1_select(BatchImpl* b, cudaStream_t st) {
  const int n = b->count;
  const int src[4] = {kSlotM, 0x7fffffff, 0x7fffffff, 0x7fffffff};
  const double a[4] = {1.0, 0.0, 0.0, 0.0};
  BCK(launch_bcombine(b->d_phi, b->d_elem_prefix, n, b->elem_blocks, sX, src, a, 0.0, 1, -1, st));  // X = lambda M
  BCK(launch_bnorm1(b->d_phi, n, b->max_m, sX, b->d_norms, st));
  BCK(launch_bselect(b->d_phi, n, b->d_norms, kThetaT16, kMaxSquarings, b->d_sv, st));
  BCK(cudaMemcpyAsync(b->h_sv, b->d_sv, (size_t)(n + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(b->h_norms, b->d_norms, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
  return RFD_OK;
}

// Step a4, second part: phi1 at X = 2^-s_c lambda M by its Taylor polynomial of
// degree 16, sum_k X^k / (k+1)!, in Paterson-Stockmeyer form with blocks of 4:
// with B_j = sum_{i<4} c_{4j+i} X^i (c_k = 1/(k+1)!),
//   F = B_0 + X^4 (B_1 + X^4 (B_2 + X^4 (B_3 + c_16 X^4)))
// -- three products for X^2, X^3, X^4 and three Horner products, whose
// epilogues (D = alpha A B + beta C + diag I) add B_j (its X, X^2, X^3 part
// from one element-wise combination, c_{4j} on the diagonal); then max_s masked
// squaring steps, phi1(2Y) = (e^Y + I) phi1(Y) / 2 with e^Y = I + Y phi1(Y):
// E = I + X F, F <- (E F + F) / 2, E <- E^2; G = lambda F, and the finiteness
// flags.  Slots are swapped instead of copied.
// Moduli per product of the Taylor evaluation (see phi1_core), from the batch's
// largest scaled norm x = max ||2^-s lambda M||_1 <= theta_16 and largest m:
// {X^2, X^3 and X^4 (one count: they share operands), Horner j = 2, 1, 0}.
// An emulated product P = A B with k-bit operand integers errs by at most
// 2^(1-k) K max|A| max|B| per entry; a native FP64 product by ~K u max|A|
// max|B|.  If P's error reaches F = phi1(X) multiplied by at most S, and F's
// largest entry is at least 1/2 (its diagonal is >= phi1(-x) >= 0.6), then
// k = 55 + log2(max|A| max|B| S / (1/2)) bits keep P's share of F's error at
// half a native product's worst case or less.  Entry bounds (|M| is symmetric,
// so its row and column norms agree): |(X^i)_ab| <= x^i; the Horner partial
// sums F_j = B_j + X^4 F_(j+1) have entries <= f_j = sum_(k >= 4j) c_k x^(k-4j).
//   X^p (p = 2, 3, 4):  max|A| max|B| = x^p, S = sum_(k >= p) k c_k x^(k-p)
//     (X^p occurs at most k times in the evaluation of X^k);
//   Horner j (X^4 F_(j+1) + B_j):  x^4 f_(j+1), S = x^(4j) (the factors X^4 to come).
// The Horner products take far fewer moduli than the powers: their operands
// F_(j+1) are small (f_3 ~ c_12 = 1/13!).  The counts enter the CUDA-graph key.
void product_moduli(const BatchImpl* b, int out[4]) {
  double x = 0.0;
  for (int c = 0; c < b->count; ++c)
    if (std::isfinite(b->h_norms[c])) x = std::max(x, std::ldexp(b->h_norms[c], -std::max(b->h_sv[c], 0)));
  x = std::min(x, kThetaT16);
  double ck[kTaylorDegree + 1];
  ck[0] = 1.0;
  for (int k = 1; k <= kTaylorDegree; ++k) ck[k] = ck[k - 1] / (double)(k + 1);
  auto moduli_for = [&](double scale) {  // scale = max|A| max|B| S
    const int k = (int)std::ceil(55.0 + std::log2(std::max(scale / 0.5, 1e-300)));
    return std::min(16, std::max(4, ozaki_moduli_for_bits(std::max(b->max_m, 1), k)));
  };
  int powers = 4;
  for (int p = 2; p <= 4; ++p) {
    double S = 0.0;
    for (int k = p; k <= kTaylorDegree; ++k) S += k * ck[k] * std::pow(x, k - p);
    powers = std::max(powers, moduli_for(std::pow(x, p) * S));
  }
  out[0] = powers;
  for (int j = 2; j >= 0; --j) {
    double f = 0.0;  // f_(j+1)
    for (int k = 4 * (j + 1); k <= kTaylorDegree; ++k) f += ck[k] * std::pow(x, k - 4 * (j + 1));
    out[3 - j] = moduli_for(std::pow(x, 4) * f * std::pow(x, 4 * j));
  }
}

rfd_status phi1_core(BatchImpl* b, cudaStream_t st, int max_s, const int nmod[4]) {
  const int n = b->count;
  auto comb = [&](int dst, std::initializer_list<int> src, std::initializer_list<double> a, double diag, int kmode,
                  int mask) {
    int s4[4] = {0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff};
    double a4[4] = {0, 0, 0, 0};
    int i = 0;
    for (int v : src) s4[i++] = v;
    i = 0;
    for (double v : a) a4[i++] = v;
    return launch_bcombine(b->d_phi, b->d_elem_prefix, n, b->elem_blocks, dst, s4, a4, diag, kmode, mask, st);
  };
  // moduli per product (product_moduli); the squaring steps take all 16
  const int kfull = 16;
  // the A / B residues hold the operands of the previous product (split with the same
  // number of moduli, hence the same integer width): split only what changed
  int last_a = kNoSlot, last_b = kNoSlot, last_na = 0, last_nb = 0;
  auto gemm = [&](int a, int bb, int c, int d, double alpha, double beta, double diag, int mask, int nmod) {
    const bool sa = a != last_a || nmod != last_na, sb = bb != last_b || nmod != last_nb;
    last_a = a;
    last_b = bb;
    last_na = last_nb = nmod;
    return launch_bgemm(b->d_phi, n, b->d_rowa_prefix, b->rows_a, b->d_rexp_prefix, b->rexp_blocks, b->d_strip_prefix, b->col_strips, b->d_oz,
                        b->n_oz, b->oz_stage_bytes, b->d_grp_prefix, b->grp_blocks, nmod, b->d_maps, a,
                        bb, c, d, alpha, beta, diag, mask, sa, sb, b->d_err, st);
  };
  // a slot that is written no longer matches its residues
  auto wrote = [&](int slot) {
    if (slot == last_a) last_a = kNoSlot;
    if (slot == last_b) last_b = kNoSlot;
  };
  double ck[kTaylorDegree + 1];  // c_k = 1 / (k + 1)!
  ck[0] = 1.0;
  for (int k = 1; k <= kTaylorDegree; ++k) ck[k] = ck[k - 1] / (double)(k + 1);
  if (max_s > 0) BCK(comb(sX, {sX}, {1.0}, 0.0, 2, -1));  // X = 2^-s X
  BCK(gemm(sX, sX, kNoSlot, sX2, 1.0, 0.0, 0.0, -1, nmod[0]));
  wrote(sX2);
  BCK(gemm(sX2, sX, kNoSlot, sX3, 1.0, 0.0, 0.0, -1, nmod[0]));
  wrote(sX3);
  BCK(gemm(sX2, sX2, kNoSlot, sX4, 1.0, 0.0, 0.0, -1, nmod[0]));
  wrote(sX4);
  BCK(comb(sF, {sX, sX2, sX3, sX4}, {ck[13], ck[14], ck[15], ck[16]}, ck[12], 0, -1));  // B_3 + c_16 X^4
  wrote(sF);
  int F = sF, Fb = sFb;
  for (int j = 2; j >= 0; --j) {
    BCK(comb(sB, {sX, sX2, sX3}, {ck[4 * j + 1], ck[4 * j + 2], ck[4 * j + 3]}, 0.0, 0, -1));  // B_j - c_4j I
    wrote(sB);
    const int nm = nmod[3 - j];
    BCK(gemm(sX4, F, sB, Fb, 1.0, 1.0, ck[4 * j], -1, nm));  // F <- B_j + X^4 F
    wrote(Fb);
    std::swap(F, Fb);
  }
  if (max_s > 0) {
    int E = sE, E2 = sT1;
    BCK(gemm(sX, F, kNoSlot, E, 1.0, 0.0, 1.0, -1, kfull));  // E = I + X F
    wrote(E);
    for (int k = 0; k < max_s; ++k) {
      BCK(gemm(E, F, F, Fb, 0.5, 0.5, 0.0, k, kfull));  // F <- (E F + F) / 2 (clouds with s <= k copy F)
      wrote(Fb);
      std::swap(F, Fb);
      if (k + 1 < max_s) {
        BCK(gemm(E, E, kNoSlot, E2, 1.0, 0.0, 0.0, k + 1, kfull));  // E <- E^2 (clouds with s <= k + 1 skip)
        wrote(E2);
        std::swap(E, E2);
      }
    }
  }
  BCK(comb(kSlotG, {F}, {1.0}, 0.0, 1, -1));  // G = lambda F
  BCK(launch_bfinite(b->d_phi, b->d_elem_prefix, n, b->elem_blocks, kSlotG, st));
  return RFD_OK;
}

// Step a4 one cloud at a time (native FP64 requested).
rfd_status phi1_per_plan(BatchImpl* b) {
  for (rfd_plan_s* pl : b->plans) {
    Phi1Info info{};
    rfd_status s = phi1_fp64(pl->m, pl->p.lambda, pl->d_M, pl->d_G, pl->d_work, pl->d_ipiv, pl->d_ints + 1,
                             pl->d_scalar, pl->d_ints + 2, b->d_err, (pl->p.flags & RFD_FLAG_NATIVE_FP64) == 0, b->st,
                             &info);
    pl->stats.phi1_emulated = info.emulated;
    pl->stats.phi1_gemms = info.gemms;
    pl->stats.norm1 = info.norm1;
    pl->stats.pade_degree = info.degree;
    pl->stats.squarings = info.squarings;
    pl->stats.nonfinite = info.nonfinite;
    if (s == RFD_ENUMERIC) return fail(s, "G = lambda phi1(lambda M) is not finite");
    if (s != RFD_OK) return fail(s, std::string("phi1: ") + cudaGetErrorString(cudaGetLastError()));
  }
  return RFD_OK;
}

// Runs enqueue(stream, timing) on the batch's stream, or (kBatchGraphs) replays
// the graph captured for `key`, capturing it on first use.
template <typename Fn>
rfd_status run_segment(BatchImpl* b, const int (&key)[4], bool graph, Timing* tm, Fn enqueue) {
  if (!graph) return enqueue(b->st, tm);
  BatchImpl::Graph* g = nullptr;
  for (auto& x : b->graphs)
    if (std::equal(key, key + 4, x.key)) g = &x;
  if (!g) {
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const long long l0 = t_kernel_launches;
    rfd_status s = enqueue(b->cap, nullptr);
    const long long nl = t_kernel_launches - l0;
    t_kernel_launches = l0;
    cudaGraph_t graph_obj = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &graph_obj);
    cudaGraphExec_t exec = nullptr;
    if (s == RFD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph_obj, 0);
    if (graph_obj) cudaGraphDestroy(graph_obj);
    if (s != RFD_OK) return s;
    if (e != cudaSuccess) return cuda_fail2("CUDA graph capture", e);
    b->graphs.push_back(BatchImpl::Graph{{key[0], key[1], key[2], key[3]}, exec, nl});
    g = &b->graphs.back();
  }
  BCK(cudaGraphLaunch(g->exec, b->st));
  count_launch(g->launches);
  return RFD_OK;
}

}  // namespace

// One phase of the reductions over N of `mode`: the 2-SM pair kernel when the batch
// has pair units for the mode, else the one-SM kernel.
cudaError_t gram_phase(BatchImpl* b, int mode, int kb0, cudaStream_t s) {
  if (b->n_pair[mode] > 0)
    return launch_gram_pair_phase(b->d_maps, b->d_pair[mode], b->n_pair[mode], b->pair_stage_bytes, kb0,
                                  b->phase_blocks, b->d_err, s, b->prof);
  return launch_gram_tc_phase(b->d_maps, b->d_units[mode], b->n_units[mode], b->a_boxes, kb0, b->phase_blocks,
                              b->d_err, s, b->prof);
}
// All phases of the reductions over N of `mode`, one launch each.
cudaError_t gram_all(BatchImpl* b, int mode, cudaStream_t s) {
  const int phases = b->max_kb > 0 ? (b->max_kb + b->phase_blocks - 1) / b->phase_blocks : 1;
  for (int p = 0; p < phases; ++p) {
    const cudaError_t e = gram_phase(b, mode, p * b->phase_blocks, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Features beside the Gram: a lone cloud whose point axis takes several Gram
// phases (of a multiple of 8 blocks, so that the 512-point blocks of the
// features kernel fall in one phase) may run its features phase by phase on
// the side stream; the Gram of phase p waits for the features of phase p only,
// so the features of phase p + 1 (MUFU and HBM writes) overlap the Gram of
// phase p (tensor cores and L2 reads).  The autotuner does not choose it (at
// N = 10^6, m = 1024 it gains 1.5 - 2 % of the step, and the Gram's own time
// is no longer measurable); rfd_debug_plan_set_overlap selects it.
int gram_phases(const BatchImpl* b) {
  return b->max_kb > 0 ? (b->max_kb + b->phase_blocks - 1) / b->phase_blocks : 1;
}
bool can_overlap(const BatchImpl* b) { return b->side && gram_phases(b) >= 2 && b->phase_blocks % 8 == 0; }
bool pipelines(const BatchImpl* b) { return b->overlap && can_overlap(b); }

// The features, phase by phase, on the side stream (forked from s); ev_phase[p]
// marks phase p done.  The last event is recorded after the step's timing scope.
rfd_status pipelined_features(BatchImpl* b, cudaStream_t s, Timing* t) {
  const int phases = gram_phases(b);
  while ((int)b->ev_phase.size() < phases) {
    cudaEvent_t e = nullptr;
    BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->ev_phase.push_back(e);
  }
  const rfd_plan_s* pl = b->plans[0];
  const int bx = pl->desc.feat.bx, per = b->phase_blocks / 8;  // 512-point blocks per phase
  BCK(cudaEventRecord(b->ev_fork, s));
  BCK(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
  {
    StepScope sc(t, b->side, RFD_STEP_FEATURES);
    for (int p = 0; p < phases; ++p) {
      BCK(launch_features_range(b->d_feat, b->d_calls, pl->h, p * per, std::min(per, bx - p * per), b->side));
      if (p + 1 < phases) BCK(cudaEventRecord(b->ev_phase[p], b->side));
    }
  }
  BCK(cudaEventRecord(b->ev_phase[phases - 1], b->side));
  return RFD_OK;
}

// The Gram phases on s, each after the features of its phase (pipelined_features first).
// The step's timing scope opens after the wait for the first phase's features, so that
// it spans the Gram launches (and any later wait between them), not the features ahead.
rfd_status pipelined_gram(BatchImpl* b, int mode, cudaStream_t s, Timing* t) {
  for (int p = 0; p < gram_phases(b); ++p) {
    BCK(cudaStreamWaitEvent(s, b->ev_phase[p], 0));
    StepScope sc(t, s, RFD_STEP_GRAM);
    BCK(gram_phase(b, mode, p * b->phase_blocks, s));
  }
  return RFD_OK;
}

rfd_status batch_run(BatchImpl* b, int mode, const CloudCall* calls, Timing* tm) {
  cudaStream_t st = b->st;
  const bool gram_only = mode == kModeGram;
  if (gram_only) mode = kModeFeatures;
  const int n = b->count;
  // per-call tables: the callers' buffers, and the apply blocks (they depend on c)
  int max_c = 1;
  for (int k = 0; k < n; ++k) max_c = std::max(max_c, calls[k].c);
  const int cg = max_c <= 3 ? 3 : (max_c <= 4 ? 4 : (max_c <= 8 ? 8 : (max_c <= 16 ? 16 : 32)));
  // the apply on the tensor cores where it is the faster form: the SIMT kernel's FMAs grow with
  // c, the tensor-core form's time hardly (it has a fixed cost per 256-point tile instead), so
  // above 16 channels always, from 9 channels on when every cloud has m >= 512 (measured on
  // GB300 at N = 10^5 and 10^6, m = 128 .. 1024); up to the Z images' capacity
  const bool tc_rule = b->apply_tc_ok && max_c <= std::min(kApplyTcMaxC, b->max_channels) &&
                       (b->apply_tc_mode == 2 ||
                        (b->apply_tc_mode == 1 && (max_c > 16 || (max_c > 8 && b->min_m >= 512))));
  const bool use_tc = mode != kModeFeatures && tc_rule;
  // a pinned staging buffer whose previous upload has been consumed
  const int slot = b->stage_next;
  b->stage_next = (slot + 1) % BatchImpl::kStageRing;
  BCK(cudaEventSynchronize(b->stage_done[slot]));
  unsigned char* stage = b->h_stage[slot];
  auto* hc = reinterpret_cast<CloudCall*>(stage);
  auto* hp = reinterpret_cast<int*>(stage + (size_t)n * sizeof(CloudCall));
  hp[0] = 0;
  for (int k = 0; k < n; ++k) {
    hc[k] = calls[k];
    const int nb = (mode == kModeFeatures || use_tc) ? 0 : b->apply_bx[k] * ((calls[k].c + cg - 1) / cg);
    hp[k + 1] = hp[k] + nb;
  }
  const int apply_blocks = hp[n];
  const int* d_apply_prefix = reinterpret_cast<const int*>(reinterpret_cast<unsigned char*>(b->d_calls) +
                                                           (size_t)n * sizeof(CloudCall));
  // Phi^T F from the points: always for compact plans; for full plans in integration calls of
  // few channels, where it is faster than a pass over Psi (its cost grows with c, the pass's
  // hardly) and carries no BF16 rounding
  const bool pts = b->compact || (mode == kModeIntegrate && b->pts_ok && max_c <= kPtsMaxChannels);
  // the same on the tensor cores where the apply takes them (the two share the rule), and by
  // default only for 2^19 points or more: its persistent CTAs take whole SMs, and in a serving
  // mix of smaller concurrent requests that cost latency (p99 2.0 -> 6.4 ms measured)
  const bool use_tcf = pts && tc_rule && (b->apply_tc_mode == 2 || b->total_n >= (int64_t(1) << 19));
  // the blocks of the points-based Phi^T F (they depend on c too)
  int* hq = hp + (n + 1);
  hq[0] = 0;
  for (int k = 0; k < n; ++k)
    hq[k + 1] = hq[k] + (pts && !use_tcf ? fieldpts_blocks(b->fpts_h[k], calls[k].c, cg) : 0);
  const int fpts_blocks = hq[n];
  const int* d_fpts_prefix = d_apply_prefix + (n + 1);
  int* hr = hq + (n + 1);  // and of their sums over the chunks
  hr[0] = 0;
  for (int k = 0; k < n; ++k) hr[k + 1] = hr[k] + (pts ? fieldpts_reduce_blocks(b->fpts_h[k], calls[k].c) : 0);
  const int fred_blocks = hr[n];
  const int* d_fred_prefix = d_fpts_prefix + (n + 1);
  int* hz = hr + (n + 1);  // and of the tensor-core apply's Z images
  hz[0] = 0;
  for (int k = 0; k < n; ++k) hz[k + 1] = hz[k] + (use_tc ? apply_prep_blocks(b->apply_tc_h[k], calls[k].c) : 0);
  const int prep_blocks = hz[n];
  const int* d_prep_prefix = d_fred_prefix + (n + 1);
  if (b->compact && mode != kModeIntegrate)
    return fail(RFD_EINVAL, "a compact plan has no feature matrix: only integration runs on it");
  BCK(cudaMemcpyAsync(b->d_calls, stage, b->stage_bytes, cudaMemcpyHostToDevice, st));
  BCK(cudaEventRecord(b->stage_done[slot], st));
  const bool with_feat = mode != kModeIntegrate, with_phi = with_feat && !gram_only;
  const bool with_apply = mode != kModeFeatures;
  const bool graph = (b->options & kBatchGraphs) && (!with_phi || b->phi_batched);

  const bool pipelined = with_feat && pipelines(b);
  // F's rows of Psi: one point per thread up to 8 channels, else 8 points x 32 channels per warp
  const bool wide_fill = max_c > 8;
  auto fill = [&](cudaStream_t s) -> cudaError_t {
    return wide_fill ? launch_fill_wide_batched(b->d_fill, b->d_fillw_prefix, n, b->fillw_blocks, b->d_calls, s)
                     : launch_fill_batched(b->d_fill, b->d_fill_prefix, n, b->fill_blocks, b->d_calls, s);
  };
  auto reductions = [&](cudaStream_t s, Timing* t) -> rfd_status {
    if (pts) {  // Phi^T F from the points, summed over the chunks by the reduce kernel
      const FieldPtsJob* fj = use_tcf ? b->d_fpts_tc : b->d_fpts;
      {
        StepScope sc(t, s, RFD_STEP_FIELD);
        if (use_tcf)
          BCK(launch_fieldpts_tc(fj, b->d_item_prefix, n, b->fpts_items, std::min(b->fpts_items, b->sms), b->d_calls,
                                 b->d_err, s));
        else
          BCK(launch_fieldpts_batched(fj, d_fpts_prefix, n, fpts_blocks, cg, b->d_calls, s));
      }
      StepScope sc(t, s, RFD_STEP_REDUCE);
      BCK(launch_fieldpts_reduce(fj, d_fred_prefix, n, fred_blocks, b->d_calls, s));
      return RFD_OK;
    }
    if (pipelined) {
      if (rfd_status q = pipelined_features(b, s, t); q != RFD_OK) return q;
      if (with_apply) {
        StepScope sc(t, s, RFD_STEP_FIELD);
        BCK(fill(s));
      }
      if (rfd_status q = pipelined_gram(b, mode, s, t); q != RFD_OK) return q;
      StepScope sc(t, s, RFD_STEP_REDUCE);
      BCK(launch_reduce_batched(b->d_red[mode], b->n_red[mode], b->d_calls, s));
      return RFD_OK;
    }
    if (with_feat) {
      StepScope sc(t, s, RFD_STEP_FEATURES);
      BCK(launch_features_batched(b->d_feat, b->d_feat_prefix, n, b->feat_blocks, b->d_calls, s));
    }
    if (with_apply) {
      StepScope sc(t, s, RFD_STEP_FIELD);
      BCK(fill(s));
    }
    {
      StepScope sc(t, s, RFD_STEP_GRAM);
      BCK(gram_all(b, mode, s));
    }
    StepScope sc(t, s, RFD_STEP_REDUCE);
    BCK(launch_reduce_batched(b->d_red[mode], b->n_red[mode], b->d_calls, s));
    return RFD_OK;
  };
  auto small_apply = [&](cudaStream_t s, Timing* t) -> rfd_status {
    {
      StepScope sc(t, s, RFD_STEP_SMALL);
      if (max_c > 16)
        BCK(launch_small_wide_batched(b->d_apply, b->d_wide_prefix, n, b->wide_blocks, b->d_calls, s));
      else
        BCK(launch_small_batched(b->d_apply, b->d_small_prefix, n, b->small_rows, b->d_calls, s));
    }
    if (use_tc) {
      {
        StepScope sc(t, s, RFD_STEP_SMALL);
        BCK(launch_apply_prep(b->d_apply_tc, d_prep_prefix, n, prep_blocks, b->d_calls, s));
      }
      StepScope sc(t, s, RFD_STEP_APPLY);
      BCK(launch_apply_tc(b->d_apply_tc, b->d_tile_prefix, n, b->apply_tiles, std::min(b->apply_tiles, b->sms),
                          b->d_calls, b->d_err, s));
      return RFD_OK;
    }
    StepScope sc(t, s, RFD_STEP_APPLY);
    BCK(launch_apply_batched(b->d_apply, d_apply_prefix, n, apply_blocks, cg, b->d_calls, s));
    return RFD_OK;
  };
  // the apply's part of the graph keys: the SIMT kernel's channel group and grid, or the
  // tensor-core form's Z-image grid (its own grid is fixed per batch)
  // (a tensor-core apply: 100, + 1 with the wide fill, + 2 with the wide form of step a5;
  // the SIMT apply's channel group implies both: 16 and 32 above 8 channels, 32 above 16)
  const int akey_cg = use_tc ? 100 + (wide_fill ? 1 : 0) + (max_c > 16 ? 2 : 0) : cg;
  const int akey_blocks = use_tc ? -1 - prep_blocks : apply_blocks;

  if (gram_only) {  // steps a2-a3: M only, and G no longer matches the points
    for (rfd_plan_s* pl : b->plans) pl->have_G = false;
    const int key[4] = {mode, -3, 0, 0};
    return run_segment(b, key, graph, tm, reductions);
  }
  if (!with_phi) {
    // the points-based path: both of its launches' grids (they depend on every call's c)
    const int key[4] = {mode, pts ? (use_tcf ? -(1 << 24) - b->fpts_items : -4 - fpts_blocks) : -1,
                        pts ? akey_cg + 64 * fred_blocks : akey_cg, akey_blocks};
    return run_segment(b, key, graph, tm, [&](cudaStream_t s, Timing* t) -> rfd_status {
      rfd_status r = reductions(s, t);
      return r == RFD_OK ? small_apply(s, t) : r;
    });
  }
  for (rfd_plan_s* pl : b->plans) pl->have_G = false;
  if (!b->phi_batched) {
    rfd_status r = reductions(st, tm);
    if (r != RFD_OK) return r;
    {
      StepScope sc(tm, st, RFD_STEP_PHI1);
      r = phi1_per_plan(b);
    }
    if (r != RFD_OK) return r;
    for (rfd_plan_s* pl : b->plans) pl->have_G = true;
    return with_apply ? small_apply(st, tm) : RFD_OK;
  }
  // reductions, then the first part of a4; the host learns the largest s_c
  const int key_pre[4] = {mode, -2, with_apply && wide_fill ? 1 : 0, 0};
  rfd_status r = run_segment(b, key_pre, graph, tm, [&](cudaStream_t s, Timing* t) -> rfd_status {
    rfd_status q = reductions(s, t);
    if (q != RFD_OK) return q;
    StepScope sc(t, s, RFD_STEP_PHI1);
    return phi1_select(b, s);
  });
  if (r != RFD_OK) return r;
  BCK(cudaEventRecord(b->ev_mid, st));
  BCK(cudaEventSynchronize(b->ev_mid));
  const int max_s = std::min(std::max(b->h_sv[n], 0), kMaxSquarings);
  for (int k = 0; k < n; ++k) {
    rfd_plan_s* pl = b->plans[k];
    const int s = b->h_sv[k];
    pl->stats.norm1 = b->h_norms[k];
    pl->stats.pade_degree = kTaylorDegree;  // the Taylor degree on this path
    pl->stats.squarings = s;
    pl->stats.phi1_emulated = 1;
    pl->stats.phi1_gemms = 6 + 2 * s;
  }
  int hn[4];
  product_moduli(b, hn);
  const int key_post[4] = {mode, max_s + 64 * ((hn[0] - 1) | (hn[1] - 1) << 4 | (hn[2] - 1) << 8 | (hn[3] - 1) << 12),
                           with_apply ? akey_cg : 0, with_apply ? akey_blocks : 0};
  r = run_segment(b, key_post, graph, tm, [&](cudaStream_t s, Timing* t) -> rfd_status {
    {
      StepScope sc(t, s, RFD_STEP_PHI1);
      rfd_status q = phi1_core(b, s, max_s, hn);
      if (q != RFD_OK) return q;
    }
    return with_apply ? small_apply(s, t) : RFD_OK;
  });
  if (r != RFD_OK) return r;
  for (rfd_plan_s* pl : b->plans) pl->have_G = true;
  return RFD_OK;
}

// Step a4 alone on the plans' resident M (the batched, emulated path): what
// batch_run does between the reductions and step a5, without CUDA graphs.
rfd_status batch_phi1_only(BatchImpl* b) {
  if (!b->phi_batched) return fail(RFD_EINVAL, "the batched step a4 is not in use for this batch");
  cudaStream_t st = b->st;
  const int n = b->count;
  for (rfd_plan_s* pl : b->plans) pl->have_G = false;
  rfd_status r = phi1_select(b, st);
  if (r != RFD_OK) return r;
  BCK(cudaEventRecord(b->ev_mid, st));
  BCK(cudaEventSynchronize(b->ev_mid));
  const int max_s = std::min(std::max(b->h_sv[n], 0), kMaxSquarings);
  for (int k = 0; k < n; ++k) {
    rfd_plan_s* pl = b->plans[k];
    pl->stats.norm1 = b->h_norms[k];
    pl->stats.pade_degree = kTaylorDegree;
    pl->stats.squarings = b->h_sv[k];
    pl->stats.phi1_emulated = 1;
    pl->stats.phi1_gemms = 6 + 2 * b->h_sv[k];
  }
  int hn[4];
  product_moduli(b, hn);
  r = phi1_core(b, st, max_s, hn);
  if (r != RFD_OK) return r;
  for (rfd_plan_s* pl : b->plans) pl->have_G = true;
  return RFD_OK;
}

// ---- Timing ------------------------------------------------------------------
cudaError_t Timing::init() {
  on = true;
  ring.resize(kRing);
  for (auto& s : ring)
    for (cudaEvent_t& e : s.ev) e = nullptr;
  for (auto& s : ring)
    for (cudaEvent_t& e : s.ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
    }
  return cudaSuccess;
}
void Timing::destroy() {
  for (auto& s : ring)
    for (cudaEvent_t e : s.ev)
      if (e) cudaEventDestroy(e);
  ring.clear();
}
void Timing::fold(cudaStream_t st) {
  if (!on || pending == 0) return;
  cudaStreamSynchronize(st);
  for (int k = pending; k > 0; --k) {
    auto& s = ring[(head - k + kRing) % kRing];
    for (int i = 0; i < RFD_NUM_STEPS; ++i) {
      if (!s.used[i]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s.ev[2 * i], s.ev[2 * i + 1]) == cudaSuccess) sum[i] += ms;
    }
    ++calls;
  }
  pending = 0;
}
void Timing::begin_call(cudaStream_t st) {
  mark = t_kernel_launches;
  if (!on) return;
  if (pending == kRing) fold(st);
  cur = &ring[head];
  for (bool& u : cur->used) u = false;
}
void Timing::end_call() {
  launches += t_kernel_launches - mark;
  if (!on) return;
  cur = nullptr;
  head = (head + 1) % kRing;
  ++pending;
}
void Timing::reset(cudaStream_t st) {
  fold(st);
  for (double& v : sum) v = 0.0;
  calls = 0;
  launches = 0;
}

void batch_set_phase(BatchImpl* b, int phase_blocks) { b->phase_blocks = phase_blocks; }

void batch_set_profile(BatchImpl* b, unsigned long long* prof) { b->prof = prof; }

bool batch_set_overlap(BatchImpl* b, bool overlap) {
  b->overlap = overlap;
  return can_overlap(b);
}

rfd_status batch_time_gram(BatchImpl* b, int mode, int reps, float* ms, const CloudCall* calls) {
  // the call table of this batch: the features beside the Gram read the callers' points
  {
    const int slot = b->stage_next;
    b->stage_next = (slot + 1) % BatchImpl::kStageRing;
    BCK(cudaEventSynchronize(b->stage_done[slot]));
    std::memcpy(b->h_stage[slot], calls, (size_t)b->count * sizeof(CloudCall));
    BCK(cudaMemcpyAsync(b->d_calls, b->h_stage[slot], (size_t)b->count * sizeof(CloudCall), cudaMemcpyHostToDevice,
                        b->st));
    BCK(cudaEventRecord(b->stage_done[slot], b->st));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  // modes with features time them with the Gram, so that the serial schedule and the features
  // beside the Gram compare (there the phase length trades the first phase's exposed features
  // against the launches of more phases)
  const bool feat = mode != kModeIntegrate, pipe = feat && pipelines(b);
  auto launch = [&]() -> cudaError_t {
    if (!pipe) {
      if (feat) {
        cudaError_t f =
            launch_features_batched(b->d_feat, b->d_feat_prefix, b->count, b->feat_blocks, b->d_calls, b->st);
        if (f != cudaSuccess) return f;
      }
      return gram_all(b, mode, b->st);
    }
    if (pipelined_features(b, b->st, nullptr) != RFD_OK || pipelined_gram(b, mode, b->st, nullptr) != RFD_OK)
      return cudaErrorLaunchFailure;
    return cudaSuccess;
  };
  cudaError_t e = launch();  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, b->st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1, b->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail2("Gram timing", e);
  *ms = t / (float)reps;
  return RFD_OK;
}

int* batch_error_word(BatchImpl* b) { return b->d_err; }

bool batch_set_apply_tc(BatchImpl* b, int mode) {
  b->apply_tc_mode = mode;
  return b->apply_tc_ok;
}

rfd_status batch_check_error(BatchImpl* b, int* bad) {
  const int n = b->count;
  BCK(cudaMemcpyAsync(b->h_flags, b->d_flags, (size_t)(n + 1) * sizeof(int), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  const int err = b->h_flags[n];
  std::string clouds;
  for (int k = 0; k < n; ++k) {
    if (bad) bad[k] = b->h_flags[k] ? 1 : 0;
    if (!b->h_flags[k]) continue;
    b->plans[k]->stats.nonfinite = 1;
    b->plans[k]->have_G = false;
    clouds += (clouds.empty() ? "" : ",") + std::to_string(k);
  }
  if (err || !clouds.empty()) BCK(cudaMemsetAsync(b->d_flags, 0, (size_t)(n + 1) * sizeof(int), b->st));
  if (err) return fail(RFD_ETIMEDOUT, "a device-side wait ran out (code " + std::to_string(err) + ")");
  if (!clouds.empty())
    return fail(RFD_ENUMERIC, "G = lambda phi1(lambda M) is not finite for cloud(s) " + clouds +
                                  (n == 1 ? "" : " of the batch"));
  return RFD_OK;
}

}  // namespace rfd
