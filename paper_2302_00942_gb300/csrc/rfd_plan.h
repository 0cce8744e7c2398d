// Internal: the plan (one point cloud's integrator) and the batch (many plans
// run by shared launches), shared by rfd_api.cu and rfd_batch.cu.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include "kernels.h"
#include "rfd_internal.h"

namespace rfd {

constexpr int kRing = 64;
constexpr int kTensorMapBytes = 128;
// Gram A / B (64-row box) / F maps, Ozaki slice maps A / B, Gram B (16-row box), and the
// pair kernel's B (8-row box) and F (half-width box) maps
constexpr int kMapsPerCloud = 8;

// CUDA-event timing of the path's steps (RFD_FLAG_TIMING): a ring of per-call
// event sets, folded into per-step sums when the stream is synchronised.
struct Timing {
  struct Slot {
    cudaEvent_t ev[2 * RFD_NUM_STEPS];
    bool used[RFD_NUM_STEPS];
  };
  bool on = false;
  std::vector<Slot> ring;
  int head = 0, pending = 0;
  Slot* cur = nullptr;
  double sum[RFD_NUM_STEPS] = {};
  long long calls = 0;
  long long launches = 0;
  long long mark = 0;

  cudaError_t init();
  void destroy();
  void fold(cudaStream_t st);
  void begin_call(cudaStream_t st);
  void end_call();
  void reset(cudaStream_t st);
};

// Records CUDA events around one step on a stream (no-op when timing is off).
// A second scope of the same step in one call extends the first.
struct StepScope {
  Timing* t;
  cudaStream_t st;
  int step;
  StepScope(Timing* tt, cudaStream_t s, int k) : t(tt), st(s), step(k) {
    if (t && t->cur && !t->cur->used[step]) cudaEventRecord(t->cur->ev[2 * step], st);
  }
  ~StepScope() {
    if (t && t->cur) {
      cudaEventRecord(t->cur->ev[2 * step + 1], st);
      t->cur->used[step] = true;
    }
  }
};

// SIMT (FP32 plain form) work tables of one plan.
struct TileSet {
  std::vector<GramTile> tiles;
  std::vector<GramUnit> units;
  GramTile* d_tiles = nullptr;
  GramUnit* d_units = nullptr;
  int slots = 0;
  int n_narrow = 0;  // the last n_narrow units are field tiles of <= kSimtNarrow columns (narrow kernel)
};

enum Mode : int { kModeFeatures = 0, kModeIntegrate = 1, kModeGfi = 2 };
// batch_run only: steps a2 and a3 of kModeFeatures (M, no step a4)
constexpr int kModeGram = 3;

// Host copies of one BF16 plan's batched-path descriptors (absolute device
// pointers; tensor-map indices relative to the plan's own kMapsPerCloud maps,
// cloud index 0).  A batch concatenates them.
struct PlanDesc {
  std::vector<TcUnit> units[3];    // indexed by Mode
  std::vector<RedTile> red[3];
  // the 2-SM form of the Gram modes (features, gfi) for m >= 512: pair units and their
  // reduce tiles (partials final for the plan's own lanes; used by the plan's batch of one)
  std::vector<PairUnit> pair_units[3];
  std::vector<RedTile> pair_red[3];
  int pair_stage_bytes = 0;
  // a compact plan (rfd_plan_compact): Phi^T F from the points, into d_fpart
  FieldPtsJob fpts{};
  FeatJob feat{};
  FillJob fill{};
  ApplyJob apply{};
  ApplyTcJob apply_tc{};  // the tensor-core apply (w2pi / zimg null: the plan has none)
  PhiCloud phi{};
  unsigned char maps[kMapsPerCloud][kTensorMapBytes];
};

struct BatchImpl;  // rfd_batch.cu

// Where the device and pinned host memory of plans and batches comes from: the
// CUDA allocator (the default), or a server's pools, which hand out memory
// without cudaMalloc / cudaFree (both can synchronise the device).
struct MemSource {
  virtual ~MemSource() = default;
  virtual void* dev(size_t bytes) = 0;  // nullptr when out of memory
  virtual void dev_free(void* p) = 0;
  virtual void* pinned(size_t bytes) = 0;
  virtual void pinned_free(void* p) = 0;
};
MemSource* cuda_mem();  // cudaMalloc / cudaMallocHost, with the allocation-failure test hook

// Batch options
enum : int { kBatchGraphs = 1 };  // replay the batch's launches from CUDA graphs

// Launch parameters of the tensor-core reductions that the autotuner varies:
// the split-K lanes of a lone cloud (percent of SMs / tiles), the waves of CTAs
// a batch plans for, the phase length of the point axis, and (a lone cloud
// with m >= 512) the one-SM or the CTA-pair form of the Gram.
struct GramTuning {
  int lanes_pct = 100;
  int waves = 4;
  int phase_blocks = kGramPhaseBlocks;
  int pairs = 0;  // a lone cloud with m >= 512: the Gram modes on CTA pairs (k_gram_pair.cu)
  int overlap = 0;  // a lone cloud with several phases: its features phase by phase beside the Gram
};

}  // namespace rfd

struct rfd_plan_s {
  rfd_params p{};
  cudaStream_t stream = nullptr;
  int m = 0, h = 0, cpad = 0, sms = 0;
  int64_t n = 0, n_pad = 0;
  int rows_alloc = 0;
  bool bf16 = false;
  bool fsplit = false;  // F as hi + lo BF16 rows (BF16 form, 2 max_channels <= 256)
  std::vector<double> omega, r, oa, ob;
  float* d_omega_hi = nullptr;
  float* d_omega_lo = nullptr;
  double* d_oa = nullptr;
  double* d_ob = nullptr;
  float* d_xyz = nullptr;  // BF16 form: copy of the points, written by the features step
  void* d_psi = nullptr;
  float* d_part = nullptr;
  int part_slots = 0;
  int64_t slot_elems = 0;
  std::vector<float> omega_hi_h, omega_lo_h;  // FP32 split of omega (hi + lo)
  double* d_M = nullptr;
  double* d_Y = nullptr;
  double* d_G = nullptr;
  float* d_Z = nullptr;
  float4* d_w2pi = nullptr;    // BF16 form: the tensor-core apply's 2 pi w and Z images
  uint8_t* d_zimg = nullptr;
  double* d_work = nullptr;
  int* d_ipiv = nullptr;
  int* d_ints = nullptr;  // [0] error word, [1] LU info, [2] finite flag
  double* d_scalar = nullptr;
  rfd::TileSet gram_only, field_only, both;  // FP32 plain form
  rfd::PlanDesc desc;                         // BF16 tensor-core form
  rfd::BatchImpl* self = nullptr;             // the plan as a batch of one (BF16 form)
  bool have_G = false;
  // compact (rfd_plan_compact): Psi, the split-K partials and the phi1 workspace are released;
  // rfd_integrate recomputes the features from d_xyz (FieldPtsJob) into d_fpart
  bool compact = false;
  float* d_fpart = nullptr;
  rfd_stats stats{};
  std::vector<void*> allocs;       // temporary owners only (rfd_phi1, debug GEMM)
  rfd::MemSource* mem = nullptr;   // source of the plan's single device chunk
  rfd::GramTuning tune;            // tensor-core reduction launch parameters
  // per-block cost of each compute tile, measured by the autotuner ([form: one SM, CTA pairs][mode];
  // empty: the cost model), so that every tile's lanes sweep the point axis at one pace
  std::vector<double> tile_cost[2][3];
  double tune_form_ms[2] = {0.0, 0.0};  // the autotuner's best time of each form
  bool autotune = false, tuned = false;
  void* chunk = nullptr;
  size_t chunk_bytes = 0;
  rfd::Timing timing;
};

namespace rfd {

// Plans: validation and host set-up (no device memory), the size of the plan's
// device chunk, and the device half (chunk from `mem`, descriptors, uploads on
// the plan's stream; `self_batch` also builds the plan's batch of one).
rfd_status plan_prepare(const rfd_params& p, cudaStream_t st, rfd_plan_s** out);
size_t plan_device_bytes(rfd_plan_s* pl);
rfd_status plan_materialize(rfd_plan_s* pl, MemSource* mem, bool self_batch, bool sync_init);
// Shrinks a BF16 plan with G to its compact form (a new chunk from the plan's memory
// source, the old one released; synchronises the plan's stream).  On failure the plan
// is unchanged.  self_batch: rebuild the plan's batch of one for the compact form.
rfd_status plan_compact(rfd_plan_s* pl, bool self_batch);
size_t plan_compact_bytes(const rfd_plan_s* pl);
void plan_destroy(rfd_plan_s* pl);  // frees without synchronising (the caller has)

// Builds / frees the device tables of a batch over the given BF16 plans (one
// device and one pinned block from `mem`; uploads are asynchronous on `st`).
rfd_status batch_build(rfd_plan_s* const* plans, int count, cudaStream_t st, MemSource* mem, int options,
                       const GramTuning& tune, BatchImpl** out);
void batch_free(BatchImpl* b);  // the caller has synchronised the batch's stream
size_t batch_device_bytes(BatchImpl* b);
// Runs one batched call.  calls: one CloudCall per plan (pts / F / out as the
// mode needs).  Updates each plan's stats and have_G.  Non-finite G and
// device-side timeouts are reported by batch_check_error.
rfd_status batch_run(BatchImpl* b, int mode, const CloudCall* calls, Timing* timing);
// Step a4 alone (the batched emulated path) on the plans' resident M; synchronises.
rfd_status batch_phi1_only(BatchImpl* b);
cudaStream_t batch_stream(BatchImpl* b);
int* batch_error_word(BatchImpl* b);  // the sticky device word that batch_check_error reads
// Kernel eigenvalues (rfd_eigen.cu): argument checks, and the k smallest /
// largest eigenvalues of every plan's exp(lambda W_hat) from its resident M
// into d_out (count x k), asynchronous on st.
rfd_status check_eigen_args(rfd_plan_s* const* plans, int count, int k);
rfd_status batch_eigenvalues(rfd_plan_s* const* plans, int count, int k, int largest, float* d_out, cudaStream_t st,
                             Timing* tm);
// Synchronises the batch's stream and reads (and clears) its device error word
// and per-cloud finiteness flags: RFD_ETIMEDOUT if a bounded wait ran out,
// RFD_ENUMERIC if some cloud's G is not finite (bad[k] = 1 for those clouds when
// bad is given).
rfd_status batch_check_error(BatchImpl* b, int* bad = nullptr);
// The apply (step a6): 0 always on the SIMT kernel, 1 (the default) on the tensor cores where
// that form is the faster (by the calls' largest c and the clouds' m), 2 on the tensor cores
// wherever the calls' c fits; returns whether the batch has the tensor-core form.
bool batch_set_apply_tc(BatchImpl* b, int mode);
// Times the Gram launches of one batched call of `mode`, with the features in
// front of them (serially or beside them, as the batch is set) in modes that
// compute features, from the points of calls (one CloudCall per plan): mean ms
// over `reps` launches after one warm-up.
rfd_status batch_time_gram(BatchImpl* b, int mode, int reps, float* ms, const CloudCall* calls);
void batch_set_phase(BatchImpl* b, int phase_blocks);
// Features beside the Gram on or off; returns whether the batch can run that schedule at all
// (a lone cloud with several phases of a multiple of 8 blocks).
bool batch_set_overlap(BatchImpl* b, bool overlap);
// Gram launches record each CTA's start and end (%globaltimer) into prof (2 words per CTA;
// null: off).  The autotuner's measure of the tiles' pace.
void batch_set_profile(BatchImpl* b, unsigned long long* prof);

}  // namespace rfd
