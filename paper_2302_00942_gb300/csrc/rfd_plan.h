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
constexpr int kMapsPerCloud = 5;  // Gram A / B / F maps, Ozaki slice maps A / B

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
struct StepScope {
  Timing* t;
  cudaStream_t st;
  int step;
  StepScope(Timing* tt, cudaStream_t s, int k) : t(tt), st(s), step(k) {
    if (t && t->cur) cudaEventRecord(t->cur->ev[2 * step], st);
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
};

enum Mode : int { kModeFeatures = 0, kModeIntegrate = 1, kModeGfi = 2 };

// Host copies of one BF16 plan's batched-path descriptors (absolute device
// pointers; tensor-map indices relative to the plan's own kMapsPerCloud maps,
// cloud index 0).  A batch concatenates them.
struct PlanDesc {
  std::vector<TcUnit> units[3];    // indexed by Mode
  std::vector<RedTile> red[3];
  FeatJob feat{};
  FillJob fill{};
  ApplyJob apply{};
  PhiCloud phi{};
  std::vector<OzTile> oz;
  unsigned char maps[kMapsPerCloud][kTensorMapBytes];
};

struct BatchImpl;  // rfd_batch.cu

}  // namespace rfd

struct rfd_plan_s {
  rfd_params p{};
  cudaStream_t stream = nullptr;
  int m = 0, h = 0, cpad = 0, sms = 0;
  int64_t n = 0, n_pad = 0;
  int rows_alloc = 0;
  bool bf16 = false;
  std::vector<double> omega, r, oa, ob;
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
  int* d_ints = nullptr;  // [0] error word, [1] LU info, [2] finite flag
  double* d_scalar = nullptr;
  rfd::TileSet gram_only, field_only, both;  // FP32 plain form
  rfd::PlanDesc desc;                         // BF16 tensor-core form
  rfd::BatchImpl* self = nullptr;             // the plan as a batch of one (BF16 form)
  bool have_G = false;
  rfd_stats stats{};
  std::vector<void*> allocs;
  rfd::Timing timing;
};

namespace rfd {

// Builds / frees the device tables of a batch over the given BF16 plans.
rfd_status batch_build(rfd_plan_s* const* plans, int count, cudaStream_t st, BatchImpl** out);
void batch_free(BatchImpl* b);
// Runs one batched call.  calls: one CloudCall per plan (pts / F / out as the
// mode needs).  Updates each plan's stats and have_G.
rfd_status batch_run(BatchImpl* b, int mode, const CloudCall* calls, Timing* timing);
cudaStream_t batch_stream(BatchImpl* b);
// Reads (and clears) the batch's device error word: RFD_ETIMEDOUT if a bounded wait ran out.
rfd_status batch_check_error(BatchImpl* b);

}  // namespace rfd
