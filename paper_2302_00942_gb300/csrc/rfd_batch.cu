// Batched execution of the BF16 tensor-core path: one launch per step serves
// every cloud of a batch (Sec. 2.4 steps a2..a6 for many point clouds of uneven
// N and m); a single cloud runs as a batch of one.
//
// Step a4 runs on the FP64-accurate tensor-core GEMM for all clouds at once:
// diagonal Pade of degree 5 on the block-triangular augmented matrix, the
// denominator solved by the product (I + R)(I + R^2)...(I + R^16) (||R|| <
// 0.14 for ||X||_1 <= theta_5, see rfd_phi1.cu), and per-cloud squarings s_c
// (clouds with s_c <= k skip squaring step k).  The only host synchronisation
// of a batched call is the one that brings the clouds' ||lambda M||_1 to the
// host to choose s_c (and one for the finiteness flags).
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

constexpr double kTheta5 = 2.539398330063230e-1;  // Higham (2005), Table 2.3, degree 5
constexpr int kSolveFactors = 5;                  // (0.135)^(2^5) / (1 - 0.135) < 2^-56
// matrix slots of the phi1 evaluation (see kernels.h: slot k = work + k m^2)
enum : int { sX = 0, sX2, sX4, sSp, sVp, sUp, sR, sR2, sF, sFb, sE, sT1, sT2 };

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v, std::vector<void*>& owned) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  owned.push_back(p);
  *dst = static_cast<T*>(p);
  return cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

std::vector<int> prefix_of(const std::vector<int>& counts) {
  std::vector<int> p(counts.size() + 1, 0);
  for (size_t i = 0; i < counts.size(); ++i) p[i + 1] = p[i] + counts[i];
  return p;
}

}  // namespace

struct BatchImpl {
  std::vector<rfd_plan_s*> plans;
  int count = 0;
  cudaStream_t st = nullptr;
  std::vector<void*> owned;  // device allocations
  void* d_maps = nullptr;
  TcUnit* d_units[3] = {};
  int n_units[3] = {};
  RedTile* d_red[3] = {};
  int n_red[3] = {};
  FeatJob* d_feat = nullptr;
  int* d_feat_prefix = nullptr;
  int feat_blocks = 0;
  FillJob* d_fill = nullptr;
  int* d_fill_prefix = nullptr;
  int fill_blocks = 0;
  ApplyJob* d_apply = nullptr;
  std::vector<ApplyJob> h_apply;
  int* d_small_prefix = nullptr;
  int small_rows = 0;
  PhiCloud* d_phi = nullptr;
  std::vector<PhiCloud> h_phi;
  int* d_elem_prefix = nullptr;
  int elem_blocks = 0;
  int* d_rowa_prefix = nullptr;
  int rows_a = 0;
  int* d_rowb_prefix = nullptr;
  int rows_b = 0;
  int* d_t_prefix = nullptr;
  int t_blocks = 0;
  OzTile* d_oz = nullptr;
  int n_oz = 0;
  int max_m = 0, max_cpad = 16;
  bool phi_batched = true;  // all clouds on the emulated path (m <= 1024, no native flag)
  // per call
  CloudCall* d_calls = nullptr;
  int* d_apply_prefix = nullptr;
  static constexpr int kStageRing = 4;  // pinned per-call staging buffers, reused round-robin
  unsigned char* h_stage_ring[kStageRing] = {};
  cudaEvent_t stage_done[kStageRing] = {};
  int stage_next = 0;
  PhiCloud* h_phi_stage = nullptr;   // pinned copy of h_phi for the async upload
  double* d_norms = nullptr;
  double* h_norms = nullptr;         // pinned
  int* d_flags = nullptr;
  int* h_flags = nullptr;            // pinned
  int* d_err = nullptr;
};

cudaStream_t batch_stream(BatchImpl* b) { return b->st; }

void batch_free(BatchImpl* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  for (void* p : b->owned) cudaFree(p);
  for (int i = 0; i < BatchImpl::kStageRing; ++i) {
    if (b->h_stage_ring[i]) cudaFreeHost(b->h_stage_ring[i]);
    if (b->stage_done[i]) cudaEventDestroy(b->stage_done[i]);
  }
  if (b->h_phi_stage) cudaFreeHost(b->h_phi_stage);
  if (b->h_norms) cudaFreeHost(b->h_norms);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  delete b;
}

rfd_status batch_build(rfd_plan_s* const* plans, int count, cudaStream_t st, BatchImpl** out) {
  *out = nullptr;
  auto* b = new (std::nothrow) BatchImpl();
  if (!b) return fail(RFD_ENOMEM, "host allocation failed");
  b->plans.assign(plans, plans + count);
  b->count = count;
  b->st = st;
  auto bail = [&](rfd_status s, const std::string& msg) {
    batch_free(b);
    return fail(s, msg);
  };
  int sms = plans[0]->sms;
  // --- Gram lanes: each cloud's lanes share the batch's CTAs in proportion to its work
  double work = 0.0;
  for (int k = 0; k < count; ++k)
    work += (double)plans[k]->desc.units[kModeGfi].size() * (double)(plans[k]->n_pad / kTcBK);
  const double target = (count == 1) ? 1e300 : std::max(1.0, work / (4.0 * sms));  // k-blocks per CTA
  std::vector<TcUnit> units[3];
  std::vector<RedTile> red[3];
  std::vector<unsigned char> maps((size_t)count * kMapsPerCloud * kTensorMapBytes);
  std::vector<FeatJob> feat;
  std::vector<FillJob> fill;
  std::vector<int> feat_n, fill_n, small_n, elem_n, rowa_n, rowb_n, t_n;
  std::vector<OzTile> oz;
  for (int k = 0; k < count; ++k) {
    rfd_plan_s* pl = plans[k];
    const PlanDesc& d = pl->desc;
    b->max_m = std::max(b->max_m, pl->m);
    b->max_cpad = std::max(b->max_cpad, pl->cpad);
    if (pl->m > 1024 || (pl->p.flags & RFD_FLAG_NATIVE_FP64)) b->phi_batched = false;
    std::memcpy(maps.data() + (size_t)k * kMapsPerCloud * kTensorMapBytes, d.maps, sizeof(d.maps));
    const int64_t kb = pl->n_pad / kTcBK;
    for (int mode = 0; mode < 3; ++mode) {
      // the plan's own units use nlanes = L_plan; the batch may use fewer lanes
      const std::vector<TcUnit>& pu = d.units[mode];
      if (pu.empty()) continue;
      const int L_plan = pu[0].nlanes;
      const int T = (int)pu.size() / L_plan;
      int L = L_plan;
      if (count > 1) L = (int)std::max<int64_t>(1, std::min<int64_t>(L_plan, (int64_t)std::ceil(kb / target)));
      for (int t = 0; t < T; ++t)
        for (int l = 0; l < L; ++l) {
          TcUnit u = pu[(size_t)t * L_plan];
          u.lane = l;
          u.nlanes = L;
          u.map += k * kMapsPerCloud;
          u.out = pl->d_part + (int64_t)(t * L + l) * pl->slot_elems;
          units[mode].push_back(u);
        }
      for (RedTile r : d.red[mode]) {
        // red tiles of the plan are per compute tile t (stored in .count as t): remap to lanes
        const int t = r.count;
        r.part = pl->d_part + (int64_t)t * L * pl->slot_elems;
        r.count = L;
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
    fill_n.push_back(fl.bx * ((fl.cpad + 31) / 32));
    ApplyJob aj = d.apply;
    aj.cloud = k;
    b->h_apply.push_back(aj);
    small_n.push_back(pl->m);
    PhiCloud pc = d.phi;
    pc.map_a += k * kMapsPerCloud;
    pc.map_b += k * kMapsPerCloud;
    b->h_phi.push_back(pc);
    elem_n.push_back((int)(((int64_t)pl->m * pl->m + 255) / 256));
    rowa_n.push_back(pc.mpa);
    rowb_n.push_back(pc.mpb);
    t_n.push_back(((pl->m + 31) / 32) * ((pl->m + 31) / 32));
    for (OzTile o : d.oz) {
      o.cloud = k;
      oz.push_back(o);
    }
  }
  cudaError_t e = cudaSuccess;
  {
    void* p = nullptr;
    if ((e = cudaMalloc(&p, maps.size())) != cudaSuccess) return bail(RFD_ENOMEM, "batch tables");
    b->owned.push_back(p);
    b->d_maps = p;
    if ((e = cudaMemcpy(p, maps.data(), maps.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(RFD_ECUDA, "batch tables");
  }
  auto up_prefix = [&](int** d, const std::vector<int>& n, int* total) {
    std::vector<int> pre = prefix_of(n);
    *total = pre.back();
    return upload(d, pre, b->owned);
  };
  for (int mode = 0; mode < 3 && e == cudaSuccess; ++mode) {
    b->n_units[mode] = (int)units[mode].size();
    b->n_red[mode] = (int)red[mode].size();
    if ((e = upload(&b->d_units[mode], units[mode], b->owned)) != cudaSuccess) break;
    e = upload(&b->d_red[mode], red[mode], b->owned);
  }
  if (e == cudaSuccess) e = upload(&b->d_feat, feat, b->owned);
  if (e == cudaSuccess) e = up_prefix(&b->d_feat_prefix, feat_n, &b->feat_blocks);
  if (e == cudaSuccess) e = upload(&b->d_fill, fill, b->owned);
  if (e == cudaSuccess) e = up_prefix(&b->d_fill_prefix, fill_n, &b->fill_blocks);
  if (e == cudaSuccess) e = upload(&b->d_apply, b->h_apply, b->owned);
  if (e == cudaSuccess) e = up_prefix(&b->d_small_prefix, small_n, &b->small_rows);
  if (e == cudaSuccess) e = up_prefix(&b->d_elem_prefix, elem_n, &b->elem_blocks);
  if (e == cudaSuccess) e = up_prefix(&b->d_rowa_prefix, rowa_n, &b->rows_a);
  if (e == cudaSuccess) e = up_prefix(&b->d_rowb_prefix, rowb_n, &b->rows_b);
  if (e == cudaSuccess) e = up_prefix(&b->d_t_prefix, t_n, &b->t_blocks);
  if (e == cudaSuccess) e = upload(&b->d_oz, oz, b->owned);
  b->n_oz = (int)oz.size();
  // per-call buffers
  auto dev = [&](void** p, size_t bytes) {
    cudaError_t r = cudaMalloc(p, bytes);
    if (r == cudaSuccess) b->owned.push_back(*p);
    return r;
  };
  void* p = nullptr;
  if (e == cudaSuccess && (e = dev(&p, (size_t)count * sizeof(CloudCall) + (size_t)(count + 1) * sizeof(int))) == cudaSuccess) {
    b->d_calls = static_cast<CloudCall*>(p);
    b->d_apply_prefix = reinterpret_cast<int*>(static_cast<unsigned char*>(p) + (size_t)count * sizeof(CloudCall));
  }
  if (e == cudaSuccess && (e = dev(&p, (size_t)count * sizeof(PhiCloud))) == cudaSuccess) b->d_phi = static_cast<PhiCloud*>(p);
  if (e == cudaSuccess && (e = dev(&p, (size_t)count * sizeof(double))) == cudaSuccess) b->d_norms = static_cast<double*>(p);
  if (e == cudaSuccess && (e = dev(&p, (size_t)count * sizeof(int) + 256)) == cudaSuccess) {
    b->d_flags = static_cast<int*>(p);
    b->d_err = reinterpret_cast<int*>(static_cast<unsigned char*>(p) + (((size_t)count * sizeof(int) + 127) & ~size_t(127)));
  }
  for (int i = 0; i < BatchImpl::kStageRing && e == cudaSuccess; ++i) {
    e = cudaMallocHost(&b->h_stage_ring[i], (size_t)count * sizeof(CloudCall) + (size_t)(count + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->stage_done[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_phi_stage, (size_t)count * sizeof(PhiCloud));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_norms, (size_t)count * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_flags, (size_t)count * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(e == cudaErrorMemoryAllocation ? RFD_ENOMEM : RFD_ECUDA,
                std::string("batch set-up: ") + cudaGetErrorString(e));
  }
  for (int k = 0; k < count; ++k) b->h_phi[k].flag = b->d_flags + k;
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

// Step a4 for every cloud of the batch (emulated FP64 on the tensor cores).
rfd_status phi1_batched(BatchImpl* b) {
  cudaStream_t st = b->st;
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
  int gemms = 0;
  auto gemm = [&](int a, int bb, int c, double alpha, double beta, int mask) {
    ++gemms;
    return launch_bgemm(b->d_phi, n, b->d_rowa_prefix, b->rows_a, b->d_rowb_prefix, b->rows_b, b->d_t_prefix,
                        b->t_blocks, b->d_oz, b->n_oz, b->d_maps, a, bb, c, alpha, beta, mask, b->d_err, st);
  };
  // the per-call fields of the cloud descriptors are not known yet: upload with s = 0
  for (int k = 0; k < n; ++k) {
    b->h_phi[k].s = 0;
    b->h_phi[k].scale = 1.0;
  }
  std::memcpy(b->h_phi_stage, b->h_phi.data(), (size_t)n * sizeof(PhiCloud));
  BCK(cudaMemcpyAsync(b->d_phi, b->h_phi_stage, (size_t)n * sizeof(PhiCloud), cudaMemcpyHostToDevice, st));
  BCK(comb(sX, {kSlotM}, {1.0}, 0.0, 1, -1));  // X = lambda M
  BCK(launch_bnorm1(b->d_phi, n, b->max_m, sX, b->d_norms, st));
  BCK(cudaMemcpyAsync(b->h_norms, b->d_norms, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  int max_s = 0;
  std::string bad;
  for (int k = 0; k < n; ++k) {
    const double nrm = b->h_norms[k];
    rfd_plan_s* pl = b->plans[k];
    pl->stats.norm1 = nrm;
    pl->stats.nonfinite = 0;
    if (!std::isfinite(nrm)) {
      pl->stats.nonfinite = 1;
      bad += (bad.empty() ? "" : ",") + std::to_string(k);
      continue;
    }
    int s = 0;
    if (nrm > kTheta5) s = (int)std::ceil(std::log2(nrm / kTheta5));
    if (s > 1000) {
      pl->stats.nonfinite = 1;
      bad += (bad.empty() ? "" : ",") + std::to_string(k);
      continue;
    }
    b->h_phi[k].s = s;
    b->h_phi[k].scale = std::ldexp(1.0, -s);
    max_s = std::max(max_s, s);
    pl->stats.pade_degree = 5;
    pl->stats.squarings = s;
    pl->stats.phi1_emulated = 1;
  }
  if (!bad.empty()) return fail(RFD_ENUMERIC, "||lambda M||_1 is not finite for cloud(s) " + bad);
  std::memcpy(b->h_phi_stage, b->h_phi.data(), (size_t)n * sizeof(PhiCloud));
  BCK(cudaMemcpyAsync(b->d_phi, b->h_phi_stage, (size_t)n * sizeof(PhiCloud), cudaMemcpyHostToDevice, st));
  // diagonal Pade, degree 5: b_k = (10-k)! 5! / (10! k! (5-k)!) with b_0 = 1
  double pb[6];
  pb[0] = 1.0;
  for (int k = 0; k < 5; ++k) pb[k + 1] = pb[k] * double(5 - k) / (double(10 - k) * double(k + 1));
  if (max_s > 0) BCK(comb(sX, {sX}, {1.0}, 0.0, 2, -1));  // X = 2^-s X
  BCK(gemm(sX, sX, sX2, 1.0, 0.0, -1));
  BCK(gemm(sX2, sX2, sX4, 1.0, 0.0, -1));
  BCK(comb(sSp, {sX4, sX2}, {pb[5], pb[3]}, pb[1], 0, -1));
  BCK(comb(sVp, {sX4, sX2}, {pb[4], pb[2]}, pb[0], 0, -1));
  BCK(gemm(sX, sSp, sUp, 1.0, 0.0, -1));
  BCK(comb(sR, {sVp, sUp}, {-1.0, 1.0}, 1.0, 0, -1));  // R = I - (Vp - Up)
  BCK(comb(sF, {sSp}, {2.0}, 0.0, 0, -1));             // F = 2 Sp
  int F = sF, Fb = sFb, R = sR, R2 = sR2;
  for (int j = 0; j < kSolveFactors; ++j) {
    BCK(comb(Fb, {F}, {1.0}, 0.0, 0, -1));
    BCK(gemm(R, F, Fb, 1.0, 1.0, -1));  // F <- F + R^(2^j) F
    std::swap(F, Fb);
    if (j + 1 < kSolveFactors) {
      BCK(gemm(R, R, R2, 1.0, 0.0, -1));
      std::swap(R, R2);
    }
  }
  if (max_s > 0) {
    BCK(comb(sE, {}, {}, 1.0, 0, -1));
    BCK(gemm(sX, F, sE, 1.0, 1.0, -1));  // E = I + X F
    for (int k = 0; k < max_s; ++k) {
      BCK(gemm(sE, F, sT1, 1.0, 0.0, k));
      BCK(comb(F, {F, sT1}, {0.5, 0.5}, 0.0, 0, k));  // F <- (F + E F) / 2
      if (k + 1 < max_s) {
        BCK(gemm(sE, sE, sT2, 1.0, 0.0, k + 1));
        BCK(comb(sE, {sT2}, {1.0}, 0.0, 0, k + 1));
      }
    }
  }
  BCK(comb(kSlotG, {F}, {1.0}, 0.0, 1, -1));  // G = lambda F
  BCK(cudaMemsetAsync(b->d_flags, 0, (size_t)n * sizeof(int), st));
  BCK(launch_bfinite(b->d_phi, b->d_elem_prefix, n, b->elem_blocks, kSlotG, st));
  BCK(cudaMemcpyAsync(b->h_flags, b->d_flags, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, st));
  int err = 0;
  BCK(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  if (err) {
    cudaMemsetAsync(b->d_err, 0, sizeof(int), st);
    return fail(RFD_ETIMEDOUT, "a device-side wait ran out in the batched phi1 (code " + std::to_string(err) + ")");
  }
  for (int k = 0; k < n; ++k) {
    rfd_plan_s* pl = b->plans[k];
    const int s = b->h_phi[k].s;
    pl->stats.phi1_gemms = 3 + 2 * kSolveFactors - 1 + (s > 0 ? 2 * s : 0);
    if (b->h_flags[k]) {
      pl->stats.nonfinite = 1;
      bad += (bad.empty() ? "" : ",") + std::to_string(k);
    }
  }
  (void)gemms;
  if (!bad.empty()) return fail(RFD_ENUMERIC, "G = lambda phi1(lambda M) is not finite for cloud(s) " + bad);
  return RFD_OK;
}

// Step a4 one cloud at a time (native FP64, or clouds beyond the emulated path's m <= 1024).
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

}  // namespace

rfd_status batch_run(BatchImpl* b, int mode, const CloudCall* calls, Timing* tm) {
  cudaStream_t st = b->st;
  const int n = b->count;
  // per-call tables: the callers' buffers, and the apply blocks (they depend on c)
  int max_c = 1;
  for (int k = 0; k < n; ++k) max_c = std::max(max_c, calls[k].c);
  const int cg = max_c <= 4 ? 4 : (max_c <= 8 ? 8 : (max_c <= 16 ? 16 : 32));
  // a pinned staging buffer whose previous upload has been consumed
  const int slot = b->stage_next;
  b->stage_next = (slot + 1) % BatchImpl::kStageRing;
  BCK(cudaEventSynchronize(b->stage_done[slot]));
  unsigned char* stage = b->h_stage_ring[slot];
  auto* hc = reinterpret_cast<CloudCall*>(stage);
  auto* hp = reinterpret_cast<int*>(stage + (size_t)n * sizeof(CloudCall));
  hp[0] = 0;
  for (int k = 0; k < n; ++k) {
    hc[k] = calls[k];
    const int nb = (mode == kModeFeatures) ? 0 : b->h_apply[k].bx * ((calls[k].c + cg - 1) / cg);
    hp[k + 1] = hp[k] + nb;
  }
  const int apply_blocks = hp[n];
  BCK(cudaMemcpyAsync(b->d_calls, stage, (size_t)n * sizeof(CloudCall) + (size_t)(n + 1) * sizeof(int),
                      cudaMemcpyHostToDevice, st));
  BCK(cudaEventRecord(b->stage_done[slot], st));
  if (mode != kModeIntegrate) {
    StepScope t(tm, st, RFD_STEP_FEATURES);
    BCK(launch_features_batched(b->d_feat, b->d_feat_prefix, n, b->feat_blocks, b->d_calls, st));
  }
  if (mode != kModeFeatures) {
    StepScope t(tm, st, RFD_STEP_FIELD);
    BCK(launch_fill_batched(b->d_fill, b->d_fill_prefix, n, b->fill_blocks, b->d_calls, st));
  }
  {
    StepScope t(tm, st, RFD_STEP_GRAM);
    BCK(launch_gram_tc(b->d_maps, b->d_units[mode], b->n_units[mode], b->max_cpad, b->d_err, st));
  }
  {
    StepScope t(tm, st, RFD_STEP_REDUCE);
    BCK(launch_reduce_batched(b->d_red[mode], b->n_red[mode], b->d_calls, st));
  }
  if (mode != kModeIntegrate) {
    for (rfd_plan_s* pl : b->plans) pl->have_G = false;
    rfd_status s;
    {
      StepScope t(tm, st, RFD_STEP_PHI1);
      s = b->phi_batched ? phi1_batched(b) : phi1_per_plan(b);
    }
    if (s != RFD_OK) return s;
    for (rfd_plan_s* pl : b->plans) pl->have_G = true;
  }
  if (mode != kModeFeatures) {
    {
      StepScope t(tm, st, RFD_STEP_SMALL);
      BCK(launch_small_batched(b->d_apply, b->d_small_prefix, n, b->small_rows, b->d_calls, st));
    }
    StepScope t(tm, st, RFD_STEP_APPLY);
    BCK(launch_apply_batched(b->d_apply, b->d_apply_prefix, n, apply_blocks, cg, b->d_calls, st));
  }
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

rfd_status batch_check_error(BatchImpl* b) {
  int err = 0;
  BCK(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  if (err) {
    cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st);
    return fail(RFD_ETIMEDOUT, "a device-side wait ran out (code " + std::to_string(err) + ")");
  }
  return RFD_OK;
}

}  // namespace rfd
