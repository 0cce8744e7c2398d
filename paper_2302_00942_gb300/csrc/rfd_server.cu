// Serving loop for GFI requests (Sec. 2.4 graph field integration, one
// request = one point cloud and one field F): rfd_server_create / rfd_submit /
// rfd_poll / rfd_server_destroy.
//
// Memory: the whole budget is allocated once and carved by a host-side
// first-fit allocator, so admitting, evicting and finishing requests never
// calls cudaMalloc / cudaFree.  Plans (features Phi, G, partials, phi1
// workspace) come from the plan pool; batch tables from a small table pool;
// pinned staging from a pinned pool.
//
// Scheduling: `executors` threads, each with its own non-blocking stream.  A
// free executor takes every queued request it can admit (arrival order; a
// request waits while its resident cloud is busy in another batch or while
// memory is short after evicting idle resident clouds), up to max_batch,
// builds one batch of the new clouds (steps a2-a6) and one of the reused
// clouds (steps a3(Y)-a6), runs them, and waits for them on its stream.  The
// other executors keep admitting and launching meanwhile, so batches of
// requests that arrived while others run overlap on the device.
//
// Residency: a cloud kept for later requests (keep = 1) is compacted after its
// first pass to its points, frequencies, M and G (plan_compact: the feature
// matrix, partials and phi1 workspace go back to the pool), so the budget holds
// ~50x more resident clouds; a request on it recomputes the features from the
// points (FP32) for B^T F and the apply.  A cloud's id is the ticket of the
// request that keeps it, so a request may name a cloud whose keeping request
// has not finished yet: it waits in the queue behind it.
#include <cuda_runtime.h>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>
#include "kernels.h"
#include "rfd_internal.h"
#include "rfd_plan.h"

using namespace rfd;
using Clock = std::chrono::steady_clock;

namespace {

constexpr size_t kGran = 256;

// First-fit allocator over one block, coalescing on free.  Thread-safe.
class Pool {
 public:
  void init(void* base, size_t bytes) {
    base_ = static_cast<unsigned char*>(base);
    cap_ = bytes / kGran * kGran;
    free_.clear();
    if (cap_) free_[0] = cap_;
  }
  void* alloc(size_t bytes) {
    bytes = std::max<size_t>(kGran, (bytes + kGran - 1) / kGran * kGran);
    std::lock_guard<std::mutex> g(mu_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, left = it->second - bytes;
      free_.erase(it);
      if (left) free_[off + bytes] = left;
      live_[off] = bytes;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return base_ + off;
    }
    return nullptr;
  }
  void release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(mu_);
    const size_t off = static_cast<size_t>(static_cast<unsigned char*>(p) - base_);
    auto lv = live_.find(off);
    if (lv == live_.end()) return;
    size_t size = lv->second;
    live_.erase(lv);
    used_ -= size;
    auto next = free_.find(off + size);  // merge with the following free block
    if (next != free_.end()) {
      size += next->second;
      free_.erase(next);
    }
    auto it = free_.lower_bound(off);  // and with the preceding one
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == off) {
        prev->second += size;
        return;
      }
    }
    free_[off] = size;
  }
  size_t capacity() const { return cap_; }
  size_t used() {
    std::lock_guard<std::mutex> g(mu_);
    return used_;
  }
  size_t peak() {
    std::lock_guard<std::mutex> g(mu_);
    return peak_;
  }

 private:
  std::mutex mu_;
  unsigned char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;             // offset -> bytes
  std::unordered_map<size_t, size_t> live_;   // offset -> bytes
};

// Device memory from one pool, pinned memory from another.
struct PoolMem final : MemSource {
  Pool* dpool = nullptr;
  Pool* hpool = nullptr;
  void* dev(size_t bytes) override { return dpool->alloc(bytes); }
  void dev_free(void* p) override { dpool->release(p); }
  void* pinned(size_t bytes) override { return hpool->alloc(bytes); }
  void pinned_free(void* p) override { hpool->release(p); }
};

struct Cloud {
  uint64_t id = 0;
  rfd_plan_s* plan = nullptr;
  bool busy = false;
};

struct Req {
  rfd_request r{};
  rfd_plan_s* plan = nullptr;  // new cloud: prepared at submit, materialised at admission
  Cloud* cloud = nullptr;      // reused resident cloud
  bool done = false;
  rfd_result res{};
  Clock::time_point t_submit, t_start;
};

rfd_params request_params(const rfd_request& r) {
  rfd_params p{};
  p.n = r.n;
  p.m = r.m;
  p.max_channels = std::max(r.c, r.keep ? r.max_channels : 0);
  p.eps = r.eps;
  p.lambda = r.lambda;
  p.seed = r.seed;
  p.precision = RFD_BF16_TC;
  return p;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct rfd_server_s {
  rfd_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::unordered_map<uint64_t, std::unique_ptr<Cloud>> clouds;
  std::list<uint64_t> lru;  // idle resident clouds, least recently used first
  uint64_t next_ticket = 1;
  int64_t outstanding = 0;
  bool stop = false, paused = false;
  rfd_server_stats st{};
  void* dbase = nullptr;
  void* tbase = nullptr;
  void* hbase = nullptr;
  Pool plans, tables, pinned;
  PoolMem plan_mem, table_mem;
  std::vector<std::thread> threads;
  std::vector<cudaStream_t> streams;
};

namespace {

void finish(rfd_server_s* s, Req& q, rfd_status status, Clock::time_point t_done, int batch) {
  q.res.status = status;
  q.res.latency_ms = ms_between(q.t_submit, t_done);
  q.res.queue_ms = ms_between(q.t_submit, q.t_start == Clock::time_point{} ? t_done : q.t_start);
  q.res.batch_size = batch;
  q.done = true;
  --s->outstanding;
  ++s->st.completed;
}

// Evicts idle resident clouds (least recently used first) until `bytes` can be
// allocated from the plan pool; returns the allocation or nullptr.  Lock held.
void* reserve(rfd_server_s* s, size_t bytes) {
  void* p = s->plans.alloc(bytes);
  while (!p && !s->lru.empty()) {
    const uint64_t id = s->lru.front();
    s->lru.pop_front();
    auto it = s->clouds.find(id);
    if (it != s->clouds.end()) {
      plan_destroy(it->second->plan);
      s->clouds.erase(it);
      ++s->st.evicted;
    }
    p = s->plans.alloc(bytes);
  }
  return p;
}

// Runs one group (all new clouds, or all reused clouds) as batches on `stream`;
// statuses[k] receives each request's outcome.  Splits the group when its
// tables do not fit the table pool.
void run_group(rfd_server_s* s, std::vector<Req*>& group, int mode, cudaStream_t stream, rfd_status* statuses) {
  if (group.empty()) return;
  std::vector<rfd_plan_s*> plans;
  std::vector<CloudCall> calls;
  for (Req* q : group) {
    rfd_plan_s* pl = q->cloud ? q->cloud->plan : q->plan;
    plans.push_back(pl);
    calls.push_back(CloudCall{q->r.d_points, q->r.d_F, q->r.d_out, q->r.ldF, q->r.ldOut, q->r.c, 0});
  }
  BatchImpl* b = nullptr;
  rfd_status bs = batch_build(plans.data(), (int)plans.size(), stream, &s->table_mem, 0, GramTuning{}, &b);
  if (bs == RFD_ENOMEM && group.size() > 1) {
    const size_t h = group.size() / 2;
    std::vector<Req*> a(group.begin(), group.begin() + h), c(group.begin() + h, group.end());
    run_group(s, a, mode, stream, statuses);
    run_group(s, c, mode, stream, statuses + h);
    return;
  }
  if (bs != RFD_OK) {
    for (size_t k = 0; k < group.size(); ++k) statuses[k] = bs;
    return;
  }
  rfd_status rs = batch_run(b, mode, calls.data(), nullptr);
  std::vector<int> bad(group.size(), 0);
  rfd_status cs = batch_check_error(b, bad.data());  // waits for the batch
  for (size_t k = 0; k < group.size(); ++k) {
    if (rs != RFD_OK)
      statuses[k] = rs;
    else if (cs == RFD_ETIMEDOUT)
      statuses[k] = cs;
    else
      statuses[k] = bad[k] ? RFD_ENUMERIC : RFD_OK;
  }
  batch_free(b);
}

// A request with keep = 1 that has not finished: its ticket names the cloud it will
// leave resident, so requests that reuse that cloud wait behind it.  Lock held.
bool root_pending(rfd_server_s* s, uint64_t ticket) {
  auto it = s->reqs.find(ticket);
  return it != s->reqs.end() && it->second.r.keep && !it->second.done;
}

void executor(rfd_server_s* s, int idx) {
  cudaSetDevice(s->device);
  cudaStream_t stream = s->streams[idx];
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_work.wait(lk, [&] { return s->stop || (!s->paused && !s->queue.empty()); });
    if (s->stop) break;
    // ---- admission: arrival order, up to max_batch
    std::vector<Req*> fresh, reuse;
    std::vector<uint64_t> fresh_t, reuse_t;
    const Clock::time_point now = Clock::now();
    bool mem_blocked = false;
    bool finished_here = false;  // requests refused during admission: their pollers are woken below
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)(fresh.size() + reuse.size()) < s->cfg.max_batch;) {
      const uint64_t t = *it;
      Req& q = s->reqs[t];
      if (q.r.cloud && !q.plan && !s->clouds.count(q.r.cloud) && root_pending(s, q.r.cloud)) {
        ++it;  // its cloud is still being made by the request that keeps it
        continue;
      }
      if (q.r.cloud && !q.plan) {
        auto c = s->clouds.find(q.r.cloud);
        if (c == s->clouds.end()) {  // evicted since rfd_submit: rebuild it from the points, if given
          rfd_status ps = RFD_EINVAL;
          if (q.r.d_points) ps = plan_prepare(request_params(q.r), nullptr, &q.plan);
          if (ps != RFD_OK) {
            q.t_start = now;
            finish(s, q, ps, now, 0);
            finished_here = true;
            it = s->queue.erase(it);
            continue;
          }
        }
      }
      if (q.r.cloud && !q.plan) {
        auto c = s->clouds.find(q.r.cloud);
        Cloud* cl = c->second.get();
        if (cl->busy) {  // in another batch: stays queued
          ++it;
          continue;
        }
        if (!cl->plan->have_G || q.r.c > cl->plan->p.max_channels || (q.r.n && q.r.n != cl->plan->n)) {
          q.t_start = now;
          finish(s, q, cl->plan->have_G ? RFD_EINVAL : RFD_ENUMERIC, now, 0);
          finished_here = true;
          it = s->queue.erase(it);
          continue;
        }
        cl->busy = true;
        s->lru.remove(cl->id);
        q.cloud = cl;
        reuse.push_back(&q);
        reuse_t.push_back(t);
        it = s->queue.erase(it);
        continue;
      }
      if (mem_blocked) {  // new clouds wait behind the first one that did not fit
        ++it;
        continue;
      }
      void* chunk = reserve(s, plan_device_bytes(q.plan));
      if (!chunk) {
        mem_blocked = true;
        ++it;
        continue;
      }
      q.plan->chunk = chunk;
      q.plan->mem = &s->plan_mem;
      fresh.push_back(&q);
      fresh_t.push_back(t);
      it = s->queue.erase(it);
    }
    if (finished_here) s->cv_done.notify_all();
    if (fresh.empty() && reuse.empty()) {
      // everything queued waits for memory or a busy cloud: sleep until something finishes
      s->cv_work.wait(lk);
      continue;
    }
    for (Req* q : fresh) q->t_start = now;
    for (Req* q : reuse) q->t_start = now;
    ++s->st.batches;
    lk.unlock();
    // ---- run (no lock held)
    const long long l0 = t_kernel_launches;
    std::vector<rfd_status> fs(fresh.size(), RFD_OK), rs(reuse.size(), RFD_OK);
    std::vector<Req*> ready;
    std::vector<size_t> ready_idx;
    for (size_t k = 0; k < fresh.size(); ++k) {
      rfd_plan_s* pl = fresh[k]->plan;
      pl->stream = stream;
      const rfd_status m = plan_materialize(pl, &s->plan_mem, false, false);
      if (m != RFD_OK) {  // plan_materialize destroyed the plan (and released its chunk)
        fresh[k]->plan = nullptr;
        fs[k] = m;
        continue;
      }
      ready.push_back(fresh[k]);
      ready_idx.push_back(k);
    }
    std::vector<rfd_status> rstat(ready.size(), RFD_OK);
    run_group(s, ready, kModeGfi, stream, rstat.data());
    for (size_t i = 0; i < ready.size(); ++i) fs[ready_idx[i]] = rstat[i];
    run_group(s, reuse, kModeIntegrate, stream, rs.data());
    const Clock::time_point t_done = Clock::now();
    // clouds that stay resident keep only their compact form (points, frequencies, M, G):
    // later requests on them recompute the features from the points
    for (size_t k = 0; k < fresh.size(); ++k)
      if (fresh[k]->plan && fs[k] == RFD_OK && fresh[k]->r.keep) plan_compact(fresh[k]->plan, false);
    const long long launches = t_kernel_launches - l0;
    lk.lock();
    s->st.kernel_launches += launches;
    const int bsz = (int)(fresh.size() + reuse.size());
    for (size_t k = 0; k < fresh.size(); ++k) {
      Req& q = *fresh[k];
      if (q.plan && fs[k] == RFD_OK && q.r.keep) {
        auto cl = std::make_unique<Cloud>();
        cl->id = fresh_t[k];  // the ticket of the request that keeps it
        cl->plan = q.plan;
        q.res.cloud = cl->id;
        s->lru.push_back(cl->id);
        s->clouds[cl->id] = std::move(cl);
      } else if (q.plan) {
        plan_destroy(q.plan);
      }
      q.plan = nullptr;
      finish(s, q, fs[k], t_done, bsz);
    }
    for (size_t k = 0; k < reuse.size(); ++k) {
      Req& q = *reuse[k];
      q.cloud->busy = false;
      s->lru.push_back(q.cloud->id);
      q.res.cloud = q.cloud->id;
      q.res.reused = 1;
      ++s->st.reused;
      finish(s, q, rs[k], t_done, bsz);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

rfd_status rfd_server_create(size_t mem_budget, const rfd_server_config* cfg, rfd_server_t* out) {
  if (!out) return fail(RFD_EINVAL, "null output pointer");
  *out = nullptr;
  rfd_server_config c = cfg ? *cfg : rfd_server_config{};
  if (!cfg) c.mem_budget = mem_budget;
  if (c.mem_budget == 0) c.mem_budget = mem_budget;
  if (c.max_queue <= 0) c.max_queue = 4096;
  if (c.max_batch <= 0) c.max_batch = 256;
  if (c.executors <= 0) c.executors = 2;
  if (c.executors > 8) return fail(RFD_EINVAL, "executors must be <= 8");
  const size_t table_bytes = (size_t)c.executors * (32u << 20), pinned_bytes = (size_t)c.executors * (32u << 20);
  if (c.mem_budget < table_bytes + (64u << 20))
    return fail(RFD_EINVAL, "mem_budget must be at least " + std::to_string((table_bytes + (64u << 20)) >> 20) + " MiB");
  auto s = std::make_unique<rfd_server_s>();
  s->cfg = c;
  if (cudaGetDevice(&s->device) != cudaSuccess) return fail(RFD_ECUDA, "no CUDA device");
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, s->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, s->device);
  if (!(major == 10 && minor == 3)) return fail(RFD_ENOTSUP, "the server runs the BF16 tensor-core form: sm_103 only");
  auto cleanup = [&](rfd_status st, const std::string& msg) {
    for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
    if (s->dbase) cudaFree(s->dbase);
    if (s->hbase) cudaFreeHost(s->hbase);
    cudaGetLastError();
    return fail(st, msg);
  };
  if (cudaMalloc(&s->dbase, c.mem_budget) != cudaSuccess)
    return cleanup(RFD_ENOMEM, "device allocation of the " + std::to_string(c.mem_budget) + "-byte budget failed");
  if (cudaMallocHost(&s->hbase, pinned_bytes) != cudaSuccess) return cleanup(RFD_ENOMEM, "pinned allocation failed");
  s->tbase = static_cast<unsigned char*>(s->dbase) + (c.mem_budget - table_bytes) / kGran * kGran;
  s->plans.init(s->dbase, static_cast<unsigned char*>(s->tbase) - static_cast<unsigned char*>(s->dbase));
  s->tables.init(s->tbase, table_bytes);
  s->pinned.init(s->hbase, pinned_bytes);
  s->plan_mem.dpool = &s->plans;
  s->plan_mem.hpool = &s->pinned;
  s->table_mem.dpool = &s->tables;
  s->table_mem.hpool = &s->pinned;
  s->st.mem_budget = (int64_t)c.mem_budget;
  for (int i = 0; i < c.executors; ++i) {
    cudaStream_t x = nullptr;
    if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(RFD_ECUDA, "stream creation failed");
    s->streams.push_back(x);
  }
  rfd_server_s* raw = s.get();
  for (int i = 0; i < c.executors; ++i) raw->threads.emplace_back(executor, raw, i);
  *out = s.release();
  return RFD_OK;
}

rfd_status rfd_server_destroy(rfd_server_t s) {
  if (!s) return RFD_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  for (cudaStream_t x : s->streams) cudaStreamSynchronize(x);
  for (auto& kv : s->reqs)
    if (kv.second.plan) plan_destroy(kv.second.plan);  // queued, never materialised
  for (auto& kv : s->clouds) plan_destroy(kv.second->plan);
  for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
  cudaFree(s->dbase);
  cudaFreeHost(s->hbase);
  delete s;
  return RFD_OK;
}

rfd_status rfd_submit(rfd_server_t s, const rfd_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return fail(RFD_EINVAL, "null server, request or ticket pointer");
  const rfd_request& r = *req;
  if (r.c < 1 || r.c > 256) return fail(RFD_EINVAL, "c must be in [1, 256]");
  if (!r.d_F || !r.d_out) return fail(RFD_EINVAL, "null field or output pointer");
  if (r.ldF < r.c || r.ldOut < r.c) return fail(RFD_EINVAL, "leading dimensions must be >= c");
  if (r.d_F == r.d_out && r.ldF != r.ldOut) return fail(RFD_EINVAL, "in-place integration needs ldOut == ldF");
  if (r.keep && r.max_channels && r.max_channels < r.c) return fail(RFD_EINVAL, "max_channels must be >= c");
  bool resident = false;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->outstanding >= s->cfg.max_queue) {
      ++s->st.rejected;
      return fail(RFD_EBUSY, "admission refused: " + std::to_string(s->outstanding) + " requests outstanding");
    }
    resident = r.cloud && (s->clouds.count(r.cloud) || root_pending(s, r.cloud));
  }
  rfd_plan_s* pl = nullptr;
  if (!resident) {
    if (r.cloud && !r.d_points) return fail(RFD_EINVAL, "cloud " + std::to_string(r.cloud) + " is not resident and no points were given");
    if (!r.d_points) return fail(RFD_EINVAL, "null points");
    rfd_status ps = plan_prepare(request_params(r), nullptr, &pl);
    if (ps != RFD_OK) return ps;
    const size_t need = plan_device_bytes(pl);
    if (need > s->plans.capacity()) {
      plan_destroy(pl);
      std::lock_guard<std::mutex> g(s->mu);
      ++s->st.rejected;
      return fail(RFD_EBUSY, "admission refused: the request needs " + std::to_string(need) +
                                 " device bytes, more than the budget");
    }
  }
  std::lock_guard<std::mutex> g(s->mu);
  const uint64_t t = s->next_ticket++;
  Req& q = s->reqs[t];
  q.r = r;
  q.plan = pl;
  q.t_submit = Clock::now();
  s->queue.push_back(t);
  ++s->outstanding;
  ++s->st.submitted;
  *ticket = t;
  s->cv_work.notify_one();
  return RFD_OK;
}

rfd_status rfd_poll(rfd_server_t s, uint64_t ticket, int32_t timeout_us, rfd_result* out) {
  if (!s || !out) return fail(RFD_EINVAL, "null server or result pointer");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(RFD_EINVAL, "unknown or retired ticket " + std::to_string(ticket));
  Req* q = &it->second;
  if (!q->done) {
    if (timeout_us <= 0) return RFD_ENOTREADY;
    if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return q->done; }))
      return fail(RFD_ETIMEDOUT, "ticket " + std::to_string(ticket) + " not done after " +
                                     std::to_string(timeout_us) + " us");
  }
  *out = q->res;
  s->reqs.erase(ticket);
  return RFD_OK;
}

rfd_status rfd_server_stats_get(rfd_server_t s, rfd_server_stats* out) {
  if (!s || !out) return fail(RFD_EINVAL, "null server or output");
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->st;
  out->resident = (int64_t)s->clouds.size();
  out->mem_used = (int64_t)(s->plans.used() + s->tables.used());
  out->mem_peak = (int64_t)(s->plans.peak() + s->tables.peak());
  return RFD_OK;
}

// Test hook: while paused, executors start no new batch (running ones finish).
void rfd_debug_server_pause(rfd_server_t s, int32_t paused) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->paused = paused != 0;
  }
  s->cv_work.notify_all();
}

}  // extern "C"
