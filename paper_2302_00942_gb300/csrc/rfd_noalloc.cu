// rfd_phi1_noalloc: step a4 (G = lambda phi1(lambda M)) for callers that must
// not allocate device memory -- e.g. a latency-critical loop in which a
// cudaMalloc/cudaFree (which can synchronise the whole device) is not allowed,
// or a host process whose device memory is handed out by another allocator.
//
// The workspace lives in one file-scope __device__ array of fixed size, shared
// by every call: it covers m <= kNoAllocMaxM and stays resident on every GPU
// that loads the library until the process exits.  Host code may not use the
// array's name as a device address (it is a host-side stand-in), so the first
// call on each device resolves the real address with cudaGetSymbolAddress,
// with that device current, and caches it together with the identity of the
// device's context: after a cudaDeviceReset the module is loaded again, maybe
// elsewhere, and the next call resolves the address anew.  Because every call
// uses the same memory, calls whose device work overlaps (different streams,
// or different host threads) race; serialise them on one stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include "kernels.h"
#include "rfd_internal.h"
#include "rfd_phi1.h"

namespace rfd {

namespace {

constexpr int kNoAllocMaxM = 128;
// phi1_workspace_doubles(128) doubles (FP64 Pade buffers + the tensor-core
// GEMM's residue buffers) plus pivots and a few status words, rounded up: 3.75 MiB.
constexpr size_t kNoAllocScratchBytes = (size_t)15 << 18;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_phi1_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
struct Resolved {
  unsigned long long ctx_id = 0;  // the context the address belongs to (0: none yet)
  void* ptr = nullptr;
};
Resolved g_scratch[kMaxDevices];

// The unique id of the current context (cuCtxGetId, through the runtime's driver entry points).
bool current_context_id(unsigned long long* id) {
  static const auto fns = [] {  // once per process (thread-safe initialisation)
    void* get = nullptr;
    void* gid = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &get, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      get = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &gid, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      gid = nullptr;
    return std::make_pair(reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(get), reinterpret_cast<PFN_cuCtxGetId_v12000>(gid));
  }();
  CUcontext ctx = nullptr;
  if (!fns.first || !fns.second || fns.first(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return fns.second(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_phi1_scratch on the current device: resolved on the first call on a
// device, and again whenever that device's context has changed (a cudaDeviceReset).
rfd_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RFD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(RFD_ENOTSUP, "device index beyond the supported range");
  e = cudaSetDevice(dev);  // makes the device's primary context current (no allocation)
  if (e != cudaSuccess) return fail(RFD_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  unsigned long long id = 0;
  if (!current_context_id(&id)) return fail(RFD_ECUDA, "no current CUDA context");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  Resolved& r = g_scratch[dev];
  if (!r.ptr || r.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_phi1_scratch);
    if (e != cudaSuccess || !p)
      return fail(RFD_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    r.ptr = p;
    r.ctx_id = id;
  }
  *out = r.ptr;
  return RFD_OK;
}

}  // namespace

}  // namespace rfd

using namespace rfd;

extern "C" rfd_status rfd_phi1_noalloc(int32_t m, double lambda, const double* d_M, double* d_G, int32_t flags,
                                       void* cuda_stream, rfd_stats* stats_out) {
  if (m < 1 || m > kNoAllocMaxM)
    return fail(RFD_EINVAL, "rfd_phi1_noalloc: m = " + std::to_string(m) + " is outside [1, " +
                                std::to_string(kNoAllocMaxM) + "] (the fixed scratch covers m <= " +
                                std::to_string(kNoAllocMaxM) + "; use rfd_phi1 for larger m)");
  if (!d_M || !d_G || d_M == d_G) return fail(RFD_EINVAL, "null or aliased M / G");
  if (!std::isfinite(lambda)) return fail(RFD_EINVAL, "lambda must be finite");
  if (flags & ~RFD_FLAG_NATIVE_FP64) return fail(RFD_EINVAL, "unknown bits in flags");
  // carve: [work | ipiv | ints (16 words) | scalar (2 doubles)], each part 256-byte aligned;
  // the size check uses the same offsets
  auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t off_ipiv = a256(phi1_workspace_doubles(m) * sizeof(double));
  const size_t off_ints = off_ipiv + a256((size_t)m * sizeof(int));
  const size_t off_scalar = off_ints + a256(16 * sizeof(int));
  const size_t end = off_scalar + 2 * sizeof(double);
  if (end > kNoAllocScratchBytes) return fail(RFD_EINVAL, "rfd_phi1_noalloc: scratch too small for this m");
  void* base = nullptr;
  rfd_status s = scratch_for_current_device(&base);
  if (s != RFD_OK) return s;
  uint8_t* p = static_cast<uint8_t*>(base);
  double* work = reinterpret_cast<double*>(p);
  int* ipiv = reinterpret_cast<int*>(p + off_ipiv);
  int* ints = reinterpret_cast<int*>(p + off_ints);  // [0] error word, [1] LU info, [2] finite flag
  double* scalar = reinterpret_cast<double*>(p + off_scalar);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the array keeps the previous call's contents: clear the status words
  cudaError_t e = cudaMemsetAsync(ints, 0, 16 * sizeof(int), st);
  if (e != cudaSuccess) return fail(RFD_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  Phi1Info info{};
  s = phi1_fp64(m, lambda, d_M, d_G, work, ipiv, ints + 1, scalar, ints + 2, ints, (flags & RFD_FLAG_NATIVE_FP64) == 0,
                st, &info);
  e = cudaStreamSynchronize(st);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, ints, sizeof(int), cudaMemcpyDeviceToHost);
  if (stats_out) {
    *stats_out = rfd_stats{};
    stats_out->norm1 = info.norm1;
    stats_out->pade_degree = info.degree;
    stats_out->squarings = info.squarings;
    stats_out->nonfinite = info.nonfinite;
    stats_out->phi1_emulated = info.emulated;
    stats_out->phi1_gemms = info.gemms;
  }
  if (e != cudaSuccess) return fail(RFD_ECUDA, std::string("rfd_phi1_noalloc: ") + cudaGetErrorString(e));
  if (s == RFD_ECUDA) return fail(s, std::string("phi1: ") + cudaGetErrorString(cudaGetLastError()));
  if (s == RFD_ENUMERIC) return fail(s, "G is not finite");
  if (s == RFD_OK && err) return fail(RFD_ETIMEDOUT, "a device-side wait ran out in phi1 (code " + std::to_string(err) + ")");
  return s;
}
