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
// with that device current, and caches it.  Because every call uses the same
// memory, calls whose device work overlaps (different streams, or different
// host threads) race; serialise them on one stream.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
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
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_phi1_scratch on the current device (set up once per device).
rfd_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RFD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(RFD_ENOTSUP, "device index beyond the supported range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_phi1_scratch);
    if (e != cudaSuccess || !p)
      return fail(RFD_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
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
  const size_t mm = (size_t)m * m;
  const size_t work_bytes = phi1_workspace_doubles(m) * sizeof(double);
  const size_t need = work_bytes + 256 + (size_t)m * sizeof(int) + 16 * sizeof(int) + 4 * sizeof(double);
  if (need > kNoAllocScratchBytes) return fail(RFD_EINVAL, "rfd_phi1_noalloc: scratch too small for this m");
  (void)mm;
  void* base = nullptr;
  rfd_status s = scratch_for_current_device(&base);
  if (s != RFD_OK) return s;
  // carve: [work | ipiv | ints | scalar]
  uint8_t* p = static_cast<uint8_t*>(base);
  double* work = reinterpret_cast<double*>(p);
  uint8_t* q = p + ((work_bytes + 255) & ~size_t(255));
  int* ipiv = reinterpret_cast<int*>(q);
  q += ((size_t)m * sizeof(int) + 255) & ~size_t(255);
  int* ints = reinterpret_cast<int*>(q);  // [0] error word, [1] LU info, [2] finite flag
  q += 256;
  double* scalar = reinterpret_cast<double*>(q);
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
