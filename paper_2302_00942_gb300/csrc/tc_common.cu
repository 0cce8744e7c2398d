// Host-side helpers shared by the tcgen05 kernels: tensor-map encoding through
// the CUDA driver API entry point (no link-time dependency on libcuda) and the
// device check; and the probe of the kernels' bounded-wait unwind path.
#include "tc_common.cuh"
#include "kernels.h"

namespace rfd {
namespace tc {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {  // once per process (thread-safe initialisation)
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
  return fn;
}

bool make_map_bf16(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t row_stride,
                   uint32_t box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {row_stride * 2};
  const cuuint32_t box[2] = {64u, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_map_bf16_blocked(CUtensorMap* map, const void* base, uint64_t rows, uint64_t rows_alloc, uint64_t nblocks,
                           uint32_t box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {64, rows, nblocks};
  const cuuint64_t strides[2] = {64 * 2, rows_alloc * 64 * 2};
  const cuuint32_t box[3] = {64u, box_rows, 1u};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_map_bf16_3d(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint64_t planes,
                      uint32_t box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {cols, rows, planes};
  const cuuint64_t strides[2] = {cols * 2, rows * cols * 2};
  const cuuint32_t box[3] = {64u, box_rows, 1u};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool sm103_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

}  // namespace tc

namespace {

constexpr int kWaitProbeCode = 21;

// The unwind path of the tcgen05 kernels on its own: warp 1 allocates TMEM as
// the Gram and residue-GEMM kernels do, thread 0 waits on an mbarrier that no
// thread and no copy ever arrives on, with the caller's limit; when the wait
// runs out it records kWaitProbeCode in *err (unless an earlier code is
// there), and the CTA frees its TMEM and returns.  No TMA copy is issued, so
// there is nothing in flight to drain.
__global__ void __launch_bounds__(64, 1) wait_probe_kernel(unsigned long long limit_ns, int* err) {
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tc::smem_u32(&tmem_base), 32);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (threadIdx.x == 0) tc::mbar_wait(tc::smem_u32(&bar), 0u, err, kWaitProbeCode, limit_ns);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem_base, 32);
}

}  // namespace

cudaError_t launch_wait_probe(unsigned long long limit_ns, int* err, cudaStream_t st) {
  wait_probe_kernel<<<1, 64, 0, st>>>(limit_ns, err);
  return launched();
}

}  // namespace rfd
