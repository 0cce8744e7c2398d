/*
 * rfd_testing.h -- host-side fault injection for the RFD library's tests.
 *
 * The paper has no counterpart: these hooks exist so that failure paths (a
 * device allocation that fails) can be exercised without faulting a GPU.
 */
#ifndef RFD_TESTING_H_
#define RFD_TESTING_H_

#include "rfd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Make the k-th device or pinned allocation performed by the library from
 * now on fail (k = 0: the next one), as if cudaMalloc had returned out-of-memory; the
 * failing entry point returns RFD_ENOMEM and releases what it had allocated.
 * k < 0 disables the hook.  Process-wide, not thread-safe; tests only. */
RFD_API void rfd_debug_fail_alloc_after(int32_t k);

/* The FP64 GEMM building block of step a4 on its own:
 * C = alpha A B + beta C for row-major float64 DEVICE buffers (A: M x K, lda;
 * B: K x N, ldb; C: M x N, ldc).  method 0: native FP64 kernel; method 1: the
 * FP64-accurate Ozaki-split emulation on the BF16 tensor cores (K <= 4096,
 * sm_103 only, else RFD_ENOTSUP).  Allocates its workspace, synchronises
 * `cuda_stream`, and returns RFD_ETIMEDOUT if a bounded device wait ran out. */
RFD_API rfd_status rfd_debug_dgemm(int32_t method, int32_t M, int32_t N, int32_t K, double alpha, const double* A,
                                   int32_t lda, const double* B, int32_t ldb, double beta, double* C, int32_t ldc,
                                   void* cuda_stream);

/* Step a4 of a BF16 plan alone, on a given m x m FP64 DEVICE matrix M (copied
 * into the plan's M): the batched emulated evaluation of G = lambda phi1(lambda M)
 * that rfd_features runs (Taylor degree 16 in Paterson-Stockmeyer form with
 * scaling and squaring), leaving G resident for rfd_plan_export.  Synchronises
 * the plan's stream; RFD_EINVAL for FP32 plans or plans on the native-FP64
 * path, RFD_ENUMERIC if G is not finite. */
RFD_API rfd_status rfd_debug_plan_phi1(rfd_plan_t plan, const double* d_M);

/* The form of the Gram reductions that plans created from now on start with
 * (process-wide): enable = 1 puts a BF16 plan with m >= 512 (m a multiple of
 * 16, at most 64 field channels) on CTA pairs (tcgen05.mma.cta_group::2, half
 * of B loaded by each SM of the pair); enable = 0 (the default) on the one-SM
 * kernel.  The autotuner (RFD_FLAG_AUTOTUNE) times both and may change it.
 * A test compares the two forms on the same inputs with it.  Not thread-safe
 * against concurrent plan creation; tests only. */
RFD_API void rfd_debug_gram_pairs(int32_t enable);

/* Set the point-axis phase length of a BF16 plan's tensor-core reductions:
 * the reductions run as one launch per phase of phase_blocks 64-point blocks,
 * each later phase adding to the split-K lanes' partials (step a3).  A short
 * phase makes a modest cloud take the multi-phase accumulation that the large
 * workload takes.  Plans without RFD_FLAG_GRAPH and RFD_FLAG_AUTOTUNE only
 * (RFD_EINVAL otherwise, for FP32 plans, or for phase_blocks < 1).  Host only. */
RFD_API rfd_status rfd_debug_plan_set_phase(rfd_plan_t plan, int32_t phase_blocks);

/* Run a BF16 plan's features phase by phase beside its Gram (enable = 1) or
 * before it (0): the schedule the autotuner may choose for a lone cloud whose
 * point axis takes several phases.  Takes effect with the plan's current phase
 * length (rfd_debug_plan_set_phase); RFD_EINVAL when that schedule cannot run
 * (one phase, or a phase length that is not a multiple of 8 blocks), for FP32
 * plans, or for plans with RFD_FLAG_GRAPH or RFD_FLAG_AUTOTUNE.  Host only. */
RFD_API rfd_status rfd_debug_plan_set_overlap(rfd_plan_t plan, int32_t enable);

/* Which form step a6 of a BF16 plan takes (Sec. 2.4, the apply of the low-rank
 * factors), and with it a compact plan's B^T F from the points.  enable = 0:
 * the FP32 SIMT kernels in every call.  1 (the default): the tensor-core forms
 * where they are the faster -- calls of 17..64 channels, or 9..16 channels when
 * m >= 512; for B^T F from the points, clouds of 2^19 points or more -- else
 * the SIMT kernels.  2: the tensor-core forms in every call of
 * c <= min(64, max_channels): Phi recomputed in FP32 and split into BF16 hi and
 * lo parts, out = F + Phi_hi Z_hi + Phi_hi Z_lo + Phi_lo Z_hi (and B^T F
 * likewise) with FP32 accumulation.  RFD_EINVAL for FP32 plans, plans with
 * RFD_FLAG_GRAPH or another value; RFD_ENOTSUP (enable = 2) off sm_103.
 * Host only. */
RFD_API rfd_status rfd_debug_plan_set_apply_tc(rfd_plan_t plan, int32_t enable);

/* The bounded device-side wait on its own.  Every wait of the library's
 * kernels on an mbarrier gives up after a %globaltimer limit, records a code
 * in a device error word, frees its TMEM and returns, and the host reports
 * RFD_ETIMEDOUT instead of hanging.  This hook launches, on the plan's stream,
 * one CTA that allocates TMEM and waits on an mbarrier that nothing ever
 * arrives on, with a limit of limit_us microseconds (1 .. 10^6), recording
 * into the plan's own error word: the next rfd_sync(plan) returns
 * RFD_ETIMEDOUT (and clears the word), and the plan stays usable.  No copy is
 * issued and nothing faults.  Asynchronous; RFD_ENOTSUP off sm_103. */
RFD_API rfd_status rfd_debug_plan_wait_timeout(rfd_plan_t plan, int32_t limit_us);

/* Hold (paused = 1) or release (0) a server's executors: while held they
 * start no new batch (batches already running finish), so a test can make a
 * poll wait run out deterministically. */
RFD_API void rfd_debug_server_pause(rfd_server_t server, int32_t paused);

#ifdef __cplusplus
}
#endif

#endif /* RFD_TESTING_H_ */
