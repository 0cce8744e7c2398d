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

/* Make the k-th device allocation performed by the library from now on fail
 * (k = 0: the next one), as if cudaMalloc had returned out-of-memory; the
 * failing entry point returns RFD_ENOMEM and releases what it had allocated.
 * k < 0 disables the hook.  Process-wide, not thread-safe; tests only. */
RFD_API void rfd_debug_fail_alloc_after(int32_t k);

#ifdef __cplusplus
}
#endif

#endif /* RFD_TESTING_H_ */
