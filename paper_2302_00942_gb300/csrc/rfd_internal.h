// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cstddef>
#include <string>
#include "../../include/rfd.h"
#include "../../include/rfd_testing.h"

namespace rfd {

// thread-local last-error message (rfd_last_error)
void set_error(const std::string& msg);
rfd_status fail(rfd_status st, const std::string& msg);

// Step a1 on the host (Sec. 2.4): frequencies from the truncated Gaussian and
// weights r = tau/p for the threshold function `kernel` (rfd_kernel).
// Returns RFD_OK or RFD_EINVAL.
rfd_status sample_frequencies_host(int m, double eps, uint64_t seed, double sigma,
                                   double radius, int kernel, double* omega, double* r);
double default_sigma(double eps);
double default_radius(double eps);

}  // namespace rfd
