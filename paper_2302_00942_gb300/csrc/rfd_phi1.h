// Step a4 entry point: G = lambda phi1(lambda M), FP64, on the device.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include "../../include/rfd.h"

namespace rfd {

struct Phi1Info {
  double norm1;   // ||lambda M||_1
  int degree;     // Pade degree q
  int squarings;  // s
  int nonfinite;
  int emulated;   // 1: the m x m x m products ran on the Ozaki-split tensor-core GEMM
  int gemms;      // m x m x m products evaluated
  int lu;         // 1: the Pade denominator was solved by LU (native path)
  int solve_factors;  // emulated path: factors (I + R^(2^j)) of the denominator solve
};

// FP64 doubles of workspace needed for an m x m problem.
size_t phi1_workspace_doubles(int m);

// Number of m x m x m GEMMs of the evaluation for degree q and s squarings
// (besides them: one LU factorisation and a solve with m, or 2m when s > 0,
// right-hand sides).
int phi1_gemm_count(int q, int s);

// d_M, d_G: m x m row-major FP64 device buffers.  work: phi1_workspace_doubles(m)
// doubles; d_ipiv: m ints; d_info, d_flag, d_err: one int each (d_err: error
// word of bounded device waits); d_scalar: one double.  emulated: use the
// Ozaki-split tensor-core GEMM for the m x m x m products (FP64-accurate),
// else native FP64.  Synchronises `st` (norm -> host; finiteness flag -> host).
rfd_status phi1_fp64(int m, double lambda, const double* d_M, double* d_G, double* work, int* d_ipiv, int* d_info,
                     double* d_scalar, int* d_flag, int* d_err, bool emulated, cudaStream_t st, Phi1Info* info);

}  // namespace rfd
