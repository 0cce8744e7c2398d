// Kernel launchers and work descriptors of the RFD GPU path.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace rfd {

// Kernels launched by this thread (every launcher adds its count); the plan
// reports the difference around its calls.
extern thread_local long long t_kernel_launches;
inline void count_launch(long long k = 1) { t_kernel_launches += k; }
inline cudaError_t launched(long long k = 1) {
  t_kernel_launches += k;
  return cudaGetLastError();
}

// One output tile of the reductions over N (step a3).  Rows i0.. of the
// feature matrix Psi form the M side (features f), rows j0.. the N side
// (features g, or field channels when kind == kTileField).
enum : int32_t { kTileGram = 0, kTileField = 1 };

struct GramTile {
  int32_t i0, j0;      // first Psi row on each side (j0 >= m for field tiles)
  int32_t ni, nj;      // valid rows on each side
  int32_t kind;        // kTileGram (Phi^T Phi, upper triangle) or kTileField (Phi^T F)
  int32_t unit_first;  // first partial slot of this tile (its split-K pieces use consecutive slots)
  int32_t unit_count;  // number of split-K pieces
  int32_t ld;          // row stride (floats) of this tile's partials
  int32_t col_off;     // column of this tile's first entry within a partial row
  int32_t pad_;
};

// One split-K piece of the reductions over N.
//  SIMT form: a tile over the point range [k0, k1).
//  Tensor-core form: one persistent CTA; a Gram part (rows i0.. x rows j0.., N = nj_mma,
//  absent when nj_mma == 0) and/or a field part (rows i0.. x the cpad field rows,
//  when has_f), accumulated over the 64-point blocks kb = lane, lane + nlanes, ...
struct GramUnit {
  int32_t tile;
  int32_t kind;
  int32_t i0, j0, nj_mma;
  int32_t has_f;
  int64_t k0, k1;
  int64_t out;             // float offset of this unit's partial tile
  int32_t lane, nlanes;
};

// ---- step a2: features ---------------------------------------------------
cudaError_t launch_features(const float* pts, int64_t n, int64_t n_pad, const float* omega_hi,
                            const float* omega_lo, int h, bool bf16, void* psi, cudaStream_t st);
cudaError_t launch_fill_field_rows(const float* F, int64_t ldF, int c, int64_t n, int64_t n_pad,
                                   int cpad, bool bf16, void* rows, cudaStream_t st);

// ---- step a3: reductions over N --------------------------------------------
// FP32 SIMT form: 128 x 128 tiles, chunked + Kahan-compensated accumulation.
constexpr int kSimtTile = 128;
constexpr int kSimtK = 16;
cudaError_t launch_gram_simt(const float* psi, int64_t n_pad, const GramUnit* units, int num_units,
                             float* partials, cudaStream_t st);

// BF16 tensor-core form (tcgen05 + TMA): one CTA per (tile, lane); a tile is
// 128 rows x (<= 256 Gram columns + cpad field columns).  Partial rows have
// kTcLd floats: Gram part at column 0, field part at column kTcBNMax.
constexpr int kTcBM = 128;
constexpr int kTcBNMax = 256;
constexpr int kTcBK = 64;
constexpr int kTcLd = 512;
struct TcGramArgs {
  const void* psi;       // bf16 [rows][n_pad]
  int64_t n_pad;
  int32_t m, cpad;
  const GramUnit* units;
  int32_t num_units;
  float* partials;
  int* err;              // device error word (bounded waits record here)
};
cudaError_t launch_gram_tc(const TcGramArgs& a, int grid, cudaStream_t st);
bool tc_gram_supported();

// Sum the split-K partials of every tile in a fixed order (Kahan) and apply
// the column scales: M = diag(ob) K diag(oa) (both triangles), Y = diag(ob) Y'.
// Partials of tile t, split s live at partials + (t.unit_first + s) * slot_elems.
cudaError_t launch_reduce(const GramTile* tiles, int num_tiles, const float* partials, int64_t slot_elems,
                          const double* oa, const double* ob, int m, int c, double* M, double* Y,
                          int tile_rows, int tile_cols, cudaStream_t st);

// ---- step a5: Z = diag(oa) G Y ------------------------------------------------
cudaError_t launch_small_product(const double* G, const double* Y, const double* oa, int m, int c,
                                 float* Z, cudaStream_t st);

// ---- step a6: out = F + Phi Z ---------------------------------------------------
cudaError_t launch_apply_simt(const void* psi, bool bf16, int64_t n, int64_t n_pad, int m, const float* Z,
                              int c, const float* F, int64_t ldF, float* out, int64_t ldOut, cudaStream_t st);

// ---- step a4: FP64 dense toolkit for phi1 --------------------------------------
// C = alpha A B + beta C   (row-major, leading dimensions in elements)
cudaError_t dgemm(int M, int N, int K, double alpha, const double* A, int lda, const double* B, int ldb,
                  double beta, double* C, int ldc, cudaStream_t st);
// D = a0 X0 + a1 X1 + a2 X2 + a3 X3 + diag * I   (any Xi may be null)
cudaError_t dcombine(int m, int n, double* D, int ldd, double a0, const double* X0, double a1,
                     const double* X1, double a2, const double* X2, double a3, const double* X3,
                     double diag, int ldx, cudaStream_t st);
cudaError_t dnorm1(int m, const double* X, int ldx, double* out, cudaStream_t st);  // max column abs-sum
cudaError_t dfinite_check(int m, int n, const double* X, int ldx, int* flag, cudaStream_t st);
// FP64-accurate C = alpha A B + beta C on the BF16 tensor cores (Ozaki
// splitting, k_ozaki.cu); K <= 1024.  `work` holds ozaki_workspace_bytes(M, N, K).
size_t ozaki_workspace_bytes(int M, int N, int K);
bool ozaki_supported(int K);
cudaError_t dgemm_ozaki(int M, int N, int K, double alpha, const double* A, int lda, const double* B, int ldb,
                        double beta, double* C, int ldc, void* work, int* err, cudaStream_t st);
// LU with partial pivoting (in place), then solve for nrhs right-hand sides
cudaError_t dgetrf(int m, double* A, int lda, int* ipiv, double* work, int* info, cudaStream_t st);
cudaError_t dgetrs(int m, int nrhs, const double* LU, int lda, const int* ipiv, double* B, int ldb,
                   cudaStream_t st);

}  // namespace rfd
