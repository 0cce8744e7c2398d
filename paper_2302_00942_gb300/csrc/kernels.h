// Kernel launchers and work descriptors of the RFD GPU path.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cuda_bf16.h>
#include <vector>

namespace rfd {

// Kernels launched by this thread (every launcher adds its count); the plan
// reports the difference around its calls.
extern thread_local long long t_kernel_launches;
inline void count_launch(long long k = 1) { t_kernel_launches += k; }
inline cudaError_t launched(long long k = 1) {
  t_kernel_launches += k;
  return cudaGetLastError();
}

// Compensated FP32 summation (Knuth's TwoSum per term, the lost low parts kept
// in a second FP32 word): the split-K partials and the small products are
// summed this way.  wide() keeps both words (the compensated sum carries more
// bits than one FP32 word holds) for the reduction's final column scaling.
struct Fp32Sum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + c; }
  __device__ __forceinline__ double wide() const { return (double)s + (double)c; }
};

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
// Field tiles of at most kSimtNarrow columns: 128 x 16 tiles (same partial layout).
constexpr int kSimtNarrow = 16;
cudaError_t launch_gram_simt_narrow(const float* psi, int64_t n_pad, const GramUnit* units, int num_units,
                                    float* partials, cudaStream_t st);

// BF16 tensor-core form (tcgen05 + TMA): one CTA per (tile pair, lane).  A
// logical tile is 128 rows x (Gram columns + field columns <= 256); partial
// rows have kTcLd floats: Gram part at column 0, field part at column kTcBNMax.
constexpr int kTcBM = 128;
constexpr int kTcBNMax = 256;
constexpr int kTcBK = 64;
constexpr int kTcLd = 512;
// One CTA of the tensor-core reductions: rows i0 .. i0+127 (half 0) and, when
// out1 is set, rows i0+128 .. i0+255 (half 1) of one cloud's Psi against the
// same B rows -- Gram rows j0 .. j0 + nj_mma (nj_mma a multiple of 16, may be
// 0) followed by the cloud's cpad field rows (has_f) -- over the 64-point
// blocks kb = lane, lane + nlanes, ... < kb_total.  Half 0 is one MMA of
// N = nj_mma (+ cpad) per 16 points; half 1 skips the first skip1 B rows (the
// part of a diagonal tile below the diagonal), N = nj_mma - skip1 (+ cpad).
// maps[map + 0/1/2/5]: the cloud's A (box 128 rows), B (64 rows), F (cpad rows)
// and B (16 rows) maps; b_rows: rows of the B map (m).  slot: the logical tile
// index of half 0 (half 1: slot + 1); out / out1 point at this lane's partials.
struct TcUnit {
  float* out;   // half 0 partial: 128 rows x kTcLd floats
  float* out1;  // half 1 partial, or null when the unit has one half
  int32_t map;
  int32_t i0, j0, nj_mma, has_f, cpad;
  int32_t lane, nlanes, kb_total, a_rows, b_rows;
  int32_t slot, skip1;
  int32_t work;  // the tile's cost per 64-point block (SM clocks; sets its share of the lanes)
};
// One CTA pair of the 2-SM reductions (k_gram_pair.cu, m >= 512, m % 16 == 0):
// feature rows r0 .. r0 + 511 (S0 = r0.., S1 = r0 + 256..) against the nc
// columns c0 .. c0 + nc - 1 (nc a multiple of 16, <= 256), and, on the first
// column tile of the row block (c0 = r0, no S1 x B part), the cpad field rows
// (has_f).  CTA rank k of the pair holds the logical halves S0 + 128 k and
// S1 + 128 k: out0[k] / out1[k] are this lane's partials of them (out1 null
// when the pair tile has no S1 part).  g2: the S1 x B MMA; a1: S1 rows are
// loaded (g2 or the field with S1 rows); m: rows of the cloud (loads of rows
// >= m are skipped).  maps[map + 0/1/5/6/7]: A (128-row box), B (64-, 16-,
// 8-row boxes), the field rows (box cpad / 2 rows).
struct PairUnit {
  float* out0[2];
  float* out1[2];
  int32_t map, r0, c0, nc, cpad, m;
  int32_t g2, has_f, a1;
  int32_t lane, nlanes, kb_total;
  int32_t work, pad_;
};
// Stage size of the pair kernel for the largest column tile and field width of a launch.
int gram_pair_stage_bytes(int max_nc, int max_cpad);
// One phase of the pair reductions: grid 2 x num_units in clusters of two.
// prof (optional, 2 x 2 num_units words): each CTA's %globaltimer at the start of its pipeline
// and at its end, for the autotuner's measure of every tile's pace.
cudaError_t launch_gram_pair_phase(const void* maps_dev, const PairUnit* units, int num_units, int stage_bytes,
                                   int kb0, int phase_blocks, int* err, cudaStream_t st,
                                   unsigned long long* prof = nullptr);
cudaError_t gram_pair_prepare();
// CTA pairs of the pair kernel that fit on the GPU at once (0 if unknown).
int gram_pair_max_clusters();
// Encodes the three tensor maps of a cloud's bf16 feature matrix Psi
// ([rows_alloc][n_pad], rows 0..m-1 features, m..m+cpad-1 field) into maps[0..2].
// maps_host3[0..2]: A (box min(128, m) rows), B (box min(64, m) rows), F rows (box cpad rows);
// map_b16: B with a box of min(16, m) rows; maps_pair2[0..1] (the pair kernel's): B with a
// box of min(8, m) rows, and the F rows with a box of cpad / 2 rows.
bool make_gram_maps(void* maps_host3, void* map_b16, void* maps_pair2, const void* psi, int64_t n_pad, int m,
                    int cpad, int rows_alloc);
// One launch per phase of phase_blocks 64-point blocks (max_kb: the largest
// point-block count of the units' clouds); later phases add to the partials.
constexpr int kGramPhaseBlocks = 4096;  // default phase length
// a_boxes: 2 when some unit has a second half (stages hold two A boxes), else 1.
cudaError_t launch_gram_tc(const void* maps_dev, const TcUnit* units, int num_units, int a_boxes, int max_kb,
                           int phase_blocks, int* err, cudaStream_t st);
// One phase alone: the 64-point blocks [kb0, kb0 + phase_blocks) (kb0 > 0 adds to the partials).
// prof: as launch_gram_pair_phase's (2 x num_units words)
cudaError_t launch_gram_tc_phase(const void* maps_dev, const TcUnit* units, int num_units, int a_boxes, int kb0,
                                 int phase_blocks, int* err, cudaStream_t st,
                                 unsigned long long* prof = nullptr);
bool tc_gram_supported();
// One CTA that allocates TMEM, waits on an mbarrier nothing arrives on for
// limit_ns, records its code in *err, frees the TMEM and returns: the bounded
// wait's unwind path on its own (a test hook).
cudaError_t launch_wait_probe(unsigned long long limit_ns, int* err, cudaStream_t st);

// Sum the split-K partials of every tile in a fixed order (compensated FP32)
// and apply the column scales: M = diag(ob) K diag(oa) (both triangles),
// Y = diag(ob) Y', stored as FP64 for step a4 (the scaling is the only FP64
// arithmetic of step a3: three multiplies per entry, with the commutative
// product ob_f ob_g so that M diag(sgn r) is exactly symmetric).
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
// FP64-accurate C = alpha A B + beta C on the BF16 tensor cores (the modular
// form of the Ozaki scheme, k_ozaki.cu); K <= 4096.  `work` holds
// ozaki_workspace_bytes(M, N, K).
// Workspace layout of the emulated FP64 GEMM (byte offsets from a 256-byte
// aligned base): A residues [16][mp][kp] and B^T residues [16][np][kp] (BF16),
// exponents, residues of the product [16][mp][np] (bytes).  The single source
// of the padded sizes.
struct OzLayout {
  int mp, np, kp;
  size_t sa, sb, ea, eb, eap, ebp, res, bytes;  // eap: raw row exponents [mp]; ebp: per-64-row column exponents [kp / 64][np]
};
OzLayout ozaki_layout(int M, int N, int K);
size_t ozaki_workspace_bytes(int M, int N, int K);  // layout bytes + alignment slack
int ozaki_col_split_blocks(int m);  // blocks of the batched column split of an m x m operand
int ozaki_combine_blocks(int m);    // blocks of the batched reconstruction of an m x m product
int ozaki_row_split_warps(int m);   // warps of the batched row split of an m x m operand
int ozaki_row_exponent_blocks(int m);  // blocks (8 rows each) of the batched row-exponent pass
int ozaki_kbits(int K, int nmod);   // bits of the scaled integers (length-K contractions, first nmod moduli)
int ozaki_moduli_for_bits(int K, int k);  // fewest moduli that give k bits at length K (16 at most)
bool ozaki_supported(int K);
cudaError_t dgemm_ozaki(int M, int N, int K, double alpha, const double* A, int lda, const double* B, int ldb,
                        double beta, double* C, int ldc, void* work, int* err, cudaStream_t st);
// LU with partial pivoting (in place), then solve for nrhs right-hand sides
cudaError_t dgetrf(int m, double* A, int lda, int* ipiv, double* work, int* info, cudaStream_t st);
cudaError_t dgetrs(int m, int nrhs, const double* LU, int lda, const int* ipiv, double* B, int ldb,
                   cudaStream_t st);

// ===========================================================================
// Batched path: many clouds per launch (and a single cloud as a batch of one).
// Each launcher takes device tables; kernels with a per-cloud block count find
// their cloud by binary search over a prefix array of block counts.
// ===========================================================================

// Per call and cloud: the caller's buffers and channel count.
struct CloudCall {
  const float* pts;
  const float* F;
  float* out;
  int64_t ldF, ldOut;
  int32_t c, pad_;
};

// Step a2 (features) for one cloud, BF16 form.
// BF16 feature buffer layout (blocked): 64-point blocks, each holding all of
// its rows contiguously, so that a 64-point slab of every row is one
// contiguous span: element (row, point p) at ((p / 64) rows_alloc + row) 64 + p % 64.
__host__ __device__ inline size_t psi_index(int64_t p, int row, int rows_alloc) {
  return ((size_t)(p >> 6) * (size_t)rows_alloc + (size_t)row) * 64 + (size_t)(p & 63);
}
struct FeatJob {
  int64_t n, n_pad;
  const float* omega;   // h x 3 FP32 frequencies
  __nv_bfloat16_raw* psi;
  float* xyz;           // the plan's copy of the points (N x 3), read by the apply
  int32_t h, bx, cloud, rows_alloc;  // bx: 512-point blocks; the job has bx * ceil(h / 32) blocks
};
// F^T rows of a cloud's Psi (rows m .. m + cpad - 1), BF16.
// With fsplit, channel ch of F is written as two BF16 rows, hi = bf16(F) at
// row ch and lo = bf16(F - hi) at row c + ch, so Phi^T F carries no BF16
// rounding of F (the reduction adds the two columns).
struct FillJob {
  int64_t n, n_pad;
  __nv_bfloat16_raw* psi;
  int32_t cpad, bx, cloud, fsplit;  // bx: 256-point blocks (fill_batched)
  int32_t row0, rows_alloc;         // F rows start at row0 (= m) of the blocked buffer
  int32_t bxw, cgw;                 // fill_wide_batched: 64-point blocks x channel groups of 32
};
// Y' = Phi^T F from the points, for a compact plan (no feature matrix): per
// chunk of `pts` points, part[chunk][f][ch] = sum_n Phi(n, f) F[n, ch] with
// Phi recomputed in FP32 exactly as the apply does (rows f < h cos, h + f sin);
// part is [chunks][m][ld] floats, summed over the chunks into Y[f][ch] =
// ob[f] sum_chunks part by fieldpts_reduce.
struct FieldPtsJob {
  const float* xyz;       // the plan's copy of the points (N x 3)
  const float* omega_hi;  // h x 3
  float* part;
  int64_t n, pts;
  int32_t h, m, chunks, ld, cloud, pad_;
  double* Y;              // m x c (the call's c), the plan's Y
  const double* ob;       // m column scales s
};
// One output tile of the split-K reduction (absolute pointers).
struct RedTile {
  const float* part;    // partial of lane 0; lane l at part + l * slot_elems
  double* M;
  double* Y;
  const double* oa;
  const double* ob;
  int64_t slot_elems;
  int32_t i0, j0, ni, nj, kind, count, ld, col_off, m, cloud;
  int32_t fsplit, pad_;  // field tiles: columns c..2c-1 hold the lo parts of F (see FillJob)
};
// Steps a5 / a6 for one cloud.
struct ApplyJob {
  const float* xyz;       // the plan's copy of the points (N x 3)
  const float* omega_hi;  // h x 3 frequencies, FP32 hi + lo parts
  const float* omega_lo;
  const double* G;
  const double* Y;
  const double* oa;
  float* Z;
  int64_t n, n_pad;
  int32_t m, cloud, bx, pad_;  // bx: 512-point blocks (apply), m rows (small product)
};
// Step a4 (phi1) for one cloud on the emulated-FP64 path.  Matrix "slots":
// slot k >= 0 is work + k m^2; kSlotM is M, kSlotG is G.
constexpr int kSlotM = -1, kSlotG = -2, kNoSlot = -3;
struct PhiCloud {
  double* work;
  const double* M;
  double* G;
  __nv_bfloat16_raw* sa;  // A-operand residues [16][mpa][kp]
  __nv_bfloat16_raw* sb;  // B^T-operand residues [16][mpb][kp]
  int* ea;                // row exponents of A (mpa)
  int* eb;                // column exponents of B (mpb)
  int* ebp;               // column exponents of B per 64 rows of K ([kp / 64][mpb])
  int* eap;               // largest biased exponents of A's rows (mpa)
  uint8_t* res;           // residues of the product [16][mpa][mpb]
  int* flag;              // finiteness flag
  double lambda, scale;   // scale = 2^-s (set per call)
  int32_t m, mpa, mpb, kp;
  int32_t map_a, map_b;   // tensor maps of sa / sb
  int32_t s, pad_;        // squarings (set per call)
  int8_t kbits_n[16];     // bits of the scaled integers with the first n moduli: ozaki_kbits(m, n), n = 1..16
};
// One tile of the residue GEMM: rows m0 .. m0 + 127, columns
// n0 .. n0 + nb of one cloud's product (kp: the padded K, for ordering the tiles
// by cost); a launch with nmod moduli has the work items (tile, modulus g < nmod).
struct OzTile {
  int32_t cloud, m0, n0, nb, kp, g0, ng, pad_;
};
// The residue-GEMM tiles of a batch of m x m products (cloud k of size ms[k]),
// longest first: one per (row tile, column tile of <= 256).
// *stage_bytes: the pipeline stage size.
void ozaki_batch_tiles(const std::vector<int>& ms, int sms, std::vector<OzTile>* out, int* stage_bytes);

cudaError_t launch_features_batched(const FeatJob* jobs, const int* prefix, int count, int total_blocks,
                                    const CloudCall* calls, cudaStream_t st);
// Step a2 for one cloud (job 0 of jobs), its 512-point blocks blk0 .. blk0 + blk_n - 1 only
// (the features of one phase of the point axis; h: the cloud's frequencies).
cudaError_t launch_features_range(const FeatJob* jobs, const CloudCall* calls, int h, int blk0, int blk_n,
                                  cudaStream_t st);
cudaError_t launch_fill_batched(const FillJob* jobs, const int* prefix, int count, int total_blocks,
                                const CloudCall* calls, cudaStream_t st);
// the same for calls whose largest c is above 8 (prefix over bxw * cgw blocks per cloud)
cudaError_t launch_fill_wide_batched(const FillJob* jobs, const int* prefix, int count, int total_blocks,
                                     const CloudCall* calls, cudaStream_t st);
cudaError_t launch_reduce_batched(const RedTile* tiles, int num_tiles, const CloudCall* calls, cudaStream_t st);
// Y' partials of compact plans from their points: cg channels per block (3, 4, 8, 16 or 32),
// fieldpts_fpt(cg) frequencies per thread; prefix over chunks x ceil(h / (256 fpt)) x
// ceil(c / cg) blocks per cloud.
cudaError_t launch_fieldpts_batched(const FieldPtsJob* jobs, const int* prefix, int count, int total_blocks, int cg,
                                    const CloudCall* calls, cudaStream_t st);
constexpr int fieldpts_fpt(int cg) { return cg <= 8 ? 2 : 1; }
// Y of compact plans from their fieldpts partials (one warp per feature row and group of 4
// channels, 8 warps per block); prefix over fieldpts_reduce_blocks per cloud.
cudaError_t launch_fieldpts_reduce(const FieldPtsJob* jobs, const int* prefix, int count, int total_blocks,
                                   const CloudCall* calls, cudaStream_t st);
inline int fieldpts_reduce_blocks(const FieldPtsJob& j, int c) { return (j.m * ((c + 3) / 4) + 7) / 8; }
// blocks of one cloud's fieldpts launch for c channels, cg per block
inline int fieldpts_blocks(const FieldPtsJob& j, int c, int cg) {
  const int fb = 256 * fieldpts_fpt(cg);
  return j.chunks * ((j.h + fb - 1) / fb) * ((c + cg - 1) / cg);
}
// Z = diag(oa) G Y per cloud (one block per matrix row: prefix over m)
cudaError_t launch_small_batched(const ApplyJob* jobs, const int* prefix, int count, int total_rows,
                                 const CloudCall* calls, cudaStream_t st);
// the same for calls whose largest c is above 16: blocks of 8 rows x 64 channels, prefix over
// small_wide_blocks per cloud
cudaError_t launch_small_wide_batched(const ApplyJob* jobs, const int* prefix, int count, int total_blocks,
                                      const CloudCall* calls, cudaStream_t st);
inline int small_wide_blocks(int m, int max_channels) { return (m + 7) / 8 * ((max_channels + 63) / 64); }
// out = F + Phi Z per cloud; cg: channels per thread (3, 4, 8, 16 or 32); a block covers
// kApplyPts points, two per thread; prefix over bx * ceil(c / cg) blocks per cloud
// (bx = ceil(n / kApplyPts))
constexpr int kApplyPts = 512;
cudaError_t launch_apply_batched(const ApplyJob* jobs, const int* prefix, int count, int total_blocks, int cg,
                                 const CloudCall* calls, cudaStream_t st);
// Step a6 on the tensor cores (k_apply_tc.cu), for 1 <= c <= kApplyTcMaxC channels:
// per cloud, 2 pi w as float4 (zero past h) and Z split into BF16 hi / lo parts,
// laid out per chunk of 64 features as the MMA's B operand (apply_prep, from
// the FP32 Z of step a5); the apply then recomputes Phi per 256-point tile.
struct ApplyTcJob {
  const float* xyz;       // the plan's copy of the points (N x 3)
  const float* omega_hi;  // h x 3
  const float* Z;         // m x c FP32 (the call's c), step a5's output
  float4* w2pi;           // 32 kchunks frequencies
  uint8_t* zimg;          // kchunks x 2 cp rows x 128 B (cp = apply_tc_cpad(c))
  int64_t n;
  int32_t h, kchunks, cloud, tiles;  // kchunks = ceil(h / 32), tiles = ceil(n / 256)
};
constexpr int kApplyTcMaxC = 64;
__host__ __device__ constexpr int apply_tc_cpad(int c) { return (c + 15) / 16 * 16; }
inline size_t apply_tc_zimg_bytes(int h, int max_c) {
  const int c = max_c < kApplyTcMaxC ? max_c : kApplyTcMaxC;
  return (size_t)((h + 31) / 32) * 2 * apply_tc_cpad(c) * 128;
}
inline int apply_prep_blocks(const ApplyTcJob& j, int c) { return (j.kchunks * 2 * apply_tc_cpad(c) * 8 + 255) / 256; }
bool apply_tc_supported();
// Y' of compact plans from their points on the tensor cores (k_apply_tc.cu): work items of one
// chunk of points (jobs[k].pts a multiple of 64) and one tile of 128 frequencies, item_prefix over
// chunks * ceil(h / 128) per cloud; persistent CTAs (at most one per SM).  The partials are laid
// out as the SIMT kernel's (launch_fieldpts_reduce sums them).
cudaError_t launch_fieldpts_tc(const FieldPtsJob* jobs, const int* item_prefix, int count, int total_items, int grid,
                               const CloudCall* calls, int* err, cudaStream_t st);
inline int fieldpts_tc_items(const FieldPtsJob& j) { return j.chunks * ((j.h + 127) / 128); }
cudaError_t apply_tc_prepare();
cudaError_t launch_apply_prep(const ApplyTcJob* jobs, const int* prefix, int count, int total_blocks,
                              const CloudCall* calls, cudaStream_t st);
// grid: persistent CTAs (at most one per SM) over total_tiles = tile_prefix[count]
cudaError_t launch_apply_tc(const ApplyTcJob* jobs, const int* tile_prefix, int count, int total_tiles, int grid,
                            const CloudCall* calls, int* err, cudaStream_t st);
// phi1 building blocks over all clouds (elements: prefix over ceil(m^2 / 256) blocks)
// D = k (a0 X0 + a1 X1 + a2 X2 + a3 X3 + diag I), k = 1, lambda or scale (kmode 0/1/2);
// clouds with s <= mask_k are skipped (mask_k < 0: none).
cudaError_t launch_bcombine(const PhiCloud* pc, const int* prefix, int count, int total_blocks, int dst,
                            const int* src4, const double* a4, double diag, int kmode, int mask_k, cudaStream_t st);
cudaError_t launch_bnorm1(const PhiCloud* pc, int count, int max_m, int slot, double* norms, cudaStream_t st);
// squarings per cloud from the norms (see bselect_kernel); sv: count + 1 ints
cudaError_t launch_bselect(PhiCloud* pc, int count, const double* norms, double theta, int max_s, int* sv,
                           cudaStream_t st);
// sets a cloud's flag when an entry of the slot is not finite (flags are sticky)
cudaError_t launch_bfinite(const PhiCloud* pc, const int* prefix, int count, int total_blocks, int slot,
                           cudaStream_t st);
// D = alpha A B + beta C + diag I on every cloud (emulated FP64): exponent pass
// (A's rows: prefix over ozaki_row_exponent_blocks(m) per cloud), row split of
// A (warp prefix over ozaki_row_split_warps(m) per cloud), column split of B (prefix over
// ozaki_col_split_blocks(m) per cloud), the residue GEMM over the tiles and the
// reconstruction (prefix over ozaki_combine_blocks(m) per cloud).
// nmod: the moduli used (the first nmod; fewer when the product only needs
// k = kbits(m, nmod) bits relative to its operands' row and column maxima).
// c_slot kNoSlot: no C.  Clouds with s <= mask_k (mask_k >= 0) skip the
// product and copy C to D.  split_a / split_b false: the residues already hold
// that operand (split by the previous product over the same or a larger set of
// clouds).
cudaError_t launch_bgemm(const PhiCloud* pc, int count, const int* row_prefix_a, int rows_a, const int* rexp_prefix,
                         int rexp_blocks, const int* strip_prefix,
                         int col_strips, const OzTile* tiles, int num_tiles, int stage_bytes,
                         const int* group_prefix, int group_blocks, int nmod,
                         const void* maps_dev, int a_slot, int b_slot, int c_slot, int d_slot, double alpha,
                         double beta, double diag, int mask_k, bool split_a, bool split_b, int* err, cudaStream_t st);
// one-time kernel attribute set-up of launch_gram_tc / launch_bgemm (call before a stream capture)
cudaError_t gram_tc_prepare();
cudaError_t bgemm_prepare();
// tensor maps of a cloud's residue buffers (A: box 64 x 128 rows, B: box 64 x 64 rows, one modulus)
bool make_ozaki_maps(void* map_a_host, void* map_b_host, const void* sa, const void* sb, int mpa, int mpb, int kp);

}  // namespace rfd
