/*
 * rfd.h -- C ABI of the GB300 RFDiffusion (RFD) graph-field integrator.
 *
 * RFD (Sec. 2.4, "RFDiffusion") approximates graph-field integration
 *     i(v) = sum_w K(w, v) F(w)                  (Sec. 1, Eq. base_integ)
 * with the graph diffusion kernel K = exp(lambda W) (Sec. 2, Eq. diffusion)
 * on the eps-nearest-neighbour graph of a point cloud, W(i,j) = f(n_i - n_j)
 * (Sec. 2.4, Eq. w), by a random-feature factorisation W ~ A B^T and
 *     out = F + A ([exp(lambda B^T A) - I] (B^T A)^{-1} (B^T F))   (Sec. 2.4)
 * evaluated here as out = F + A (G (B^T F)), G = lambda phi1(lambda B^T A),
 * phi1(X) = sum_k X^k / (k+1)!  (the same matrix whenever B^T A is
 * invertible; no inverse is ever formed).
 *
 * Conventions used by every entry point
 *   - Kernel f: indicator of the L-infinity cube ||z||_inf <= eps; its Fourier
 *     transform is tau(w) = prod_d sin(2 pi eps w_d)/(pi w_d) (Sec. 2.4).
 *   - m = number of REAL columns of A and B (even): m/2 frequencies w_j in R^3,
 *     each giving a cos and a sin column (the real-part estimator of App. A.4).
 *   - Frequencies: per-coordinate N(0, sigma^2) truncated to [-R, R], drawn by
 *     rejection from a SplitMix64 stream seeded with `seed` (rfd_sample_frequencies
 *     documents the exact order); r_j = tau(w_j)/p(w_j).
 *   - A = Phi diag(s sgn r), B = Phi diag(s), s_j = sqrt(2 |r_j| / m), where
 *     Phi = [cos 2 pi X w^T | sin 2 pi X w^T] (N x m).
 *   - Points: N x 3 float32, row-major (x, y, z), DEVICE memory unless stated.
 *   - Fields F and outputs: N x c float32, row-major with leading dimension
 *     ld >= c (elements), DEVICE memory unless stated.
 *   - Every call returns an rfd_status; nothing aborts or throws across the
 *     ABI.  On failure rfd_last_error() returns a thread-local message and the
 *     plan stays usable (unless the CUDA context itself is lost).
 *   - Device work is asynchronous on the plan's stream unless stated; the caller
 *     keeps device buffers alive until rfd_sync() (or rfd_poll()) reports
 *     completion.
 */
#ifndef RFD_H_
#define RFD_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RFD_API __attribute__((visibility("default")))
#else
#define RFD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RFD_OK = 0,
  RFD_EINVAL = 1,      /* invalid argument (sizes, null pointers, parameters)      */
  RFD_ENOMEM = 2,      /* device or host allocation failed                          */
  RFD_ECUDA = 3,       /* a CUDA runtime/driver call failed                         */
  RFD_ENOTREADY = 4,   /* rfd_poll: the request has not finished yet                */
  RFD_ETIMEDOUT = 5,   /* a bounded wait ran out (host poll or device-side wait)    */
  RFD_ENUMERIC = 6,    /* G or the output is not finite (overflow of exp(lambda W)) */
  RFD_EBUSY = 7,       /* serving: admission refused (memory budget / queue full)   */
  RFD_ENOTSUP = 8      /* feature not available in this build / on this device      */
} rfd_status;

typedef enum {
  RFD_FP32_PLAIN = 0,  /* FP32 features, SIMT FP32 reductions (compensated), FP64 G */
  RFD_BF16_TC = 1      /* BF16 features, tcgen05 BF16 x BF16 -> FP32 GEMMs, FP64 G  */
} rfd_precision;

/* Parameters of one point cloud's integrator (Sec. 2.4: points, eps, lambda,
 * m random features, seed).  Zero for freq_sigma / freq_radius selects the
 * defaults sigma = 1/(2 eps), R = 1/eps. */
typedef struct {
  int64_t n;             /* number of points N >= 1                               */
  int32_t m;             /* real feature columns, even, 2 <= m <= 4096            */
  int32_t max_channels;  /* largest c passed to rfd_integrate / rfd_gfi, 1..256   */
  double eps;            /* L-infinity radius of the eps-NN graph, > 0            */
  double lambda;         /* diffusion parameter, any finite real; 0 => out == F   */
  uint64_t seed;         /* seed of the frequency stream                          */
  int32_t precision;     /* rfd_precision                                         */
  int32_t flags;         /* RFD_FLAG_* bits (0 = none)                            */
  double freq_sigma;     /* sigma of the truncated Gaussian (0 => 1/(2 eps))      */
  double freq_radius;    /* truncation half-width R (0 => 1/eps)                  */
  int32_t kernel;        /* rfd_kernel: the eps-NN indicator f (0 = L-infinity cube) */
  int32_t reserved_;     /* must be 0                                             */
} rfd_params;

/* The threshold function f of the eps-NN graph, W(i, j) = f(x_i - x_j) (Sec. 2.4),
 * and with it tau = the Fourier transform of f (2 pi convention):
 *   RFD_KERNEL_CUBE: f = 1[||z||_inf <= eps], tau(w) = prod_d sin(2 pi eps w_d) / (pi w_d)
 *                    (the product of per-coordinate sincs printed in Sec. 2.4);
 *   RFD_KERNEL_BALL: f = 1[||z||_2 <= eps], tau(w) = 4 pi (sin(q eps) - q eps cos(q eps)) / q^3,
 *                    q = 2 pi ||w||_2 (the Bessel-function case of Sec. 2.4 in d = 3:
 *                    4 pi eps^3 j_1(q eps) / (q eps));
 *   RFD_KERNEL_CUBE_L1: f = ||z||_1 1[||z||_inf <= eps] (the distance-weighted adjacency of the
 *                    paper's brute-force baseline, on the cube of RFD_KERNEL_CUBE):
 *                    tau(w) = sum_d g(w_d) prod_{e != d} sin(2 pi eps w_e) / (pi w_e) with
 *                    g(w) = int_{-eps}^{eps} |z| cos(2 pi w z) dz = 2 eps^2 (sin x / x + (cos x - 1) / x^2),
 *                    x = 2 pi eps w (eps^2 at w = 0);
 *   RFD_KERNEL_L1_BALL: f = 1[||z||_1 <= eps] (the L1 ball of Sec. 2.4, an octahedron; its transform
 *                    does not factor over coordinates): the sum over the 8 simplices
 *                    conv(0, +-eps e_1, +-eps e_2, +-eps e_3) of eps^3 times the divided difference
 *                    of exp at 0, -2 pi i eps s_d w_d (d = 1..3), the corner entry of exp of the
 *                    bidiagonal matrix of those nodes (value 4 eps^3 / 3, the volume, at w = 0). */
typedef enum { RFD_KERNEL_CUBE = 0, RFD_KERNEL_BALL = 1, RFD_KERNEL_CUBE_L1 = 2, RFD_KERNEL_L1_BALL = 3 } rfd_kernel;

typedef struct rfd_plan_s* rfd_plan_t;

/* rfd_params.flags bits */
#define RFD_FLAG_TIMING 1       /* record CUDA events around every step (see rfd_stats.step_ms) */
#define RFD_FLAG_NATIVE_FP64 2  /* step a4 products in native FP64 instead of the FP64-accurate
                                   modular (Chinese-remainder) emulation on the BF16 tensor cores
                                   (the default) */
#define RFD_FLAG_GRAPH 4        /* BF16 plans and batches: replay each call's launches from CUDA
                                   graphs, captured on first use per call shape (per-step timings
                                   are then not recorded; ignored by FP32 plain plans) */
#define RFD_FLAG_AUTOTUNE 8     /* BF16 plans and batches: after the first features pass, time the
                                   tensor-core reductions for a few split-K lane counts (plans) or
                                   wave targets (batches), point-axis phase lengths and (a plan with
                                   m >= 512) the one-SM or CTA-pair form of the Gram on the
                                   cloud's own features, and keep the fastest (cached per bucket:
                                   m, point count and field width for plans; cloud count and work
                                   for batches).  That first call returns after the tuning. */

/* Indices of rfd_stats.step_ms */
enum {
  RFD_STEP_FEATURES = 0,  /* a2: feature map                      */
  RFD_STEP_FIELD = 1,     /* F^T rows of the feature matrix        */
  RFD_STEP_GRAM = 2,      /* a3: reductions over N (GEMMs)         */
  RFD_STEP_REDUCE = 3,    /* a3: split-K reduction and scaling     */
  RFD_STEP_PHI1 = 4,      /* a4: G = lambda phi1(lambda M), FP64   */
  RFD_STEP_SMALL = 5,     /* a5: Z = diag(s sgn r) G Y             */
  RFD_STEP_APPLY = 6,     /* a6: out = F + Phi Z                   */
  RFD_STEP_EIGEN = 7,     /* kernel eigenvalues (m x m problem)    */
  RFD_NUM_STEPS = 8
};

/* Statistics of a plan.  norm1 .. splits describe the last rfd_features /
 * rfd_gfi call.  With RFD_FLAG_TIMING, step_ms holds the mean device time of
 * each step (CUDA events on the plan's stream) over the `timed_calls` calls
 * since the last rfd_plan_stats_reset; kernel_launches counts every kernel
 * the plan launched since then.  rfd_plan_stats synchronises the stream. */
typedef struct {
  double norm1;          /* ||lambda M||_1                                         */
  int32_t pade_degree;   /* degree of the approximant of step a4: Taylor degree (16) on the
                            batched emulated path, diagonal Pade degree q on the native path */
  int32_t squarings;     /* scaling-and-squaring steps s                          */
  int32_t nonfinite;     /* 1 if G was not finite                                 */
  int32_t splits;        /* split-K pieces per tile (mean) of the reductions over N */
  int32_t phi1_emulated; /* 1: the m x m x m products of step a4 used the FP64-accurate tensor-core emulation */
  int32_t phi1_gemms;    /* m x m x m products evaluated by step a4 (LU solve not included) */
  double step_ms[RFD_NUM_STEPS];
  int64_t timed_calls;
  int64_t kernel_launches;
  int32_t tune_lanes_pct;    /* reductions' launch parameters in use (RFD_FLAG_AUTOTUNE picks them): */
  int32_t tune_waves;        /*   split-K lanes (% of SMs per tile), waves a batch plans for, */
  int32_t tune_phase_blocks; /*   point-axis phase length (64-point blocks)                  */
  int32_t tuned;             /* 1 once the autotuner has chosen them                        */
  int32_t tune_pair_gram;    /* 1: the reductions run on CTA pairs (2-SM MMAs; a lone BF16  */
                             /*    cloud with m >= 512, chosen by the autotuner)           */
  int32_t tune_overlap;      /* 1: a lone cloud's features run phase by phase beside the    */
                             /*    Gram (a test hook selects it; the autotuner does not)    */
  double tune_form_ms[2];    /* the autotuner's best time (ms) of features + reductions with */
                             /*    one SM per tile [0] and CTA pairs [1] (0: not timed)     */
} rfd_stats;

/* ---------------------------------------------------------------------------
 * Step a1 (host only, no device work): the random frequencies and weights.
 * Sec. 2.4: w_1..w_{m/2} iid ~ P, nu_j^2 = tau(w_j)/p(w_j).
 *
 * Draw order: a SplitMix64 stream (state += 0x9E3779B97F4A7C15, finaliser
 * shifts 30/27/31) seeded with `seed` yields uniforms u = ((x >> 11) + 0.5)
 * 2^-53.  For j = 0..m/2-1, d = 0..2: repeat { u1, u2 from the stream;
 * w = R (2 u1 - 1); accept if u2 < exp(-(w/sigma)^2 / 2) } (at most 2^20
 * tries per coordinate, else RFD_EINVAL).
 *   omega_out: host, (m/2) x 3 doubles, row-major, caller-owned (may be NULL)
 *   r_out:     host, m/2 doubles r_j = tau(w_j)/p(w_j), caller-owned (may be NULL)
 * --------------------------------------------------------------------------- */
RFD_API rfd_status rfd_sample_frequencies(int32_t m, double eps, uint64_t seed, double freq_sigma,
                                  double freq_radius, double* omega_out, double* r_out);

/* The same draw for the threshold function `kernel` (rfd_kernel): omega_out is
 * identical for every kernel, r_out = tau_kernel(w_j)/p(w_j).  RFD_EINVAL for an
 * unknown kernel. */
RFD_API rfd_status rfd_sample_weights(int32_t m, double eps, uint64_t seed, double freq_sigma, double freq_radius,
                                      int32_t kernel, double* omega_out, double* r_out);

/* Create a plan: validate params, run step a1 on the host, upload the
 * frequencies and column scales, and allocate every device buffer the plan
 * will use (the feature matrix, split-K partials, M, G and the FP64 phi1
 * workspace).  `cuda_stream` is a cudaStream_t (NULL = legacy default
 * stream); all of the plan's device work runs on it.  *out receives the plan
 * (owned by the caller, released with rfd_plan_destroy).  RFD_ENOMEM if a
 * device allocation fails (nothing is leaked). */
RFD_API rfd_status rfd_plan(const rfd_params* params, void* cuda_stream, rfd_plan_t* out);

/* Release a plan and its device memory (synchronises the plan's stream). */
RFD_API rfd_status rfd_plan_destroy(rfd_plan_t plan);

/* Pre-processing (Sec. 2.4: "linear in N, cubic in m"), steps a2-a4:
 * features Phi of d_points (N x 3 float32, device), M = B^T A by split-K
 * reduction over N, and G = lambda phi1(lambda M) in FP64 (scaling-and-
 * squaring diagonal Pade on the block-triangular augmented matrix
 * [[lambda M, I], [0, 0]]).  Phi and G stay resident in the plan for later
 * rfd_integrate calls.  The host waits once on the stream, for the number of
 * squarings (chosen from ||lambda M||_1).  A G that is not finite is reported
 * as RFD_ENUMERIC: by this call in the FP32 plain form or with
 * RFD_FLAG_NATIVE_FP64, by the next rfd_sync in the BF16 tensor-core form. */
RFD_API rfd_status rfd_features(rfd_plan_t plan, const float* d_points);

/* Inference (Sec. 2.4: "linear in N, quadratic in m"), steps a3(Y)-a6, on
 * the resident Phi and G: Y = B^T F, Z = diag(s sgn r) G Y, out = F + Phi Z.
 * d_F: N x c float32 device, leading dimension ldF >= c; d_out: N x c float32
 * device, leading dimension ldOut >= c.  d_out == d_F (same ld) is allowed.
 * 1 <= c <= params.max_channels.  Asynchronous on the plan's stream. */
RFD_API rfd_status rfd_integrate(rfd_plan_t plan, const float* d_F, int32_t c, int64_t ldF,
                         float* d_out, int64_t ldOut);

/* Entropic Wasserstein barycenter on the resident plan (App. C, Algorithm
 * wass_barycenter; the steps of Solomon et al. 2015, Algorithm 2): for k input
 * distributions mu^i (columns of d_mu: N x k float32 device, leading dimension
 * ld_mu >= k), weights alpha (host, k doubles >= 0), area weights d_area (N
 * float32 device) and `iters` passes, with the kernel action x -> exp(lambda
 * W_hat) x of rfd_integrate on all k columns at once:
 *   v^i = 1;  repeat: mu = 1;  w^i = mu^i / K(a v^i);  d^i = v^i K(a w^i);
 *             mu = prod_i (d^i)^alpha_i;  then v^i = v^i mu / d^i.
 * d_out (N float32 device) receives mu (1 everywhere for iters = 0).  Kernel
 * outputs are lifted to 1e-30 before they divide or enter a power (the
 * random-feature kernel need not be positive).  Requires rfd_features (or
 * rfd_gfi) first and 1 <= k <= min(32, max_channels).  Asynchronous on the
 * plan's stream (temporaries of 4 N k floats from the stream-ordered
 * allocator); RFD_ENOMEM if they cannot be had. */
RFD_API rfd_status rfd_barycenter(rfd_plan_t plan, const float* d_mu, int32_t k, int64_t ld_mu, const double* alpha,
                                  const float* d_area, int32_t iters, float* d_out);

/* Gromov-Wasserstein building blocks with implicit structure matrices (App.
 * C.2).  The structure matrix of a cloud is its kernel C = exp(lambda W_hat),
 * applied by its resident plan, never formed; matrices are float32 device,
 * row-major.  Both plans must have run rfd_features (or rfd_gfi) and share
 * one stream; n1, n2 are their point counts.
 *   rfd_fm_apply: d_Y = C d_X for an n x ncols matrix (ldX, ldY >= ncols),
 *     rfd_integrate over column chunks of at most max_channels; asynchronous.
 *   rfd_gw_tensor_product: Algorithm tensor_prod with the square loss,
 *     d_L (n1 x n2) = (C^{(.)2} p) 1^T + 1 (D^{(.)2} q)^T - 2 C T D^T, with
 *     C^{(.)2} p = diag(C D_p C^T) (Eq. sq); d_T n1 x n2, d_p (n1), d_q (n2);
 *     asynchronous.  When both clouds have m <= 32 the sums are taken through
 *     the low-rank factors (C = I + Psi K Psi^T: the Hadamard squares in
 *     O(N m^2), one pass over T for its two projections, one for L;
 *     temporaries O((n1 + n2) mf) plus 16 n2 mf + n1 n2 mf / 256 floats, mf = 16
 *     or 32 the padded m); otherwise
 *     as four actions on n x n matrices (temporaries of 2 max(n1, n2)^2 +
 *     3 n1 n2 floats).  Temporaries come from the stream-ordered allocator
 *     (RFD_ENOMEM if it fails).
 *   rfd_gw_line_search: Algorithm line_search, the optimal step of a
 *     conditional-gradient (F)GW iteration for the transport G, direction dG,
 *     feature cost M (all n1 x n2) and trade-off alpha: with c_CD = steps 1-2 of
 *     tensor_prod, a1 = C dG D, b1 = C G D, a = -2 alpha <a1, dG>,
 *     b = <(1 - alpha) M + alpha c_CD, dG> - 2 alpha (<a1, G> + <b1, dG>);
 *     tau = clamp(-b / 2a, 0, 1) if a > 0, else 1 if a + b < 0, else 0.
 *     The inner products are accumulated in FP64 (the low-rank form for
 *     m <= 32 as in rfd_gw_tensor_product, reading G, dG and M once more).
 *     out3 (host, 3 doubles) = {tau, a, b}; waits for the stream. */
RFD_API rfd_status rfd_fm_apply(rfd_plan_t plan, const float* d_X, int64_t ncols, int64_t ldX, float* d_Y,
                                int64_t ldY);
RFD_API rfd_status rfd_gw_tensor_product(rfd_plan_t plan_C, rfd_plan_t plan_D, const float* d_T, const float* d_p,
                                         const float* d_q, float* d_L);
RFD_API rfd_status rfd_gw_line_search(rfd_plan_t plan_C, rfd_plan_t plan_D, double alpha, const float* d_G,
                                      const float* d_dG, const float* d_M, const float* d_p, const float* d_q,
                                      double* out3);

/* Eigenvalues of the cloud's RFD kernel exp(lambda W_hat) (Sec. 3.3: point-
 * cloud classification by the kernel's k smallest eigenvalues, computed from
 * the low-rank factorisation; App. E: graph classification by the k largest).
 * W_hat = A B^T is symmetric of rank <= m: its nonzero eigenvalues are those
 * of the m x m matrix M = B^T A, so exp(lambda W_hat) has the eigenvalues
 * exp(lambda mu) for the m eigenvalues mu of M and 1 with multiplicity N - m
 * (when N < m, the m - N eigenvalues of M of smallest modulus are the rank
 * deficiency and are dropped).  Writes the k smallest (largest = 0,
 * ascending) or the k largest (largest = 1, descending) of these N values to
 * d_out (k float32, device).  Needs the resident M of rfd_features / rfd_gfi;
 * 1 <= k <= N and m <= 128 (RFD_EINVAL otherwise).  Asynchronous on the
 * plan's stream; M is unchanged.  Cholesky of M diag(sgn r), cyclic Jacobi
 * in FP32 on the symmetric m x m matrix L^T diag(sgn r) L; for an FP32-plain
 * plan the Cholesky factor is FP64 and each eigenvalue is the FP64 Rayleigh
 * quotient of its eigenvector (~1e-10 relative), for a BF16 plan (M good to
 * ~1e-4) FP32 throughout (~1e-6 of the largest |eigenvalue| of lambda M). */
RFD_API rfd_status rfd_eigenvalues(rfd_plan_t plan, int32_t k, int32_t largest, float* d_out);

/* One cold pass of the whole path (a2-a6) when F is known up front: the
 * reductions B^T A and B^T F share one pass over the feature matrix.
 * Arguments as rfd_features + rfd_integrate; leaves Phi and G resident. */
RFD_API rfd_status rfd_gfi(rfd_plan_t plan, const float* d_points, const float* d_F, int32_t c,
                   int64_t ldF, float* d_out, int64_t ldOut);

/* Keep a BF16 plan resident at a fraction of its memory (inference on a resident
 * cloud, Sec. 2.4: "linear in N, quadratic in m").  After rfd_features or
 * rfd_gfi, the plan's feature matrix Phi (2 (m + field rows) N bytes), its
 * split-K partials and its FP64 phi1 workspace are released; it keeps its copy
 * of the points, the frequencies and column scales, M and G, and a small
 * partial buffer (at most 16 MB).  Later rfd_integrate calls recompute the
 * features from the points in FP32 for both B^T F and the apply (the BF16
 * rounding of Phi in B^T F is then gone: results agree with the full plan's
 * within the BF16 form's tolerance and with the FP64 oracle more closely).
 * rfd_features / rfd_gfi on a compact plan return RFD_EINVAL (create a new
 * plan); rfd_integrate, rfd_barycenter, rfd_fm_apply, the GW calls and
 * rfd_eigenvalues work as before.  Allocates the compact chunk before
 * releasing the full one (RFD_ENOMEM leaves the plan unchanged); synchronises
 * the plan's stream.  RFD_EINVAL for FP32 plain plans or before G exists;
 * a compact plan stays compact (a second call does nothing). */
RFD_API rfd_status rfd_plan_compact(rfd_plan_t plan);

/* Device bytes the plan holds now (its chunk: the full or the compact form). */
RFD_API rfd_status rfd_plan_device_bytes(rfd_plan_t plan, int64_t* bytes_out);

/* Step a4 alone: G = lambda phi1(lambda M) for an m x m FP64 matrix M
 * (Sec. 2.4: [exp(lambda M) - I] M^{-1}, evaluated without the inverse),
 * by the same scaling-and-squaring Pade evaluation rfd_features uses.
 * d_M, d_G: m x m row-major float64 DEVICE buffers (may not alias); flags:
 * RFD_FLAG_NATIVE_FP64 or 0;
 * 1 <= m <= 4096.  Allocates (and frees) its own FP64 workspace, about
 * 24 m^2 doubles; synchronises `cuda_stream`.  stats_out (host, may be NULL)
 * receives ||lambda M||_1, the Pade degree and the squaring count.
 * RFD_ENUMERIC if G is not finite. */
RFD_API rfd_status rfd_phi1(int32_t m, double lambda, const double* d_M, double* d_G, int32_t flags, void* cuda_stream,
                            rfd_stats* stats_out);

/* Step a4 for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of rfd_phi1 (same arguments, same
 * result) for code in which cudaMalloc/cudaFree are not allowed -- a
 * latency-critical loop where an allocation could synchronise the device, or a
 * process whose device memory is owned by another allocator.  It calls no
 * allocating routine: its workspace is a fixed 3.75 MiB __device__ array that
 * every GPU loading the library holds until the process exits, so it only
 * serves 1 <= m <= 128 (RFD_EINVAL with a message beyond that).  The first call
 * on each device looks up that array's device address (cudaGetSymbolAddress),
 * and so does the first call after the device's context changed (after a
 * cudaDeviceReset the module is loaded anew); make such a call before any
 * stream capture.  All calls share the array
 * and it keeps the previous call's contents: calls whose device work overlaps
 * (other streams or threads) race and must be serialised by the caller.
 * Synchronises `cuda_stream`. */
RFD_API rfd_status rfd_phi1_noalloc(int32_t m, double lambda, const double* d_M, double* d_G, int32_t flags,
                                    void* cuda_stream, rfd_stats* stats_out);

/* Wait for all of the plan's queued device work.  Reports (and clears) what
 * the device recorded since the last rfd_sync: RFD_ETIMEDOUT if a bounded
 * device-side wait ran out, RFD_ENUMERIC if G was not finite (BF16 form). */
RFD_API rfd_status rfd_sync(rfd_plan_t plan);

/* Copy the plan's random features and (if computed) G to HOST buffers:
 * omega (m/2 x 3), r (m/2), G (m x m, row-major FP64; pass NULL to skip, or
 * if rfd_features has not run).  Synchronises the stream. */
RFD_API rfd_status rfd_plan_export(rfd_plan_t plan, double* omega, double* r, double* G);

/* Statistics of the plan (host struct; synchronises the plan's stream). */
RFD_API rfd_status rfd_plan_stats(rfd_plan_t plan, rfd_stats* out);

/* Zero the accumulated step timings and launch count of a plan. */
RFD_API rfd_status rfd_plan_stats_reset(rfd_plan_t plan);

/* ---------------------------------------------------------------------------
 * Batches: many point clouds of uneven N and m integrated by shared launches
 * (one launch per step for all clouds; step a4 of every cloud on the
 * FP64-accurate tensor-core emulation with per-cloud scaling).  A batch is a
 * fixed list of BF16 plans (RFD_BF16_TC, each listed once) and uses their
 * device buffers; it runs on its own stream, and a plan in a batch must not
 * be used on its own while a batch call on it may be in flight.
 * --------------------------------------------------------------------------- */
typedef struct rfd_batch_s* rfd_batch_t;

/* Per-cloud arguments of a batched call (device pointers; see rfd_gfi). */
typedef struct {
  const float* d_points;  /* N x 3 (features / gfi)                       */
  const float* d_F;       /* N x c, leading dimension ldF (integrate / gfi) */
  float* d_out;           /* N x c, leading dimension ldOut; may equal d_F */
  int32_t c;
  int32_t reserved_;
  int64_t ldF, ldOut;
} rfd_batch_item;

/* Build a batch over `count` plans (caller-owned array, copied).  flags:
 * RFD_FLAG_TIMING, RFD_FLAG_GRAPH or 0.  Allocates the batch's device tables
 * (one block) and pinned staging (one block); RFD_EINVAL for FP32 plans or a
 * repeated plan. */
RFD_API rfd_status rfd_batch_create(const rfd_plan_t* plans, int32_t count, int32_t flags, void* cuda_stream,
                                    rfd_batch_t* out);
RFD_API rfd_status rfd_batch_destroy(rfd_batch_t batch);
/* Batched rfd_features / rfd_integrate / rfd_gfi: items[k] belongs to plans[k].
 * features and gfi wait once on the batch stream for the largest per-cloud
 * squaring count of step a4 (each cloud's count is chosen on the device).
 * rfd_batch_sync returns RFD_ENUMERIC naming the clouds whose G was not
 * finite since the last rfd_batch_sync (the other clouds' results stand),
 * or RFD_ETIMEDOUT if a bounded device-side wait ran out. */
RFD_API rfd_status rfd_batch_features(rfd_batch_t batch, const rfd_batch_item* items);
RFD_API rfd_status rfd_batch_integrate(rfd_batch_t batch, const rfd_batch_item* items);
RFD_API rfd_status rfd_batch_gfi(rfd_batch_t batch, const rfd_batch_item* items);
RFD_API rfd_status rfd_batch_sync(rfd_batch_t batch);
/* Step timings / launch count of the batch (RFD_FLAG_TIMING), as rfd_plan_stats. */
RFD_API rfd_status rfd_batch_stats(rfd_batch_t batch, rfd_stats* out);
RFD_API rfd_status rfd_batch_stats_reset(rfd_batch_t batch);
/* Batched rfd_eigenvalues from points: steps a2-a3 for every cloud
 * (items[k].d_points; d_F, d_out and c unused), no step a4 (each plan's G is
 * left invalid: run rfd_batch_features before integrating), then the k
 * smallest / largest eigenvalues of every cloud's exp(lambda W_hat) into
 * d_out (count x k float32, device, row k per cloud).  Every plan needs
 * m <= 128 and N >= k.  Asynchronous on the batch stream. */
RFD_API rfd_status rfd_batch_eigenvalues(rfd_batch_t batch, const rfd_batch_item* items, int32_t k, int32_t largest,
                                         float* d_out);

/* ---------------------------------------------------------------------------
 * Serving: a request loop for GFI requests (the paper's graph field
 * integration, Sec. 2.4, one request = one point cloud and one field F).
 * rfd_submit only queues; executor threads admit queued requests in arrival
 * order as device memory allows (a fixed budget, allocated once, from which
 * plans and batch tables are carved), batch the admitted requests of all sizes
 * that are waiting when an executor is free, and run them on the BF16
 * tensor-core batched path.  Several batches are in flight at once on
 * separate streams, so requests that arrive while others run are started as
 * soon as an executor and memory free up.  A request that names a resident
 * cloud reuses its G (only steps a3(Y)-a6 run); clouds submitted with keep = 1
 * stay resident, in the compact form of rfd_plan_compact (points, frequencies,
 * M, G), until memory is needed (least recently used first) or the server is
 * destroyed.
 * --------------------------------------------------------------------------- */
typedef struct rfd_server_s* rfd_server_t;

typedef struct {
  size_t mem_budget;   /* device bytes for plans, resident clouds and batch tables   */
  int32_t max_queue;   /* queued + running requests before RFD_EBUSY (0: 4096)       */
  int32_t max_batch;   /* requests per batch (0: 256)                                */
  int32_t executors;   /* batches in flight at once, one stream each (0: 2, max 8)   */
  int32_t reserved_;
} rfd_server_config;

typedef struct {
  const float* d_points; /* N x 3 float32 device; may be NULL when `cloud` is resident   */
  const float* d_F;      /* N x c float32 device, leading dimension ldF                 */
  float* d_out;          /* N x c float32 device, leading dimension ldOut; may equal d_F */
  int64_t n;
  int64_t ldF, ldOut;
  int32_t m;             /* random features (even); ignored for a resident cloud       */
  int32_t c;             /* 1 <= c <= 256                                               */
  double eps, lambda;    /* as rfd_params                                               */
  uint64_t seed;
  uint64_t cloud;        /* 0, or a resident cloud to reuse: its id is the ticket of the
                            request that kept it (keep = 1), which may still be pending:
                            this request then waits for it                             */
  int32_t keep;          /* 1: keep this request's cloud resident (id = this ticket)   */
  int32_t max_channels;  /* channel capacity of a kept cloud for later requests (0: c)  */
} rfd_request;

typedef struct {
  int32_t status;        /* the request's own outcome (an rfd_status)                   */
  int32_t reused;        /* 1 if a resident cloud's G (and its points) were reused     */
  uint64_t cloud;        /* id of the resident cloud (keep = 1: this ticket; reuse), else 0 */
  double queue_ms;       /* rfd_submit -> its batch's launch                            */
  double latency_ms;     /* rfd_submit -> the server saw its batch complete            */
  int32_t batch_size;    /* requests in the batch that ran it                          */
  int32_t reserved_;
} rfd_result;

typedef struct {
  int64_t submitted, completed, rejected, batches, reused, evicted, resident;
  int64_t mem_used, mem_peak, mem_budget;  /* device bytes */
  int64_t kernel_launches;
} rfd_server_stats;

/* Create a server on the current device.  cfg: host, may be NULL (then a
 * budget of mem_budget bytes and the defaults above).  Allocates the whole
 * budget up front (RFD_ENOMEM if it cannot) and starts the executor threads. */
RFD_API rfd_status rfd_server_create(size_t mem_budget, const rfd_server_config* cfg, rfd_server_t* out);

/* Stop the server: queued requests that have not started complete with
 * status RFD_EBUSY; running batches finish first.  Frees all of its memory. */
RFD_API rfd_status rfd_server_destroy(rfd_server_t server);

/* Queue one request (host struct, copied).  Never blocks on the device.
 * *ticket receives the id to poll.  RFD_EINVAL for invalid arguments or an
 * unknown cloud id with no points; RFD_EBUSY when admission is refused: the
 * queue is full, or the request alone needs more than the memory budget.
 * The request's device buffers must stay valid until rfd_poll reports it. */
RFD_API rfd_status rfd_submit(rfd_server_t server, const rfd_request* request, uint64_t* ticket);

/* Wait up to timeout_us microseconds (0: do not wait) for a ticket.
 * RFD_OK: done, *out holds its result and the ticket is retired;
 * RFD_ENOTREADY: not done and timeout_us == 0; RFD_ETIMEDOUT: not done when
 * the wait ran out; RFD_EINVAL: unknown or retired ticket. */
RFD_API rfd_status rfd_poll(rfd_server_t server, uint64_t ticket, int32_t timeout_us, rfd_result* out);

/* Counters of the server (host struct). */
RFD_API rfd_status rfd_server_stats_get(rfd_server_t server, rfd_server_stats* out);

/* Thread-local description of the last error on this thread ("" if none). */
RFD_API const char* rfd_last_error(void);

/* Library version string. */
RFD_API const char* rfd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RFD_H_ */
