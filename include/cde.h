/*
 * cde.h -- C ABI of the GB300 (sm_103a) library for the double-kernel
 * conditional density estimator of Holmes, Gray & Isbell, "Fast Nonparametric
 * Conditional Density Estimation".
 *
 * Notation (the paper's h1/h2 roles are swapped here; this library uses):
 *   h1 = bandwidth of the x kernel (d_x dimensions, isotropic),
 *   h2 = bandwidth of the y kernel (scalar y).
 *   K_h(t) = h^{-d} K(t/h) (Sec. 2), K one of two radial kernel families,
 *   chosen per dataset at creation:
 *     Gaussian (default): K the standard normal density;
 *     Epanechnikov (CDE_KERNEL_EPANECHNIKOV, the kernel of all the paper's
 *     experiments, Sec. 4): K(t) = c_d (1 - |t|^2) for |t| < 1, else 0,
 *     c_d = (d + 2) / (2 V_d), V_d = pi^{d/2} / Gamma(d/2 + 1).
 *   fhat(y|x) = sum_i K_h1(|x-x_i|) K_h2(y-y_i) / sum_i K_h1(|x-x_i|)   (Eq. 1)
 *   A_j = sum_{i!=j} K_h1(|x_j-x_i|) K_h2(y_j-y_i),
 *   B_j = sum_{i!=j} K_h1(|x_j-x_i|)                          (Sec. 3.2)
 *   L_cond(h1,h2) = sum_j ln(A_j / B_j)      (conditional LOO log-likelihood)
 *   L_eq3(h1,h2)  = (1/N) sum_j ln A_j - ln(N-1)   (Eq. 3 and its expansion)
 *   With the Epanechnikov kernel sums can be exactly zero: A_j = 0 (and the
 *   0/0 case B_j = 0) give ln(A_j/B_j) = -inf, so a score is -inf at
 *   bandwidths where some left-out point has no neighbour inside the supports
 *   (the divergence at small bandwidths of Sec. 4.1); a density query with no
 *   x-neighbour inside h1 gets fhat = 0.
 *
 * Conventions for every entry point:
 *   - Returns a cde_status; never aborts the process.  On failure the
 *     thread-local message from cde_last_error() says what went wrong.
 *   - Inputs are copied or only read; the caller keeps ownership of every
 *     pointer it passes.  Outputs go to caller-owned buffers.
 *   - Pointers are host pointers unless a flag or argument says device.
 *     Device pointers must be CUDA device memory on the context's device.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the context's own
 *     stream.  Calls whose outputs are host memory are synchronous; calls
 *     with CDE_OUT_DEVICE only enqueue work on the stream.
 *   - Invalid sizes or non-finite values give CDE_EINVAL; a bandwidth must be
 *     finite and in [1e-12, 1e12].
 *   - A context may be used from several host threads; calls are serialised
 *     internally except the request queue, which is thread-safe by design.
 */
#ifndef CDE_H
#define CDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cde_ctx cde_ctx;   /* opaque: device, streams, datasets */
typedef int64_t cde_dataset;      /* handle of a device-resident dataset */

typedef enum {
    CDE_OK = 0,
    CDE_EINVAL = 1,     /* bad argument */
    CDE_ENOMEM = 2,     /* memory budget or device allocation refused */
    CDE_ECUDA = 3,      /* CUDA runtime error (message has the CUDA text) */
    CDE_EBUSY = 4,      /* request queue full */
    CDE_ETIMEOUT = 5,   /* cde_wait ran out before the request finished, or a tensor-core
                           kernel's bounded on-device wait ran out (results invalid) */
    CDE_ENOTFOUND = 6,  /* unknown dataset handle or ticket */
    CDE_ECANCELED = 7   /* request cancelled before it ran */
} cde_status;

enum { CDE_OUT_DEVICE = 1,    /* output pointers are device memory; call is async */
       CDE_IN_DEVICE = 2,     /* input arrays (x, y, queries, grids) are device memory */
       CDE_KERNEL_EPANECHNIKOV = 4 };  /* cde_create_dataset: Epanechnikov kernels (Sec. 4) */

enum { CDE_KERNEL_GAUSS = 0, CDE_KERNEL_EPAN = 1 };  /* values reported by cde_dataset_kernel */

/* Library version string (static storage). */
const char *cde_version(void);

/* Message of the last failed call on this host thread (static/thread storage,
 * valid until the next call on the same thread). */
const char *cde_last_error(void);

/* Create a context on CUDA device `device`.  `mem_budget_bytes` caps the
 * device memory held by resident datasets and admitted serving jobs
 * (0 = 90% of the device's free memory).  *ctx receives the context. */
int cde_init(cde_ctx **ctx, int device, size_t mem_budget_bytes);

/* Stop the request loop (if running), free every dataset and the context. */
void cde_shutdown(cde_ctx *ctx);

/*
 * Make a dataset resident on the device.
 *   x: N x d_x row-major float32; y: N float32 (host, or device with
 *   CDE_IN_DEVICE in `flags`).  standardize != 0 centres each x dimension and
 *   divides it by its sample standard deviation (ddof = 1), in FP64 (Sec. 4);
 *   y is never scaled.  Requires N >= 2, d_x >= 1, finite values, and a
 *   non-zero spread in every dimension when standardising.
 *   CDE_KERNEL_EPANECHNIKOV in `flags` makes every score, gradient and
 *   density on this dataset use Epanechnikov kernels on x and y (default:
 *   Gaussian).  For Gaussian datasets the call also computes, once, each row's
 *   nearest squared distance to any other row in x and in y (the per-row
 *   shifts used to keep exp2 in range); Epanechnikov sums need no shift.
 *   *out receives the handle.  Memory: about (d_x + 3) * 4 * N bytes.
 */
int cde_create_dataset(cde_ctx *ctx, const float *x, const float *y, int64_t N, int d_x,
                       int standardize, int flags, cde_dataset *out);

/* Release a dataset's device memory.  CDE_ENOTFOUND for an unknown handle. */
int cde_destroy_dataset(cde_ctx *ctx, cde_dataset ds);

/* Size, dimension and (when standardised) per-dimension mean and sd of a
 * dataset; mean/sd may be NULL, otherwise arrays of d_x doubles. */
int cde_dataset_info(cde_ctx *ctx, cde_dataset ds, int64_t *N, int *d_x, double *mean,
                     double *sd);

/*
 * Device index checks of a checked build (libcde_checked.so, compiled with
 * -DCDE_CHECKS; the closed sanitizers' stand-in): *enabled = 1 there, and
 * *code receives the first failed check's code since the last call (0: none)
 * and clears it -- a failed check redirects its access to index 0 instead of
 * faulting.  In the normal library *enabled = 0.  In both builds a
 * tensor-core kernel whose bounded on-device wait ran out reports
 * CDE_CHECK_TENSOR_WAIT | (which waits) here when no index check failed, and
 * the report is cleared: bits 0x1 and 0x2 for cde_density, 0x100 ... 0x1000
 * for the d_x >= 16 gradient (cde_loo_grad, cde_loo_grad_rows), 64 for
 * cde_selftest_wait.  The synchronous calls also return CDE_ETIMEOUT then.
 * Waits for the device to be idle.
 * enabled may be NULL.
 */
#define CDE_CHECK_TENSOR_WAIT 0x10000u

/* Self-test of the bounded on-device waits (failure detection without a GPU
 * fault): one thread waits on an mbarrier that nothing arrives on, with the
 * limit the tensor-core kernels use (about 2^31 SM cycles, a second), then
 * records wait code 64; returns CDE_OK once the kernel has finished.  A
 * following cde_check_status reports CDE_CHECK_TENSOR_WAIT | 64. */
int cde_selftest_wait(cde_ctx *ctx);
int cde_check_status(cde_ctx *ctx, unsigned int *code, int *enabled);

/* Per-row nearest squared distances of a Gaussian dataset, the exp2 shifts:
 * nn_x2[j] = min_{i != j} |x_j - x_i|^2 (stored, possibly standardised x; FP32,
 * accumulated dimension by dimension with fused multiply-adds as in every pair
 * kernel), nn_y2[j] = min_{i != j} (y_j - y_i)^2.  Host arrays of N floats;
 * either may be NULL.  Zeros for Epanechnikov datasets (no shift). */
int cde_dataset_nn(cde_ctx *ctx, cde_dataset ds, float *nn_x2, float *nn_y2);

/* The other coordinate's distance of each row's nearest neighbours, stored
 * with the shifts of a Gaussian dataset: other_y2[j] = (y_j - y_i)^2 for the
 * x-nearest point i of row j, other_x2[j] = |x_j - x_i|^2 for its y-nearest
 * point (when several points are nearest, the smallest such distance).  Every
 * minimiser over i of a1 |x_j - x_i|^2 + a2 (y_j - y_i)^2 (a1, a2 > 0), the
 * dominant term of A_j in Eq. 3 at any bandwidths, lies within both bounds:
 * the exact recomputation of cells whose separably shifted sum underflowed
 * uses them to skip points.  Host arrays of N floats, either may be NULL;
 * zeros for Epanechnikov datasets. */
int cde_dataset_nn_other(cde_ctx *ctx, cde_dataset ds, float *other_x2, float *other_y2);

/*
 * The tile partition of a LOO launch (host query, no GPU needed): n_units units
 * (rows / rows per unit), units_per_tile units per small tile, ctas resident
 * CTAs of the launch.  Writes the number of tiles; for tile >= 0 also its units
 * unit_first + m * unit_stride, m < unit_count, added to the tile's FP64 slot in
 * that order.  Every tile's units are distinct and together they are 0 ..
 * n_units - 1.  Any output may be NULL.  (The same code the kernels run; the
 * result of a launch depends on this partition only.)
 */
int cde_loo_tile_partition(int64_t n_units, int units_per_tile, int ctas, int tile, int *n_tiles,
                           int *unit_first, int *unit_stride, int *unit_count);

/*
 * Kernel timing (a profiling aid).  With timing on, these calls record CUDA
 * events on their stream around their dominant kernel: cde_loo_loglik and
 * cde_loo_rows (the exact-LOO tile kernel, from the first to the last launch
 * of the call for grids wider than 32), cde_density (the tensor-core
 * kernel), cde_loo_grad (the pair kernel), cde_cond_stats (the pair kernel)
 * and cde_loo_loglik_batch (the replay of its captured graph).
 * cde_timing_last waits for the latest recorded end event and returns the
 * milliseconds between the pair; CDE_EINVAL when nothing has been recorded
 * since timing was (re)enabled.  The request queue's jobs are not timed.
 */
int cde_timing_enable(cde_ctx *ctx, int on);
int cde_timing_last(cde_ctx *ctx, double *ms);

/* Kernel family of a dataset: *kernel = CDE_KERNEL_GAUSS or CDE_KERNEL_EPAN. */
int cde_dataset_kernel(cde_ctx *ctx, cde_dataset ds, int *kernel);

/*
 * Exact LOO log-likelihood over a bandwidth grid (Eq. 3 and Sec. 3.2),
 * every pair (j, i != j) evaluated once for all G1 x G2 bandwidth pairs.
 *   h1[G1], h2[G2]: host arrays of bandwidths (any order, G1,G2 >= 1).
 *   L_cond_out, L_eq3_out: G1 x G2 row-major (h1 major) doubles; either may be
 *   NULL.  Host memory unless flags has CDE_OUT_DEVICE.
 * Numerics: pair sums in FP32 with per-row shifts (exp2 on the SFU),
 * exact joint-shift recomputation of any cell whose shifted numerator falls
 * below 2^(ceil(log2 N) - 91) (so that terms lost to the FP32 range stay
 * below 2^-24 of it), log-ratio and the sum over j in FP64 in a fixed order (the
 * result is bitwise reproducible).  Epanechnikov datasets: the kernel
 * profile (1 - t^2/h^2)_+ by one saturating FP32 FMA per factor, no shifts,
 * and -inf scores where a sum is zero (see the notation above).
 */
int cde_loo_loglik(cde_ctx *ctx, cde_dataset ds, const double *h1, int G1, const double *h2,
                   int G2, double *L_cond_out, double *L_eq3_out, int flags, void *stream);

/*
 * cde_loo_loglik without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * a process whose device memory is owned by another allocator (for example a
 * framework's caching allocator that has reserved most of HBM, so a
 * cudaMalloc here could fail or fragment its pool), a latency-bound service
 * loop in which cudaMalloc/cudaFree may synchronise the device and stall other
 * work, or a host that forbids allocation calls to the plugins it loads.
 *   Same scores as cde_loo_loglik (up to the order of FP64 additions) for one
 *   grid of at most 32 x 32 bandwidths; larger grids give CDE_EINVAL.  For
 *   d_x >= 16 this entry point forms the squared distances directly (the
 *   Gram-form kernel of cde_loo_loglik needs a per-CTA buffer larger than the
 *   fixed scratch), so the two agree within the FP32 distance precision there.
 *   d_L_cond, d_L_eq3: caller-owned DEVICE arrays of G1 x G2 doubles (either
 *   may be NULL); the call only enqueues work on `stream` (NULL: the context's
 *   stream) and returns.
 *   Scratch: the tile partials and the tile counter live in one fixed 16 MiB
 *   array in the library's device memory, held on every GPU that loads the
 *   library until the process exits; tiles are enlarged so that any N fits.
 *   The first call on a device looks up that array's address (set-up); make
 *   it before any stream capture.  Every call uses the same array and it keeps
 *   the last call's contents (the counter is cleared by each call), so calls
 *   whose work overlaps on the GPU -- on different streams or contexts, or
 *   from different host threads -- race and give wrong results: order them.
 *   Calls no cudaMalloc, cudaFree or other allocating routine.
 */
int cde_loo_loglik_noalloc(cde_ctx *ctx, cde_dataset ds, const double *h1, int G1,
                           const double *h2, int G2, double *d_L_cond, double *d_L_eq3,
                           void *stream);

/*
 * Per-row terms ell_j(k,l) = ln(A_j/B_j) for a list of rows (Eq. 1 at the
 * left-out point), for checking full-size runs row by row.
 *   rows[n_rows]: host int64 row indices in [0, N); ell_out: n_rows x G1 x G2
 *   doubles (host).
 */
int cde_loo_rows(cde_ctx *ctx, cde_dataset ds, const double *h1, int G1, const double *h2,
                 int G2, const int64_t *rows, int64_t n_rows, double *ell_out, void *stream);

/*
 * L_cond and its gradient with respect to (ln h1, ln h2) at one bandwidth
 * pair (derivative of the Sec. 3.2 sums for the Gaussian kernel):
 *   dL/dln h1 = sum_j (E_Aj[|dx|^2] - E_Bj[|dx|^2]) / h1^2,
 *   dL/dln h2 = sum_j (E_Aj[dy^2] / h2^2 - 1),
 * E_Aj weighting i by K_h1 K_h2 and E_Bj by K_h1.
 *   out3 = {L_cond, dL/dln h1, dL/dln h2} (host, or device with CDE_OUT_DEVICE).
 * For d_x >= 16 the squared distances come from the Gram form
 * n_j + n_i - 2 x_j.x_i with 3xTF32 dot products on the tensor cores (absolute
 * error up to about 2^-19 (n_j + n_i)); CDE_ETIMEOUT if one of that kernel's
 * bounded device waits ran out (results invalid).
 */
int cde_loo_grad(cde_ctx *ctx, cde_dataset ds, double h1, double h2, double *out3, int flags,
                 void *stream);

/* Per-row terms of cde_loo_grad for every row: rows_out is N x 3 doubles
 * (host) holding {ell_j, d ell_j/d ln h1, d ell_j/d ln h2} (for checking). */
int cde_loo_grad_rows(cde_ctx *ctx, cde_dataset ds, double h1, double h2, double *rows_out,
                      void *stream);

/*
 * Conditional density fhat(y|x) of Eq. 1 (all N points, no leave-one-out) at
 * Q query points and a G_y-point y grid.
 *   xq: Q x d_x row-major float32 in the dataset's ORIGINAL units (the
 *   dataset's standardisation is applied to the queries); ygrid: G_y float32;
 *   f_out: Q x G_y float32.  CDE_IN_DEVICE: xq and ygrid are device memory;
 *   CDE_OUT_DEVICE: f_out is device memory.  Q >= 0 (Q = 0 is a no-op).
 */
int cde_density(cde_ctx *ctx, cde_dataset ds, double h1, double h2, const float *xq, int64_t Q,
                const float *ygrid, int G_y, float *f_out, int flags, void *stream);

/*
 * Many datasets in one persistent launch inside a captured CUDA graph.
 *   n datasets ds[n]; per dataset b: h1[b] (G1[b] doubles), h2[b] (G2[b]
 *   doubles), outputs L_cond_out[b] / L_eq3_out[b] (G1[b] x G2[b] doubles, host;
 *   either array of pointers, or an entry, may be NULL).  Every G must be
 *   <= 32.  The result of each dataset is bitwise identical to
 *   cde_loo_loglik on that dataset alone.  Datasets with d_x >= 16 (whose
 *   single launch uses the Gram-form distance kernel) are run by that launch,
 *   one per dataset, before the batched graph of the others.
 */
int cde_loo_loglik_batch(cde_ctx *ctx, int n, const cde_dataset *ds, const double *const *h1,
                         const int *G1, const double *const *h2, const int *G2,
                         double *const *L_cond_out, double *const *L_eq3_out, void *stream);

/*
 * Autotuner of the LOO launch for one grid shape class (grids are padded to
 * 16 or 32 in G1 and 8, 16 or 32 in G2).  It times every tile configuration
 * -- units per tile (rows per tile = units x 1024 / (T1 T2); the d >= 16
 * kernel's units are fixed) and resident CTAs per SM (1 or 2) -- with the
 * single-dataset launch on dataset `ds`, keeps the fastest in the context and
 * marks the class tuned.  cde_loo_loglik, the chunked and no-alloc launches
 * and cde_loo_loglik_batch all read the kept configuration, so their results
 * stay bitwise identical to each other.  Outputs may be NULL.
 *
 * cde_loo_loglik_batch tunes, by default, every shape class of its batch that
 * is not yet tuned (on the class's largest dataset, before building the
 * batch's graph) and then writes the tuning cache named by CDE_TUNING_CACHE,
 * if set.  cde_autotune_enable(ctx, 0), or CDE_AUTOTUNE=0 in the environment
 * at cde_init, turns this off (untuned classes then run the defaults).
 */
int cde_autotune(cde_ctx *ctx, cde_dataset ds, const double *h1, int G1, const double *h2, int G2,
                 int *units_per_tile, int *ctas_per_sm, double *best_ms);
int cde_autotune_enable(cde_ctx *ctx, int on);
/* Read / set the tile parameters for the shape of a G1 x G2 grid (0 = default:
 * 8 rows per tile, halved while a dataset's grid would give fewer than 64 tiles
 * per resident CTA; cde_tuning_get reports the 8-row value then).  Setting any
 * non-zero value marks the class tuned; setting both to 0 returns it to its
 * defaults and to untuned.  cde_tuning_get_ex also reports the tuned flag. */
int cde_tuning_get(cde_ctx *ctx, int G1, int G2, int *units_per_tile, int *ctas_per_sm);
int cde_tuning_get_ex(cde_ctx *ctx, int G1, int G2, int *units_per_tile, int *ctas_per_sm, int *tuned);
int cde_tuning_set(cde_ctx *ctx, int G1, int G2, int units_per_tile, int ctas_per_sm);
/*
 * Tuning cache on disk: cde_tuning_save writes all shape classes' parameters
 * (units per tile, CTAs per SM, tuned flag) with the device's name, compute
 * capability and SM count (atomically, via a temporary file and rename);
 * cde_tuning_load applies a file written for the same device (CDE_EINVAL for
 * another device, another format version or a malformed file, CDE_ENOTFOUND
 * when it cannot be read).  cde_init loads the file named by the environment
 * variable CDE_TUNING_CACHE when it exists and matches.
 */
int cde_tuning_save(cde_ctx *ctx, const char *path);
int cde_tuning_load(cde_ctx *ctx, const char *path);

/* ------------------------------------------------------------------ */
/* Bandwidth selection as in the paper (Sec. 3.5, Sec. 4)              */
/* ------------------------------------------------------------------ */
enum { CDE_L_COND = 0, CDE_L_EQ3 = 1 };   /* which score a selector maximises */

/*
 * Random-search selection (Sec. 3.5; bandwidths sampled from [0, h_max],
 * Sec. 4).  Each of `rounds` rounds draws G1 values of h1 uniformly from
 * (0, h1_max] and G2 values of h2 from (0, h2_max], scores all G1 x G2 pairs
 * exactly (one grid evaluation, as cde_loo_loglik) and keeps the pair with the
 * largest score `objective` (CDE_L_EQ3: the paper's Eq. 3; CDE_L_COND: the
 * conditional score).  Draws: value k of the SplitMix64 stream of `seed`
 * (Steele, Lea & Flood 2014; counter form z = seed + (k+1) 0x9E3779B97F4A7C15,
 * then the published mixing steps) gives u = (z >> 11) 2^-53 and
 * h = h_max (1 - u), raised to at least 1e-6 h_max; round r uses k = r (G1 + G2)
 * + 0 .. G1-1 for h1, then the next G2 values for h2.
 *   best[4] (host) = {h1, h2, L_cond, L_eq3} of the first strict maximum in
 *   (round, k, l) order; scores of -inf never win (all -inf: best h = NaN).
 *   Optional host outputs (NULL to skip): h1_out[rounds x G1],
 *   h2_out[rounds x G2], Lc_out / Le_out[rounds x G1 x G2].
 *   1 <= G1, G2 <= 32; h_max in [1e-6, 1e6].  Synchronous.
 */
int cde_select_random(cde_ctx *ctx, cde_dataset ds, double h1_max, double h2_max, int rounds,
                      int G1, int G2, uint64_t seed, int objective, double *best,
                      double *h1_out, double *h2_out, double *Lc_out, double *Le_out);

/*
 * Reference-rule bandwidths (the paper's baseline, Sec. 4.2, after Silverman):
 * each kernel gets the AMISE-optimal bandwidth of an unconditional KDE of a
 * normal density with the data's spread, h = A(K, d) sigma n^{-1/(d+4)}, with
 * A^{d+4} = 4/(d+2) for the Gaussian and 8 (d+4) (2 sqrt(pi))^d / V_d for the
 * Epanechnikov kernel (V_d the unit-ball volume).  h1: the dataset's d_x
 * dimensions as stored (standardised if it was created so), sigma^2 their mean
 * sample variance; h2: d = 1, sigma the sample sd of y.  Synchronous.
 */
int cde_reference_rule(cde_ctx *ctx, cde_dataset ds, double *h1, double *h2);

/* ------------------------------------------------------------------ */
/* Products of fhat(.|x) used by the paper's evaluation (Sec. 4.2)     */
/* ------------------------------------------------------------------ */
/*
 * Per query q (all N data points, no leave-one-out), with the x weights
 * u_qi = K_h1(x_q - x_i) of Eq. 1:
 *   mean_out[q] = E[y | x_q] = sum_i u_qi y_i / sum_i u_qi   (the y kernel is
 *                 symmetric; NaN when the x-support is empty -- Epanechnikov);
 *   fat_out[q]  = fhat(yq[q] | x_q), Eq. 1 at one point (0 when the x-support
 *                 is empty; Gaussian values below about 2^-126 of the
 *                 conditional peak flush to 0).
 *   xq: Q x d_x row-major float32 in the dataset's original units; yq: Q
 *   float32 (needed for fat_out only).  Either output may be NULL.  Outputs
 *   are doubles, host unless CDE_OUT_DEVICE; CDE_IN_DEVICE: xq/yq on device.
 * Sums in FP32 per data-range split, splits combined in FP64.
 */
int cde_cond_stats(cde_ctx *ctx, cde_dataset ds, double h1, double h2, const float *xq,
                   const float *yq, int64_t Q, double *mean_out, double *fat_out, int flags,
                   void *stream);

/*
 * Prediction intervals (Sec. 4): for each query, S draws from fhat(.|x_q)
 * and the narrowest window [lo, hi] of ceil((1 - alpha) S) consecutive sorted
 * draws.  A draw picks data index i with probability u_qi / sum u (inverse
 * CDF over the cumulative weights in a fixed order) and adds h2 e, e drawn
 * from the y kernel by inverse CDF (Gaussian: Phi^{-1}(V); Epanechnikov:
 * 2 sin(asin(2V - 1)/3)).  Random numbers: value k of the SplitMix64 stream of
 * `seed` (as in cde_select_random), k = 2 (q S + s) for draw s of query q and
 * k + 1 for its kernel offset, u = ((z >> 40) + 1/2) 2^-24.
 *   1 <= S <= 4096, 0 < alpha < 1.  lo_out, hi_out: Q floats; samples_out
 *   (optional): Q x S sorted draws.  NaN for a query whose x-support is empty.
 *   Host outputs unless CDE_OUT_DEVICE; CDE_IN_DEVICE: xq on device.
 */
int cde_cond_interval(cde_ctx *ctx, cde_dataset ds, double h1, double h2, const float *xq,
                      int64_t Q, int S, double alpha, uint64_t seed, float *lo_out, float *hi_out,
                      float *samples_out, int flags, void *stream);

/* ------------------------------------------------------------------ */
/* Request queue (continuous batching of density and selection jobs)   */
/* ------------------------------------------------------------------ */
enum { CDE_REQ_DENSITY = 0, CDE_REQ_SELECT = 1 };

typedef struct {
    int kind;              /* CDE_REQ_DENSITY or CDE_REQ_SELECT */
    cde_dataset ds;
    /* density: bandwidths, queries (host, Q x d_x, original units), y grid, output */
    double h1, h2;
    const float *xq;
    int64_t Q;
    const float *ygrid;
    int G_y;
    float *f_out;          /* Q x G_y, host, written when the ticket completes */
    /* selection: a G1 x G2 grid search followed by n_steps gradient-ascent
     * steps in (ln h1, ln h2) from the best grid cell (step size `lr`). */
    const double *h1_grid;
    int G1;
    const double *h2_grid;
    int G2;
    int n_steps;
    double lr;
    double *sel_out;       /* 4 doubles: best h1, best h2, L at best, L of the grid best */
    double *L_grid_out;    /* optional G1 x G2 L_cond of the grid (host) */
} cde_request;

typedef struct {
    int n_streams;          /* concurrent jobs on the device (default 4) */
    int queue_capacity;     /* pending requests before cde_submit returns CDE_EBUSY */
    size_t job_mem_budget;  /* device bytes admitted jobs may hold at once (0 = ctx budget) */
} cde_server_config;

/* Start the request loop (a native scheduler thread).  cfg may be NULL. */
int cde_server_start(cde_ctx *ctx, const cde_server_config *cfg);
/* Stop the loop after the running jobs finish; pending jobs are cancelled. */
int cde_server_stop(cde_ctx *ctx);
/* Queue a request; *ticket identifies it.  The request's buffers must stay
 * valid until the ticket completes.  CDE_EBUSY when the queue is full. */
int cde_submit(cde_ctx *ctx, const cde_request *req, int64_t *ticket);
/* *done = 1 when finished (then *status holds the job's cde_status). */
int cde_poll(cde_ctx *ctx, int64_t ticket, int *done, int *status);
/* Wait up to timeout_us microseconds (< 0: no limit); CDE_ETIMEOUT if not
 * finished.  On completion returns the job's own status.  Never hangs. */
int cde_wait(cde_ctx *ctx, int64_t ticket, int64_t timeout_us);
/* Cancel a queued request (CDE_OK) -- running ones finish normally. */
int cde_cancel(cde_ctx *ctx, int64_t ticket);

typedef struct {
    int64_t completed, cancelled, failed;
    double p50_ms, p99_ms, mean_ms;     /* submit -> completion latency */
    double p50_density_ms, p99_density_ms, p50_select_ms, p99_select_ms;
    double busy_s;                       /* wall time with >= 1 job on the device */
    int64_t peak_concurrent;             /* most jobs admitted at once */
    int64_t peak_selection;              /* most selection jobs admitted at once (at most half
                                            of the stream slots, at least one) */
} cde_server_stats;

int cde_server_stats_get(cde_ctx *ctx, cde_server_stats *out);
/* Forget collected latencies (counters restart at zero). */
int cde_server_stats_reset(cde_ctx *ctx);

/* ------------------------------------------------------------------ */
/* Measured pipe rates of this GPU (roofline denominators)             */
/* ------------------------------------------------------------------ */
typedef struct {
    int sm_count;
    double sm_clock_mhz;        /* clock seen by the micro-benchmark kernels */
    double ffma_per_clk_sm;     /* FP32 FMA lanes per clock per SM */
    double ex2_per_clk_sm;      /* MUFU ex2 results per clock per SM */
    double ffma_tops;           /* FP32 FMA per second, whole GPU (1e12) */
    double ex2_tops;            /* ex2 per second, whole GPU (1e12) */
    double umma_bf16_mac_per_clk_sm;  /* tcgen05.mma kind::f16, BF16 in / FP32 accumulate,
                                         M = 128, N = 256, K = 16, back to back from one
                                         thread: multiply-adds per clock per SM */
    double umma_bf16_tflops;    /* the same, whole GPU at the clock seen (2 flop per MAC, 1e12) */
    double mma_tf32_mac_per_clk_sm;   /* legacy mma.sync m16n8k8 TF32, FP32 accumulate */
    double mma_bf16_mac_per_clk_sm;   /* legacy mma.sync m16n8k16 BF16, FP32 accumulate */
    double umma_tf32_mac_per_clk_sm;  /* tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, back to
                                         back from one thread (the d >= 16 gradient's dot products) */
} cde_peaks;

int cde_measure_peaks(cde_ctx *ctx, cde_peaks *out);

#ifdef __cplusplus
}
#endif
#endif /* CDE_H */
