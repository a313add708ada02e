/*
 * geo.h -- C ABI of the mixed-precision Gaussian log-likelihood library (libgeo.so).
 *
 * The library evaluates, on one CUDA device (sm_103a), the Gaussian
 * log-likelihood of Eq. 2,
 *     l(theta) = -n/2 log(2 pi) - 1/2 log|Sigma(theta)| - 1/2 Z' Sigma(theta)^-1 Z,
 * for the Matern covariance of Eq. 1 over 2D locations, by the mixed-precision
 * tile Cholesky factorization of Algorithm 1: tiles within `band` (the paper's
 * diag_thick) tiles of the diagonal are held and updated in FP64, all others in
 * FP32 storage with FP32-accurate arithmetic.
 *
 * Conventions shared by every call
 *  - Memory: the caller owns every buffer.  Pointers named d_* are device
 *    pointers, h_* host pointers.  The library never allocates device memory and
 *    never frees a caller's buffer (exception: geo_tiles_bind creates two CUDA
 *    events and one stream, released by geo_tiles_release).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated otherwise.
 *  - Layout: locations are structure-of-arrays FP64 x[n], y[n]; Z is FP64[n].
 *    Inputs are expected in Morton order (geo_morton_order), which the
 *    likelihood does not depend on but the mixed-precision error does.
 *    Tiles: p = ceil(n/nb) tiles per side; the n x n matrix is padded to p*nb
 *    with decoupled identity rows (which add 0 to log|Sigma| and to Z'Sigma^-1 Z).
 *    Lower tile (i,j), i >= j, is FP64 iff i - j < band.  Every tile is stored
 *    contiguously, column-major, leading dimension nb, in the FP64 store
 *    (band tiles) or the FP32 store (off-band tiles).
 *  - Errors: 0 = GEO_OK; a negative value -k means argument k (1-based) was
 *    invalid (nothing was launched); positive values are the GEO_ERR_* codes.
 *    Device-side failures (non-SPD pivot, scheduler timeout) are recorded in the
 *    status words of the bound workspace and returned by the blocking calls or
 *    read with geo_status.
 */
#ifndef GEO_H
#define GEO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GEO_OK 0
#define GEO_ERR_NOT_SPD 1      /* a diagonal pivot was <= 0 (or NaN); info = 1-based global row */
#define GEO_ERR_TIMEOUT 2      /* a device-side wait exceeded its bound; work was abandoned */
#define GEO_ERR_CUDA 3         /* a CUDA runtime call failed */
#define GEO_ERR_UNSUPPORTED 4  /* a valid but unimplemented configuration */
#define GEO_ERR_TOO_LARGE 5    /* the problem exceeds a fixed-size internal buffer */

/* LP (off-band) arithmetic.  GEO_LP_SPLIT_BF16 (the name of the tensor-core
 * slice mode) runs the off-band updates on the tcgen05 tensor cores: each
 * panel row is scaled by a power of two and cut exactly into an 8-bit and two
 * 12-bit integer slices held in FP16 planes; six FP16 slice products (those of
 * weight >= 2^-24 of the leading one) are accumulated in FP32 tensor memory,
 * the leading product exactly.  In-band updates use seven 8-bit slices held in
 * BF16.  GEO_LP_FP32 runs the off-band updates as FP32 FMA on the CUDA cores.
 * Both store off-band tiles in FP32. */
#define GEO_LP_SPLIT_BF16 0
#define GEO_LP_FP32 1

/* Matern parameters (Eq. 1): theta1 = sigma2 (variance), theta2 = beta (range),
 * theta3 = nu (smoothness); nugget tau2 >= 0 is added to the diagonal. */
typedef struct geo_theta {
    double sigma2, beta, nu, nugget;
} geo_theta;

/* Sizes of one problem's tile store and workspace, computed by geo_layout_init.
 * All byte counts are for caller-allocated device buffers (256-byte aligned). */
typedef struct geo_layout {
    int n, nb, p, band, lp_mode;
    int pp;                       /* BF16 plane edge: nb rounded up to a multiple of 64 */
    long long n_dp_tiles, n_sp_tiles, n_slots;
    size_t bytes_dp;              /* FP64 tile store */
    size_t bytes_sp;              /* FP32 tile store */
    size_t bytes_planes;          /* BF16 slice planes + row exponents of panel tiles (0 for GEO_LP_FP32) */
    size_t bytes_meta;            /* offset tables and status words */
} geo_layout;

/* A bound problem: layout + the caller's device buffers + library stream/events. */
typedef struct geo_tiles {
    geo_layout lay;
    double* d_dp;
    float* d_sp;
    void* d_planes;
    void* d_meta;
    void* aux_stream;             /* library-created stream for concurrent off-band work */
    void* ev_fork;
    void* ev_join;
    unsigned long long tmap[48];  /* library-private: three TMA descriptors of the BF16 planes */
    int flags;                    /* GEO_FLAG_* options, set with geo_tiles_set_flags */
    void* trace;                  /* optional device trace buffer (geo_tiles_set_trace) */
    long long trace_cap;          /* its capacity in records */
    long long timeout_ns;         /* bound of every device-side wait (geo_tiles_set_timeout_ns); 0 = default */
    int far_products;             /* far tier (geo_tiles_set_far): 0 = off, else 1 or 3 products */
} geo_tiles;

/* One record of the device-side task trace (tensor-core mode scheduler):
 * type 0..4 = potrf sub-block factor / solve / update, panel trsm, FP64 (DMMA)
 * update item; 5, 6 = forward-solve diagonal / block-row task; 7, 8 = the
 * dpotrf chain tasks PC, PC2 (a = 0); 10 = tensor-core off-band update item
 * (t_claim = its epilogue started, t_ready = its products were done),
 * 11 = tensor-core in-band (FP64-accurate) update item; 12, 13 = one sub-step
 * s (in a) of PC: the factor of (s,s), the solve of (s+1,s), with t_claim =
 * sub-step start, t_ready = its dependencies met, t_end = done; 14 = one
 * (column slice, contraction part) of an in-band item (c = slice * parts +
 * part), t_ready = its products done, t_end = drained; 15 = the MMA
 * thread's view of an off-band item (t_claim = began waiting for its first
 * stage, t_ready = that stage arrived, t_end = its last MMA issued); 16 = the
 * copy thread's view (t_claim = before taking it from the queue, t_ready =
 * its panel tiles were solved, t_end = its first stage's copies issued).  Times are
 * %globaltimer nanoseconds: t_claim when the task was taken, t_ready when its
 * dependencies were met, t_end when it finished. */
typedef struct geo_trace_rec {
    int type, sm, k, a, b, c;
    long long t_claim, t_ready, t_end;
} geo_trace_rec;

/* Generation option: compute off-band (FP32-stored) covariance entries in FP64
 * and round them to FP32 (Algorithm 1's dlag2s of the FP64 value) instead of
 * computing them in compensated FP32 arithmetic (the default, ~8x fewer FP64
 * operations; entries within 8 2^-24 relative for nu in {1/2, 3/2, 5/2} and
 * (16 + 4 nu |ln x|) 2^-24 otherwise, x = r/theta2). */
#define GEO_FLAG_FP64_OFFBAND_GEN 1
/* Scheduling option (tensor-core mode only): run Algorithm 1 as host-sequenced
 * outer steps (per step: potrf, trsm, slicing, then the FP64 and tensor-core
 * updates concurrently) instead of the persistent device-side task scheduler.
 * Same arithmetic; kept for comparison. */
#define GEO_FLAG_STEPWISE 2
/* Arithmetic option (tensor-core mode only): run the in-band (FP64 target)
 * dsyrk/dgemm updates of Algorithm 1 on the FP64 pipe (DMMA) instead of the
 * default FP64-accurate tensor-core products.  The default splits each operand
 * into seven 8-bit fixed-point slices, forms the 28 slice products of weight
 * >= 2^-48 with exact integer accumulation for the leading 15 and drains every
 * 256-long part of the contraction into the FP64 tile: its rounding error is
 * no larger than that of FP64 accumulation (measured against exact sums). */
#define GEO_FLAG_FP64_DMMA 4
/* Approximation option (tensor-core mode, default scheduler): the Diagonal
 * Super-Tile (DST) method of Section V-B, the tile form of the independent-
 * blocks (IND) approximation.  Tile (i,j) of the covariance is kept, in FP64,
 * when i - j < band and set to zero otherwise; the factorization, log-
 * determinant and solve then follow Eq. 2 for that matrix.  Its Cholesky
 * factor has the same tile band, so no task is scheduled for the zero tiles:
 * the work falls from O(n^3) to O(n nb^2 band^2).  With band = 1 the tiles are
 * independent blocks.  The zeroed matrix need not be positive definite: a
 * failing pivot reports GEO_ERR_NOT_SPD as for any other matrix.  Not with
 * GEO_FLAG_STEPWISE or GEO_FLAG_FP64_DMMA (geo_tiles_set_flags returns -2). */
#define GEO_FLAG_DST 8
/* Test hook (persistent scheduler only): the tensor-core update items of the
 * first step wait for one more solved row chunk of their panel tile than the
 * tile has, so that dependency can never be met; that wait's bound is half the
 * store's, so it gives up before the waits downstream of it.  The bounded wait
 * then ends the launch: the status words record GEO_ERR_TIMEOUT with the
 * wait's location code (31, read back by geo_status), every worker leaves, the
 * tensor-core group returns its tensor memory, and the store can be evaluated
 * again once the flag is cleared.  Used with a short geo_tiles_set_timeout_ns
 * bound to exercise the failure path without faulting or hanging the device. */
#define GEO_FLAG_TEST_STALL 16
/* Default bound of a device-side wait of the persistent scheduler. */
#define GEO_DEFAULT_TIMEOUT_NS 10000000000LL
/* Fewest CTAs a partial launch (geo_batch_set_ctas) may use: three CUDA-core
 * groups carry a diagonal tile's two chain tasks and the sub-tasks those wait
 * for, and one more serves the FP64 bulk queue. */
#define GEO_MIN_CTAS 4

/* A1, "appropriate ordering" (Section VI): Z-order permutation of n locations.
 * Each coordinate c (expected in [0,1]) is quantised to q = clamp(floor(c*2^16),
 * 0, 2^16-1); the key interleaves qx (even bits) and qy (odd bits); perm[new] =
 * old index, sorted by (key, old index).  Host-only; x, y, perm are host arrays.
 * Returns 0 or -k for a bad argument k. */
int geo_morton_order(const double* x, const double* y, int n, int* perm);

/* Fill *out with the tile geometry and buffer sizes for n locations, tile size
 * nb (16 <= nb <= 768) and band (1 <= band; band >= p means all tiles FP64).
 * Pure host arithmetic. */
int geo_layout_init(int n, int nb, int band, int lp_mode, geo_layout* out);

/* Bind caller-owned device buffers (sizes from *lay) to t and write the offset
 * tables into d_meta.  Blocks until the tables are on the device.  Creates one
 * non-blocking stream and two events (released by geo_tiles_release).
 * d_planes may be NULL when lay->bytes_planes == 0. */
int geo_tiles_bind(geo_tiles* t, const geo_layout* lay, void* d_dp, void* d_sp,
                   void* d_planes, void* d_meta, void* stream);
int geo_tiles_release(geo_tiles* t);
int geo_tiles_set_flags(geo_tiles* t, int flags);
/* Bound, in nanoseconds of %globaltimer, of every wait inside the persistent
 * factorization kernel on this store (a dependency counter, a queue claim, a
 * copy or tensor-core hand-off): a wait that exceeds it abandons the launch
 * with GEO_ERR_TIMEOUT and a location code in the status words (geo_status),
 * and the store stays usable.  Batched launches use the bound of their first
 * item's store.  ns = 0 restores the default GEO_DEFAULT_TIMEOUT_NS; otherwise
 * 1e5 <= ns <= 1e12 (returns -2 outside).  Legitimate waits last at most as
 * long as the factorization itself. */
int geo_tiles_set_timeout_ns(geo_tiles* t, long long ns);
/* Record every scheduler task of the following factorizations into d_trace
 * (device memory: one unsigned long long record counter, padded to 64 bytes,
 * then `capacity` geo_trace_rec).  The caller zeroes the counter; records past
 * the capacity are dropped (the counter keeps counting).  NULL disables. */
int geo_tiles_set_trace(geo_tiles* t, void* d_trace, long long capacity);

/* Three-precision extension (the paper's future work, Section IX: a third,
 * lower precision for the tiles farthest from the diagonal).  Off-band tiles
 * marked far keep their FP32 storage and FP32 panel solve, but their
 * trailing updates use fewer fixed-point slice products on the tensor cores:
 * each panel row, scaled by its power of two, is cut into an 8-bit slice a0
 * and a 12-bit slice a1 (the same planes the FP32-accurate tier reads), and
 *   products = 3: a0 b0 + 2^-12 (a0 b1 + a1 b0)   (terms of weight >= 2^-12;
 *                 relative error ~2^-16 per product term, half the MMAs),
 *   products = 1: a0 b0                           (8-bit operands, 1/6 of the MMAs).
 * A tile (i, j) is far when i - j >= far_band (far_band >= 1; 0: no band rule),
 * or, with far_dist > 0, when the smallest distance between the bounding boxes
 * of the two tiles' locations (d_x, d_y: device FP64[n], the locations the
 * store is evaluated on, Morton-ordered) is at least far_dist; in-band (FP64)
 * tiles are never far.  The tile map is computed once here (on `stream`,
 * asynchronously) and kept in the store's meta buffer until the next call;
 * far_band = 0 and far_dist <= 0 turn the tier off.  Tensor-core mode with the
 * persistent scheduler only (the GEO_LP_FP32 mode and GEO_FLAG_STEPWISE return
 * GEO_ERR_UNSUPPORTED).  Returns 0, -k for a bad argument k, or GEO_ERR_CUDA. */
int geo_tiles_set_far(geo_tiles* t, int far_band, const double* d_x, const double* d_y, double far_dist,
                      int products, void* stream);

/* A2, Eq. 1: write Sigma_ab = C(||s_a - s_b||; theta) (+ nugget if a == b) into
 * every lower tile, each directly in its own precision (the FP64 -> FP32
 * conversion of Algorithm 1's first loop is fused into generation).  The
 * strictly upper triangle of a diagonal tile, which no later step reads, is
 * written as 0.  d_x, d_y: device FP64[n].  Asynchronous. */
int geo_matern_tiles(geo_tiles* t, const double* d_x, const double* d_y, geo_theta theta, void* stream);

/* Scatter a dense symmetric n x n FP64 matrix (device, column-major, ld = n,
 * lower triangle read) into the tile store, rounding off-band tiles to FP32.
 * Test utility for factor parity.  Asynchronous. */
int geo_tiles_load_dense(geo_tiles* t, const double* d_a, void* stream);

/* Gather the lower triangle of the tile store into a dense n x n FP64 matrix
 * (device, column-major, ld = n; FP32 tiles promoted exactly, upper triangle
 * set to 0).  Asynchronous. */
int geo_tiles_to_dense(const geo_tiles* t, double* d_out, void* stream);

/* A3-A9, Algorithm 1: factor the tile store in place, A = L L', with the
 * precision map of the bound layout (its band; band >= p is the all-FP64
 * path).  In GEO_LP_SPLIT_BF16 mode the tile tasks run in one persistent
 * cooperative kernel that schedules them on the device by dependency counters
 * (one CTA per SM; the device must be otherwise idle enough to host it).  On a non-positive pivot the factorization stops early and the status
 * words record GEO_ERR_NOT_SPD with info = 1-based global row.  Asynchronous;
 * read the outcome with geo_status. */
int geo_potrf_mp(geo_tiles* t, void* stream);

/* A10-A11, Eq. 2: from the factored store and Z (device FP64[n]), write
 * d_logdet[0] = log|Sigma| = 2 sum log L_ii and d_quad[0] = ||L^-1 Z||^2
 * (device FP64 scalars), and, if d_y != NULL, y = L^-1 Z (device FP64[p*nb]).
 * FP64 accumulation.  When the store's status records a failed factorization
 * (not positive definite, timeout) both scalars are set to NaN.  Asynchronous. */
int geo_logdet_trsv(const geo_tiles* t, const double* d_z, double* d_logdet, double* d_quad,
                    double* d_y, void* stream);

/* Allocation-free variant of geo_logdet_trsv (the paper has no counterpart:
 * this is an interface for callers that cannot allocate device memory).
 * Callers that cannot call cudaMalloc -- code running while a CUDA graph is
 * being captured, or inside a framework whose memory pool owns the device and
 * forbids side allocations -- would otherwise have to size and pass the
 * solve's scratch themselves.  Here the scratch (the forward-solve vector and
 * the per-tile partial sums) lives in a fixed array in the library's device
 * memory: at most GEO_NOALLOC_MAX_N padded locations (p * nb) and
 * GEO_NOALLOC_MAX_P tiles per side; larger problems return GEO_ERR_TOO_LARGE
 * without launching anything.  The caller still passes the factored store, Z
 * and the two output scalars (device FP64), exactly as for geo_logdet_trsv.
 * When the store's factorization failed both scalars are set to NaN (never a
 * stale value left in the array by an earlier call).
 * The array is shared by every call in the process: calls whose work overlaps
 * on the GPU (different streams, no ordering between them) race on it.  The
 * first call on each device looks up the array's device address (no
 * allocation); make that first call before any stream capture.  Asynchronous. */
#define GEO_NOALLOC_MAX_N 262144
#define GEO_NOALLOC_MAX_P 4096
int geo_logdet_trsv_noalloc(const geo_tiles* t, const double* d_z, double* d_logdet, double* d_quad,
                            void* stream);

/* Copy the status words to the host (blocking on `stream`): *h_code = GEO_OK or
 * a GEO_ERR_* code; *h_info = the 1-based failing row for GEO_ERR_NOT_SPD, the
 * location code of the wait that gave up for GEO_ERR_TIMEOUT. */
int geo_status(const geo_tiles* t, int* h_code, int* h_info, void* stream);

/* A2-A12: generation, Algorithm 1, log-determinant, forward solve and
 * assembly of Eq. 2 (Section IV, Eq. 1-2; Algorithm 1), enqueued on `stream`
 * without waiting.  d_res (caller-owned device FP64[3]) receives
 *   d_res[0] = log|Sigma|, d_res[1] = Z' Sigma^-1 Z,
 *   d_res[2] = l(theta) = -n/2 log(2 pi) - d_res[0]/2 - d_res[1]/2,
 * all computed on the device.  d_x, d_y, d_z: device FP64[n], Morton-ordered,
 * read only.  On the persistent tile-DAG path (split-BF16 stores) the forward
 * solve runs inside the factorization launch, per element the same arithmetic
 * as geo_logdet_trsv.  A failure (not positive definite, timeout) is recorded
 * in the status words (geo_status) and leaves NaN in all three entries.
 * Returns GEO_OK or a negative argument index / GEO_ERR_CUDA. */
int geo_loglik_async(geo_tiles* t, const double* d_x, const double* d_y, const double* d_z, geo_theta theta,
                     double* d_res, void* stream);

/* A2-A12: full evaluation of Eq. 2 (generation, Algorithm 1, log-det, solve,
 * assembly).  Blocking: returns after the scalars are on the host.
 * h_out[0] = l(theta), h_out[1] = log|Sigma|, h_out[2] = Z' Sigma^-1 Z.
 * Returns GEO_OK, GEO_ERR_NOT_SPD (with *h_info set, h_out undefined), or an error. */
int geo_loglik(geo_tiles* t, const double* d_x, const double* d_y, const double* d_z,
               geo_theta theta, double* h_out, int* h_info, void* stream);

/* Maximum likelihood estimation (Section IV-C).  theta-hat maximises Eq. 2
 * over (sigma2, beta, nu), or, with profile = 1, Eq. 3 over (beta, nu) with
 * theta1 = Z' S~^-1 Z / n (S~ the covariance at unit variance, the nugget taken
 * relative to theta1).  The paper drives this with NLopt at tolerance 1e-3
 * without naming the method; the reading here is the Nelder-Mead simplex
 * (Nelder & Mead 1965) over the logarithms of the free parameters:
 * simplex theta0 and theta0 * e^step in each free parameter; each iteration
 * orders the vertices by -l (ties: the earlier position first), stops when
 * every vertex is within xtol of the best (max norm), and replaces the worst
 * by the reflection (coefficient 1), expansion (2), outside or inside
 * contraction (1/2) or shrinks towards the best (1/2); trial points are
 * clamped to [lo, hi]; an evaluation that is not positive definite counts as
 * l = -inf.  At most max_evals likelihood evaluations (each a full A2-A12
 * pass on t, blocking), and the best point evaluated is returned. */
typedef struct geo_mle_opts {
    int max_evals;        /* evaluation budget (default 60) */
    int profile;          /* 0: Eq. 2 over 3 parameters; 1: Eq. 3 over (beta, nu) */
    int fix_nu;           /* 1: nu stays at theta0.nu */
    double xtol;          /* simplex-size stop in log-parameter space (default 1e-3) */
    double step;          /* initial simplex step in log space (default 0.1) */
    double lo[3], hi[3];  /* box on (sigma2, beta, nu) (defaults [1e-3,1e2], [1e-4,2], [0.05,3]) */
    /* Optional evaluation journal (host memory, default NULL), for runs split
     * over several calls: journal_cap records of 4 doubles (sigma2, beta, nu,
     * f = -l, +inf when not positive definite), in evaluation order.  On entry
     * *journal_len records are already present: the estimator's first
     * *journal_len evaluations take their values from them instead of the
     * device (the simplex is deterministic, so it retraces the same points; a
     * point that differs from its record returns -6).  Every new evaluation is
     * appended while there is room, and *journal_len is updated.  A run with
     * max_evals = E and the journal of an earlier run with a smaller budget
     * therefore gives the same estimate as one uninterrupted run of E. */
    double* journal;
    int journal_cap;
    int* journal_len;
} geo_mle_opts;

typedef struct geo_mle_result {
    geo_theta theta;      /* theta-hat (nugget as given in theta0) */
    double loglik;        /* l at theta-hat: Eq. 2, or Eq. 3 with profile = 1 */
    int evals;            /* likelihood evaluations made */
    int iterations;       /* completed simplex iterations */
    int not_spd;          /* evaluations that were not positive definite */
} geo_mle_result;

/* Fill *o with the defaults above.  Returns 0, or -1 for NULL. */
int geo_mle_default_opts(geo_mle_opts* o);
/* Run the estimator on the bound store t (its layout fixes n, nb, band and
 * the arithmetic).  Locations and Z are caller-owned device arrays.  Returns
 * GEO_OK with *out filled, -k for a bad argument k, or the first error other
 * than GEO_ERR_NOT_SPD that an evaluation returned. */
int geo_mle(geo_tiles* t, const double* d_x, const double* d_y, const double* d_z, geo_theta theta0,
            const geo_mle_opts* opts, geo_mle_result* out, void* stream);

/* Batched evaluation: many problems of their own n, tile size, band and theta
 * through one persistent factorization launch (the tasks of all problems share
 * the device-side queues, merged step by step, each problem keeping its own
 * dependency order).  Each item is a bound store with its Morton-ordered
 * locations and Z (device arrays).  Per problem the arithmetic is that of
 * geo_loglik, operation for operation, so a problem's result is the same
 * alone and in any batch.
 *
 * geo_batch_workspace: bytes of device workspace for these items (host only).
 * geo_batch_bind: write the merged task queues (factorization and forward
 *   solve), the per-problem views, tensor maps and generator table into d_work
 *   (blocking); GEO_ERR_TOO_LARGE if the problems' generation needs more than
 *   2^31 - 1 CTAs.  The stores' flags are read here.
 * geo_loglik_batch: enqueue one evaluation (asynchronous, two kernel
 *   launches and three memsets, no host synchronization, so it can be captured
 *   in a CUDA graph): one launch generating every problem's tiles from
 *   d_theta[b] (device memory: a replay of a captured graph may use new
 *   values; the problems' CTAs share the launch), then one
 *   persistent launch that factors every problem and runs its forward solve,
 *   log-determinant and assembly as soon as its own factor is ready, writing
 *   d_out[3b .. 3b+2] = (l, log|Sigma|, Z' Sigma^-1 Z) (device FP64[3 nprob]);
 *   NaN for a problem that is not positive definite (its store's status says
 *   which row).  d_done_ns (optional, device int64[nprob + 1]): [0] = the
 *   launch's start and [1 + b] = when problem b's result was written, in
 *   %globaltimer nanoseconds (0 if it failed), for per-problem latency.  A
 *   timeout ends the launch and marks every unfinished problem with
 *   GEO_ERR_TIMEOUT.  A trace enabled on the first item's store
 *   (geo_tiles_set_trace) records the tasks of all problems; the wait bound is
 *   the first item's (geo_tiles_set_timeout_ns).
 * geo_batch_set_ctas: run this workspace's factorization launches on `ctas`
 *   CTAs (one per SM at most) instead of one per SM (ctas = 0, the default, a
 *   cooperative launch of every SM).  With GEO_MIN_CTAS <= ctas < SM count the
 *   launch is a plain one: launches on other streams (another batch, kriging)
 *   run beside it on the remaining SMs.  The schedule needs no co-residency
 *   beyond GEO_MIN_CTAS workers: the queues are claimed in a topological
 *   order, at most a third of the CUDA-core groups (at least three) work in
 *   the priority queue while FP64 bulk items exist, and the forward-solve
 *   queue is taken only when ready, so every wait is on a task a running
 *   worker holds or can take.  1 <= ctas < GEO_MIN_CTAS is refused (-2).
 * geo_batch_release: forget the workspace's binding (host bookkeeping only;
 *   the caller frees d_work).
 * All return 0, -k for a bad argument k, or GEO_ERR_CUDA. */
typedef struct geo_batch_item {
    geo_tiles* t;
    const double* d_x;
    const double* d_y;
    const double* d_z;
} geo_batch_item;

int geo_batch_workspace(int nprob, const geo_batch_item* items, size_t* bytes);
int geo_batch_bind(int nprob, const geo_batch_item* items, void* d_work, size_t bytes, void* stream);
int geo_loglik_batch(int nprob, const geo_batch_item* items, const geo_theta* d_theta, void* d_work,
                     double* d_out, long long* d_done_ns, void* stream);
int geo_batch_set_ctas(const void* d_work, int ctas);
int geo_batch_release(const void* d_work);

/* A13, prediction (Section VIII-D; simple kriging reading): with t holding the
 * factor of Sigma(theta) over the observed locations (d_x, d_y, n = t->lay.n)
 * and observations d_z, write d_zhat[m] = Sigma_new,obs Sigma^-1 Z for the m
 * new locations (d_xnew, d_ynew).  With GEO_FLAG_DST on t (Section V-B) the
 * factor is that of the truncated covariance, and Sigma_new,obs is truncated
 * the same way: a new location keeps its covariances with the observed
 * points whose tile is within `band` tiles of its own tile, the tile of its
 * nearest observed point (lowest index on a tie).  d_work: device FP64
 * scratch of 2 * p * nb doubles.  Asynchronous. */
int geo_krige(const geo_tiles* t, const double* d_x, const double* d_y, const double* d_z,
              geo_theta theta, const double* d_xnew, const double* d_ynew, int m,
              double* d_zhat, double* d_work, void* stream);

/* Instrumentation.  geo_kernel_launches returns the number of kernel launches
 * this library has issued in the process (all entry points, all devices).
 * geo_profile_enable(1) makes geo_potrf_mp (and the evaluation calls) bracket
 * each launch of its kernels with CUDA events on the stream it launches them on;
 * geo_profile_read (blocking: synchronizes those events) returns, for
 * kind 0 = FP64 update (dsyrk/dgemm), 1 = off-band update (tensor-core or
 * FP32), 2 = diagonal-tile potrf, 3 = panel trsm (kinds 0-3: the step-by-step
 * driver), 4 = the persistent tile-DAG kernel (the whole factorization in one
 * launch), 5 = the covariance generation of geo_loglik / geo_loglik_async, the
 * summed event time in ms and the launch count since the last
 * geo_profile_reset.  An unknown kind returns -1. */
unsigned long long geo_kernel_launches(void);
int geo_profile_enable(int on);
int geo_profile_reset(void);
int geo_profile_read(int kind, double* h_ms, long long* h_launches);

#ifdef __cplusplus
}
#endif
#endif /* GEO_H */
